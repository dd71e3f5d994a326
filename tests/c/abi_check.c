/* C99 client of the MTPT C ABI (include/mtpt.h): takes the address of every
 * entry point (so a missing symbol fails the link) and exercises the calls
 * that need no GPU -- parameter validation, handle creation and destruction,
 * state errors before particles are set, status strings.  Prints "ok" and
 * returns 0 when every expectation holds. */
#include <stdio.h>
#include <string.h>

#include "mtpt.h"

typedef void (*any_fn)(void);
#define ENTRY(f) ((any_fn)(f))

static int failures = 0;
#define EXPECT(cond)                                                    \
    do {                                                                \
        if (!(cond)) {                                                  \
            fprintf(stderr, "line %d: expectation failed: %s\n", __LINE__, #cond); \
            ++failures;                                                 \
        }                                                               \
    } while (0)

int main(void) {
    const any_fn entries[] = {
        ENTRY(mtpt_check_word), ENTRY(mtpt_create), ENTRY(mtpt_destroy),
        ENTRY(mtpt_set_stream), ENTRY(mtpt_set_particles), ENTRY(mtpt_set_particles_device),
        ENTRY(mtpt_create_batch), ENTRY(mtpt_set_particles_batch),
        ENTRY(mtpt_get_realisation_info), ENTRY(mtpt_step), ENTRY(mtpt_step_ex),
        ENTRY(mtpt_get_masses), ENTRY(mtpt_get_masses_device), ENTRY(mtpt_get_positions),
        ENTRY(mtpt_get_positions_device), ENTRY(mtpt_get_row_sums), ENTRY(mtpt_get_pairs),
        ENTRY(mtpt_get_info), ENTRY(mtpt_set_step), ENTRY(mtpt_sync),
        ENTRY(mtpt_timing_enable), ENTRY(mtpt_timing_read), ENTRY(mtpt_timing_reset),
        ENTRY(mtpt_step_noalloc), ENTRY(mtpt_adjoint_forward), ENTRY(mtpt_adjoint_backward),
        ENTRY(mtpt_set_tuning), ENTRY(mtpt_get_tuning), ENTRY(mtpt_autotune),
        ENTRY(mtpt_status_string), ENTRY(mtpt_set_particles_async),
        ENTRY(mtpt_get_masses_async)};
    for (size_t k = 0; k < sizeof(entries) / sizeof(entries[0]); ++k) EXPECT(entries[k] != NULL);

    mtpt_params p;
    memset(&p, 0, sizeof(p));
    p.dim = 2;
    p.precision = MTPT_FP32W;
    p.D = 1.0;
    p.kappa = 0.5;
    p.dt = 0.1;
    p.beta = 1.0;
    p.lambda = 3.0;
    p.hi[0] = 100.0;
    p.hi[1] = 100.0;
    p.seed = 2204037561u;

    mtpt_handle* h = NULL;
    EXPECT(mtpt_create(&p, &h) == MTPT_OK && h != NULL);
    EXPECT(mtpt_step(h, 1) == MTPT_ERR_STATE);              /* no particles yet */
    EXPECT(mtpt_step(h, -1) == MTPT_ERR_INVALID_ARG);
    double m = 0.0;
    EXPECT(mtpt_get_masses(h, &m) == MTPT_ERR_STATE);
    EXPECT(mtpt_get_masses_async(h, &m) == MTPT_ERR_STATE);
    EXPECT(mtpt_set_particles_async(h, 1, &m, &m) == MTPT_ERR_STATE);
    EXPECT(mtpt_set_particles_async(NULL, 1, &m, &m) == MTPT_ERR_INVALID_ARG);
    EXPECT(mtpt_destroy(h) == MTPT_OK);
    EXPECT(mtpt_destroy(NULL) == MTPT_OK);

    mtpt_params bad = p;
    bad.dim = 4;
    h = NULL;
    EXPECT(mtpt_create(&bad, &h) == MTPT_ERR_INVALID_ARG && h == NULL);
    bad = p;
    bad.lambda = 21.0;
    EXPECT(mtpt_create(&bad, &h) == MTPT_ERR_INVALID_ARG);
    EXPECT(mtpt_create(NULL, &h) == MTPT_ERR_INVALID_ARG);

    /* normal build: no checks (MTPT_ERR_STATE, word 0); checked build: the
     * word, or a CUDA error when no device is present */
    uint32_t word = 1u;
    const int rc = mtpt_check_word(&word, 0);
    EXPECT((rc == MTPT_ERR_STATE && word == 0u) || rc == MTPT_OK || rc == MTPT_ERR_CUDA);

    for (int s = 0; s <= MTPT_ERR_TOO_LARGE; ++s)
        EXPECT(mtpt_status_string(s) != NULL && mtpt_status_string(s)[0] != '\0');

    if (failures == 0) printf("ok\n");
    return failures == 0 ? 0 : 1;
}
