/*
 * mtpt.h -- C ABI of the GB300 mass-transfer particle-tracking (MTPT) step.
 *
 * One time step of the method of Schauer et al., "Parallelized Domain
 * Decomposition for Multi-Dimensional Lagrangian Random Walk, Mass-Transfer
 * Particle Tracking Schemes" (arXiv:2204.03756), Sec. 3:
 *   1. random walk  X_i <- X_i + xi_i sqrt(2 D_RW dt), D_RW = kappa D, with
 *      elastic reflection at the walls of the box (zero-flux boundary);
 *   2. every pair with ||x_i - x_j|| <= psi, psi = lambda sqrt(4 D_MT dt / beta)
 *      (Eq. "cutoff"), D_MT = (1 - kappa) D;
 *   3. Gaussian kernel K_ij of variance h^2 = 2 D_MT dt / beta per axis
 *      (simplified Eq. "kernel");
 *   4. W_ij = K_ij / (1/2 (sum_i K_ij + sum_j K_ij)) = 2 K_ij / (r_i + r_j),
 *      r the row sums of K including the self term;
 *   5. M_i <- M_i + sum_j beta (M_j - M_i) W_ij  (Eq. "changemass", explicit).
 *
 * Conventions shared by every entry point:
 *   - Return value: an mtpt_status code; 0 is success.  No call aborts or
 *     exits the process; no C++ exception crosses the ABI.
 *   - Ownership: the library copies caller buffers in and out; the caller
 *     keeps ownership of its own memory.  The handle owns every device
 *     allocation it makes until mtpt_destroy.
 *   - Positions are structure-of-arrays float64: pos[a * n + i] is axis a of
 *     particle i, a < dim.  Masses are float64, length n.  Particle i of the
 *     last mtpt_set_particles* call keeps index i in every output.
 *   - Stream: all device work of a handle is ordered on the handle's stream
 *     (the legacy default stream unless mtpt_set_stream was called).  Calls
 *     that read host buffers return once the buffers are no longer read (the
 *     rest of their work may still be queued); calls that write host buffers
 *     synchronise the stream before returning; *_device calls only enqueue
 *     work.  The two *_async calls are the exception: they only enqueue
 *     copies, and their host buffers belong to the copy until mtpt_sync.
 *   - Device errors found inside kernels (non-finite positions) are latched
 *     in a device status word and reported by the next synchronising call.
 *   - Threads: a handle is not safe for concurrent calls; use one thread per
 *     handle at a time.  Distinct handles are independent (mtpt_step_noalloc
 *     shares one scratch array per device; see there).
 */
#ifndef MTPT_H
#define MTPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum mtpt_status {
    MTPT_OK = 0,
    MTPT_ERR_INVALID_ARG = 1,     /* null pointer, bad dimension, bad parameter */
    MTPT_ERR_OUT_OF_DOMAIN = 2,   /* a particle outside [lo, hi] or not finite */
    MTPT_ERR_CUDA = 3,            /* a CUDA runtime call failed */
    MTPT_ERR_NO_MEMORY = 4,       /* device or host allocation failed */
    MTPT_ERR_STATE = 5,           /* call not valid in the handle's state */
    MTPT_ERR_CAPACITY = 6,        /* a caller buffer is too small */
    MTPT_ERR_TOO_LARGE = 7        /* problem exceeds mtpt_step_noalloc's fixed scratch */
} mtpt_status;

/* Precision forms of the pair arithmetic. */
typedef enum mtpt_precision {
    /* Every pair weight, sum and flux in binary64 (the paper's method). */
    MTPT_FP64 = 0,
    /* Pair kernel and weights in binary32 with the hardware exp; row sums and
     * per-particle mass accumulation in compensated binary32, the mass update
     * itself in binary64.  The neighbour test stays exact binary64, so the pair
     * set equals MTPT_FP64's, and W_ij = W_ji bit for bit, so every pair flux is
     * exactly antisymmetric. */
    MTPT_FP32W = 1
} mtpt_precision;

/* Flags of mtpt_step_ex. */
enum {
    MTPT_DO_WALK = 1,       /* step 1 (random walk + reflection) */
    MTPT_DO_TRANSFER = 2    /* steps 2-5 (search, kernel, normalise, exchange) */
};

/* Parameters of Sec. 2-3.  dim in {1, 2, 3}; D >= 0; 0 <= kappa <= 1;
 * dt > 0; beta > 0 (the paper takes 1); lambda > 0 (the paper's Eq. "cutoff"
 * prints 6, its cost analysis uses 3 in this notation; see the design notes);
 * lo[a] < hi[a] for a < dim (entries a >= dim are ignored); seed keys the
 * counter-based generator of the walk.  The create and set calls also reject
 * (MTPT_ERR_INVALID_ARG) lambda > 20, |lo[a]| or |hi[a]| above 1e15, and a
 * kernel variance h^2 = 2 (1 - kappa) D dt / beta that is positive but below
 * 1e-35. */
typedef struct mtpt_params {
    int32_t dim;
    int32_t precision;      /* an mtpt_precision */
    double D;
    double kappa;
    double dt;
    double beta;
    double lambda;
    double lo[3];
    double hi[3];
    uint64_t seed;
    double v[3];            /* uniform velocity (the advection term of the model
                             * equation, Sec. 2; the paper's runs take 0): each
                             * axis moves by v[a] dt + sigma xi before the
                             * reflection.  Finite, |v[a] dt| <= 1e15. */
} mtpt_params;

/* Derived quantities and counters of a handle. */
typedef struct mtpt_info {
    int64_t n;                /* particles */
    uint64_t step;            /* walk steps taken so far (the generator's step counter) */
    uint64_t pair_count;      /* ordered neighbour pairs (i != j) summed over transfer steps */
    double D_RW, D_MT;        /* kappa D, (1 - kappa) D */
    double sigma;             /* sqrt(2 D_RW dt) */
    double h2;                /* 2 D_MT dt / beta */
    double psi, psi2;         /* cutoff and its square (as used by the pair test) */
    double kernel_norm;       /* (2 pi h^2)^(-d/2) */
    int32_t cells[3];         /* cell-list grid (1 on unused axes) */
    double cell_width[3];
} mtpt_info;

typedef struct mtpt_handle mtpt_handle;

/* Bounds-check word of the checked build (the library compiled with
 * MTPT_CHECKED, which verifies index invariants of every kernel at run time
 * and skips any access that violates one): *out receives the OR of the
 * violated checks since the last reset on the current device (0: none), after
 * a device synchronisation; reset != 0 clears it.  The normal build compiles
 * the checks out and returns MTPT_ERR_STATE with *out = 0.  No counterpart in
 * the paper: it stands in for a memory checker in the tests. */
int mtpt_check_word(uint32_t* out, int32_t reset);

/* Create a handle on the current CUDA device.  *out receives the handle.
 * Defining passage: the parameters of Sec. 3 -- the split D_RW = kappa D,
 * D_MT = (1 - kappa) D of the diffusion coefficient, the search radius psi of
 * Eq. "cutoff", the kernel bandwidth h^2 = 2 D_MT dt / beta that follows
 * Eq. "kernel", and the domain with zero-flux (reflecting) walls; v is the
 * velocity of the model equation of Sec. 2.
 * Validates the parameters (MTPT_ERR_INVALID_ARG).  Allocates nothing on the
 * device until particles are set. */
int mtpt_create(const mtpt_params* params, mtpt_handle** out);

/* Release every device allocation and the handle.  Synchronises the stream.
 * Passing NULL is a no-op returning MTPT_OK.  Resource management: no
 * counterpart in the paper. */
int mtpt_destroy(mtpt_handle* h);

/* Order all later device work of the handle on `stream` (a cudaStream_t;
 * NULL selects the legacy default stream).  Execution control: no
 * counterpart in the paper. */
int mtpt_set_stream(mtpt_handle* h, void* stream);

/* Load n particles from HOST buffers: pos (dim x n, SoA float64) and mass (n
 * float64).  Defining passage: the particle state of Sec. 2.1 and Sec. 3 --
 * positions X_i inside the domain and masses M_i at the current time (the
 * paper's test problem scatters the particles uniformly and gives them a
 * Heaviside mass, Sec. 2.1).  Every coordinate must be finite and inside [lo, hi] of its axis
 * (MTPT_ERR_OUT_OF_DOMAIN otherwise) and every mass finite, in the precision
 * form at most 1e30 in magnitude (MTPT_ERR_INVALID_ARG otherwise); on either
 * error the handle keeps its old state.  The buffers are copied to the device
 * and checked there: into the free half of the handle's double-buffered state
 * when its capacity already holds n particles, else into a staging area kept
 * by the handle ((dim + 1) n float64).  The call returns once the host buffers
 * are no longer read.
 * Particle ids are 0..n-1 in input order; they key the walk's generator.
 * Resets the step counter and pair counter to 0.  n = 0 is allowed. */
int mtpt_set_particles(mtpt_handle* h, int64_t n, const double* pos, const double* mass);

/* As mtpt_set_particles with DEVICE buffers, enqueued on the stream.
 * The domain check runs on the device; a violation is reported by the next
 * synchronising call. */
int mtpt_set_particles_device(mtpt_handle* h, int64_t n, const double* pos_dev,
                              const double* mass_dev);

/* Batch of independent realisations stepped together (the ensemble form).
 * Defining passage: each realisation is one run of the Sec. 3 step; the
 * paper averages its timings over an ensemble of five independent runs
 * (Sec. 2.3), which a batch steps in one launch per kernel.
 * params[k] holds realisation k's parameters (D, kappa, dt, beta, lambda,
 * box, seed may all differ); dim and precision must be equal across the
 * batch (MTPT_ERR_INVALID_ARG otherwise), 1 <= count <= 2^20.  Every time
 * step is one launch per kernel over all realisations' particles, and
 * realisation k evolves bit for bit as a handle created with params[k] on the
 * same particles would. */
int mtpt_create_batch(const mtpt_params* params, int32_t count, mtpt_handle** out);

/* Load the particles of every realisation of a batch from HOST buffers
 * (the particle state of Sec. 2.1 and Sec. 3, per realisation):
 * counts[k] particles for realisation k (count entries), concatenated in
 * realisation order.  pos is dim x total (SoA over the concatenation: axis a
 * of particle i of realisation k at pos[a * total + offset_k + i], offset_k
 * the sum of the earlier counts), mass is total doubles.  Realisation k's
 * particles must lie inside its own box.  Outputs (masses, positions, row
 * sums) use the same concatenated order; the generator id of a particle is
 * its index within its realisation. */
int mtpt_set_particles_batch(mtpt_handle* h, const int64_t* counts, const double* pos,
                             const double* mass);

/* Derived quantities (Sec. 3) of realisation k of a batch (n is that realisation's
 * particle count; pair_count is not filled). */
int mtpt_get_realisation_info(mtpt_handle* h, int32_t k, mtpt_info* out);

/* Advance nsteps full time steps (walk, then mass transfer on the moved
 * positions).  Defining passage: the time step of Sec. 3 -- the random walk
 * X_i(t + dt) = X_i(t) + xi_i sqrt(2 D_RW dt) with elastic reflection at the
 * walls, every pair within psi of Eq. "cutoff", the simplified kernel that
 * follows Eq. "kernel", the normalisation W_ij = K_ij / (1/2 (column sum +
 * row sum)), and M_i(t + dt) = M_i(t) + delta_i with delta_i of
 * Eq. "changemass", all M_j taken at time t.  Enqueued on the stream;
 * returns the launch status.  Calls of four or more steps replay a CUDA graph
 * captured on first use; in the precision form of a plain handle, the mass
 * transfer of every step of a call but its last also walks the particles for
 * the next step (one kernel instead of two).  Either way the results equal
 * step-by-step launches bit for bit. */
int mtpt_step(mtpt_handle* h, int64_t nsteps);

/* As mtpt_step with a subset of the step: flags is a combination of
 * MTPT_DO_WALK and MTPT_DO_TRANSFER.  The walk's step counter advances only
 * when MTPT_DO_WALK is set. */
int mtpt_step_ex(mtpt_handle* h, int64_t nsteps, int32_t flags);

/* Copy the masses, in input order, to a HOST buffer of n doubles.  Defining
 * passage: the particle masses M_i(t) of Sec. 3 (the paper turns them into
 * concentrations as C = N M / L^d, end of Sec. 3).  Syncs and reports any
 * latched device error. */
int mtpt_get_masses(mtpt_handle* h, double* out);

/* As mtpt_get_masses into a DEVICE buffer of n doubles (stream-ordered). */
int mtpt_get_masses_device(mtpt_handle* h, double* out_dev);

/* Copy the positions, in input order, to a HOST buffer of dim x n doubles
 * (SoA).  Defining passage: the positions X_i(t) produced by the random walk
 * with reflection of Sec. 3.  Syncs. */
int mtpt_get_positions(mtpt_handle* h, double* out);

/* As mtpt_get_positions into a DEVICE buffer of dim x n doubles. */
int mtpt_get_positions_device(mtpt_handle* h, double* out_dev);

/* Row sums r_i = sum_j K_ij of the normalisation of W (Sec. 3; self term
 * included, in the paper's units, i.e.
 * with the factor (2 pi h^2)^(-d/2)) of the most recent transfer step, in
 * input order, to a HOST buffer of n doubles.  MTPT_ERR_STATE before the first
 * transfer step. */
int mtpt_get_row_sums(mtpt_handle* h, double* out);

/* Neighbour pairs of the CURRENT positions -- the neighbour list within psi
 * (Eq. "cutoff") that the search of Sec. 3 provides: every ordered pair (i, j), i != j,
 * with ||x_i - x_j||^2 <= psi^2, as input-order indices, written to the HOST
 * arrays pair_i / pair_j of capacity `cap` (in no particular order).
 * *count receives the number of pairs; if it exceeds cap, only cap pairs are
 * written and MTPT_ERR_CAPACITY is returned.  Syncs.  Intended for tests. */
int mtpt_get_pairs(mtpt_handle* h, int64_t cap, int64_t* count, uint32_t* pair_i,
                   uint32_t* pair_j);

/* Derived quantities of Sec. 3 (D_RW, D_MT, h^2, psi of Eq. "cutoff", the
 * kernel's constant) and counters.  Syncs. */
int mtpt_get_info(mtpt_handle* h, mtpt_info* out);

/* Overwrite the walk's step counter (checkpoint resume, no counterpart in the
 * paper: a run restarted from
 * saved positions and masses with the saved counter reproduces the
 * uninterrupted run bit for bit). */
int mtpt_set_step(mtpt_handle* h, uint64_t step);

/* Wait for the handle's stream (and the copy streams of the *_async calls)
 * and report any latched device error.  Execution control: no counterpart in
 * the paper. */
int mtpt_sync(mtpt_handle* h);

/* Pipelined host I/O (no counterpart in the paper: host traffic around the
 * Sec. 3 step).  A loop that feeds every step from host memory and reads
 * every result back,
 *     repeat: mtpt_set_particles_async; mtpt_step(h, 1); mtpt_get_masses_async
 *     then:   mtpt_sync,
 * overlaps the host-to-device copy of one step's input and the device-to-host
 * copy of another step's masses with the device work of a third.  The copies
 * run on two streams the handle creates for them, ordered against the
 * handle's stream by events, through two device staging slots each way
 * ((dim + 1) n and n float64 per slot, kept by the handle).  Both calls
 * return once the work is enqueued: the host buffers must stay allocated and
 * unchanged (pos, mass) or unread (out) until mtpt_sync returns.  Overlap
 * needs page-locked host memory; pageable memory gives the same results with
 * the copies serialised by the driver. */

/* Pipelined host I/O (no counterpart in the paper).  Enqueue a load of n
 * particles from HOST buffers laid out as for
 * mtpt_set_particles.  n must equal the handle's current particle count
 * (MTPT_ERR_INVALID_ARG otherwise, also for a handle of more than one
 * realisation; MTPT_ERR_STATE before the first load).  The device checks the
 * copy as mtpt_set_particles does and, if it passes, makes it the state that
 * the next step queued on the handle's stream advances (ids 0..n-1, step
 * counter 0).  A rejected load leaves the previous state and step counter in
 * place and is reported once, by the next synchronising call (mtpt_sync or
 * any other call that syncs): MTPT_ERR_OUT_OF_DOMAIN for a position,
 * MTPT_ERR_INVALID_ARG for a mass. */
int mtpt_set_particles_async(mtpt_handle* h, int64_t n, const double* pos, const double* mass);

/* Pipelined host I/O (no counterpart in the paper).  Enqueue a copy of the
 * masses, in input order, into a HOST buffer of n
 * doubles: the masses as they stand after the work queued on the handle so
 * far.  The values are in `out` once mtpt_sync returns.  MTPT_ERR_STATE
 * before the first load; MTPT_ERR_INVALID_ARG for a null `out` with n > 0. */
int mtpt_get_masses_async(mtpt_handle* h, double* out);

/* Per-kernel timing (tracing).  While enabled, every kernel the handle
 * launches is bracketed by two CUDA events on the handle's stream; the
 * elapsed times are summed per kernel name.  Enabling adds two event records
 * per launch and nothing else. */
typedef struct mtpt_kernel_stat {
    char name[40];          /* kernel name, NUL-terminated */
    int64_t launches;       /* launches timed since the last reset */
    double total_ms;        /* summed event-to-event time of those launches */
} mtpt_kernel_stat;

/* Start (on != 0) or stop timing; stopping keeps the collected figures.
 * Tracing: no counterpart in the paper (which profiles with gprof, Sec. 6). */
int mtpt_timing_enable(mtpt_handle* h, int32_t on);

/* Tracing (no counterpart in the paper).  Synchronise, fold pending events
 * into the per-kernel sums, and copy up to
 * `cap` entries into `out`; *count receives the number of distinct kernels. */
int mtpt_timing_read(mtpt_handle* h, int32_t cap, mtpt_kernel_stat* out, int32_t* count);

/* Clear the per-kernel sums (tracing: no counterpart in the paper). */
int mtpt_timing_reset(mtpt_handle* h);

/* One full time step (walk, then mass transfer) on caller-owned DEVICE
 * buffers, without allocating any memory.
 *
 * This entry point has no counterpart in the paper; it exists for callers
 * that cannot allocate device memory when they step the particles: code
 * whose GPU memory is owned entirely by another allocator (a framework's
 * caching allocator, or a host application that reserves the whole device up
 * front), where a cudaMalloc from this library could fail or fragment that
 * pool, and time-critical loops that cannot pay for cudaMalloc/cudaFree
 * (cudaFree synchronises the device).  It creates no handle and calls no
 * cudaMalloc, cudaFree or other allocating routine: its working memory is a
 * fixed file-scope device array of MTPT_NOALLOC_SCRATCH_BYTES (12 MiB) that
 * every GPU which loads this library holds until the process exits.
 *
 * pos_dev (dim x n SoA float64) and mass_dev (n float64) hold the state in
 * the caller's order and are updated in place; particle i is id i for the
 * walk's generator and `step` is the generator's step counter, so the result
 * equals mtpt_set_particles + mtpt_set_step(step) + mtpt_step(1) on the same
 * state.  params is read as in mtpt_create.  Work is enqueued on `stream`
 * (a cudaStream_t; NULL = legacy default stream) and, after the first call
 * on a device, the call does not wait for it: everything the GPU needs from
 * the host travels as kernel arguments.
 *
 * Errors: the return value covers the arguments and the launches only.
 * Positions are not range-checked, and a non-finite or out-of-box position
 * that the step meets is latched in a status word inside the scratch array
 * that no call reads back, so it goes unreported: pass finite particles
 * inside the box.
 *
 * Limits: n <= MTPT_NOALLOC_MAX_PARTICLES (65,536); larger n returns
 * MTPT_ERR_TOO_LARGE before any work is enqueued.  The cell grid is capped
 * at 4 n + 64 cells however sparse the box, so n alone bounds the working
 * memory: the largest layout (3-d, binary32 form, n = 65,536, the cell cap
 * reached) needs about 10.8 MiB of the 12.
 *
 * Shared scratch: every call uses the same array, which keeps the last
 * call's contents (each call clears what must start at zero).  Calls whose
 * GPU work overlaps -- on different streams, or from different threads
 * without ordering -- race on that array and give wrong results; order them
 * on one stream.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current, caches it, and writes a
 * 2 KiB table of the binary64 kernel exponential into the array with one
 * synchronous copy; make that first call on a device before any stream
 * capture begins. */
#define MTPT_NOALLOC_MAX_PARTICLES 65536
#define MTPT_NOALLOC_SCRATCH_BYTES (12u << 20)
int mtpt_step_noalloc(const mtpt_params* params, int64_t n, uint64_t step, double* pos_dev,
                      double* mass_dev, void* stream);

/* Adjoint of a run (no counterpart in the paper, which has no gradient).  For a
 * loss L(M_T) of the final masses, gives dL/dM_0 and dL/dD along the run's own
 * random path (the normals xi stay fixed: pathwise derivative).  The mass
 * update is linear, M_{t+1} = A_t M_t with A_t = I + beta (W_t - diag(W_t 1))
 * symmetric, so dL/dM_0 = A_0 ... A_{T-1} dL/dM_T; D enters through the walk
 * scale (positions) and the kernel bandwidth h^2, and bin or pair-set changes
 * contribute zero almost everywhere.  Single-realisation handles with D > 0
 * and D_MT > 0 only (MTPT_ERR_INVALID_ARG otherwise).  The adjoint passes run
 * in binary64 in both precision forms (for MTPT_FP32W they differentiate the
 * binary64 model at the run's positions, which are the same in both forms). */

/* Adjoint (no counterpart in the paper).  Advance nsteps full steps from the
 * loaded state, as mtpt_step does, while
 * recording a checkpoint of the state every `checkpoint_every` steps and the
 * position tangents dX/dD.  Memory: (nsteps / checkpoint_every +
 * checkpoint_every + 1) snapshots of (4 dim + 12) bytes per particle.
 * Synchronises. */
int mtpt_adjoint_forward(mtpt_handle* h, int64_t nsteps, int64_t checkpoint_every);

/* Adjoint (no counterpart in the paper).  Reverse sweep of the run recorded
 * by mtpt_adjoint_forward: gmass_dev holds
 * dL/dM_T (n doubles, DEVICE, input order); gmass0_dev receives dL/dM_0 (n
 * doubles, DEVICE, input order); *dldD receives dL/dD (HOST).  Recomputes
 * each segment forward from its checkpoint, then steps back through it.
 * Leaves the handle in the final state of the forward run.  Deterministic
 * (fixed summation orders).  Synchronises.  MTPT_ERR_STATE without a recorded
 * run. */
int mtpt_adjoint_backward(mtpt_handle* h, const double* gmass_dev, double* gmass0_dev,
                          double* dldD);

/* Launch tuning.  cell_scale >= 1 widens every cell to cell_scale x psi
 * (fewer, fuller cells; more candidates per particle); cell_scale = 0.5 makes
 * the cells half the cutoff wide, a neighbour then up to two cells away per
 * axis (more, narrower candidate windows closer to the cutoff ball);
 * pair_block is the thread-block size of the binary32 pair passes (128 or
 * 256).  Results do not depend on the tuning beyond rounding (the neighbour
 * sums visit the same pairs in a different order). */
typedef struct mtpt_tuning {
    double cell_scale;
    int32_t pair_block;
    int32_t pad;
} mtpt_tuning;

/* Launch tuning (no counterpart in the paper).  Apply a tuning
 * (MTPT_ERR_INVALID_ARG outside the ranges above); the cell
 * list is rebuilt on the next step. */
int mtpt_set_tuning(mtpt_handle* h, const mtpt_tuning* t);

/* Current tuning (no counterpart in the paper). */
int mtpt_get_tuning(mtpt_handle* h, mtpt_tuning* out);

/* Autotuner (no counterpart in the paper): times `trial_steps` full steps
 * (after one warm-up step) of the
 * loaded particles for every cell_scale in {0.5, 1, 1.25, 1.5, 2} and pair_block
 * in {128, 256}, keeps the fastest, and restores the particles, masses, step
 * counter and pair counter to their state before the call.  Allocates a
 * temporary snapshot of the state.  *chosen (may be NULL) receives the pick.
 * Synchronises. */
int mtpt_autotune(mtpt_handle* h, int32_t trial_steps, mtpt_tuning* chosen);

/* Split domain (Secs. 4-5): one handle per tile of a checkerboard over the
 * box, the tiles exchanging particles once per time step.
 *
 * The box is cut into tiles[a] equal slabs per axis (Sec. 4.2); a particle
 * is native to the tile that contains it (coordinate a in tile
 * floor((x_a - lo_a) / width_a), clamped to the last tile at the upper
 * wall).  Besides its natives a tile holds, for the mass transfer, ghost
 * copies of the particles of other tiles within a pad of its box (Sec. 5).
 * The pad is 2 psi (the paper's is psi): every ghost within psi of the tile
 * then has all its own neighbours in the tile too, so its row sum, which
 * enters the weights W_ij of the natives it touches, is the undivided run's.
 * The tile's cell grid is the undivided run's grid restricted to the tile
 * and its pad, so with ghosts exchanged every step the natives' positions,
 * masses and pair counts are those of one handle holding all n_global
 * particles, bit for bit (the paper's equivalence of the decomposed and the
 * single-domain runs, Sec. 5).  Only natives walk and only natives' masses
 * are kept (Sec. 5).  Generator ids are global, below 2^31.
 *
 * One time step of every tile:
 *   mtpt_step_ex(h, 1, MTPT_DO_WALK);            walk the natives
 *   mtpt_tile_pack(h, cap, send, counts);         records for the other tiles
 *   (the caller moves the records between tiles: all-to-all)
 *   mtpt_tile_transfer(h, n_recv, recv);          mass transfer, natives kept
 * A record is dim + 2 doubles: the coordinates, the mass, the generator id
 * (an integer-valued double).
 *
 * A tiled handle is a single realisation; it refuses the calls that need
 * its whole particle set at once (mtpt_step / mtpt_step_ex with
 * MTPT_DO_TRANSFER, the other loads, mtpt_get_pairs, tuning, autotuning, the
 * adjoint) with MTPT_ERR_STATE.  mtpt_get_masses / mtpt_get_positions /
 * mtpt_get_ids give its natives in the handle's own order, which changes
 * from step to step; mtpt_get_info's n and pair_count are the natives'. */

/* Tiles per axis of a checkerboard of `ntiles` tiles over the box [lo, hi]
 * of `dim` axes, into factors[3] (1 on unused axes).  Defining passage:
 * Eq. "minimization" (Sec. 4.2) in 2-d: f1 <= f2 with f1 f2 = ntiles and
 * |f2 / f1 - A| least for the box's aspect ratio A >= 1, the longer side
 * cut into f2 tiles (the smallest f1 among equals).  In 3-d, where the paper
 * asks only for tiles closest to cubes, the triple whose largest tile edge
 * over its smallest is least (the first in lexicographic order among
 * equals); in 1-d, ntiles slices (Sec. 4.1).  Host arithmetic only. */
int mtpt_tiling_factors(int32_t dim, const double* lo, const double* hi, int32_t ntiles,
                        int32_t* factors);

/* Tile of a checkerboard. */
typedef struct mtpt_tiling {
    int32_t tiles[3];       /* tiles per axis (1 on unused axes) */
    int32_t tile;           /* this tile: t0 + tiles[0] (t1 + tiles[1] t2) */
    int64_t n_global;       /* particles in the whole box (fixes the cell grid) */
} mtpt_tiling;

/* Make h (a single realisation without particles; MTPT_ERR_STATE otherwise)
 * hold one tile of a checkerboard over its box (the subdomains of Sec. 4.2
 * with the ghost pad of Sec. 5).  Every tile must
 * be at least the pad 2 psi wide on each axis cut into more than one tile
 * (MTPT_ERR_INVALID_ARG otherwise); n_global must be below 2^31. */
int mtpt_set_tiling(mtpt_handle* h, const mtpt_tiling* t);

/* Load the tile's natives from HOST buffers: pos (dim x n SoA), mass (n),
 * ids (n global generator ids).  Defining passage: the particle state of
 * Sec. 2.1 and Sec. 3, of one subdomain (Sec. 4).  Every particle must be
 * native to the tile (MTPT_ERR_OUT_OF_DOMAIN otherwise), every mass finite
 * and, in the precision form, at most 1e30 in magnitude, every id below
 * 2^31 (MTPT_ERR_INVALID_ARG otherwise); a rejected load leaves the handle
 * without particles.  Resets the step and pair counters.  Syncs. */
int mtpt_set_particles_tile(mtpt_handle* h, int64_t n, const double* pos, const double* mass,
                            const uint32_t* ids);

/* After the walk of a step: pack, for every other tile, the particles it
 * owns or holds in its pad (Sec. 5) into the DEVICE buffer send_dev of `cap`
 * records -- tile 0's first, then tile 1's and so on, each tile's natives
 * before its ghosts -- and keep this tile's own share on the device for
 * mtpt_tile_transfer.  counts (HOST, 2 x number of tiles) receives for tile t
 * the natives counts[2 t] and ghosts counts[2 t + 1] packed for it; this
 * tile's own entries count what it keeps, and nothing is packed for it.
 * When the records exceed cap, nothing is packed, counts still holds the
 * numbers, and MTPT_ERR_CAPACITY is returned: call again with a larger
 * buffer.  The packed buffer is complete when the handle's stream reaches
 * this point.  Syncs once (for the counts). */
int mtpt_tile_pack(mtpt_handle* h, int64_t cap, double* send_dev, int64_t* counts);

/* Finish a step: the tile's set is what mtpt_tile_pack kept plus the n_recv
 * records received from the other tiles (DEVICE buffer, any order); the
 * mass transfer of Sec. 3 runs on natives and ghosts alike, then the ghosts
 * are dropped (Sec. 5: only natives are updated).  A received record outside
 * the tile's pad box or with a bad id gives MTPT_ERR_INVALID_ARG (it was
 * treated as a ghost and changed no native).  Syncs once. */
int mtpt_tile_transfer(mtpt_handle* h, int64_t n_recv, const double* recv_dev);

/* Bimolecular reaction A + B -> 0, the extension Sec. 8 names (the paper
 * gives no model; this is the library's reading).  Every particle carries a
 * mass of species A (the masses of the other calls) and of species B; each
 * step walks the particles, transfers both species with the same weights
 * W_ij (Sec. 3, Eq. "changemass" for each species), then lets every particle
 * react well mixed over dt: with concentrations C = N M / V (V the box
 * volume; the mass-concentration relation of Sec. 3) the rate law
 * dC_A/dt = dC_B/dt = -k C_A C_B, solved exactly over dt on the particle's
 * masses (rate k N / V).  A particle with a negative mass of either species
 * does not react.  The binary64 form reacts in binary64; the precision form
 * computes the two reaction factors in binary32 and applies them to the
 * binary64 masses.
 *
 * mtpt_set_reaction: turn the reaction on (or change k >= 0, finite;
 * MTPT_ERR_INVALID_ARG otherwise) for a single-run handle that is not a
 * tile (MTPT_ERR_STATE for a batch or a tile).  Species B starts at zero on
 * the loaded particles and on every later load.  Allocates species B's
 * buffers (MTPT_ERR_NO_MEMORY; the handle is then unchanged).  Reaction runs
 * refuse the adjoint and tiling (MTPT_ERR_STATE). */
int mtpt_set_reaction(mtpt_handle* h, double k);

/* Species B's masses from a HOST buffer of n doubles in input order, each
 * finite and >= 0 (in the precision form at most 1e30; MTPT_ERR_INVALID_ARG
 * otherwise, nothing changed).  MTPT_ERR_STATE without mtpt_set_reaction or
 * before the first load.  Syncs.  The particle state of the reaction
 * extension of Sec. 8 (see mtpt_set_reaction). */
int mtpt_set_masses_b(mtpt_handle* h, const double* mass_b);

/* Species B's masses in input order to a HOST buffer of n doubles (the
 * reaction extension of Sec. 8; MTPT_ERR_STATE as mtpt_set_masses_b).
 * Syncs. */
int mtpt_get_masses_b(mtpt_handle* h, double* out);

/* Generator ids of the particles in the order mtpt_get_masses and
 * mtpt_get_positions use, to a HOST buffer of n: i for particle i of a plain
 * handle, the global ids of a tile's natives.  Identification: no
 * counterpart in the paper.  Syncs. */
int mtpt_get_ids(mtpt_handle* h, uint32_t* out);

/* Failure injection for tests (no counterpart in the paper): from this call
 * on, the nth device allocation that the library attempts (in this process,
 * on any handle) fails as if the device were out of memory; nth = 0 turns the
 * injection off.  *remaining (may be NULL) receives how many allocations the
 * previous setting still had to go (0: it fired or was off).  A call that
 * meets the failure returns MTPT_ERR_NO_MEMORY: loads, retuning and the
 * autotuner leave the handle's particles, counters and tuning as they were;
 * the adjoint's recording allocates before it steps; time steps allocate
 * nothing. */
int mtpt_debug_fail_alloc(int64_t nth, int64_t* remaining);

/* Wait-limit test hook (no counterpart in the paper).  The cell-count scan of
 * every step is one launch in which each tile of 16384 cells publishes its
 * total and then waits, polling, for the totals of the tiles before it; after
 * a bounded number of polls (tens of milliseconds) a tile stops waiting for
 * one and sums that tile's counts directly, which gives the same result.
 * From this call on, scans this process launches never publish tile `tile`
 * (-1: off; launches already captured in a CUDA graph keep the setting they
 * were captured with), so every tile after it runs out of polls.  *gave_up
 * (may be NULL) receives how many times, on the current device since the
 * library was loaded, a tile stopped waiting for an earlier one, after a
 * device synchronisation.  MTPT_ERR_INVALID_ARG for tile < -1. */
int mtpt_debug_scan_hold(int32_t tile, uint64_t* gave_up);

/* Human-readable text of a status code (static storage).  Error reporting:
 * no counterpart in the paper. */
const char* mtpt_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* MTPT_H */
