/*
 * mtpt_oracle.c -- serial FP64 CPU oracle of one MTPT time step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of the mass-transfer particle-tracking (MTPT) step of Schauer et
 * al., "Parallelized Domain Decomposition for Multi-Dimensional Lagrangian
 * Random Walk, Mass-Transfer Particle Tracking Schemes" (arXiv:2204.03756).
 * Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * may load it.  It shares no code, header, table or constant with the CUDA
 * library: every formula below is written from the paper (and, for the
 * random numbers the paper leaves unspecified, from the published
 * definitions named at each function).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math), so every
 * floating-point operation is a single IEEE-754 round-to-nearest operation
 * in the order written here.
 *
 * Step (Sec. 3, in the paper's order):
 *   1. random walk   X_i <- X_i + xi_i * sqrt(2 D_RW dt), D_RW = kappa D,
 *      then elastic reflection at every wall (zero-flux boundary);
 *   2. neighbour search: every pair with ||x_i - x_j||^2 <= psi^2, with
 *      psi = lambda sqrt(4 D_MT dt / beta) (Eq. "cutoff"), found with a
 *      K-D tree (the paper's structure) or by brute force;
 *   3. kernel K_ij = (2 pi h^2)^(-d/2) exp(-||x_i-x_j||^2 / (2 h^2)),
 *      h^2 = 2 D_MT dt / beta (simplified Eq. "kernel");
 *   4. W_ij = K_ij / (1/2 (sum_i K_ij + sum_j K_ij))  (column + row sums);
 *   5. delta_i = sum_j beta (M_j - M_i) W_ij, M_i <- M_i + delta_i
 *      (Eq. "changemass", explicit: all M_j taken at time t).
 *
 * Parity status per function is listed in oracle/__init__.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,        */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11).  The paper names   */
/* no generator; the random walk of Sec. 3 only needs i.i.d. N(0,1) draws.   */
/* Round: two 32x32->64 products with the published multipliers, the high    */
/* halves xor'ed with the other words and the round key; key bumped by the   */
/* published Weyl increments between rounds.                                 */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += ORC_PHILOX_W0; k1 += ORC_PHILOX_W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_many(int64_t n, const uint32_t* ctr /* n x 4 */,
                     const uint32_t* key /* 2 */, uint32_t* out /* n x 4 */) {
    for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Normal variates.  Reading of the paper (which specifies only "standard    */
/* normal"): uniforms u = (k)/2^24 with k = (word >> 8) + 1 in [1, 2^24], so */
/* u lies in (0, 1]; two uniforms give two normals by the Box-Muller         */
/* transform (Box & Muller 1958): R = sqrt(-2 ln u_a), theta = 2 pi u_b,     */
/* n = (R cos theta, R sin theta).  ln, sin and cos are evaluated in binary32 */
/* with the methods below, using only correctly rounded +, -, *, /, sqrt and  */
/* fused multiply-add, so the result is a pure function of the input bits.   */
/* ------------------------------------------------------------------------ */

/* ln(u) for normal binary32 u > 0: split u = 2^e m with m in [sqrt(1/2),
 * sqrt(2)], then ln m = 2 atanh(f), f = (m-1)/(m+1), summed by the odd power
 * series of atanh through f^11 (|f| <= 0.1716 so the next term is below
 * 2^-29 relative); e ln 2 is added as e*ln2_hi + e*ln2_lo with ln2_hi holding
 * few enough bits that e*ln2_hi is exact (Cody & Waite 1980 splitting). */
float orc_log_f32(float u) {
    union { float f; uint32_t b; } v;
    v.f = u;
    int e = (int)((v.b >> 23) & 0xffu) - 127;
    v.b = (v.b & 0x007fffffu) | 0x3f800000u;     /* m in [1, 2) */
    float m = v.f;
    if (m > 1.41421354f) { m = m * 0.5f; e += 1; }
    float f = (m - 1.0f) / (m + 1.0f);
    float s = f * f;
    float q = fmaf(s, 1.0f / 11.0f, 1.0f / 9.0f);
    q = fmaf(s, q, 1.0f / 7.0f);
    q = fmaf(s, q, 1.0f / 5.0f);
    q = fmaf(s, q, 1.0f / 3.0f);
    float two_f = 2.0f * f;
    float t = two_f * s;
    float ln_m = fmaf(t, q, two_f);
    const float ln2_hi = 0.693145752f;      /* 0x3f317200: 16 significant bits */
    const float ln2_lo = 1.42860677e-06f;   /* ln 2 - ln2_hi */
    float fe = (float)e;
    return fmaf(fe, ln2_hi, fmaf(fe, ln2_lo, ln_m));
}

/* sin and cos of theta = 2 pi k / 2^24 for an integer k in [0, 2^24].  The
 * range reduction is exact integer arithmetic: quadrant q = k / 2^22, offset
 * r = k mod 2^22, and offsets past half a quadrant are folded by the
 * complementary-angle identities.  On the reduced angle x in [0, pi/4] the
 * Taylor series of sin (through x^9) and cos (through x^10) are summed by
 * Horner's rule; the first omitted terms are below 2^-26 relative. */
void orc_sincos_2pi_f32(uint32_t k, float* s_out, float* c_out) {
    uint32_t q = (k >> 22) & 3u;
    uint32_t r = k & 0x3fffffu;
    int folded = 0;
    if (r > 0x200000u) { r = 0x400000u - r; folded = 1; }
    const float step = 3.74507028e-07f;     /* binary32 nearest to pi / 2^23 */
    float x = (float)r * step;
    float z = x * x;
    float ps = fmaf(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = fmaf(z, ps, 1.0f / 120.0f);
    ps = fmaf(z, ps, -1.0f / 6.0f);
    float sin_x = fmaf(x * z, ps, x);
    float pc = fmaf(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = fmaf(z, pc, -1.0f / 720.0f);
    pc = fmaf(z, pc, 1.0f / 24.0f);
    pc = fmaf(z, pc, -0.5f);
    float cos_x = fmaf(z, pc, 1.0f);
    float sa = folded ? cos_x : sin_x;   /* sin of the in-quadrant angle */
    float ca = folded ? sin_x : cos_x;   /* cos of the in-quadrant angle */
    float s, c;
    switch (q) {
        case 0: s = sa;  c = ca;  break;
        case 1: s = ca;  c = -sa; break;
        case 2: s = -sa; c = -ca; break;
        default: s = -ca; c = sa; break;
    }
    *s_out = s;
    *c_out = c;
}

void orc_log_f32_many(int64_t n, const float* u, float* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_log_f32(u[i]);
}

void orc_sincos_2pi_many(int64_t n, const uint32_t* k, float* s, float* c) {
    for (int64_t i = 0; i < n; ++i) orc_sincos_2pi_f32(k[i], s + i, c + i);
}

/* Four N(0,1) draws from one block of four generator words: normals 0,1
 * come from words (0,1) and normals 2,3 from words (2,3). */
void orc_box_muller4(const uint32_t w[4], float out[4]) {
    for (int pair = 0; pair < 2; ++pair) {
        uint32_t ka = (w[2 * pair] >> 8) + 1u;        /* in [1, 2^24] */
        uint32_t kb = (w[2 * pair + 1] >> 8) + 1u;
        float ua = (float)ka * 5.9604644775390625e-08f;  /* * 2^-24, exact */
        float radius = sqrtf(-2.0f * orc_log_f32(ua));
        float sn, cs;
        orc_sincos_2pi_f32(kb, &sn, &cs);
        out[2 * pair] = radius * cs;
        out[2 * pair + 1] = radius * sn;
    }
}

void orc_box_muller_many(int64_t n, const uint32_t* w /* n x 4 */, float* out /* n x 4 */) {
    for (int64_t i = 0; i < n; ++i) orc_box_muller4(w + 4 * i, out + 4 * i);
}

/* Four N(0,1) draws for (particle id, step).  Counter (id, step mod 2^32,
 * step div 2^32, 0), key (seed mod 2^32, seed div 2^32); axis a of the walk
 * uses normal a. */
void orc_normals4(uint64_t seed, uint32_t id, uint64_t step, float out[4]) {
    uint32_t ctr[4] = { id, (uint32_t)step, (uint32_t)(step >> 32), 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    orc_box_muller4(w, out);
}

void orc_normals_many(uint64_t seed, int64_t n, const uint32_t* id, uint64_t step,
                      float* out /* n x 4 */) {
    for (int64_t i = 0; i < n; ++i) orc_normals4(seed, id[i], step, out + 4 * i);
}

/* ------------------------------------------------------------------------ */
/* Derived parameters (Sec. 3).                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim;
    double D, kappa, dt, beta, lambda;
    double lo[3], hi[3];
    uint64_t seed;
    double v[3];      /* uniform velocity of the model equation (Sec. 2); 0 in the paper's runs */
} orc_params;

typedef struct {
    double D_RW, D_MT, sigma, h2, psi, psi2, kernel_norm;
} orc_derived;

void orc_derive(const orc_params* p, orc_derived* d) {
    d->D_RW = p->kappa * p->D;                       /* D_RW = kappa D */
    d->D_MT = (1.0 - p->kappa) * p->D;               /* D_MT = (1 - kappa) D */
    d->sigma = sqrt(2.0 * d->D_RW * p->dt);          /* walk scale sqrt(2 D_RW dt) */
    d->h2 = 2.0 * d->D_MT * p->dt / p->beta;         /* bandwidth h^2 = 2 D_MT dt / beta */
    d->psi = p->lambda * sqrt(4.0 * d->D_MT * p->dt / p->beta);  /* Eq. "cutoff" */
    d->psi2 = d->psi * d->psi;
    /* (2 pi h^2)^(-d/2) */
    d->kernel_norm = (d->h2 > 0.0) ? pow(2.0 * M_PI * d->h2, -0.5 * (double)p->dim) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Random walk + reflecting walls (Sec. 3).                                  */
/* ------------------------------------------------------------------------ */

/* Elastic reflection: a coordinate past a wall is mirrored in that wall,
 * repeatedly while it is outside; after 64 mirrors (a displacement of more
 * than 64 box lengths) it is put on the nearest wall.  A coordinate equal to
 * a wall is inside. */
double orc_reflect(double x, double lo, double hi) {
    for (int it = 0; it < 64; ++it) {
        if (x < lo) x = 2.0 * lo - x;
        else if (x > hi) x = 2.0 * hi - x;
        else return x;
    }
    if (x < lo) return lo;
    if (x > hi) return hi;
    return x;
}

/* pos is structure-of-arrays: pos[a * n + i] is axis a of particle i.
 * Each axis moves by sigma xi; with a velocity v (the advection term of the
 * model equation, Sec. 2, where the paper itself takes v = 0) the move is
 * v dt + sigma xi, the advective part applied as a plain translation. */
void orc_random_walk(const orc_params* p, int64_t n, double* pos, const uint32_t* id,
                     uint64_t step) {
    orc_derived dv;
    orc_derive(p, &dv);
    for (int64_t i = 0; i < n; ++i) {
        float xi[4];
        orc_normals4(p->seed, id[i], step, xi);
        for (int a = 0; a < p->dim; ++a) {
            double x = pos[a * n + i];
            double disp = dv.sigma * (double)xi[a];
            if (p->v[a] != 0.0) disp = p->v[a] * p->dt + disp;
            x = x + disp;
            pos[a * n + i] = orc_reflect(x, p->lo[a], p->hi[a]);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Neighbour search.                                                         */
/* The pair distance is evaluated as dx*dx + dy*dy (+ dz*dz), left to right, */
/* dx = x_i - x_j, each operation rounded once (no fused multiply-add); the  */
/* pair is a neighbour pair when that value is <= psi^2 (inclusive).         */
/* ------------------------------------------------------------------------ */
static double orc_dist2(int dim, int64_t n, const double* pos, int64_t i, int64_t j) {
    double s = 0.0;
    for (int a = 0; a < dim; ++a) {
        double dx = pos[a * n + i] - pos[a * n + j];
        double sq = dx * dx;
        s = (a == 0) ? sq : s + sq;
    }
    return s;
}

/* Growable list of ordered pairs (i, j). */
typedef struct { int64_t* i; int64_t* j; int64_t len, cap; } orc_pairlist;

static int orc_pl_push(orc_pairlist* pl, int64_t i, int64_t j) {
    if (pl->len == pl->cap) {
        int64_t nc = pl->cap ? 2 * pl->cap : 1024;
        int64_t* ni = (int64_t*)realloc(pl->i, (size_t)nc * sizeof(int64_t));
        if (!ni) return -1;
        pl->i = ni;
        int64_t* nj = (int64_t*)realloc(pl->j, (size_t)nc * sizeof(int64_t));
        if (!nj) return -1;
        pl->j = nj;
        pl->cap = nc;
    }
    pl->i[pl->len] = i;
    pl->j[pl->len] = j;
    pl->len++;
    return 0;
}

/* Brute force O(N^2): every ordered pair i != j, rows in increasing i,
 * columns in increasing j. */
static int orc_search_brute(int dim, int64_t n, const double* pos, double psi2,
                            orc_pairlist* pl) {
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            if (j != i && orc_dist2(dim, n, pos, i, j) <= psi2)
                if (orc_pl_push(pl, i, j)) return -1;
    return 0;
}

/* K-D tree (Bentley 1975): each internal node splits its points at the
 * median of the axis with the widest extent; points left of the split have
 * coordinate <= split, points right have coordinate >= split.  Leaves hold
 * at most ORC_LEAF points. */
#define ORC_LEAF 8
typedef struct {
    int64_t begin, end;    /* range in the permutation */
    int axis;              /* -1 for a leaf */
    double split;
    int64_t left, right;   /* child node indices */
} orc_kdnode;

typedef struct {
    orc_kdnode* nodes;
    int64_t nnodes, cap;
    int64_t* perm;
} orc_kdtree;

static double orc_coord(int64_t n, const double* pos, int a, int64_t i) { return pos[a * n + i]; }

/* Reorder perm[begin, end) so that perm[k] holds the element of rank k - begin
 * along axis a, with smaller-or-equal elements before and greater-or-equal
 * after (Hoare's FIND / quickselect). */
static void orc_select(int64_t n, const double* pos, int a, int64_t* perm, int64_t begin,
                       int64_t end, int64_t k) {
    int64_t l = begin, r = end - 1;
    while (r > l) {
        int64_t mid = l + (r - l) / 2;
        /* median of three as the pivot */
        double va = orc_coord(n, pos, a, perm[l]), vb = orc_coord(n, pos, a, perm[mid]),
               vc = orc_coord(n, pos, a, perm[r]);
        double pivot = (va < vb) ? ((vb < vc) ? vb : ((va < vc) ? vc : va))
                                 : ((va < vc) ? va : ((vb < vc) ? vc : vb));
        int64_t i = l, j = r;
        while (i <= j) {
            while (orc_coord(n, pos, a, perm[i]) < pivot) ++i;
            while (orc_coord(n, pos, a, perm[j]) > pivot) --j;
            if (i <= j) {
                int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
                ++i; --j;
            }
        }
        if (k <= j) r = j;
        else if (k >= i) l = i;
        else return;
    }
}

static int64_t orc_kd_newnode(orc_kdtree* t) {
    if (t->nnodes == t->cap) {
        int64_t nc = t->cap ? 2 * t->cap : 1024;
        orc_kdnode* nn = (orc_kdnode*)realloc(t->nodes, (size_t)nc * sizeof(orc_kdnode));
        if (!nn) return -1;
        t->nodes = nn;
        t->cap = nc;
    }
    return t->nnodes++;
}

static int64_t orc_kd_build(orc_kdtree* t, int dim, int64_t n, const double* pos,
                            int64_t begin, int64_t end) {
    int64_t id = orc_kd_newnode(t);
    if (id < 0) return -1;
    t->nodes[id].begin = begin;
    t->nodes[id].end = end;
    t->nodes[id].axis = -1;
    if (end - begin <= ORC_LEAF) return id;
    int best_axis = 0;
    double best_extent = -1.0;
    for (int a = 0; a < dim; ++a) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t k = begin; k < end; ++k) {
            double v = orc_coord(n, pos, a, t->perm[k]);
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        if (mx - mn > best_extent) { best_extent = mx - mn; best_axis = a; }
    }
    int64_t mid = begin + (end - begin) / 2;
    orc_select(n, pos, best_axis, t->perm, begin, end, mid);
    double split = orc_coord(n, pos, best_axis, t->perm[mid]);
    int64_t l = orc_kd_build(t, dim, n, pos, begin, mid);
    if (l < 0) return -1;
    int64_t r = orc_kd_build(t, dim, n, pos, mid, end);
    if (r < 0) return -1;
    t->nodes[id].axis = best_axis;
    t->nodes[id].split = split;
    t->nodes[id].left = l;
    t->nodes[id].right = r;
    return id;
}

/* Range query: every j != i with dist2(i, j) <= psi2, appended to pl (order
 * within the row follows the tree walk).  A subtree on the far side of a
 * split is skipped only when (q - split)^2 > psi2: each of its points is at
 * least that far along the split axis, and rounding is monotone, so its
 * computed dist2 is at least the computed (q - split)^2. */
static int orc_kd_query(const orc_kdtree* t, int dim, int64_t n, const double* pos,
                        int64_t i, double psi2, orc_pairlist* pl, int64_t* stack) {
    int64_t sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const orc_kdnode* nd = &t->nodes[stack[--sp]];
        if (nd->axis < 0) {
            for (int64_t k = nd->begin; k < nd->end; ++k) {
                int64_t j = t->perm[k];
                if (j != i && orc_dist2(dim, n, pos, i, j) <= psi2)
                    if (orc_pl_push(pl, i, j)) return -1;
            }
            continue;
        }
        double q = orc_coord(n, pos, nd->axis, i);
        double ds = q - nd->split;
        double ds2 = ds * ds;
        int64_t nearc = (q <= nd->split) ? nd->left : nd->right;
        int64_t farc = (q <= nd->split) ? nd->right : nd->left;
        if (ds2 <= psi2) stack[sp++] = farc;
        stack[sp++] = nearc;
    }
    return 0;
}

static int orc_search_kdtree(int dim, int64_t n, const double* pos, double psi2,
                             orc_pairlist* pl) {
    if (n == 0) return 0;
    orc_kdtree t = {0};
    t.perm = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!t.perm) return -1;
    for (int64_t k = 0; k < n; ++k) t.perm[k] = k;
    if (orc_kd_build(&t, dim, n, pos, 0, n) < 0) { free(t.perm); free(t.nodes); return -1; }
    /* depth is O(log n); the stack never holds more than 2 * depth + 2 nodes */
    int64_t* stack = (int64_t*)malloc((size_t)(t.nnodes + 2) * sizeof(int64_t));
    if (!stack) { free(t.perm); free(t.nodes); return -1; }
    int rc = 0;
    for (int64_t i = 0; i < n && rc == 0; ++i) rc = orc_kd_query(&t, dim, n, pos, i, psi2, pl, stack);
    free(stack);
    free(t.perm);
    free(t.nodes);
    return rc;
}

/* Exported pair search.  method 0 = brute force, 1 = K-D tree.  Returns the
 * number of ordered pairs (i != j) found, or -1 on allocation failure.  The
 * pair arrays are malloc'ed here and released by orc_free. */
int64_t orc_pairs(int dim, int64_t n, const double* pos, double psi2, int method,
                  int64_t** out_i, int64_t** out_j) {
    orc_pairlist pl = {0};
    int rc = (method == 0) ? orc_search_brute(dim, n, pos, psi2, &pl)
                           : orc_search_kdtree(dim, n, pos, psi2, &pl);
    if (rc) { free(pl.i); free(pl.j); return -1; }
    *out_i = pl.i;
    *out_j = pl.j;
    return pl.len;
}

void orc_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Mass transfer (Sec. 3).                                                   */
/* ------------------------------------------------------------------------ */

/* One mass-transfer update on fixed positions.  Fills, when non-NULL,
 * row_sum[i] = sum_j K_ij and col_sum[j] = sum_i K_ij (the self term K_ii is
 * part of both, since the sums run over all particles) and writes the new
 * masses to mass_out (mass_in is read only: explicit update).  Returns the
 * number of ordered neighbour pairs i != j, or -1 on allocation failure.
 * With D_MT = 0 (h = 0) the kernel degenerates and no transfer happens:
 * mass_out = mass_in and 0 is returned. */
int64_t orc_mass_transfer(const orc_params* p, int64_t n, const double* pos,
                          const double* mass_in, double* mass_out, int method,
                          double* row_sum, double* col_sum) {
    orc_derived dv;
    orc_derive(p, &dv);
    if (!(dv.h2 > 0.0)) {
        memcpy(mass_out, mass_in, (size_t)n * sizeof(double));
        if (row_sum) memset(row_sum, 0, (size_t)n * sizeof(double));
        if (col_sum) memset(col_sum, 0, (size_t)n * sizeof(double));
        return 0;
    }
    orc_pairlist pl = {0};
    int rc = (method == 0) ? orc_search_brute(p->dim, n, pos, dv.psi2, &pl)
                           : orc_search_kdtree(p->dim, n, pos, dv.psi2, &pl);
    if (rc) { free(pl.i); free(pl.j); return -1; }

    double* K = (double*)malloc((size_t)(pl.len ? pl.len : 1) * sizeof(double));
    double* rs = (double*)calloc((size_t)(n ? n : 1), sizeof(double));
    double* cs = (double*)calloc((size_t)(n ? n : 1), sizeof(double));
    double* delta = (double*)calloc((size_t)(n ? n : 1), sizeof(double));
    if (!K || !rs || !cs || !delta) {
        free(K); free(rs); free(cs); free(delta); free(pl.i); free(pl.j);
        return -1;
    }
    const double inv_2h2 = 1.0 / (2.0 * dv.h2);
    const double K_self = dv.kernel_norm;   /* K_ii = (2 pi h^2)^(-d/2) exp(0) */

    /* K_ij on the sparse pattern (Eq. "kernel", simplified form). */
    for (int64_t e = 0; e < pl.len; ++e) {
        double r2 = orc_dist2(p->dim, n, pos, pl.i[e], pl.j[e]);
        K[e] = dv.kernel_norm * exp(-r2 * inv_2h2);
    }
    /* Row sums sum_j K_ij and column sums sum_i K_ij, self term included. */
    for (int64_t i = 0; i < n; ++i) { rs[i] = K_self; cs[i] = K_self; }
    for (int64_t e = 0; e < pl.len; ++e) {
        rs[pl.i[e]] += K[e];
        cs[pl.j[e]] += K[e];
    }
    /* delta_i = sum_j beta (M_j - M_i) W_ij with
     * W_ij = K_ij / (1/2 (col_sum_j + row_sum_i)); the j = i term is zero. */
    for (int64_t e = 0; e < pl.len; ++e) {
        int64_t i = pl.i[e], j = pl.j[e];
        double W = K[e] / (0.5 * (cs[j] + rs[i]));
        delta[i] += p->beta * (mass_in[j] - mass_in[i]) * W;
    }
    for (int64_t i = 0; i < n; ++i) mass_out[i] = mass_in[i] + delta[i];
    if (row_sum) memcpy(row_sum, rs, (size_t)n * sizeof(double));
    if (col_sum) memcpy(col_sum, cs, (size_t)n * sizeof(double));
    int64_t npairs = pl.len;
    free(K); free(rs); free(cs); free(delta); free(pl.i); free(pl.j);
    return npairs;
}

/* Full time steps: for s in [0, nsteps): random walk with step counter
 * step0 + s, then mass transfer on the moved positions.  pos and mass are
 * updated in place.  Returns the total number of ordered neighbour pairs
 * over all steps, or -1 on allocation failure. */
int64_t orc_run(const orc_params* p, int64_t n, double* pos, double* mass,
                const uint32_t* id, uint64_t step0, int64_t nsteps, int method) {
    double* tmp = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    if (!tmp) return -1;
    int64_t total = 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_random_walk(p, n, pos, id, step0 + (uint64_t)s);
        int64_t np = orc_mass_transfer(p, n, pos, mass, tmp, method, NULL, NULL);
        if (np < 0) { free(tmp); return -1; }
        total += np;
        memcpy(mass, tmp, (size_t)n * sizeof(double));
    }
    free(tmp);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Bimolecular reaction A + B -> 0.  The paper names reactions only as an    */
/* extension (Sec. 8) and gives no model; the reading taken here: every      */
/* particle carries a mass of each species; both species move by the same    */
/* random walk and exchange mass with the same weights W_ij (the transfer of  */
/* Sec. 3 applied to each species); then each particle reacts well mixed     */
/* over dt.  A particle's concentrations are C = N M / V (V the box volume,  */
/* the mass-concentration relation of Sec. 3), so the rate law               */
/* dC_A/dt = dC_B/dt = -k C_A C_B becomes da/dt = db/dt = -k_p a b with      */
/* k_p = k N / V, whose exact solution over dt keeps a - b and gives, for    */
/* a >= b, with x = k_p (a - b) dt and phi(x) = (1 - exp(-x)) / x (phi(0) = 1) */
/*   a' = a / q,  b' = b exp(-x) / q,  q = 1 + k_p b dt phi(x),               */
/* and the mirror image for b > a.  (The closed form                          */
/* a(t) = D a / (a - b exp(-k_p D t)), D = a - b, rearranged so that neither  */
/* D -> 0 nor the species in deficit loses digits.)                          */
/* ------------------------------------------------------------------------ */

static double orc_phi(double x) {
    return (x > 0.0) ? -expm1(-x) / x : 1.0;
}

/* One reaction substep of length dt for the masses a, b in place.  A
 * particle with a negative mass of either species does not react (the rate
 * law is for non-negative concentrations). */
void orc_react(int64_t n, double* a, double* b, double kp, double dt) {
    for (int64_t i = 0; i < n; ++i) {
        const double ai = a[i], bi = b[i];
        if (ai < 0.0 || bi < 0.0) continue;
        if (ai >= bi) {
            const double x = kp * (ai - bi) * dt;
            const double q = 1.0 + kp * bi * dt * orc_phi(x);
            a[i] = ai / q;
            b[i] = bi * exp(-x) / q;
        } else {
            const double x = kp * (bi - ai) * dt;
            const double q = 1.0 + kp * ai * dt * orc_phi(x);
            b[i] = bi / q;
            a[i] = ai * exp(-x) / q;
        }
    }
}

/* The rate on particle masses: k_p = k N / V, V the product of the box's
 * edge lengths. */
double orc_particle_rate(const orc_params* p, int64_t n, double k) {
    double vol = 1.0;
    for (int a = 0; a < p->dim; ++a) vol *= p->hi[a] - p->lo[a];
    return k * (double)n / vol;
}

/* Reactive time steps: walk, transfer of each species with the same
 * weights, reaction.  pos, ma and mb are updated in place.  Returns the total
 * number of ordered neighbour pairs, or -1 on allocation failure. */
int64_t orc_run_reactive(const orc_params* p, int64_t n, double* pos, double* ma, double* mb,
                         const uint32_t* id, uint64_t step0, int64_t nsteps, int method,
                         double k) {
    double* ta = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* tb = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    if (!ta || !tb) { free(ta); free(tb); return -1; }
    const double kp = orc_particle_rate(p, n, k);
    int64_t total = 0;
    for (int64_t s = 0; s < nsteps; ++s) {
        orc_random_walk(p, n, pos, id, step0 + (uint64_t)s);
        const int64_t np = orc_mass_transfer(p, n, pos, ma, ta, method, NULL, NULL);
        const int64_t nq = orc_mass_transfer(p, n, pos, mb, tb, method, NULL, NULL);
        if (np < 0 || nq < 0) { free(ta); free(tb); return -1; }
        total += np;
        orc_react(n, ta, tb, kp, p->dt);
        memcpy(ma, ta, (size_t)n * sizeof(double));
        memcpy(mb, tb, (size_t)n * sizeof(double));
    }
    free(ta);
    free(tb);
    return total;
}

void orc_derived_values(const orc_params* p, double out[7]) {
    orc_derived d;
    orc_derive(p, &d);
    out[0] = d.D_RW; out[1] = d.D_MT; out[2] = d.sigma; out[3] = d.h2;
    out[4] = d.psi; out[5] = d.psi2; out[6] = d.kernel_norm;
}
