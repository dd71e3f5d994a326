// kernels.cuh -- CUDA kernels of one MTPT time step (Sec. 3) for sm_103a.
//
// GB300 issues every binary64 instruction (arithmetic, compares, f32<->f64
// conversions) at about 1/70 of the binary32 rate, so the kernels keep
// binary64 to the operations whose results must match the binary64 method
// bit for bit (the walk's x + sigma xi, and the pair test inside a narrow
// band around the cutoff) or carry the binary64 form's accuracy (its pair
// terms and sums), and do everything else in binary32 and integer
// arithmetic.
//
// Data layout (structure of arrays, `stride` = capacity >= n):
//   pos[a * stride + s]  binary64 coordinates, particles in cell order
//   mass[s], id[s]       binary64 mass, uint32 input index (keys the walk)
//   cell[s]              linear cell index of particle s (written and read in 3-d
//                        only: below 3-d the record carries the cell coordinates)
//   rec[s]               float4: binary32 offsets of the particle from its
//                        cell's lower corner (x, y, z), and in .w the cell's
//                        x index (a small integer, exact in binary32); in
//                        2-d, .z (no offset there) holds the cell's y index
//   start[c]             first particle of cell c (exclusive prefix sum)
// Cells are row-major (x fastest), so the three cells (cx-1..cx+1) of one
// neighbour row are one contiguous particle range; inside a cell particles
// are ordered by x (then id), so that range is sorted by x up to rounding.
#pragma once
#include <cstdint>
#include <type_traits>

#include "expneg.cuh"
#include "rng.cuh"

namespace mtpt {

enum : uint32_t { kStatusNonFinite = 1u, kStatusOutOfDomain = 2u };

// Generator ids are below 2^31; a tile marks its ghost copies of other tiles'
// particles with this bit (see tiles.cuh).
constexpr uint32_t kGhostBit = 0x80000000u;

// Bounds-checked build (compiled with -DMTPT_CHECKED; the tests load it as a
// second library): index invariants that hold by construction are verified at
// run time; a violation sets its bit in a device word and the access is
// skipped.  The normal build compiles every check to `true`.
enum : uint32_t {
    kChkCell = 1u,       // walk: cell index inside the realisation's cells
    kChkSlot = 2u,       // scatter: counting-sort slot inside [0, n)
    kChkGather = 4u,     // gather: source and in-cell rank inside the cell's range
    kChkRow = 8u,        // pair search: neighbour row inside the realisation's cells
    kChkSegment = 16u,   // segment engine: entries within the segments' capacity
    kChkOutput = 32u,    // outputs: particle id inside [0, n)
};
#ifdef MTPT_CHECKED
__device__ uint32_t g_check_word;
__device__ __forceinline__ bool check(bool ok, uint32_t bit) {
    if (!ok) atomicOr(&g_check_word, bit);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool check(bool, uint32_t) { return true; }
#endif

constexpr int kBlock = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 16;                        // cells per scan thread
constexpr int kScanTile = kScanPerThread * kScanThreads;  // cells per scan block

struct Box {
    double lo[3], hi[3];
    long long lo_key[3], hi_key[3];   // order-preserving integer images of lo, hi
};

struct Grid {
    int n[3];          // cells per axis of this grid (1 on unused axes)
    int nglob[3];      // cells per axis of the whole box's grid (equal to n unless
                       // the grid is one tile's part of it)
    int off[3];        // global index of this grid's first cell per axis (0 unless tiled)
    double lo[3];      // lower corner of the box
    double w[3];       // cell width per axis, >= psi
    double inv_w[3];   // 1 / w
    float wf[3];       // w rounded to binary32
    float lo_f[3];     // lo rounded to binary32 (binary32 cell index)
    float inv_w_f[3];  // 1 / w in binary32
    int cell_f32;      // 1: cell index from binary32 arithmetic (margin in w), 0: binary64
    int reach;         // cells a neighbour can be away per axis: 1 (w >= psi) or 2 (w >= psi / 2)
    int corner_off[3]; // offset of axis a's corner table in `corners`
};

struct PairParams {
    double psi2;       // cutoff squared: the exact binary64 test d2 <= psi2
    float band_lo;     // binary32 d2 below this: certainly a neighbour
    float band_hi;     // binary32 d2 above this: certainly not a neighbour
    float reach2;      // band_hi (1 + 2^-16): bounds dx^2 + dy^2 (+ dz^2) of a neighbour
    float trim_eps;    // slack of the per-row candidate windows (see for_each_row)
    double a;          // 1 / (2 h^2)
    float a_log2e;     // a * log2(e) in binary32 (precision form)
    double beta;
    ExpNegConsts ec;
};

// Everything one realisation's kernels need.  A single run passes one by
// value (SingleView); a batch of independent realisations keeps a table in
// device memory and a realisation index per particle (BatchView).
struct RealParams {
    Box box;
    Grid g;
    PairParams pp;
    double sigma;        // walk scale sqrt(2 D_RW dt)
    double kernel_norm;  // (2 pi h^2)^(-d/2)
    uint64_t seed;       // generator key of the walk
    uint32_t id_offset;  // first global particle index of the realisation
    uint32_t cell_base;  // first global cell of the realisation
    int32_t transfer;    // 1 when D_MT > 0 (pair passes run)
    int32_t walk;        // 1 when sigma > 0 or a velocity component is nonzero
    double vdt[3];       // v dt per axis (advection)
    uint32_t advect;     // bit a set when v[a] != 0
    double dsigma_dD;    // d sigma / dD = sigma / (2 D) (adjoint)
    double h2;           // 2 D_MT dt / beta (adjoint)
    double inv_2D;       // 1 / (2 D) (adjoint)
    double inv_h2;       // 1 / h^2 (adjoint)
};

struct SingleView {
    static constexpr bool kBatch = false;
    RealParams p;
    __device__ __forceinline__ const RealParams& of_input(uint32_t) const { return p; }
    __device__ __forceinline__ const RealParams& of_sorted(uint32_t) const { return p; }
};

struct BatchView {
    static constexpr bool kBatch = true;
    const RealParams* tbl;
    const uint32_t* rid_input;    // realisation of each particle before the sort
    const uint32_t* rid_sorted;   // realisation of each particle in cell order
    __device__ __forceinline__ const RealParams& of_input(uint32_t i) const {
        return tbl[__ldg(rid_input + i)];
    }
    __device__ __forceinline__ const RealParams& of_sorted(uint32_t s) const {
        return tbl[__ldg(rid_sorted + s)];
    }
};

// ---------------------------------------------------------------------------
// Integer helpers for binary64 values.
// ---------------------------------------------------------------------------

// Order-preserving image of a binary64 value in int64: for non-NaN x, y,
// key(x) < key(y) implies x <= y (-0 sorts below +0).
__device__ __forceinline__ long long order_key(double x) {
    const long long b = __double_as_longlong(x);
    return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// x split as hi + lo with hi = x truncated to binary32 (integer operations
// only: no binary64 instruction) and lo the binary32 nearest to the exact
// remainder x - hi (|lo| < 2^-23 |x|).  Values below 2^-126 in magnitude give
// hi = lo = 0; |x| must be below 2^127.
__device__ __forceinline__ void split_double(double x, float* hi, float* lo) {
    const uint32_t whi = uint32_t(__double2hiint(x));
    const uint32_t wlo = uint32_t(__double2loint(x));
    const int e = int((whi >> 20) & 0x7ffu);
    const uint32_t sign = whi & 0x80000000u;
    if (e < 949) {   // |x| < 2^-74: residual below binary32's normal range
        *hi = e < 897 ? __uint_as_float(sign)
                      : __uint_as_float(sign | (uint32_t(e - 896) << 23) | ((whi & 0xfffffu) << 3) | (wlo >> 29));
        *lo = __uint_as_float(sign);
        return;
    }
    *hi = __uint_as_float(sign | (uint32_t(e - 896) << 23) | ((whi & 0xfffffu) << 3) | (wlo >> 29));
    const float m = __uint2float_rn(wlo & 0x1fffffffu);           // remainder mantissa
    const float scale = __uint_as_float(uint32_t(e - 948) << 23);  // 2^(e - 1075)
    *lo = __uint_as_float(__float_as_uint(__fmul_rn(m, scale)) | sign);
}

// Exact binary32 -> binary64 conversion by integer operations (no binary64
// pipe instruction) for zero and normal values; subnormal inputs take the
// hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t sign = b & 0x80000000u;
    const uint32_t mag = b & 0x7fffffffu;
    if (mag == 0u) return __hiloint2double(int(sign), 0);
    const uint32_t e = mag >> 23;
    if (e == 0u || e == 255u) return double(f);
    const uint32_t m = mag & 0x7fffffu;
    return __hiloint2double(int(sign | ((e + 896u) << 20) | (m >> 3)), int(m << 29));
}

// num / den for num >= 0 and 1 <= den < 2^127 with binary64 fma only: a
// binary32 reciprocal seed (relative error below 2^-21 after the head
// truncation), one Newton-Raphson step for 1/den (error below 2^-41), then
// the quotient and one residual correction q + (num - den q) / den (P.
// Markstein, "IA-64 and Elementary Functions", 2000, ch. 8), which leaves an
// error below one unit in the last place.  Five binary64 operations.
__device__ __forceinline__ double quot_pos(double num, double den) {
    float y0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y0) : "f"(head_f32(den)));
    double y = f32_to_f64(y0);
    y = __fma_rn(y, __fma_rn(-den, y, 1.0), y);
    const double q = __dmul_rn(num, y);
    return __fma_rn(__fma_rn(-den, q, num), y, q);
}

// True when x is an infinity or a NaN (integer test on the exponent field).
__device__ __forceinline__ bool not_finite(double x) {
    return (uint32_t(__double2hiint(x)) & 0x7ff00000u) == 0x7ff00000u;
}

// ---------------------------------------------------------------------------
// Step 1: random walk with reflecting walls, then the particle's cell.
// ---------------------------------------------------------------------------

// Elastic reflection in the walls lo and hi; more than 64 mirrors (a jump of
// over 64 box lengths) puts the coordinate on the nearest wall.
__device__ __forceinline__ double reflect(double x, double lo, double hi) {
    for (int it = 0; it < 64; ++it) {
        if (x < lo) x = __dsub_rn(__dmul_rn(2.0, lo), x);
        else if (x > hi) x = __dsub_rn(__dmul_rn(2.0, hi), x);
        else return x;
    }
    return x < lo ? lo : (x > hi ? hi : x);
}

// As reflect(), also reporting the derivative of the result with respect to
// the unreflected coordinate: -1 after an odd number of mirrors, +1 after an
// even number, 0 when the coordinate was put on a wall.
__device__ __forceinline__ double reflect_parity(double x, double lo, double hi, double* sign) {
    double sg = 1.0;
    for (int it = 0; it < 64; ++it) {
        if (x < lo) x = __dsub_rn(__dmul_rn(2.0, lo), x);
        else if (x > hi) x = __dsub_rn(__dmul_rn(2.0, hi), x);
        else { *sign = sg; return x; }
        sg = -sg;
    }
    *sign = 0.0;
    return x < lo ? lo : (x > hi ? hi : x);
}

__device__ __forceinline__ int clamp_cell(float u, int n) {
    // u is finite here; truncation equals floor for u >= 0
    return u <= 0.0f ? 0 : (u >= float(n - 1) ? n - 1 : int(u));
}

template <int DIM>
__device__ __forceinline__ uint32_t cell_of(const double* x, const Grid& g, bool* bad) {
    uint32_t lin = 0, mult = 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int c = 0;
        if (g.cell_f32) {
            float hi, lo;
            split_double(x[a], &hi, &lo);
            const float u = __fmul_rn(__fsub_rn(hi, g.lo_f[a]), g.inv_w_f[a]);
            if (!not_finite(x[a])) c = clamp_cell(u, g.nglob[a]);
        } else {
            const double u = __dmul_rn(__dsub_rn(x[a], g.lo[a]), g.inv_w[a]);
            if (u == u) c = u <= 0.0 ? 0 : (u >= double(g.nglob[a] - 1) ? g.nglob[a] - 1 : __double2int_rz(u));
            else *bad = true;
        }
        // the whole box's cell index, then this grid's part of it
        c -= g.off[a];
        c = c < 0 ? 0 : (c >= g.n[a] ? g.n[a] - 1 : c);
        if (not_finite(x[a])) *bad = true;
        lin += uint32_t(c) * mult;
        mult *= uint32_t(g.n[a]);
    }
    return lin;
}

// One particle's move of the random walk (Sec. 3: x + sigma xi per axis,
// then the reflecting walls), in place on x[DIM].  With TANGENT, also
// carries the pathwise derivative of the positions with respect to D (tan,
// same layout as pos, particle i): the walk adds dsigma/dD xi and a mirror
// flips the sign, exactly as it maps the coordinate.  ADVECT compiles the
// velocity term in (launched when some realisation has v != 0), so the
// binary64 pipe of a walk without one carries only its two operations per
// axis.
template <int DIM, bool TANGENT, bool ADVECT>
__device__ __forceinline__ void walk_particle(const RealParams& P, uint32_t gen_id, uint64_t step,
                                              double* x, double* __restrict__ tan, int64_t stride,
                                              int i) {
    const float4 z4 = normals4(P.seed, gen_id, step);
    const float z[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double za = f32_to_f64(z[a]);
        // move sigma xi, or v dt + sigma xi with a velocity on this axis
        double disp = __dmul_rn(P.sigma, za);
        if constexpr (ADVECT) {
            if (P.advect & (1u << a)) disp = __dadd_rn(P.vdt[a], disp);
        }
        double xv = __dadd_rn(x[a], disp);
        const long long k = order_key(xv);
        // strictly inside in the integer order => inside in binary64, no
        // mirror needed; anything else (walls, outside, NaN) takes the
        // binary64 reflection
        if constexpr (TANGENT) {
            double sign = 1.0;
            if (!(k > P.box.lo_key[a] && k < P.box.hi_key[a]))
                xv = reflect_parity(xv, P.box.lo[a], P.box.hi[a], &sign);
            const double t = __fma_rn(P.dsigma_dD, za, tan[a * stride + i]);
            tan[a * stride + i] = __dmul_rn(sign, t);
        } else {
            if (!(k > P.box.lo_key[a] && k < P.box.hi_key[a]))
                xv = reflect(xv, P.box.lo[a], P.box.hi[a]);
        }
        x[a] = xv;
    }
}

// The particle's cell (global index) into *key_out and its cell count; a
// coordinate that is not finite sets the status bit.
template <int DIM>
__device__ __forceinline__ void key_particle(const RealParams& P, const double* x,
                                             uint32_t* __restrict__ status,
                                             uint32_t* __restrict__ key_out,
                                             uint32_t* __restrict__ count) {
    bool bad = false;
    const uint32_t c = P.cell_base + cell_of<DIM>(x, P.g, &bad);
    if (bad) atomicOr(status, kStatusNonFinite);
    if (!check(c - P.cell_base < uint32_t(P.g.n[0]) * uint32_t(P.g.n[1]) * uint32_t(P.g.n[2]),
               kChkCell))
        return;
    *key_out = c;
    atomicAdd(&count[c], 1u);
}

// Step 1 over all particles, in place: the walk (with do_walk) and the
// cell keys and counts of the counting sort (with do_key).
template <int DIM, class View, bool TANGENT = false, bool ADVECT = false>
__global__ void __launch_bounds__(kBlock)
k_walk_key(int n, int64_t stride, double* __restrict__ pos, const uint32_t* __restrict__ id,
           const unsigned long long* __restrict__ step_dev, int do_walk, int do_key,
           const __grid_constant__ View v, uint32_t* __restrict__ key,
           uint32_t* __restrict__ count, uint32_t* __restrict__ status,
           double* __restrict__ tan = nullptr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t step = *step_dev;
    const RealParams& P = v.of_input(uint32_t(i));
    double x[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = pos[a * stride + i];
    if (do_walk && P.walk) {
        walk_particle<DIM, TANGENT, ADVECT>(P, id[i] - P.id_offset, step, x, tan, stride, i);
#pragma unroll
        for (int a = 0; a < DIM; ++a) pos[a * stride + i] = x[a];
    }
    if (do_key) key_particle<DIM>(P, x, status, key + i, count);
}

// Check of host-loaded input in its device copy (positions dim x n with
// stride `stride`, masses n): a position outside its realisation's box
// [lo, hi] (NaN included) sets bit 1, a mass that is not finite or above
// mass_limit in magnitude sets bit 2.  box holds lo[3], hi[3] per
// realisation; first[k] is realisation k's first particle (first[nreal] = n).
// With id_out, also writes the particle ids 0..n-1 there.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_check_input(int n, int64_t stride, int nreal, const double* __restrict__ pos,
              const double* __restrict__ mass, const double* __restrict__ box,
              const uint32_t* __restrict__ first, double mass_limit,
              uint32_t* __restrict__ flags, uint32_t* __restrict__ id_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bad = 0;
    if (i < n) {
        int k = 0;
        if (nreal > 1) {   // last k with first[k] <= i
            int lo = 0, hi = nreal - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (first[mid] <= uint32_t(i)) lo = mid; else hi = mid - 1;
            }
            k = lo;
        }
        const double* b = box + 6 * k;
        // integer tests only (the binary64 unit is slow): x inside [lo, hi]
        // through the order keys (a NaN fails the finiteness test), |m| <=
        // mass_limit through the magnitude bits (ordered like the values)
        // (-0 and +0 compare equal, so both map to key 0)
        auto key0 = [](double v) {
            return (__double_as_longlong(v) & 0x7fffffffffffffffLL) == 0 ? 0LL : order_key(v);
        };
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double x = pos[int64_t(a) * stride + i];
            const long long kx = key0(x);
            if (not_finite(x) || kx < key0(b[a]) || kx > key0(b[3 + a])) bad |= 1u;
        }
        const double m = mass[i];
        const long long mag = __double_as_longlong(m) & 0x7fffffffffffffffLL;
        if (not_finite(m) || mag > __double_as_longlong(mass_limit)) bad |= 2u;
        if (id_out) id_out[i] = uint32_t(i);
    }
    const uint32_t any = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && any) atomicOr(flags, any);
}

// Domain check of positions loaded from device memory.
template <int DIM, class View>
__global__ void k_check_domain(int n, int64_t stride, const double* __restrict__ pos,
                               const __grid_constant__ View v, uint32_t* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const RealParams& P = v.of_input(uint32_t(i));
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double x = pos[a * stride + i];
        if (!(x >= P.box.lo[a] && x <= P.box.hi[a])) atomicOr(status, kStatusOutOfDomain);
    }
}

// Cell-corner tables: entry P.g.corner_off[a] + c holds lo_a + c w_a of
// realisation P as a binary32 head (nearest) and tail (nearest to the
// remainder).  One thread per (realisation, axis, cell) entry; `first[k]` is
// the first entry of realisation k (first[nreal] = total).
__global__ void k_corners(int total, int nreal, int dim, const RealParams* __restrict__ tbl,
                          const int* __restrict__ first, float2* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int lo = 0, hi = nreal - 1;            // realisation: last k with first[k] <= t
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const Grid& g = tbl[lo].g;
    int a = 0;
    while (a + 1 < dim && t >= g.corner_off[a + 1]) ++a;
    const int c = t - g.corner_off[a];
    const double corner = __dadd_rn(g.lo[a], __dmul_rn(double(c + g.off[a]), g.w[a]));
    const float hi_f = __double2float_rn(corner);
    out[t] = make_float2(hi_f, __double2float_rn(__dsub_rn(corner, double(hi_f))));
}

__global__ void k_iota(int n, uint32_t* __restrict__ id) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = uint32_t(i);
}

// ---------------------------------------------------------------------------
// Step 2a: exclusive prefix sum of the cell counts in one launch.  Each block
// scans a tile of 16 cells per thread, publishes the tile's total, and adds
// the totals of all tiles before it, which every block publishes before it
// waits on anyone (so no wait is chained behind another: the reduce-then-scan
// pair of launches fused by single-pass publication, in the manner of D.
// Merrill and M. Garland's decoupled look-back, NVIDIA technical report
// NVR-2016-002).  The count array is padded with zeros to whole tiles, so
// start[n_cells] = n.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t block_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t ws = lane < nw ? warp_sums[lane] : 0u;
        uint32_t wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) warp_sums[lane] = wi - ws;
        if (lane == 31) block_total = wi;     // lane 31's inclusive sum covers every warp
    }
    __syncthreads();
    const uint32_t excl = warp_sums[warp] + inc - v;
    *total = block_total;
    __syncthreads();
    return excl;
}

// A tile's published word: tag << 32 | total.  The tag is the launch's number
// (ticket / tiles) mod 2^32 - 1, plus one: every launch rewrites every tile's
// word, so a word still holding the previous launch's tag, or the zero the
// host writes when the grid changes, is told apart from this launch's.
constexpr unsigned long long kScanTagMod = 0xffffffffull;
// Polls before a block stops waiting for an earlier tile's total and sums
// that tile's counts itself (tens of milliseconds; the tiles it waits on took
// their tickets first, so they are running: a safety net, not a path the
// scan takes).
constexpr int kScanWaitLimit = 1 << 17;
__device__ unsigned long long g_scan_waits_given_up;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// state[0, ntiles) are the tiles' words, state[ntiles] the ticket (both zeroed
// by the host whenever the grid changes).  The block of the last tile
// advances the walk's step counter (device-resident, so a captured graph of
// steps replays with the right counters) when `advance` is set: every kernel
// of the step that reads it has completed.  A tile equal to `hold` never
// publishes (a test hook: the tiles after it then run out of polls).
__global__ void __launch_bounds__(kScanThreads)
k_scan(const uint4* __restrict__ count4, uint4* __restrict__ start4,
       unsigned long long* __restrict__ state, int ntiles,
       unsigned long long* __restrict__ step_dev, int advance, int hold) {
    constexpr int kVec = kScanPerThread / 4;
    __shared__ uint32_t s_tile;
    __shared__ unsigned long long s_tag;
    if (threadIdx.x == 0) {
        // tiles in ticket order: a block only ever waits on blocks that started
        const unsigned long long t = atomicAdd(state + ntiles, 1ull);
        s_tile = uint32_t(t % unsigned(ntiles));
        s_tag = (t / unsigned(ntiles)) % kScanTagMod + 1ull;
    }
    __syncthreads();
    const uint32_t tile = s_tile;
    const unsigned long long tag = s_tag;
    // this thread's 16 consecutive cells
    const size_t base = (size_t(tile) * kScanThreads + threadIdx.x) * kVec;
    uint4 c[kVec];
    uint32_t own = 0;
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
        c[k] = count4[base + k];
        own += c[k].x + c[k].y + c[k].z + c[k].w;
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(own, &total);
    if (threadIdx.x == 0 && int(tile) != hold) st_relaxed_u64(state + tile, (tag << 32) | total);
    // the totals of every earlier tile, one word per thread at a time
    uint32_t part = 0;
    bool gave_up = false;
    for (uint32_t p = threadIdx.x; p < tile; p += kScanThreads) {
        unsigned long long w = ld_relaxed_u64(state + p);
        for (int polls = 0; (w >> 32) != tag && polls < kScanWaitLimit; ++polls) {
            __nanosleep(64);
            w = ld_relaxed_u64(state + p);
        }
        if ((w >> 32) == tag) {
            part += uint32_t(w);
        } else {
            gave_up = true;
            const uint4* q = count4 + size_t(p) * (kScanTile / 4);
            for (int k = 0; k < kScanTile / 4; ++k) part += q[k].x + q[k].y + q[k].z + q[k].w;
        }
    }
    if (gave_up) atomicAdd(&g_scan_waits_given_up, 1ull);
    uint32_t prefix;
    block_exclusive_scan(part, &prefix);
    if (advance && threadIdx.x == 0 && tile == uint32_t(ntiles - 1)) *step_dev += 1ull;
    uint32_t e = prefix + excl;
#pragma unroll
    for (int k = 0; k < kVec; ++k) {
        start4[base + k] = make_uint4(e, e + c[k].x, e + c[k].x + c[k].y, e + c[k].x + c[k].y + c[k].z);
        e += c[k].x + c[k].y + c[k].z + c[k].w;
    }
}

// Step counter updates for steps without a scan (walk only) and for resets.
__global__ void k_advance_step(unsigned long long* __restrict__ step_dev) { *step_dev += 1ull; }
__global__ void k_set_step(unsigned long long* __restrict__ step_dev, unsigned long long value) {
    *step_dev = value;
}

// Realisation index of every particle of a batch: the last k with
// first[k] <= i (first[nreal] = n).
__global__ void k_fill_rid(int n, int nreal, const uint32_t* __restrict__ first,
                           uint32_t* __restrict__ rid) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nreal - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= uint32_t(i)) lo = mid; else hi = mid - 1;
    }
    rid[i] = uint32_t(lo);
}

// ---------------------------------------------------------------------------
// Step 2b: counting-sort scatter.  Each particle takes a slot of its cell
// (decrementing the count returns every count to zero for the next step) and
// stores there its index and a 16-byte sort key: x, and id | cell << 32, all
// that the in-cell ranking of the gather reads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock)
k_scatter(int n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ start,
          uint32_t* __restrict__ count, const double* __restrict__ x,
          const uint32_t* __restrict__ id, uint32_t* __restrict__ perm,
          double2* __restrict__ sortkey) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = key[i];
    const double xi = x[i];
    const uint32_t idi = id[i];
    const uint32_t left = atomicSub(&count[c], 1u);
    const uint32_t slot = start[c] + left - 1u;
    if (!check(left >= 1u && slot < uint32_t(n), kChkSlot)) return;
    perm[slot] = uint32_t(i);
    sortkey[slot] = make_double2(xi, __longlong_as_double((long long)(uint64_t(idi) |
                                                                      (uint64_t(c) << 32))));
}

// Cell coordinates of a realisation-local cell index (the last axis needs
// no modulo).
template <int DIM>
__device__ __forceinline__ void cell_coords_of(uint32_t local, const Grid& g, int* c) {
    c[0] = c[1] = c[2] = 0;
    if constexpr (DIM == 1) {
        c[0] = int(local);
    } else if constexpr (DIM == 2) {
        const uint32_t q = local / uint32_t(g.n[0]);
        c[0] = int(local - q * uint32_t(g.n[0]));
        c[1] = int(q);
    } else {
        const uint32_t q = local / uint32_t(g.n[0]);
        c[0] = int(local - q * uint32_t(g.n[0]));
        const uint32_t r = q / uint32_t(g.n[1]);
        c[1] = int(q - r * uint32_t(g.n[1]));
        c[2] = int(r);
    }
}

// The same from a particle's record: its x (and, in 2-d, y) cell index is
// there, so only 3-d reads the cell array (`cell` is cell[s], unused below 3-d).
template <int DIM>
__device__ __forceinline__ void cell_coords_rec(uint32_t cell, const float4& me, const RealParams& P,
                                                int* c) {
    if constexpr (DIM == 3) {
        cell_coords_of<3>(cell - P.cell_base, P.g, c);
    } else {
        c[0] = int(me.w);
        c[1] = DIM == 2 ? int(me.z) : 0;
        c[2] = 0;
    }
}

// cell[s] where the pair searches need it (3-d), else nothing is read.
template <int DIM>
__device__ __forceinline__ uint32_t cell_arg(const uint32_t* __restrict__ cell, uint32_t s) {
    return DIM == 3 ? cell[s] : 0u;
}

// Step 2c: gather into cell order.  The slot order the atomics gave inside a
// cell is replaced by the rank of (x, id) -- binary64 x in its integer order,
// the id breaking ties -- so the layout (and every sum over it) is identical
// run to run, and each neighbour row (cells cx-1..cx+1 of one y (, z)) is
// sorted by x up to the cells' rounding slack, which the pair search uses.
// The rank reads the sort keys of the cell's slots, next to the particle's
// own; the rest of the payload comes from the source index.  Also writes the
// particle's cell, its binary32 offset from the cell corner (from the
// binary32 head/tail split of the coordinate and of the corner: error below
// 2^-23 w, no binary64 instruction).
template <int DIM, class View, bool TANGENT = false>
__global__ void __launch_bounds__(kBlock)
k_gather(int n, int64_t stride, const uint32_t* __restrict__ perm,
         const double2* __restrict__ sortkey, const uint32_t* __restrict__ start,
         const double* __restrict__ pos_in, const double* __restrict__ mass_in,
         uint32_t* __restrict__ id_out, double* __restrict__ pos_out,
         double* __restrict__ mass_out, uint32_t* __restrict__ cell_out,
         float4* __restrict__ rec_out,
         const float2* __restrict__ corners, uint32_t* __restrict__ rid_out,
         const __grid_constant__ View v, const double* __restrict__ tan_in = nullptr,
         double* __restrict__ tan_out = nullptr, const double* __restrict__ mass_b_in = nullptr,
         double* __restrict__ mass_b_out = nullptr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t src = perm[s];
    const double2 me = sortkey[s];
    if (!check(src < uint32_t(n), kChkGather)) return;
    // payload loads first: independent of the ranking below
    double xa[3] = {me.x, 0.0, 0.0};
#pragma unroll
    for (int a = 1; a < DIM; ++a) xa[a] = pos_in[a * stride + src];
    const double m = mass_in[src];
    const unsigned long long idc = (unsigned long long)__double_as_longlong(me.y);
    const uint32_t my_id = uint32_t(idc), c = uint32_t(idc >> 32);
    const uint32_t b = start[c], e = start[c + 1];
    if (!check(b <= uint32_t(s) && uint32_t(s) < e && e <= uint32_t(n), kChkGather)) return;
    const long long my_x = order_key(me.x);
    const uint32_t my_rank_id = my_id & ~kGhostBit;   // ghosts rank by their own id
    uint32_t rank = 0;
    for (uint32_t k = b; k < e; ++k) {
        const double2 q = sortkey[k];
        const long long xo = order_key(q.x);
        const uint32_t ido = uint32_t(__double_as_longlong(q.y)) & ~kGhostBit;
        rank += (xo < my_x || (xo == my_x && ido < my_rank_id)) ? 1u : 0u;
    }
    const uint32_t dst = b + rank;
    if (!check(dst < e, kChkGather)) return;
    id_out[dst] = my_id;
    if constexpr (DIM == 3) cell_out[dst] = c;   // only the 3-d searches read it
    if constexpr (View::kBatch) rid_out[dst] = __ldg(v.rid_input + src);
    if (mass_b_out) mass_b_out[dst] = mass_b_in[src];   // second species (reactions)
    const RealParams& P = v.of_input(src);
    mass_out[dst] = m;
    float off[3] = {0.0f, 0.0f, 0.0f};
    int cc[3];
    cell_coords_of<DIM>(c - P.cell_base, P.g, cc);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const uint32_t ca = uint32_t(cc[a]);
        const double x = xa[a];
        pos_out[a * stride + dst] = x;
        if constexpr (TANGENT) tan_out[a * stride + dst] = tan_in[a * stride + src];
        if (P.transfer) {
            float xh, xlo;
            split_double(x, &xh, &xlo);
            const float2 cr = __ldg(corners + P.g.corner_off[a] + ca);
            off[a] = __fadd_rn(__fsub_rn(xh, cr.x), __fsub_rn(xlo, cr.y));
        }
    }
    rec_out[dst] = make_float4(off[0], off[1], DIM == 2 ? float(cc[1]) : off[2], float(cc[0]));
}

// Sort of a freshly loaded single run, whose particles arrive in input order
// rather than cell order: the same counting sort and the same cell order, but
// the scatter stores each particle's whole payload as one record of 16-byte
// chunks at its slot, so the gather reads only records in slot order.  A
// record fills whole 32-byte sectors, which the scattered stores of an
// unsorted input then write without a read (the sort keys plus a separate
// payload read through the permutation cost more there; in steady state,
// where the slots barely move, the opposite holds).  Eight-byte lanes:
//   0: x   1: id | cell << 32   2..DIM: the other axes   DIM + 1: mass
//   then DIM position tangents (TANGENT)
template <int DIM, bool TANGENT>
struct SortRec {
    static constexpr int kLanes = 2 + DIM + (TANGENT ? DIM : 0);
    static constexpr int kChunks = (kLanes + 1) / 2;
    static constexpr int kTan = DIM + 2;
};

template <int DIM, bool TANGENT>
__global__ void __launch_bounds__(kBlock)
k_scatter_rec(int n, int64_t stride, const uint32_t* __restrict__ key,
              const uint32_t* __restrict__ start, uint32_t* __restrict__ count,
              const double* __restrict__ pos, const double* __restrict__ mass,
              const uint32_t* __restrict__ id, const double* __restrict__ tan,
              double2* __restrict__ recs) {
    using R = SortRec<DIM, TANGENT>;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = key[i];
    double lane[2 * R::kChunks];
    lane[0] = pos[i];
    lane[1] = __longlong_as_double((long long)(uint64_t(id[i]) | (uint64_t(c) << 32)));
#pragma unroll
    for (int a = 1; a < DIM; ++a) lane[1 + a] = pos[a * stride + i];
    lane[DIM + 1] = mass[i];
    if constexpr (TANGENT) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) lane[R::kTan + a] = tan[a * stride + i];
    }
    if constexpr (R::kLanes % 2 == 1) lane[R::kLanes] = 0.0;
    const uint32_t left = atomicSub(&count[c], 1u);
    const uint32_t slot = start[c] + left - 1u;
    if (!check(left >= 1u && slot < uint32_t(n), kChkSlot)) return;
    double2* r = recs + size_t(slot) * R::kChunks;
#pragma unroll
    for (int k = 0; k < R::kChunks; ++k) r[k] = make_double2(lane[2 * k], lane[2 * k + 1]);
}

// Gather from the records: the rank inside the cell by (x order key, id)
// reads chunk 0 of the cell's records; outputs as k_gather's.
template <int DIM, bool TANGENT>
__global__ void __launch_bounds__(kBlock)
k_gather_rec(int n, int64_t stride, const double2* __restrict__ recs,
             const uint32_t* __restrict__ start, uint32_t* __restrict__ id_out,
             double* __restrict__ pos_out, double* __restrict__ mass_out,
             uint32_t* __restrict__ cell_out, float4* __restrict__ rec_out,
             const float2* __restrict__ corners,
             const __grid_constant__ SingleView v, double* __restrict__ tan_out) {
    using R = SortRec<DIM, TANGENT>;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double lane[2 * R::kChunks];
    const double2* me = recs + size_t(s) * R::kChunks;
#pragma unroll
    for (int k = 0; k < R::kChunks; ++k) {
        const double2 q = me[k];
        lane[2 * k] = q.x;
        lane[2 * k + 1] = q.y;
    }
    const unsigned long long idc = (unsigned long long)__double_as_longlong(lane[1]);
    const uint32_t my_id = uint32_t(idc), c = uint32_t(idc >> 32);
    const uint32_t b = start[c], e = start[c + 1];
    if (!check(b <= uint32_t(s) && uint32_t(s) < e && e <= uint32_t(n), kChkGather)) return;
    const long long my_x = order_key(lane[0]);
    const uint32_t my_rank_id = my_id & ~kGhostBit;   // ghosts rank by their own id
    uint32_t rank = 0;
    for (uint32_t k = b; k < e; ++k) {
        const double2 q = recs[size_t(k) * R::kChunks];
        const long long xo = order_key(q.x);
        const uint32_t ido = uint32_t(__double_as_longlong(q.y)) & ~kGhostBit;
        rank += (xo < my_x || (xo == my_x && ido < my_rank_id)) ? 1u : 0u;
    }
    const uint32_t dst = b + rank;
    if (!check(dst < e, kChkGather)) return;
    id_out[dst] = my_id;
    if constexpr (DIM == 3) cell_out[dst] = c;   // only the 3-d searches read it
    const RealParams& P = v.p;
    const double m = lane[DIM + 1];
    mass_out[dst] = m;
    float off[3] = {0.0f, 0.0f, 0.0f};
    int cc[3];
    cell_coords_of<DIM>(c - P.cell_base, P.g, cc);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const uint32_t ca = uint32_t(cc[a]);
        const double x = lane[a == 0 ? 0 : 1 + a];
        pos_out[a * stride + dst] = x;
        if constexpr (TANGENT) tan_out[a * stride + dst] = lane[R::kTan + a];
        if (P.transfer) {
            float xh, xlo;
            split_double(x, &xh, &xlo);
            const float2 cr = __ldg(corners + P.g.corner_off[a] + ca);
            off[a] = __fadd_rn(__fsub_rn(xh, cr.x), __fsub_rn(xlo, cr.y));
        }
    }
    rec_out[dst] = make_float4(off[0], off[1], DIM == 2 ? float(cc[1]) : off[2], float(cc[0]));
}

// ---------------------------------------------------------------------------
// Steps 2-5: neighbour visits.  For particle s (cell order) the candidates
// are the particles of the 3^DIM surrounding cells, s itself included, each
// neighbour row cut to the window of x that can reach the cutoff (see
// for_each_row).  The
// binary32 squared distance from the cell offsets decides every candidate
// outside a narrow band around psi^2; inside the band the exact binary64 test
// dx*dx + dy*dy (+ dz*dz) <= psi^2 (no fma, dx = x_i - x_j) decides.  The
// band half-width is set on the host from an error bound of the binary32
// evaluation, so the accepted set equals the exact binary64 pair set.
//
// The binary32 difference is (off_j - off_s) + shift, which changes sign
// exactly when s and j swap, so d2f(s, j) == d2f(j, s) bit for bit and every
// quantity derived from it is symmetric in the pair.  The self pair has
// d2f = 0, K = 1 exactly: it supplies the self term of the row sum and a zero
// flux, so no candidate is skipped.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double exact_d2(const double* __restrict__ pos, int64_t stride,
                                           uint32_t i, uint32_t j) {
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double d = __dsub_rn(__ldg(pos + a * stride + i), __ldg(pos + a * stride + j));
        const double sq = __dmul_rn(d, d);
        d2 = (a == 0) ? sq : __dadd_rn(d2, sq);
    }
    return d2;
}

// Squared distance for the kernel value (not for the pair test): one fma per
// axis after the first.  Symmetric in (i, j) bit for bit (the differences
// only change sign), and within 2 ulp of the exact square sum.
template <int DIM>
__device__ __forceinline__ double kernel_d2(const double* __restrict__ pos, int64_t stride,
                                            uint32_t i, uint32_t j) {
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double d = __dsub_rn(__ldg(pos + a * stride + i), __ldg(pos + a * stride + j));
        d2 = (a == 0) ? __dmul_rn(d, d) : __fma_rn(d, d, d2);
    }
    return d2;
}

// Hardware square root approximation (relative error far below the
// windows' slack trim_eps, which covers it).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Binary32 x difference of candidate o from particle me (cells cx_o - cx_me
// apart, |cx_o - cx_me| <= reach <= 2, so the shift is a power-of-two multiple
// of wx and exact, and one fused multiply-add rounds exactly as the sum of the
// rounded offset difference and the shift would): changes sign exactly when
// the pair swaps.
__device__ __forceinline__ float dx_f32(const float4& me, const float4& o, float wx) {
    return __fmaf_rn(__fsub_rn(o.w, me.w), wx, __fsub_rn(o.x, me.x));
}

template <int DIM>
__device__ __forceinline__ float d2_f32(float dx, const float4& me, const float4& o, float sy,
                                        float sz) {
    if (DIM == 1) return __fmul_rn(dx, dx);
    const float dy = __fadd_rn(__fsub_rn(o.y, me.y), sy);
    if (DIM == 2) return __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    const float dz = __fadd_rn(__fsub_rn(o.z, me.z), sz);
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

// Lower bound of |dy_f| over the particles of the row `d` cells away along an
// axis (d = 0: the particle's own row, bound 0): the rows below hold offsets
// up to w from their cells' corners, those above offsets from 0, so the gap
// is the particle's own offset (or w minus it) plus |d| - 1 whole cells, less
// the slack that covers the roundings.
__device__ __forceinline__ float row_gap(int d, float off, float w, float eps) {
    if (d == 0) return 0.0f;
    const float near = d < 0 ? off : __fsub_rn(w, off);
    const int far = d < 0 ? -d - 1 : d - 1;
    const float gap = far == 0 ? near : __fmaf_rn(float(far), w, near);
    return fmaxf(__fsub_rn(gap, eps), 0.0f);
}

// Per-row candidate windows.  Row (dy, dz) of particle s is the particle
// range [j0, j3) of cells cx-R..cx+R at y index cy+dy (z index cz+dz), R the
// grid's reach (|dy|, |dz| <= R); the
// gather sorts it by x up to a slack.  Every accepted candidate has
// d2f <= band_hi, so with g a lower bound of |dy_f| (and |dz_f|) over the row
// its binary32 dx satisfies dx^2 <= reach2 - g^2 (reach2 carries the
// roundings).  The row is skipped when that is negative; otherwise
//   rx = sqrt(reach2 - g^2) + trim_eps
// where trim_eps (host) bounds the sqrt rounding plus the row's departure from
// x order (two dx errors and twice the cell-index error dc w).  A bisection
// finds the first j with dx_j >= -rx: every earlier candidate then has
// dx < -rx + trim_eps, too far left.  The caller's loop stops at the first
// dx_j > rx: every later one has dx > rx - trim_eps.  Neither bound drops a
// neighbour, so the accepted set is the exact binary64 one as before.
// row(j0, j3, rx, sy, sz) is called for every row that can hold a neighbour.
template <int DIM, class Row>
__device__ __forceinline__ void for_each_row(uint32_t cell, const float4& me,
                                             const float4* __restrict__ rec,
                                             const uint32_t* __restrict__ start,
                                             const RealParams& P, Row&& row) {
    const Grid& g = P.g;
    const PairParams& pp = P.pp;
    int c[3];
    cell_coords_rec<DIM>(cell, me, P, c);
    const int R = g.reach;
    const int xlo = max(c[0] - R, 0);
    const int xhi = min(c[0] + R, g.n[0] - 1);
    const int zlo = DIM == 3 ? max(-R, -c[2]) : 0;
    const int zhi = DIM == 3 ? min(R, g.n[2] - 1 - c[2]) : 0;
    const int ylo = DIM >= 2 ? max(-R, -c[1]) : 0;
    const int yhi = DIM >= 2 ? min(R, g.n[1] - 1 - c[1]) : 0;
    const float eps = pp.trim_eps;
    const float wx = g.wf[0];
    for (int dz = zlo; dz <= zhi; ++dz) {
        const float sz = DIM == 3 ? float(dz) * g.wf[2] : 0.0f;
        const float gz = DIM == 3 ? row_gap(dz, me.z, g.wf[2], eps) : 0.0f;
        for (int dy = ylo; dy <= yhi; ++dy) {
            const float sy = DIM >= 2 ? float(dy) * g.wf[1] : 0.0f;
            const float gy = DIM >= 2 ? row_gap(dy, me.y, g.wf[1], eps) : 0.0f;
            const float r2 = __fsub_rn(pp.reach2, __fmaf_rn(gy, gy, __fmul_rn(gz, gz)));
            if (r2 < 0.0f) continue;
            const float rx = __fadd_rn(sqrt_approx(r2), eps);
            const uint32_t rowc = P.cell_base + (uint32_t(c[2] + dz) * uint32_t(g.n[1]) +
                                                 uint32_t(c[1] + dy)) * uint32_t(g.n[0]);
            if (!check(rowc + uint32_t(xhi) + 1u - P.cell_base <=
                           uint32_t(g.n[0]) * uint32_t(g.n[1]) * uint32_t(g.n[2]), kChkRow))
                continue;
            uint32_t lo = __ldg(start + rowc + xlo);
            uint32_t hi = __ldg(start + rowc + xhi + 1);
            const uint32_t j3 = hi;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (dx_f32(me, __ldg(rec + mid), wx) < -rx) lo = mid + 1;
                else hi = mid;
            }
            row(lo, j3, rx, sy, sz);
        }
    }
}

// visit(j, d2f, rec_j) is called for every neighbour j of s (s included).
template <int DIM, class Visit>
__device__ __forceinline__ void visit_neighbours(uint32_t s, uint32_t cell, int64_t stride,
                                                 const float4* __restrict__ rec,
                                                 const double* __restrict__ pos,
                                                 const uint32_t* __restrict__ start,
                                                 const RealParams& P, Visit&& visit) {
    const PairParams& pp = P.pp;
    const float4 me = rec[s];
    const float wx = P.g.wf[0];
    for_each_row<DIM>(cell, me, rec, start, P,
                      [&](uint32_t j0, uint32_t j3, float rx, float sy, float sz) {
#pragma unroll 2
        for (uint32_t j = j0; j < j3; ++j) {
            const float4 o = __ldg(rec + j);
            const float dx = dx_f32(me, o, wx);
            if (dx > rx) break;
            const float d2f = d2_f32<DIM>(dx, me, o, sy, sz);
            if (d2f > pp.band_hi) continue;
            if (d2f >= pp.band_lo && exact_d2<DIM>(pos, stride, s, j) > pp.psi2) continue;
            visit(j, d2f, o);
        }
    });
}

// The exact binary64 test as a real call, so the compiler cannot if-convert
// it into every candidate's path (it runs only inside the narrow band).
template <int DIM>
__device__ __noinline__ bool exact_within(const double* __restrict__ pos, int64_t stride,
                                          uint32_t s, uint32_t j, double psi2) {
    return exact_d2<DIM>(pos, stride, s, j) <= psi2;
}

// As visit_neighbours, but calls visit(j, d2f, accept) for every candidate of
// the windows (the pass bodies run without a branch on the cutoff).  A
// candidate inside the narrow band around the cutoff gets the exact binary64
// test in place, or, with DEFER_BAND, is first visited as rejected and, if
// the particle met any, a second walk visits those the exact test accepts
// (rare: the band holds ~1e-5 of candidates; measured faster for the row
// sums, not for the exchange).
template <int DIM, bool DEFER_BAND, class Visit>
__device__ __forceinline__ void scan_neighbours(uint32_t s, uint32_t cell, int64_t stride,
                                                const float4* __restrict__ rec,
                                                const double* __restrict__ pos,
                                                const uint32_t* __restrict__ start,
                                                const RealParams& P, Visit&& visit) {
    const PairParams& pp = P.pp;
    const float4 me = rec[s];
    const float wx = P.g.wf[0];
    bool band = false;
    for_each_row<DIM>(cell, me, rec, start, P,
                      [&](uint32_t j0, uint32_t j3, float rx, float sy, float sz) {
        for (uint32_t j = j0; j < j3; ++j) {
            const float4 o = __ldg(rec + j);
            const float dx = dx_f32(me, o, wx);
            if (dx > rx) break;
            const float d2f = d2_f32<DIM>(dx, me, o, sy, sz);
            if constexpr (DEFER_BAND) {
                band |= (d2f >= pp.band_lo) & (d2f <= pp.band_hi);
                visit(j, d2f, d2f < pp.band_lo);
            } else {
                bool accept = d2f < pp.band_lo;
                if (d2f >= pp.band_lo && d2f <= pp.band_hi)
                    accept = exact_within<DIM>(pos, stride, s, j, pp.psi2);
                visit(j, d2f, accept);
            }
        }
    });
    if (DEFER_BAND && band) {
        for_each_row<DIM>(cell, me, rec, start, P,
                          [&](uint32_t j0, uint32_t j3, float rx, float sy, float sz) {
            for (uint32_t j = j0; j < j3; ++j) {
                const float4 o = __ldg(rec + j);
                const float dx = dx_f32(me, o, wx);
                if (dx > rx) break;
                const float d2f = d2_f32<DIM>(dx, me, o, sy, sz);
                if (d2f >= pp.band_lo && d2f <= pp.band_hi &&
                    exact_within<DIM>(pos, stride, s, j, pp.psi2))
                    visit(j, d2f, true);
            }
        });
    }
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Compensated summation of mixed-sign terms (Kahan-Babuska / Neumaier):
// s + c carries the sum to about twice binary32 precision whatever the order
// of magnitudes.  Used for the flux sums.
__device__ __forceinline__ void neumaier_add(float& s, float& c, float x) {
    const float t = __fadd_rn(s, x);
    const bool s_big = fabsf(s) >= fabsf(x);
    const float big = s_big ? s : x;
    const float small = s_big ? x : s;
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(big, t), small));
    s = t;
}

__device__ __forceinline__ void add_pair_count(uint32_t cnt, unsigned long long* counter) {
    const uint32_t warp_total = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && warp_total) atomicAdd(counter, (unsigned long long)warp_total);
}

// ---------------------------------------------------------------------------
// Binary64 pair passes.  A thread per particle walks its candidate windows,
// whose lengths differ from lane to lane, so work done inside that loop runs
// at a fraction of the warp's lanes, and GB300's binary64 unit charges a warp
// instruction the same whether 32 lanes or 3 are active.  These passes
// therefore split the work per warp:
//  (A) each lane walks its windows once with the binary32 prefilter and
//      appends every accepted neighbour j != s (and its binary32 d2) to its
//      own kSeg-entry segment in shared memory;
//  (B) when a lane's segment is full (checked at window ends) or the walk is
//      over, the warp evaluates the pair terms of all segments with all 32
//      lanes, one entry per lane, in lane-major order;
//  (C) each lane then adds its own results in the order it found them.
// Every sum therefore runs in candidate order and repeats bit for bit, the
// divergent loop holds only the prefilter, and the binary64 arithmetic runs
// at full width.  (The binary32 passes below keep the pair arithmetic inside
// the candidate loop: there the segment traffic costs more than the
// divergence it removes, measured at 1.5x their time.)
// ---------------------------------------------------------------------------
constexpr int kSeg = 12;                   // segment entries per lane
constexpr int kWarpsPerBlock = kBlock / 32;

__device__ __forceinline__ uint32_t warp_exclusive_scan(uint32_t v, uint32_t* total) {
    const int lane = threadIdx.x & 31;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    *total = __shfl_sync(0xffffffffu, inc, 31);
    return inc - v;
}

// Shared state of one block's warps.  V: type of the pair terms; D2: keep the
// binary32 d2 of each entry (binary32 passes).
template <int NW, class V, bool D2, int SEG = kSeg>
struct SegShared {
    static constexpr int kCap = SEG;   // entries per lane
    uint32_t j[NW][SEG][32];           // lane-owned segments, entry k of lane l at [k][l]
    float d2[NW][D2 ? SEG : 1][32];
    V v[NW][SEG * 32];                 // phase-B results, lane-major
    uint8_t owner[NW][SEG * 32];       // lane of each lane-major entry
    uint32_t off[NW][32];              // first lane-major entry of each lane
    uint32_t base[NW][32];             // entries each lane had before this flush
};

// Neighbour lists: pass 1 stores each accepted neighbour j != s and its pair
// value (the binary64 K_sj, or (K_sj, dK_sj/dD) in the adjoint) in slot k of
// s (entry at k * stride + s), up to `cap` slots; count[s] is the full
// number.  Pass 2 of a warp whose lanes all fit their lists reads them
// instead of searching and re-evaluating exp; otherwise the warp searches.
// Both paths visit the same pairs in the same order with the same values.
template <class V>
struct NbList {
    uint32_t* j;
    V* k;
    uint32_t* count;
    int cap;           // 0: no list
};
using NbList64 = NbList<double>;

// Precision-form neighbour lists: pass 1 stores each accepted neighbour
// j != s with its binary32 kernel value as {j, K bits} in slot k of s (entry
// at k * stride + s); count[s] is the full number.  Pass 2 of a warp whose
// lanes all fit their lists walks them instead of searching.
struct NbList32 {
    uint2* e;
    int cap;           // 0: no list; a particle's count is in its record ex[s].w
};

// Phases A-C for the calling warp (every lane of the warp must call it; lanes
// with valid = false walk nothing).  eval(owner_s, j, d2f) returns the pair
// term (d2f is 0 unless D2); add(term) is called by each lane for its own
// entries in order.  Returns the lane's number of accepted neighbours j != s.
template <int DIM, int NW, class V, bool D2, int SEG, class Eval, class Add>
__device__ __forceinline__ uint32_t seg_pairs(bool valid, uint32_t s, int64_t stride,
                                              const float4* __restrict__ rec,
                                              const double* __restrict__ pos,
                                              const uint32_t* __restrict__ cell,
                                              const uint32_t* __restrict__ start,
                                              const RealParams& P, SegShared<NW, V, D2, SEG>& S,
                                              Eval&& eval, Add&& add,
                                              NbList<V> store = NbList<V>{}) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t warp_s0 = s - uint32_t(lane);
    uint32_t cnt = 0, done = 0;
    auto flush = [&]() {
        uint32_t total;
        const uint32_t off = warp_exclusive_scan(cnt, &total);
        check(cnt <= uint32_t(SEG) && total <= uint32_t(SEG) * 32u, kChkSegment);
        S.off[warp][lane] = off;
        S.base[warp][lane] = done;
        for (uint32_t k = 0; k < cnt; ++k) S.owner[warp][off + k] = uint8_t(lane);
        __syncwarp();
        for (uint32_t e = uint32_t(lane); e < total; e += 32) {
            const uint32_t o = S.owner[warp][e];
            const uint32_t k = e - S.off[warp][o];
            const uint32_t j = S.j[warp][k][o];
            const V val = eval(warp_s0 + o, j, D2 ? S.d2[warp][D2 ? k : 0][o] : 0.0f);
            S.v[warp][e] = val;
            if (store.cap > 0) {
                const uint32_t slot = S.base[warp][o] + k;
                if (slot < uint32_t(store.cap)) {
                    const int64_t at = int64_t(slot) * stride + (warp_s0 + o);
                    store.j[at] = j;
                    store.k[at] = val;
                }
            }
        }
        __syncwarp();
        for (uint32_t k = 0; k < cnt; ++k) add(S.v[warp][off + k]);
        done += cnt;
        cnt = 0;
        __syncwarp();
    };

    const Grid& g = P.g;
    const PairParams& pp = P.pp;
    const float4 me = valid ? rec[s] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int c[3] = {0, 0, 0};
    if (valid) cell_coords_rec<DIM>(cell_arg<DIM>(cell, s), me, P, c);
    const int R = g.reach;
    const int xlo = max(c[0] - R, 0);
    const int xhi = min(c[0] + R, g.n[0] - 1);
    const float eps = pp.trim_eps;
    const float wx = g.wf[0];
    // rows in a fixed order for the whole warp; a lane whose row is outside
    // the grid or beyond the cutoff (see for_each_row) gets an empty window
#pragma unroll 1
    for (int dz = (DIM == 3 ? -R : 0); dz <= (DIM == 3 ? R : 0); ++dz) {
#pragma unroll 1
        for (int dy = (DIM >= 2 ? -R : 0); dy <= (DIM >= 2 ? R : 0); ++dy) {
            const float sy = DIM >= 2 ? float(dy) * g.wf[1] : 0.0f;
            const float sz = DIM == 3 ? float(dz) * g.wf[2] : 0.0f;
            uint32_t j = 0, j3 = 0;
            float rx = 0.0f;
            const bool in_grid = valid && (DIM < 2 || (c[1] + dy >= 0 && c[1] + dy < g.n[1])) &&
                                 (DIM < 3 || (c[2] + dz >= 0 && c[2] + dz < g.n[2]));
            if (in_grid) {
                const float gy = DIM >= 2 ? row_gap(dy, me.y, g.wf[1], eps) : 0.0f;
                const float gz = DIM == 3 ? row_gap(dz, me.z, g.wf[2], eps) : 0.0f;
                const float r2 = __fsub_rn(pp.reach2, __fmaf_rn(gy, gy, __fmul_rn(gz, gz)));
                if (r2 >= 0.0f) {
                    rx = __fadd_rn(sqrt_approx(r2), eps);
                    const uint32_t rowc = P.cell_base + (uint32_t(c[2] + dz) * uint32_t(g.n[1]) +
                                                         uint32_t(c[1] + dy)) * uint32_t(g.n[0]);
                    const bool row_ok = check(
                        rowc + uint32_t(xhi) + 1u - P.cell_base <=
                            uint32_t(g.n[0]) * uint32_t(g.n[1]) * uint32_t(g.n[2]), kChkRow);
                    uint32_t lo = row_ok ? __ldg(start + rowc + xlo) : 0u;
                    uint32_t hi = row_ok ? __ldg(start + rowc + xhi + 1) : 0u;
                    j3 = hi;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (dx_f32(me, __ldg(rec + mid), wx) < -rx) lo = mid + 1;
                        else hi = mid;
                    }
                    j = lo;
                }
            }
            do {
                while (j < j3 && cnt < uint32_t(SEG)) {
                    const float4 o = __ldg(rec + j);
                    const float dx = dx_f32(me, o, wx);
                    if (dx > rx) {
                        j = j3;
                        break;
                    }
                    const float d2f = d2_f32<DIM>(dx, me, o, sy, sz);
                    bool accept = d2f < pp.band_lo;
                    if (d2f >= pp.band_lo && d2f <= pp.band_hi)
                        accept = exact_within<DIM>(pos, stride, s, j, pp.psi2);
                    if (accept && j != s) {
                        S.j[warp][cnt][lane] = j;
                        if (D2) S.d2[warp][D2 ? cnt : 0][lane] = d2f;
                        ++cnt;
                    }
                    ++j;
                }
                if (__any_sync(0xffffffffu, cnt == uint32_t(SEG))) flush();
            } while (__any_sync(0xffffffffu, j < j3));
        }
    }
    if (__any_sync(0xffffffffu, cnt > 0)) flush();
    return done;
}

// Phases B-C over stored lists (the warp's lanes all fit their lists):
// eval(owner_s, j, stored value) returns the pair term, add(term) as above.
template <int NW, class V, int SEG, class VL, class Eval, class Add>
__device__ __forceinline__ void dense_listed(bool valid, uint32_t s, int64_t stride,
                                             uint32_t cnt, const NbList<VL>& nb,
                                             SegShared<NW, V, false, SEG>& S, Eval&& eval,
                                             Add&& add) {
    constexpr uint32_t kChunk = SEG * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t total;
    const uint32_t off = warp_exclusive_scan(valid ? cnt : 0u, &total);
    S.off[warp][lane] = off;
    const uint32_t warp_s0 = s - uint32_t(lane);
    for (uint32_t chunk = 0; chunk < total; chunk += kChunk) {
        const uint32_t chunk_end = chunk + kChunk;
        if (valid) {
            const uint32_t q0 = max(off, chunk), q1 = min(off + cnt, chunk_end);
            for (uint32_t q = q0; q < q1; ++q) S.owner[warp][q - chunk] = uint8_t(lane);
        }
        __syncwarp();
        const uint32_t m = min(total - chunk, kChunk);
        for (uint32_t e = uint32_t(lane); e < m; e += 32) {
            const uint32_t o = S.owner[warp][e];
            const uint32_t so = warp_s0 + o;
            const int64_t at = int64_t(chunk + e - S.off[warp][o]) * stride + so;
            S.v[warp][e] = eval(so, __ldg(nb.j + at), __ldg(nb.k + at));
        }
        __syncwarp();
        if (valid) {
            const uint32_t q0 = max(off, chunk), q1 = min(off + cnt, chunk_end);
            for (uint32_t q = q0; q < q1; ++q) add(S.v[warp][q - chunk]);
        }
        __syncwarp();
    }
}

// Pass 1, binary64 form: r_s = 1 + sum_{j != s} exp(-a d2_sj) (the kernel
// without its constant factor, which cancels in W; the self term is 1), and
// the ordered pair count.
template <int DIM, class View>
__global__ void __launch_bounds__(kBlock)
k_rowsum_f64(int n, int64_t stride, const double* __restrict__ pos, const float4* __restrict__ rec,
             const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
             const double* __restrict__ exp_table, const __grid_constant__ View v,
             double* __restrict__ r_out, unsigned long long* __restrict__ pair_counter,
             NbList64 nb, const uint32_t* __restrict__ ghost_id) {
    __shared__ double table[kExpTable];
    __shared__ SegShared<kWarpsPerBlock, double, false> seg;
    for (int t = threadIdx.x; t < kExpTable; t += blockDim.x) table[t] = exp_table[t];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const RealParams& P = v.of_sorted(uint32_t(s < n ? s : 0));
    const bool valid = s < n && P.transfer;
    double r = 1.0;
    const uint32_t cnt = seg_pairs<DIM>(
        valid, uint32_t(s), stride, rec, pos, cell, start, P, seg,
        [&](uint32_t so, uint32_t j, float) {
            const RealParams& Po = v.of_sorted(so);
            return gauss_exp(kernel_d2<DIM>(pos, stride, so, j), table, Po.pp.ec);
        },
        [&](double K) { r = __dadd_rn(r, K); }, nb);
    if (s < n) r_out[s] = r;
    if (nb.cap > 0 && s < n) nb.count[s] = valid ? cnt : 0u;
    // with ghost_id (a tile), pairs are counted for the tile's own particles only
    const bool counted = valid && !(ghost_id && (ghost_id[s] & kGhostBit));
    add_pair_count(counted ? cnt : 0u, pair_counter);
}

// The next step's walk done at the end of pass 2 (walk-ahead, for the steps of
// one call that another step follows): particle s of this step's cell order
// keeps its index, and its walked position, its id, cell key and cell count
// go to the other buffer pair, which the next step's sort then reads as its
// input order.  The walk is latency-tolerant arithmetic (binary64 pipe,
// generator) and pass 2 waits on memory, so the two overlap in one kernel.
struct WalkAhead {
    const uint32_t* id_in;              // this step's ids (cell order)
    double* pos_next;                   // walked positions, same index
    uint32_t* id_next;                  // the ids, same index
    uint32_t* key;                      // cell keys of the next sort
    uint32_t* count;                    // cell counts of the next sort
    uint32_t* status;
    const unsigned long long* step_dev; // the walk's step counter, already advanced
    const uint32_t* rid_in = nullptr;   // a batch: realisation of each particle (cell order)
    uint32_t* rid_next = nullptr;       // a batch: the same, same index
};

// WALK selects the walk-ahead instance of a pass-2 kernel: 0 none, 1 the
// walk, 2 the walk with the advection term.
template <int DIM, int WALK>
__device__ __forceinline__ void walk_ahead(const RealParams& P, int s, int64_t stride,
                                           const double* __restrict__ pos, const WalkAhead& wa) {
    double x[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = pos[a * stride + s];
    const uint32_t idv = wa.id_in[s];
    if (P.walk)
        walk_particle<DIM, false, WALK == 2>(P, idv - P.id_offset, *wa.step_dev, x, nullptr, stride, s);
#pragma unroll
    for (int a = 0; a < DIM; ++a) wa.pos_next[a * stride + s] = x[a];
    wa.id_next[s] = idv;
    if (wa.rid_next) wa.rid_next[s] = wa.rid_in[s];
    key_particle<DIM>(P, x, wa.status, wa.key + s, wa.count);
}

// Pass 2, binary64 form: M'_s = M_s + beta sum_j (M_j - M_s) 2 K_sj / (r_s + r_j).
template <int DIM, class View, int WALK = 0>
__global__ void __launch_bounds__(kBlock)
k_exchange_f64(int n, int64_t stride, const double* __restrict__ pos, const float4* __restrict__ rec,
               const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
               const double* __restrict__ exp_table, const __grid_constant__ View v,
               const double* __restrict__ r, const double* __restrict__ mass,
               double* __restrict__ mass_out, NbList64 nb, const WalkAhead wa = WalkAhead{}) {
    __shared__ double table[kExpTable];
    __shared__ SegShared<kWarpsPerBlock, double, false> seg;
    for (int t = threadIdx.x; t < kExpTable; t += blockDim.x) table[t] = exp_table[t];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const RealParams& P = v.of_sorted(uint32_t(s < n ? s : 0));
    const bool valid = s < n && P.transfer;
    double acc = 0.0;
    auto flux = [&](uint32_t so, uint32_t j, double K) {
        // 2K by an exponent increment (K is a positive normal), so
        // W = 2K / (r_s + r_j) rounds once
        const double K2 = __longlong_as_double(__double_as_longlong(K) + (1LL << 52));
        const double W = quot_pos(K2, __dadd_rn(__ldg(r + so), __ldg(r + j)));
        return __dmul_rn(__dsub_rn(__ldg(mass + j), __ldg(mass + so)), W);
    };
    const uint32_t listed = (nb.cap > 0 && valid) ? nb.count[s] : 0u;
    const bool fits = nb.cap > 0 && __all_sync(0xffffffffu, listed <= uint32_t(nb.cap));
    if (fits) {
        dense_listed(valid, uint32_t(s), stride, listed, nb, seg, flux,
                     [&](double f) { acc = __dadd_rn(acc, f); });
    } else {
        seg_pairs<DIM>(
            valid, uint32_t(s), stride, rec, pos, cell, start, P, seg,
            [&](uint32_t so, uint32_t j, float) {
                const RealParams& Po = v.of_sorted(so);
                const double K = gauss_exp(kernel_d2<DIM>(pos, stride, so, j), table, Po.pp.ec);
                return flux(so, j, K);
            },
            [&](double f) { acc = __dadd_rn(acc, f); });
    }
    if (s < n) mass_out[s] = valid ? __dadd_rn(mass[s], __dmul_rn(P.pp.beta, acc)) : mass[s];
    if constexpr (WALK > 0) {
        if (s < n) walk_ahead<DIM, WALK>(P, s, stride, pos, wa);
    }
}

// Pass 1, precision form: binary32 kernel exp2(-a log2(e) d2f) with the
// hardware ex2, compensated binary32 row sum, rounded to binary32; written
// with the binary32 head/tail split of the mass as the particle's record
// ex[s] = {m_hi, m_lo, r, list length (bits)} that pass 2 reads once per
// neighbour (.w only for the particle itself);
// with nb.cap > 0 also the neighbour lists of pass 2 (accepted j != s with
// their K, in visiting order: the band's exact accepts come last).
template <int DIM, class View, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (DIM == 3 ? 1536 : 2048) / BLOCK)
k_rowsum_f32(int n, int64_t stride, const double* __restrict__ pos, const float4* __restrict__ rec,
             const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
             const __grid_constant__ View v, const double* __restrict__ mass,
             float4* __restrict__ ex, unsigned long long* __restrict__ pair_counter,
             const uint32_t* __restrict__ ghost_id, NbList32 nb) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cnt = 0;
    if (s < n) {
        const RealParams& P = v.of_sorted(uint32_t(s));
        float rsum = 0.0f, rc = 0.0f;
        uint32_t listed = 0;
        if (P.transfer) {
            const float na = -P.pp.a_log2e;
            const uint32_t cap = uint32_t(nb.cap);
            uint2* lp = nb.e + s;          // slot `listed` of s
            scan_neighbours<DIM, true>(uint32_t(s), cell_arg<DIM>(cell, s), stride, rec, pos, start, P,
                                 [&](uint32_t j, float d2f, bool accept) {
                                     // compensated (Kahan) step for positive terms:
                                     // rsum - rc carries the sum; kept only for
                                     // accepted pairs
                                     const float K = ex2_approx(na * d2f);
                                     const float y = __fsub_rn(K, rc);
                                     const float t = __fadd_rn(rsum, y);
                                     const float cn = __fsub_rn(__fsub_rn(t, rsum), y);
                                     rsum = accept ? t : rsum;
                                     rc = accept ? cn : rc;
                                     const bool keep = accept && j != uint32_t(s);
                                     if (keep && listed < cap) *lp = make_uint2(j, __float_as_uint(K));
                                     if (keep) lp += stride;
                                     listed += keep ? 1u : 0u;
                                 });
            cnt = listed;   // the accepted pairs but the self pair
        } else {
            rsum = 1.0f;
        }
        float mhi, mlo;
        split_double(mass[s], &mhi, &mlo);
        ex[s] = make_float4(mhi, mlo, __fsub_rn(rsum, rc), __uint_as_float(listed));
        // with ghost_id (a tile), pairs are counted for the tile's own particles only
        if (ghost_id && (ghost_id[s] & kGhostBit)) cnt = 0;
    }
    add_pair_count(cnt, pair_counter);
}

// Pass 2, precision form: W = 2K / (r_s + r_j) in binary32 (symmetric bit for
// bit), mass difference from the binary32 head/tail split (exactly
// antisymmetric), flux accumulated with compensation, update in binary64.
// The flux sum of pass 2, precision form: W = 2 beta K / (r_s + r_j) in
// binary32 (symmetric bit for bit), the mass difference from the binary32
// head/tail split (exactly antisymmetric), compensated accumulation, and the
// update in binary64.  Each particle's record ex = {m_hi, m_lo, r, count} is one
// 16-byte load per neighbour.
struct FluxSum {
    float rs, two_beta;
    float2 ms;
    float acc = 0.0f, comp = 0.0f;
    // the pair's weight (shared by both species of a reaction run)
    __device__ __forceinline__ float weight(const float4& xj, float K) const {
        return __fdividef(two_beta * K, __fadd_rn(rs, xj.z));
    }
    // the flux of neighbour mass split mj under weight W
    __device__ __forceinline__ void add_w(float2 mj, float W, bool accept = true) {
        const float dm = __fadd_rn(__fsub_rn(mj.x, ms.x), __fsub_rn(mj.y, ms.y));
        // a rejected candidate (and the self pair) adds an exact zero
        neumaier_add(acc, comp, accept ? __fmul_rn(dm, W) : 0.0f);
    }
    __device__ __forceinline__ void add(const float4& xj, float K, bool accept = true) {
        add_w(make_float2(xj.x, xj.y), weight(xj, K), accept);
    }
    // two binary64 additions per particle: acc + comp is exact in binary64
    __device__ __forceinline__ double delta() const {
        return __dadd_rn(f32_to_f64(acc), f32_to_f64(comp));
    }
};

// Pass 2 of one particle by search, as pass 1 visited its candidates (the
// band's exact accepts last), for a particle whose list overflowed or when
// there are no lists.  A real call, so its registers do not weigh on the
// list loop.
template <int DIM, class View>
__device__ __noinline__ float2 search_flux(uint32_t s, int64_t stride,
                                           const double* __restrict__ pos,
                                           const float4* __restrict__ rec,
                                           const uint32_t* __restrict__ cell,
                                           const uint32_t* __restrict__ start, const View& v,
                                           const float4* __restrict__ ex, float rs, float2 ms,
                                           float two_beta) {
    const RealParams& P = v.of_sorted(s);
    const float na = -P.pp.a_log2e;
    FluxSum g{rs, two_beta, ms};
    scan_neighbours<DIM, true>(s, cell_arg<DIM>(cell, s), stride, rec, pos, start, P,
                         [&](uint32_t j, float d2f, bool accept) {
                             g.add(__ldg(ex + j), ex2_approx(na * d2f), accept);
                         });
    return make_float2(g.acc, g.comp);
}

// ---------------------------------------------------------------------------
// Bimolecular reaction A + B -> 0 (the extension Sec. 8 names; the model is
// this library's reading).  After the transfer of both species with the same
// weights, each particle reacts well mixed over dt: with concentrations
// C = N M / V the rate law dC_A/dt = dC_B/dt = -k C_A C_B is
// da/dt = db/dt = -kp a b on its masses, kp = k N / V, solved exactly over
// dt.  With `big` the larger of a and b, x = kp (big - small) dt,
// phi(x) = (1 - e^-x) / x (phi(0) = 1) and q = 1 + kp small dt phi(x):
//   big' = big / q,   small' = small e^-x / q
// (the closed form a(t) = D a / (a - b e^-kpDt), D = a - b, rearranged so
// that neither D -> 0 nor the species in deficit loses digits).  A particle
// with a negative mass of either species (sign bit set) does not react.
// ---------------------------------------------------------------------------

// The precision form's mass split of species B for its pass 2: the binary32
// head/tail of mass_b[s] (species A's is in the particle record ex).
__global__ void __launch_bounds__(kBlock)
k_split_mass(int n, const double* __restrict__ mass_b, float2* __restrict__ exb) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float hi, lo;
    split_double(mass_b[s], &hi, &lo);
    exb[s] = make_float2(hi, lo);
}

// F64: binary64 throughout (exp, expm1 and IEEE division).  Otherwise (the
// precision form) the two factors 1/q and e^-x / q in binary32 from the
// binary32 heads of the masses (kpdt_f = kp dt rounded to binary32), each
// applied to its binary64 mass with one binary64 multiply.
template <bool F64>
__device__ __forceinline__ void react_masses(double& ma, double& mb, double kp, double dt,
                                             float kpdt_f) {
    const double a = ma, b = mb;
    const long long ka = __double_as_longlong(a), kb = __double_as_longlong(b);
    if ((ka | kb) < 0) return;                       // a negative mass: no reaction
    const bool a_big = ka >= kb;                     // non-negative values order by their bits
    const double big = a_big ? a : b, small = a_big ? b : a;
    double nbig, nsmall;
    if constexpr (F64) {
        const double x = __dmul_rn(__dmul_rn(kp, __dsub_rn(big, small)), dt);
        const double phi = x > 0.0 ? -expm1(-x) / x : 1.0;
        const double q = __dadd_rn(1.0, __dmul_rn(__dmul_rn(__dmul_rn(kp, small), dt), phi));
        nbig = big / q;
        nsmall = __dmul_rn(small, exp(-x)) / q;
    } else {
        float bh, bl, sh, sl;
        split_double(big, &bh, &bl);
        split_double(small, &sh, &sl);
        const float x = __fmul_rn(kpdt_f, __fsub_rn(bh, sh));
        const float phi = x > 0.0f ? __fdiv_rn(-expm1f(-x), x) : 1.0f;
        const float rq = __frcp_rn(__fmaf_rn(__fmul_rn(kpdt_f, sh), phi, 1.0f));
        nbig = __dmul_rn(big, f32_to_f64(rq));
        nsmall = __dmul_rn(small, f32_to_f64(__fmul_rn(expf(-x), rq)));
    }
    ma = a_big ? nbig : nsmall;
    mb = a_big ? nsmall : nbig;
}

template <bool F64>
__global__ void __launch_bounds__(kBlock)
k_react(int n, double* __restrict__ ma, double* __restrict__ mb, double kp, double dt,
        float kpdt_f) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double a = ma[s], b = mb[s];
    react_masses<F64>(a, b, kp, dt, kpdt_f);
    ma[s] = a;
    mb[s] = b;
}

// As search_flux, for both species of a reaction run (species B's mass split
// in exb): {acc_A, comp_A, acc_B, comp_B}.
template <int DIM, class View>
__device__ __noinline__ float4 search_flux2(uint32_t s, int64_t stride,
                                            const double* __restrict__ pos,
                                            const float4* __restrict__ rec,
                                            const uint32_t* __restrict__ cell,
                                            const uint32_t* __restrict__ start, const View& v,
                                            const float4* __restrict__ ex,
                                            const float2* __restrict__ exb, float rs, float2 ms,
                                            float2 msb, float two_beta) {
    const RealParams& P = v.of_sorted(s);
    const float na = -P.pp.a_log2e;
    FluxSum a{rs, two_beta, ms}, b{rs, two_beta, msb};
    scan_neighbours<DIM, true>(s, cell_arg<DIM>(cell, s), stride, rec, pos, start, P,
                         [&](uint32_t j, float d2f, bool accept) {
                             const float4 xj = __ldg(ex + j);
                             const float W = a.weight(xj, ex2_approx(na * d2f));
                             a.add_w(make_float2(xj.x, xj.y), W, accept);
                             b.add_w(__ldg(exb + j), W, accept);
                         });
    return make_float4(a.acc, a.comp, b.acc, b.comp);
}

// Pass 2, precision form: each particle walks its neighbour list (the
// accepted neighbours only, with pass 1's K), two entries at a time so two
// gathers are in flight, or searches when it has none (no lists, or an
// overflowing one).  Both add the same terms in the same order.
template <int DIM, class View, int BLOCK, bool TWO = false, int WALK = 0>
__global__ void __launch_bounds__(BLOCK, 2048 / BLOCK)
k_exchange_f32(int n, int64_t stride, const double* __restrict__ pos, const float4* __restrict__ rec,
               const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
               const __grid_constant__ View v, const float4* __restrict__ ex,
               const double* __restrict__ mass, double* __restrict__ mass_out, NbList32 nb,
               const float2* __restrict__ exb = nullptr, const double* __restrict__ mass_b = nullptr,
               double* __restrict__ mass_b_out = nullptr, double kp = 0.0, double dt = 0.0,
               float kpdt_f = 0.0f, const WalkAhead wa = WalkAhead{}) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const RealParams& P = v.of_sorted(uint32_t(s));
    if (!P.transfer) {
        if constexpr (TWO) {
            double a = mass[s], b = mass_b[s];
            react_masses<false>(a, b, kp, dt, kpdt_f);
            mass_out[s] = a;
            mass_b_out[s] = b;
        } else {
            mass_out[s] = mass[s];
        }
        if constexpr (WALK > 0) walk_ahead<DIM, WALK>(P, s, stride, pos, wa);
        return;
    }
    const float4 xs = ex[s];
    FluxSum f{xs.z, float(2.0 * P.pp.beta), make_float2(xs.x, xs.y)};   // beta folded into W
    FluxSum g{xs.z, f.two_beta, TWO ? __ldg(exb + s) : make_float2(0.0f, 0.0f)};
    const uint32_t listed = nb.cap > 0 ? __float_as_uint(xs.w) : 0xffffffffu;
    if (listed <= uint32_t(nb.cap)) {
        const uint2* e = nb.e + s;
        uint32_t k = 0;
        if constexpr (TWO) {
            for (; k + 2 <= listed; k += 2, e += 2 * stride) {
                const uint2 q0 = __ldg(e), q1 = __ldg(e + stride);
                const float4 x0 = __ldg(ex + q0.x), x1 = __ldg(ex + q1.x);
                const float2 b0 = __ldg(exb + q0.x), b1 = __ldg(exb + q1.x);
                const float w0 = f.weight(x0, __uint_as_float(q0.y));
                f.add_w(make_float2(x0.x, x0.y), w0);
                g.add_w(b0, w0);
                const float w1 = f.weight(x1, __uint_as_float(q1.y));
                f.add_w(make_float2(x1.x, x1.y), w1);
                g.add_w(b1, w1);
            }
            if (k < listed) {
                const uint2 q = __ldg(e);
                const float4 x = __ldg(ex + q.x);
                const float w = f.weight(x, __uint_as_float(q.y));
                f.add_w(make_float2(x.x, x.y), w);
                g.add_w(__ldg(exb + q.x), w);
            }
        } else {
            // two entries per iteration, the next two list entries loaded
            // while this pair's neighbour records are in flight
            uint2 p0 = listed > 0u ? __ldg(e) : make_uint2(uint32_t(s), 0u);
            uint2 p1 = listed > 1u ? __ldg(e + stride) : p0;
            for (; k + 2 <= listed; k += 2, e += 2 * stride) {
                const uint2 q0 = p0, q1 = p1;
                const float4 x0 = __ldg(ex + q0.x), x1 = __ldg(ex + q1.x);
                p0 = k + 2 < listed ? __ldg(e + 2 * stride) : q0;
                p1 = k + 3 < listed ? __ldg(e + 3 * stride) : q1;
                f.add(x0, __uint_as_float(q0.y));
                f.add(x1, __uint_as_float(q1.y));
            }
            if (k < listed) f.add(__ldg(ex + p0.x), __uint_as_float(p0.y));   // p0 = entry k
        }
    } else if constexpr (TWO) {
        const float4 sum = search_flux2<DIM>(uint32_t(s), stride, pos, rec, cell, start, v, ex, exb,
                                             f.rs, f.ms, g.ms, f.two_beta);
        f.acc = sum.x;
        f.comp = sum.y;
        g.acc = sum.z;
        g.comp = sum.w;
    } else {
        const float2 sum = search_flux<DIM>(uint32_t(s), stride, pos, rec, cell, start, v, ex,
                                            f.rs, f.ms, f.two_beta);
        f.acc = sum.x;
        f.comp = sum.y;
    }
    if constexpr (TWO) {
        // both species' transfer, then the reaction on this particle
        double a = __dadd_rn(mass[s], f.delta()), b = __dadd_rn(mass_b[s], g.delta());
        react_masses<false>(a, b, kp, dt, kpdt_f);
        mass_out[s] = a;
        mass_b_out[s] = b;
    } else {
        mass_out[s] = __dadd_rn(mass[s], f.delta());
    }
    if constexpr (WALK > 0) walk_ahead<DIM, WALK>(P, s, stride, pos, wa);
}

// Test support: every accepted ordered pair j != s as (id_s, id_j).
template <int DIM, class View>
__global__ void __launch_bounds__(kBlock)
k_emit_pairs(int n, int64_t stride, const double* __restrict__ pos, const float4* __restrict__ rec,
             const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
             const uint32_t* __restrict__ id, const __grid_constant__ View v,
             unsigned long long cap, unsigned long long* __restrict__ counter,
             uint32_t* __restrict__ out_i, uint32_t* __restrict__ out_j) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const RealParams& P = v.of_sorted(uint32_t(s));
    if (!P.transfer) return;
    const uint32_t ids = id[s];
    visit_neighbours<DIM>(uint32_t(s), cell_arg<DIM>(cell, s), stride, rec, pos, start, P,
                          [&](uint32_t j, float, const float4&) {
                              if (j == uint32_t(s)) return;
                              const unsigned long long k = atomicAdd(counter, 1ull);
                              if (k < cap) {
                                  out_i[k] = ids;
                                  out_j[k] = id[j];
                              }
                          });
}

// ---------------------------------------------------------------------------
// Adjoint of the step (binary64).  The mass update is M' = A M with
// A = I + beta (W - diag(W 1)) symmetric, so the mass adjoint is
// lambda_t = A lambda_{t+1}, the same pair sum with lambda in place of M.  The
// derivative with respect to D follows the positions' pathwise tangents
// (tan = dX/dD) and h^2 = 2 D_MT dt / beta (dh^2/dD = h^2 / D):
//   dK_ij/dD = K_ij (-(x_i - x_j).(t_i - t_j) + d2_ij / (2 D)) / h^2,
//   dr_i = sum_j dK_ij,
//   dW_ij = 2 dK_ij / (r_i + r_j) - 2 K_ij (dr_i + dr_j) / (r_i + r_j)^2,
// and step t adds beta sum_i lambda_{t+1,i} sum_j dW_ij (M_j - M_i) to dL/dD.
// Pair-set and bin changes contribute zero almost everywhere.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ void pair_terms(const double* __restrict__ pos,
                                           const double* __restrict__ tan, int64_t stride,
                                           uint32_t s, uint32_t j, const RealParams& P,
                                           const double* table, double* K, double* dK) {
    double d2 = 0.0, dot = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double d = __dsub_rn(__ldg(pos + a * stride + s), __ldg(pos + a * stride + j));
        const double dt = __dsub_rn(__ldg(tan + a * stride + s), __ldg(tan + a * stride + j));
        d2 = (a == 0) ? __dmul_rn(d, d) : __fma_rn(d, d, d2);   // as kernel_d2
        dot = __fma_rn(d, dt, dot);
    }
    *K = gauss_exp(d2, table, P.pp.ec);
    *dK = __dmul_rn(*K, __dmul_rn(__fma_rn(d2, P.inv_2D, -dot), P.inv_h2));
}

// The adjoint passes run on the segment engine with two binary64 terms per
// pair (smaller segments: two values per entry).
constexpr int kAdjSeg = 8;

// Pass A: r_s = sum_j K_sj (self included) and dr_s = sum_j dK_sj / dD.
template <int DIM, class View>
__global__ void __launch_bounds__(kBlock)
k_adj_rowsum(int n, int64_t stride, const double* __restrict__ pos, const double* __restrict__ tan,
             const float4* __restrict__ rec, const uint32_t* __restrict__ cell,
             const uint32_t* __restrict__ start, const double* __restrict__ exp_table,
             const __grid_constant__ View v, double* __restrict__ r_out,
             double* __restrict__ dr_out, NbList<double2> nb) {
    __shared__ double table[kExpTable];
    __shared__ SegShared<kWarpsPerBlock, double2, false, kAdjSeg> seg;
    for (int t = threadIdx.x; t < kExpTable; t += blockDim.x) table[t] = exp_table[t];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const RealParams& P = v.of_sorted(uint32_t(s < n ? s : 0));
    const bool valid = s < n && P.transfer;
    double r = 1.0, dr = 0.0;
    const uint32_t cnt = seg_pairs<DIM>(
        valid, uint32_t(s), stride, rec, pos, cell, start, P, seg,
        [&](uint32_t so, uint32_t j, float) {
            double K, dK;
            pair_terms<DIM>(pos, tan, stride, so, j, v.of_sorted(so), table, &K, &dK);
            return make_double2(K, dK);
        },
        [&](double2 t) {
            r = __dadd_rn(r, t.x);
            dr = __dadd_rn(dr, t.y);
        }, nb);
    if (s < n) {
        r_out[s] = r;
        dr_out[s] = dr;
        if (nb.cap > 0) nb.count[s] = valid ? cnt : 0u;
    }
}

// Pass B: lambda_t,s = lambda_s + beta sum_j W_sj (lambda_j - lambda_s) and the
// step's D-gradient term g_s = beta lambda_s sum_j dW_sj (M_j - M_s), with M the
// masses entering the step.
template <int DIM, class View>
__global__ void __launch_bounds__(kBlock)
k_adj_exchange(int n, int64_t stride, const double* __restrict__ pos,
               const double* __restrict__ tan, const float4* __restrict__ rec,
               const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
               const double* __restrict__ exp_table, const __grid_constant__ View v,
               const double* __restrict__ r, const double* __restrict__ dr,
               const double* __restrict__ mass, const double* __restrict__ lam,
               double* __restrict__ lam_out, double* __restrict__ gD, NbList<double2> nb) {
    __shared__ double table[kExpTable];
    __shared__ SegShared<kWarpsPerBlock, double2, false, kAdjSeg> seg;
    for (int t = threadIdx.x; t < kExpTable; t += blockDim.x) table[t] = exp_table[t];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const RealParams& P = v.of_sorted(uint32_t(s < n ? s : 0));
    const bool valid = s < n && P.transfer;
    double lacc = 0.0, gacc = 0.0;
    auto terms = [&](uint32_t so, uint32_t j, double K, double dK) {
        const double inv = quot_pos(1.0, __dadd_rn(__ldg(r + so), __ldg(r + j)));
        const double W = __dmul_rn(__dmul_rn(2.0, K), inv);
        const double dW = __dmul_rn(
            __dmul_rn(2.0, inv),
            __fma_rn(-__dmul_rn(K, inv), __dadd_rn(__ldg(dr + so), __ldg(dr + j)), dK));
        return make_double2(__dmul_rn(W, __dsub_rn(__ldg(lam + j), __ldg(lam + so))),
                            __dmul_rn(dW, __dsub_rn(__ldg(mass + j), __ldg(mass + so))));
    };
    auto add = [&](double2 t) {
        lacc = __dadd_rn(lacc, t.x);
        gacc = __dadd_rn(gacc, t.y);
    };
    const uint32_t listed = (nb.cap > 0 && valid) ? nb.count[s] : 0u;
    const bool fits = nb.cap > 0 && __all_sync(0xffffffffu, listed <= uint32_t(nb.cap));
    if (fits) {
        dense_listed(valid, uint32_t(s), stride, listed, nb, seg,
                     [&](uint32_t so, uint32_t j, double2 kd) { return terms(so, j, kd.x, kd.y); },
                     add);
    } else {
        seg_pairs<DIM>(
            valid, uint32_t(s), stride, rec, pos, cell, start, P, seg,
            [&](uint32_t so, uint32_t j, float) {
                double K, dK;
                pair_terms<DIM>(pos, tan, stride, so, j, v.of_sorted(so), table, &K, &dK);
                return terms(so, j, K, dK);
            },
            add);
    }
    if (s < n) {
        const double ls = lam[s];
        lam_out[s] = valid ? __fma_rn(P.pp.beta, lacc, ls) : ls;
        gD[s] = valid ? __dmul_rn(__dmul_rn(P.pp.beta, ls), gacc) : 0.0;
    }
}

// Deterministic sum of x[0..n): fixed-size blocks reduce their slice in a fixed
// tree, then one block adds the block sums in index order to *acc.
constexpr int kReduceThreads = 512;

__global__ void __launch_bounds__(kReduceThreads)
k_block_sums(int n, const double* __restrict__ x, double* __restrict__ partial) {
    __shared__ double buf[kReduceThreads];
    const int i = blockIdx.x * kReduceThreads + threadIdx.x;
    buf[threadIdx.x] = i < n ? x[i] : 0.0;
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) buf[threadIdx.x] = __dadd_rn(buf[threadIdx.x], buf[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = buf[0];
}

// One block: thread t adds partial[t], partial[t + T], ... in order, then a
// fixed tree over the threads; the result is added to *acc.
__global__ void __launch_bounds__(kReduceThreads)
k_sum_into(int nparts, const double* __restrict__ partial, double* __restrict__ acc) {
    __shared__ double buf[kReduceThreads];
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += kReduceThreads) s = __dadd_rn(s, partial[k]);
    buf[threadIdx.x] = s;
    __syncthreads();
    for (int w = kReduceThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) buf[threadIdx.x] = __dadd_rn(buf[threadIdx.x], buf[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *acc = __dadd_rn(*acc, buf[0]);
}

// Input-order <-> cell-order moves of a per-particle binary64 array.
__global__ void k_take_by_id(int n, const uint32_t* __restrict__ id, const double* __restrict__ src,
                             double* __restrict__ dst) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) dst[s] = src[id[s]];
}
__global__ void k_put_by_id(int n, const uint32_t* __restrict__ id, const double* __restrict__ src,
                            double* __restrict__ dst) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) dst[id[s]] = src[s];
}

// Row sums in input order and in the paper's units:
// out[id[s]] = r_s * kernel_norm of the particle's realisation.
template <typename T, class View>
__global__ void k_row_sums_out(int n, const uint32_t* __restrict__ id, const T* __restrict__ src,
                               int src_step, const __grid_constant__ View v,
                               double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const RealParams& P = v.of_sorted(uint32_t(s));
    out[id[s]] = __dmul_rn(double(src[int64_t(s) * src_step]), P.kernel_norm);
}

// Outputs in input order: out[a * n + id[s]] = src[a * stride + s] * scale
// (binary32 sources widened exactly by integer operations; no multiply when
// scale is 1).
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return f32_to_f64(x); }

template <typename T>
__global__ void k_unpermute(int n, int64_t stride, int naxes, const uint32_t* __restrict__ id,
                            const T* __restrict__ src, int src_step, double scale,
                            double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t k = id[s];
    if (!check(k < uint32_t(n), kChkOutput)) return;
    for (int a = 0; a < naxes; ++a) {
        const double x = widen(src[(a * stride + s) * src_step]);
        out[int64_t(a) * n + k] = scale == 1.0 ? x : __dmul_rn(x, scale);
    }
}

}  // namespace mtpt
