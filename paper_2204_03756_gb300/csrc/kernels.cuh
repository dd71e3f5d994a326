// kernels.cuh -- CUDA kernels of one MTPT time step (Sec. 3) for sm_103a.
//
// Data layout (structure of arrays, `stride` = capacity >= n):
//   pos[a * stride + s]  binary64 coordinates, particles in cell order
//   mass[s], id[s]       binary64 mass, uint32 input index (keys the walk)
//   cell[s]              linear cell index of particle s
//   xl[a * stride + s]   binary32 offset of the particle from its cell's
//                        lower corner (the pair loop's prefilter operand)
//   start[c]             first particle of cell c (exclusive prefix sum)
// Cells are row-major (x fastest), so the three cells (cx-1..cx+1) of one
// neighbour row are one contiguous particle range.
#pragma once
#include <cstdint>

#include "expneg.cuh"
#include "rng.cuh"

namespace mtpt {

enum : uint32_t { kStatusNonFinite = 1u, kStatusOutOfDomain = 2u };

constexpr int kBlock = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 4 * kScanThreads;   // cells per scan block

struct Box {
    double lo[3], hi[3];
};

struct Grid {
    int n[3];          // cells per axis (1 on unused axes)
    double lo[3];      // lower corner of the box
    double w[3];       // cell width per axis, >= psi
    double inv_w[3];   // 1 / w
    float wf[3];       // w rounded to binary32
};

struct PairParams {
    double psi2;       // cutoff squared: the exact binary64 test d2 <= psi2
    float band_lo;     // binary32 d2 below this: certainly a neighbour
    float band_hi;     // binary32 d2 above this: certainly not a neighbour
    double a;          // 1 / (2 h^2)
    float a_log2e;     // a * log2(e) in binary32 (precision form)
    double beta;
    ExpNegConsts ec;
};

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

template <int DIM>
__device__ __forceinline__ uint32_t cell_of(const double* x, const Grid& g, bool* bad) {
    uint32_t lin = 0, mult = 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double u = __dmul_rn(__dsub_rn(x[a], g.lo[a]), g.inv_w[a]);
        int c = 0;
        if (u == u) {                       // not NaN
            c = u <= 0.0 ? 0 : (u >= double(g.n[a] - 1) ? g.n[a] - 1 : __double2int_rz(u));
        } else {
            *bad = true;
        }
        lin += uint32_t(c) * mult;
        mult *= uint32_t(g.n[a]);
    }
    return lin;
}

template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_walk_key(int n, int64_t stride, double* __restrict__ pos, const uint32_t* __restrict__ id,
           uint64_t seed, uint64_t step, double sigma, int do_walk, int do_key, Box box, Grid g,
           uint32_t* __restrict__ key, uint32_t* __restrict__ count, uint32_t* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = pos[a * stride + i];
    if (do_walk) {
        const float4 z4 = normals4(seed, id[i], step);
        const float z[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double v = __dadd_rn(x[a], __dmul_rn(sigma, double(z[a])));
            x[a] = reflect(v, box.lo[a], box.hi[a]);
            pos[a * stride + i] = x[a];
        }
    }
    if (do_key) {
        bool bad = false;
        const uint32_t c = cell_of<DIM>(x, g, &bad);
        if (bad) atomicOr(status, kStatusNonFinite);
        key[i] = c;
        atomicAdd(&count[c], 1u);
    }
}

// Domain check of positions loaded from device memory.
template <int DIM>
__global__ void k_check_domain(int n, int64_t stride, const double* __restrict__ pos, Box box,
                               uint32_t* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double x = pos[a * stride + i];
        if (!(x >= box.lo[a] && x <= box.hi[a])) atomicOr(status, kStatusOutOfDomain);
    }
}

__global__ void k_iota(int n, uint32_t* __restrict__ id) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = uint32_t(i);
}

// ---------------------------------------------------------------------------
// Step 2a: exclusive prefix sum of the cell counts (three launches:
// per-tile sums, scan of the tile sums, per-tile scan plus offset).  The
// count array is padded with zeros to whole tiles, so start[n_cells] = n.
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

__global__ void __launch_bounds__(kScanThreads)
k_scan_tile_sums(const uint4* __restrict__ count4, uint32_t* __restrict__ tile_sums) {
    const uint4 v = count4[size_t(blockIdx.x) * kScanThreads + threadIdx.x];
    uint32_t total;
    block_exclusive_scan(v.x + v.y + v.z + v.w, &total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tile_offsets(uint32_t* __restrict__ tile_sums, int ntiles) {
    uint32_t carry = 0;
    for (int base = 0; base < ntiles; base += kScanThreads) {
        const int t = base + threadIdx.x;
        const uint32_t v = t < ntiles ? tile_sums[t] : 0u;
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(v, &total);
        if (t < ntiles) tile_sums[t] = carry + excl;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const uint4* __restrict__ count4, const uint32_t* __restrict__ tile_offsets,
             uint4* __restrict__ start4) {
    const size_t k = size_t(blockIdx.x) * kScanThreads + threadIdx.x;
    const uint4 v = count4[k];
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(v.x + v.y + v.z + v.w, &total) + tile_offsets[blockIdx.x];
    start4[k] = make_uint4(excl, excl + v.x, excl + v.x + v.y, excl + v.x + v.y + v.z);
}

// ---------------------------------------------------------------------------
// Step 2b: counting-sort scatter.  Each particle takes a slot of its cell;
// decrementing the count returns every count to zero for the next step.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock)
k_scatter(int n, const uint32_t* __restrict__ key, const uint32_t* __restrict__ start,
          uint32_t* __restrict__ count, uint32_t* __restrict__ perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t c = key[i];
    const uint32_t slot = start[c] + atomicSub(&count[c], 1u) - 1u;
    perm[slot] = uint32_t(i);
}

// Step 2c: gather into cell order.  The slot order the atomics gave inside a
// cell is replaced by the rank of the particle id, so the layout (and every
// sum over it) is identical run to run.  Also writes the particle's cell, the
// binary32 offset from the cell corner and (precision form) the mass split
// into a binary32 head and tail.
template <int DIM, bool SPLIT_MASS>
__global__ void __launch_bounds__(kBlock)
k_gather(int n, int64_t stride, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ key,
         const uint32_t* __restrict__ start, const uint32_t* __restrict__ id_in,
         const double* __restrict__ pos_in, const double* __restrict__ mass_in,
         uint32_t* __restrict__ id_out, double* __restrict__ pos_out, double* __restrict__ mass_out,
         uint32_t* __restrict__ cell_out, float* __restrict__ xl_out, float2* __restrict__ msplit_out,
         Grid g) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t src = perm[s];
    const uint32_t c = key[src];
    const uint32_t b = start[c], e = start[c + 1];
    const uint32_t my_id = id_in[src];
    uint32_t rank = 0;
    for (uint32_t k = b; k < e; ++k) rank += (id_in[perm[k]] < my_id) ? 1u : 0u;
    const uint32_t dst = b + rank;
    id_out[dst] = my_id;
    cell_out[dst] = c;
    const double m = mass_in[src];
    mass_out[dst] = m;
    if (SPLIT_MASS) {
        const float hi = __double2float_rn(m);
        const float lo = __double2float_rn(__dsub_rn(m, double(hi)));
        msplit_out[dst] = make_float2(hi, lo);
    }
    uint32_t rest = c;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const uint32_t ca = rest % uint32_t(g.n[a]);
        rest /= uint32_t(g.n[a]);
        const double x = pos_in[a * stride + src];
        pos_out[a * stride + dst] = x;
        const double corner = __dadd_rn(g.lo[a], __dmul_rn(double(ca), g.w[a]));
        xl_out[a * stride + dst] = __double2float_rn(__dsub_rn(x, corner));
    }
}

// ---------------------------------------------------------------------------
// Steps 2-5: neighbour visits.  For particle s (cell order) every particle j
// in the 3^DIM surrounding cells is a candidate.  The binary32 squared
// distance from the cell offsets decides every candidate outside a narrow
// band around psi^2; inside the band the exact binary64 test
// dx*dx + dy*dy (+ dz*dz) <= psi^2 (no fma, dx = x_i - x_j) decides.  The
// band half-width is set on the host from an error bound of the binary32
// evaluation, so the accepted set equals the exact binary64 pair set.
//
// The binary32 difference is always evaluated in the frame of the pair's
// lower index, so d2f(i, j) == d2f(j, i) bit for bit, and every quantity
// derived from it is symmetric in the pair.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double exact_d2(const double* __restrict__ pos, int64_t stride,
                                           const double* xi, uint32_t j) {
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const double d = __dsub_rn(xi[a], __ldg(pos + a * stride + j));
        const double sq = __dmul_rn(d, d);
        d2 = (a == 0) ? sq : __dadd_rn(d2, sq);
    }
    return d2;
}

template <int DIM, class Visit>
__device__ __forceinline__ void visit_neighbours(uint32_t s, uint32_t cell, int64_t stride,
                                                 const float* __restrict__ xl,
                                                 const double* __restrict__ pos, const double* xi,
                                                 const uint32_t* __restrict__ start, const Grid& g,
                                                 const PairParams& pp, Visit&& visit) {
    int c[3] = {0, 0, 0};
    {
        uint32_t rest = cell;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            c[a] = int(rest % uint32_t(g.n[a]));
            rest /= uint32_t(g.n[a]);
        }
    }
    float xs[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xs[a] = xl[a * stride + s];
    const int xlo = c[0] > 0 ? c[0] - 1 : 0;
    const int xhi = c[0] < g.n[0] - 1 ? c[0] + 1 : c[0];
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
    const int ylo = DIM >= 2 ? -1 : 0, yhi = DIM >= 2 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        const int zz = c[2] + dz;
        if (DIM == 3 && (zz < 0 || zz >= g.n[2])) continue;
        for (int dy = ylo; dy <= yhi; ++dy) {
            const int yy = c[1] + dy;
            if (DIM >= 2 && (yy < 0 || yy >= g.n[1])) continue;
            const uint32_t row = (uint32_t(zz) * uint32_t(g.n[1]) + uint32_t(yy)) * uint32_t(g.n[0]);
            const uint32_t j0 = __ldg(start + row + xlo);
            const uint32_t b1 = __ldg(start + row + c[0]);
            const uint32_t b2 = __ldg(start + row + c[0] + 1);
            const uint32_t j3 = __ldg(start + row + xhi + 1);
            const float sh[3] = {0.0f, DIM >= 2 ? float(dy) * g.wf[1] : 0.0f,
                                 DIM == 3 ? float(dz) * g.wf[2] : 0.0f};
            for (uint32_t j = j0; j < j3; ++j) {
                if (j == s) continue;
                const bool fwd = s < j;
                float d2f = 0.0f;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    const float xj = __ldg(xl + a * stride + j);
                    float shift = a == 0 ? (j < b1 ? -g.wf[0] : (j < b2 ? 0.0f : g.wf[0])) : sh[a];
                    const float p = fwd ? xj : xs[a];
                    const float q = fwd ? xs[a] : xj;
                    shift = fwd ? shift : -shift;
                    const float d = __fsub_rn(__fadd_rn(p, shift), q);
                    const float sq = __fmul_rn(d, d);
                    d2f = (a == 0) ? sq : __fadd_rn(d2f, sq);
                }
                if (d2f > pp.band_hi) continue;
                if (d2f >= pp.band_lo && exact_d2<DIM>(pos, stride, xi, j) > pp.psi2) continue;
                visit(j, d2f);
            }
        }
    }
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Compensated summation (Kahan-Babuska / Neumaier): s + c carries the sum to
// about twice binary32 precision.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
    const float t = __fadd_rn(s, x);
    const float big = fabsf(s) >= fabsf(x) ? s : x;
    const float small = fabsf(s) >= fabsf(x) ? x : s;
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(big, t), small));
    s = t;
}

__device__ __forceinline__ void add_pair_count(uint32_t cnt, unsigned long long* counter) {
    const uint32_t warp_total = __reduce_add_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && warp_total) atomicAdd(counter, (unsigned long long)warp_total);
}

// Pass 1, binary64 form: r_s = 1 + sum_j exp(-a d2_sj) (the kernel without its
// constant factor, which cancels in W), and the ordered pair count.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_rowsum_f64(int n, int64_t stride, const double* __restrict__ pos, const float* __restrict__ xl,
             const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
             const double* __restrict__ exp_table, Grid g, PairParams pp,
             double* __restrict__ r_out, unsigned long long* __restrict__ pair_counter) {
    __shared__ double table[64];
    if (threadIdx.x < 64) table[threadIdx.x] = exp_table[threadIdx.x];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cnt = 0;
    if (s < n) {
        double xi[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) xi[a] = pos[a * stride + s];
        double r = 1.0;
        visit_neighbours<DIM>(uint32_t(s), cell[s], stride, xl, pos, xi, start, g, pp,
                              [&](uint32_t j, float) {
                                  const double d2 = exact_d2<DIM>(pos, stride, xi, j);
                                  r = __dadd_rn(r, exp_neg(__dmul_rn(d2, pp.a), table, pp.ec));
                                  ++cnt;
                              });
        r_out[s] = r;
    }
    add_pair_count(cnt, pair_counter);
}

// Pass 2, binary64 form: M'_s = M_s + beta sum_j (M_j - M_s) 2 K_sj / (r_s + r_j).
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_exchange_f64(int n, int64_t stride, const double* __restrict__ pos, const float* __restrict__ xl,
               const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
               const double* __restrict__ exp_table, Grid g, PairParams pp,
               const double* __restrict__ r, const double* __restrict__ mass,
               double* __restrict__ mass_out) {
    __shared__ double table[64];
    if (threadIdx.x < 64) table[threadIdx.x] = exp_table[threadIdx.x];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double xi[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = pos[a * stride + s];
    const double rs = r[s], ms = mass[s];
    double acc = 0.0;
    visit_neighbours<DIM>(uint32_t(s), cell[s], stride, xl, pos, xi, start, g, pp,
                          [&](uint32_t j, float) {
                              const double d2 = exact_d2<DIM>(pos, stride, xi, j);
                              const double K = exp_neg(__dmul_rn(d2, pp.a), table, pp.ec);
                              const double W = __ddiv_rn(__dmul_rn(2.0, K), __dadd_rn(rs, __ldg(r + j)));
                              acc = __fma_rn(__dsub_rn(__ldg(mass + j), ms), W, acc);
                          });
    mass_out[s] = __dadd_rn(ms, __dmul_rn(pp.beta, acc));
}

// Pass 1, precision form: binary32 kernel exp2(-a log2(e) d2f) with the
// hardware ex2, compensated binary32 row sum, rounded to binary32.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_rowsum_f32(int n, int64_t stride, const double* __restrict__ pos, const float* __restrict__ xl,
             const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start, Grid g,
             PairParams pp, float* __restrict__ r_out, unsigned long long* __restrict__ pair_counter) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cnt = 0;
    if (s < n) {
        double xi[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) xi[a] = pos[a * stride + s];
        float rsum = 1.0f, rc = 0.0f;
        visit_neighbours<DIM>(uint32_t(s), cell[s], stride, xl, pos, xi, start, g, pp,
                              [&](uint32_t, float d2f) {
                                  const float K = ex2_approx(-pp.a_log2e * d2f);
                                  const float t = __fadd_rn(rsum, K);   // rsum >= 1 >= K
                                  rc = __fadd_rn(rc, __fadd_rn(__fsub_rn(rsum, t), K));
                                  rsum = t;
                                  ++cnt;
                              });
        r_out[s] = __fadd_rn(rsum, rc);
    }
    add_pair_count(cnt, pair_counter);
}

// Pass 2, precision form: W = 2K / (r_s + r_j) in binary32 (symmetric bit for
// bit), mass difference from the binary32 head/tail split (exactly
// antisymmetric), flux accumulated with compensation, update in binary64.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_exchange_f32(int n, int64_t stride, const double* __restrict__ pos, const float* __restrict__ xl,
               const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start, Grid g,
               PairParams pp, const float* __restrict__ r, const float2* __restrict__ msplit,
               const double* __restrict__ mass, double* __restrict__ mass_out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double xi[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = pos[a * stride + s];
    const float rs = r[s];
    const float2 ms = msplit[s];
    float acc = 0.0f, comp = 0.0f;
    visit_neighbours<DIM>(uint32_t(s), cell[s], stride, xl, pos, xi, start, g, pp,
                          [&](uint32_t j, float d2f) {
                              const float K = ex2_approx(-pp.a_log2e * d2f);
                              const float W = __fdividef(2.0f * K, __fadd_rn(rs, __ldg(r + j)));
                              const float2 mj = __ldg(msplit + j);
                              const float dm = __fadd_rn(__fsub_rn(mj.x, ms.x), __fsub_rn(mj.y, ms.y));
                              comp_add(acc, comp, __fmul_rn(dm, W));
                          });
    const double delta = __dadd_rn(double(acc), double(comp));
    mass_out[s] = __dadd_rn(mass[s], __dmul_rn(pp.beta, delta));
}

// Test support: every accepted ordered pair as (id_s, id_j).
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_emit_pairs(int n, int64_t stride, const double* __restrict__ pos, const float* __restrict__ xl,
             const uint32_t* __restrict__ cell, const uint32_t* __restrict__ start,
             const uint32_t* __restrict__ id, Grid g, PairParams pp, unsigned long long cap,
             unsigned long long* __restrict__ counter, uint32_t* __restrict__ out_i,
             uint32_t* __restrict__ out_j) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double xi[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = pos[a * stride + s];
    const uint32_t ids = id[s];
    visit_neighbours<DIM>(uint32_t(s), cell[s], stride, xl, pos, xi, start, g, pp,
                          [&](uint32_t j, float) {
                              const unsigned long long k = atomicAdd(counter, 1ull);
                              if (k < cap) {
                                  out_i[k] = ids;
                                  out_j[k] = id[j];
                              }
                          });
}

// Outputs in input order: out[a * n + id[s]] = src[a * stride + s].
template <typename T>
__global__ void k_unpermute(int n, int64_t stride, int naxes, const uint32_t* __restrict__ id,
                            const T* __restrict__ src, double scale, double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t k = id[s];
    for (int a = 0; a < naxes; ++a)
        out[int64_t(a) * n + k] = __dmul_rn(double(src[a * stride + s]), scale);
}

}  // namespace mtpt
