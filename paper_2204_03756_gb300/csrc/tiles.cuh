// tiles.cuh -- kernels of the split domain (one tile of a checkerboard per
// handle), Secs. 4-5 of the paper.
//
// The global box is cut into tiles per axis (Sec. 4.2, the factors chosen by
// Eq. "minimization"); a particle belongs to ("is native to") the tile that
// contains it.  For the mass transfer each tile also holds ghost copies of the
// particles of other tiles that lie within a pad around its own box (Sec. 5).
// The pad here is 2 psi wide, not psi: a ghost within psi of the tile then
// has all of its own neighbours in the tile's set, so its row sum -- which
// enters the weights W_ij of the natives it touches -- is the single-domain
// one, and the natives' updates equal those of the undivided run.  Ghosts
// are flagged by bit 31 of their generator id and dropped after the
// transfer; only natives walk and only natives' masses are kept (Sec. 5).
//
// One step of a tile: walk the natives; pack every particle for each other
// tile that owns it or holds it in its pad (records of dim + 2 binary64
// values: the coordinates, the mass, the global id); the caller exchanges
// the packed records between tiles; assemble kept and received particles,
// natives and ghosts; run the transfer; keep the natives.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace mtpt {

enum : uint32_t { kTileErrForeign = 1u, kTileErrId = 2u, kTileErrMass = 4u };

// Checkerboard geometry, identical on every tile.  Along axis a the tile
// edges are e_t = lo_a + t width_a (binary64, t = 0..f_a, formed on the
// host); a coordinate x lies in tile t when e_t <= x < e_(t+1) (the first tile
// also holds x below e_1, the last one x from e_(f-1) on), and the tile below
// (above) holds it in its pad when x <= e_t + pad (x >= e_(t+1) - pad).  All
// three are compared through the int64 order keys of the binary64 values
// (integer instructions only); a binary32 estimate of t starts the search.
struct TileGeom {
    int f[3];                      // tiles per axis (1 on unused axes)
    int self;                      // this tile: t0 + f0 (t1 + f1 t2)
    float lo_f[3], inv_w_f[3];     // binary32 lo and 1 / width (the estimate)
    const long long* edge[3];      // order keys of e_t, t = 0..f
    const long long* near_lo[3];   // order keys of e_t + pad, t = 0..f-1
    const long long* near_hi[3];   // order keys of e_(t+1) - pad, t = 0..f-1
};

// Tile coordinate along axis a.
__device__ __forceinline__ int tile_axis(double x, long long k, const TileGeom& T, int a) {
    const int top = T.f[a] - 1;
    if (top == 0) return 0;
    float xh, xl;
    split_double(x, &xh, &xl);
    const float u = __fmul_rn(__fsub_rn(xh, T.lo_f[a]), T.inv_w_f[a]);
    int t = u >= 1.0f ? (u >= float(top) ? top : int(u)) : 0;
    // the estimate is within a tile of the answer; bounded steps regardless
    for (int it = 0; it <= top && t > 0 && k < __ldg(T.edge[a] + t); ++it) --t;
    for (int it = 0; it <= top && t < top && k >= __ldg(T.edge[a] + t + 1); ++it) ++t;
    return t;
}

// Visits every tile that needs particle x: emit(tile, native) for the owner
// (native = true) and for each other tile whose pad contains x (native =
// false).  Tiles are at least a pad wide (checked on the host), so only the
// 3^DIM tiles around the owner qualify.  Returns the owner.
template <int DIM, class Emit>
__device__ __forceinline__ int for_each_dest(const double* x, const TileGeom& T, Emit&& emit) {
    int own[3] = {0, 0, 0};
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const long long k = order_key(x[a]);
        own[a] = tile_axis(x[a], k, T, a);
        lo[a] = (own[a] > 0 && k <= __ldg(T.near_lo[a] + own[a])) ? -1 : 0;
        hi[a] = (own[a] < T.f[a] - 1 && k >= __ldg(T.near_hi[a] + own[a])) ? 1 : 0;
    }
    const int owner = own[0] + T.f[0] * (own[1] + T.f[1] * own[2]);
    for (int dz = lo[2]; dz <= hi[2]; ++dz)
        for (int dy = lo[1]; dy <= hi[1]; ++dy)
            for (int dx = lo[0]; dx <= hi[0]; ++dx) {
                const int t = (own[0] + dx) + T.f[0] * ((own[1] + dy) + T.f[1] * (own[2] + dz));
                emit(t, t == owner);
            }
    return owner;
}

// Block-wide slot allocation for the common case, a particle that stays
// native to this tile: one shared-memory atomic per warp, one global atomic
// per block.  Every thread of the block calls it; returns the slot of a
// caller with `take`, counted from the start of the region.
__device__ __forceinline__ unsigned long long block_take(bool take,
                                                         unsigned long long* __restrict__ cursor) {
    __shared__ unsigned long long blk_count, blk_base;
    if (threadIdx.x == 0) blk_count = 0;
    __syncthreads();
    const unsigned m = __ballot_sync(0xffffffffu, take);
    const int lane = threadIdx.x & 31;
    unsigned long long warp_off = 0;
    if (lane == 0 && m) warp_off = atomicAdd(&blk_count, (unsigned long long)__popc(m));
    warp_off = __shfl_sync(0xffffffffu, warp_off, 0);
    __syncthreads();
    if (threadIdx.x == 0) blk_base = blk_count ? atomicAdd(cursor, blk_count) : 0ull;
    __syncthreads();
    return blk_base + warp_off + __popc(m & ((1u << lane) - 1u));
}

// Pass 1 of the pack: per destination tile the numbers of natives and ghosts
// (counts[2 t], counts[2 t + 1]); this tile's own entries count what it keeps.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_tile_count(int n, int64_t stride, const double* __restrict__ pos, const TileGeom T,
             unsigned long long* __restrict__ counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool stays = false;
    if (i < n) {
        double x[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) x[a] = pos[a * stride + i];
        for_each_dest<DIM>(x, T, [&](int t, bool native) {
            if (t == T.self && native) stays = true;
            else atomicAdd(&counts[2 * t + (native ? 0 : 1)], 1ull);
        });
    }
    block_take(stays, &counts[2 * T.self]);
}

// Pass 2: records of dim + 2 binary64 values (coordinates, mass, global id)
// into the send buffer (region of tile t from base[2 t] for its natives and
// base[2 t + 1] for its ghosts) or, for this tile, into the keep buffer
// (natives from base[2 self], ghosts from base[2 self + 1]).  cursor (2 per
// tile) starts at zero; the order inside a region is not defined.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_tile_scatter(int n, int64_t stride, const double* __restrict__ pos,
               const double* __restrict__ mass, const uint32_t* __restrict__ id, const TileGeom T,
               const unsigned long long* __restrict__ base, unsigned long long* __restrict__ cursor,
               double* __restrict__ send, double* __restrict__ keep) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int K = DIM + 2;
    double r[K];
    bool stays = false;
    if (i < n) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) r[a] = pos[a * stride + i];
        r[DIM] = mass[i];
        r[DIM + 1] = double(id[i] & ~kGhostBit);
        for_each_dest<DIM>(r, T, [&](int t, bool native) {
            if (t == T.self && native) {
                stays = true;
                return;
            }
            const int k = 2 * t + (native ? 0 : 1);
            const unsigned long long slot = base[k] + atomicAdd(&cursor[k], 1ull);
            double* dst = (t == T.self ? keep : send) + slot * K;
#pragma unroll
            for (int c = 0; c < K; ++c) dst[c] = r[c];
        });
    }
    const unsigned long long slot = base[2 * T.self] + block_take(stays, &cursor[2 * T.self]);
    if (stays) {
        double* dst = keep + slot * K;
#pragma unroll
        for (int c = 0; c < K; ++c) dst[c] = r[c];
    }
}

// Host-loaded natives (SoA coordinates, masses, ids) as records.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_tile_records(int n, const double* __restrict__ pos, const double* __restrict__ mass,
               const uint32_t* __restrict__ ids, double* __restrict__ rec) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int K = DIM + 2;
#pragma unroll
    for (int a = 0; a < DIM; ++a) rec[int64_t(i) * K + a] = pos[int64_t(a) * n + i];
    rec[int64_t(i) * K + DIM] = mass[i];
    rec[int64_t(i) * K + DIM + 1] = double(ids[i]);
}

// The tile's particle set from the kept records (n_keep) and the received
// ones (n_recv): natives keep their id, ghosts get kGhostBit.  A record
// outside this tile's pad box (or, with strict, not native to it), with an
// id that is not an integer below 2^31, or (strict) with a mass that is not
// finite or above mass_limit in magnitude sets a bit in *flags; it is then
// stored as a ghost and changes nothing the tile keeps.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_tile_assemble(int n_keep, const double* __restrict__ keep, int n_recv,
                const double* __restrict__ recv, const TileGeom T, int strict,
                double mass_limit, int64_t stride,
                double* __restrict__ pos, double* __restrict__ mass, uint32_t* __restrict__ id,
                uint32_t* __restrict__ flags) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_keep + n_recv) return;
    constexpr int K = DIM + 2;
    const double* r = i < n_keep ? keep + int64_t(i) * K : recv + int64_t(i - n_keep) * K;
    double x[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        x[a] = r[a];
        pos[a * stride + i] = x[a];
    }
    // for_each_dest names this tile exactly when x lies in its pad box
    bool named = false, native = false;
    for_each_dest<DIM>(x, T, [&](int t, bool nat) {
        if (t == T.self) {
            named = true;
            native = nat;
        }
    });
    const double idd = r[DIM + 1];
    const bool id_ok = idd >= 0.0 && idd < 2147483648.0 && double(uint32_t(idd)) == idd;
    uint32_t bad = 0;
    if (!named || (strict && !native)) bad |= kTileErrForeign;
    if (!id_ok) bad |= kTileErrId;
    if (strict && (not_finite(r[DIM]) || !(fabs(r[DIM]) <= mass_limit))) bad |= kTileErrMass;
    if (bad) {
        atomicOr(flags, bad);
        native = false;
    }
    mass[i] = r[DIM];
    const uint32_t gid = id_ok ? uint32_t(idd) : 0u;
    id[i] = native ? gid : (gid | kGhostBit);
}

// Natives (id without kGhostBit) of the current state into the other buffer
// half, in no defined order; *count ends at their number.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_tile_compact(int n, int64_t stride, const double* __restrict__ pos,
               const double* __restrict__ mass, const uint32_t* __restrict__ id,
               double* __restrict__ pos_out, double* __restrict__ mass_out,
               uint32_t* __restrict__ id_out, unsigned long long* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool keep = i < n && !(id[i] & kGhostBit);
    const unsigned long long dst = block_take(keep, count);
    if (!keep) return;
#pragma unroll
    for (int a = 0; a < DIM; ++a) pos_out[a * stride + dst] = pos[a * stride + i];
    mass_out[dst] = mass[i];
    id_out[dst] = id[i];
}

}  // namespace mtpt
