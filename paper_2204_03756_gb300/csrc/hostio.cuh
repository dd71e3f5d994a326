// hostio.cuh -- device side of the pipelined host loads (mtpt_set_particles_async).
//
// A host load arrives in a staging slot (positions dim x n, then masses n,
// float64) by a copy on its own stream.  k_load_input checks every particle
// (the test of mtpt_set_particles: coordinates finite and inside the box,
// masses finite and at most mass_limit in magnitude) and writes it into the
// free half of the state double buffer in the same pass; k_load_settle then
// either resets the step counter (load accepted) or copies the old state back
// over the free half and latches the rejection in the status word, so a
// rejected load leaves the state as it was.  The host makes the free half
// current when it enqueues the pair, before knowing the outcome: both cases
// leave the right state there.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace mtpt {

// Rejections of a pipelined load, latched beside kStatusNonFinite and
// kStatusOutOfDomain: a position outside the box (or not finite), a mass not
// finite or beyond the precision form's limit.
enum : uint32_t { kStatusLoadPosition = 4u, kStatusLoadMass = 8u };

// Integer order key of a binary64 value with -0 and +0 on the same key (both
// compare equal as values).
__device__ __forceinline__ long long load_key(double v) {
    return (__double_as_longlong(v) & 0x7fffffffffffffffLL) == 0 ? 0LL : order_key(v);
}

// Check and copy.  in: staging slot (stride n); out: one state half (stride
// cap).  flag bit 0: a position failed, bit 1: a mass failed.  Integer tests
// only (the binary64 unit is slow): x inside [lo, hi] through the order keys
// (a NaN fails the finiteness test), |m| <= mass_limit through the magnitude
// bits, which order like the magnitudes.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_load_input(int n, const double* __restrict__ in, const double* __restrict__ box,
             double mass_limit, uint32_t* __restrict__ flag, int64_t cap,
             double* __restrict__ pos_out, double* __restrict__ mass_out,
             uint32_t* __restrict__ id_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t bad = 0;
    if (i < n) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double x = in[int64_t(a) * n + i];
            const long long kx = load_key(x);
            if (not_finite(x) || kx < load_key(box[a]) || kx > load_key(box[3 + a])) bad |= 1u;
            pos_out[int64_t(a) * cap + i] = x;
        }
        const double m = in[int64_t(DIM) * n + i];
        const long long mag = __double_as_longlong(m) & 0x7fffffffffffffffLL;
        if (not_finite(m) || mag > __double_as_longlong(mass_limit)) bad |= 2u;
        mass_out[i] = m;
        id_out[i] = uint32_t(i);
    }
    const uint32_t any = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && any) atomicOr(flag, any);
}

// Settle a checked load: accepted -> step counter 0; rejected -> the old
// state (positions, masses, ids) copied back over the new half and the
// rejection latched in the status word.  Grid-stride over the particles.
template <int DIM>
__global__ void __launch_bounds__(kBlock)
k_load_settle(int n, int64_t cap, const uint32_t* __restrict__ flag,
              const double* __restrict__ pos_old, const double* __restrict__ mass_old,
              const uint32_t* __restrict__ id_old, double* __restrict__ pos_new,
              double* __restrict__ mass_new, uint32_t* __restrict__ id_new,
              uint32_t* __restrict__ status, unsigned long long* __restrict__ step_dev) {
    const uint32_t f = *flag;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (f == 0u) {
        if (lead) *step_dev = 0ull;
        return;
    }
    if (lead)
        atomicOr(status, ((f & 1u) ? kStatusLoadPosition : 0u) | ((f & 2u) ? kStatusLoadMass : 0u));
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) pos_new[a * cap + i] = pos_old[a * cap + i];
        mass_new[i] = mass_old[i];
        id_new[i] = id_old[i];
    }
}

}  // namespace mtpt
