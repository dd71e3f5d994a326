// rng.cuh -- counter-based normal variates for the random walk (Sec. 3).
//
// The paper only asks for i.i.d. standard-normal xi_i.  This library draws
// them from Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) keyed by the
// run seed, with counter (particle id, step low word, step high word, 0), so
// a realisation is a pure function of (seed, initial state) and restarts
// reproduce it bit for bit.  Each 32-bit word w gives a uniform
// u = ((w >> 8) + 1) / 2^24 in (0, 1]; words (0,1) and (2,3) give two normals
// each by the Box-Muller transform, evaluated in binary32 with only correctly
// rounded +, -, *, /, sqrt and explicit fma (every operation below is an
// explicit _rn intrinsic, so nvcc cannot contract or reorder it):
//   ln u      : u = 2^e m, m in [sqrt(1/2), sqrt(2)], ln m = 2 atanh f with
//               f = (m - 1)/(m + 1), odd series through f^11, plus e ln 2
//               added in two parts (Cody & Waite splitting);
//   sin, cos  : of 2 pi k / 2^24, reduced exactly in integers to a quadrant
//               and an angle x in [0, pi/4], then Taylor series (sin through
//               x^9, cos through x^10) by Horner's rule.
#pragma once
#include <cstdint>

namespace mtpt {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
    constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(kMul0, c.x), lo0 = kMul0 * c.x;
        const uint32_t hi1 = __umulhi(kMul1, c.z), lo1 = kMul1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += kWeyl0;
        k.y += kWeyl1;
    }
    return c;
}

__device__ __forceinline__ float log_f32(float u) {
    uint32_t bits = __float_as_uint(u);
    int e = int((bits >> 23) & 0xffu) - 127;
    float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421354f) { m = __fmul_rn(m, 0.5f); e += 1; }
    const float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s = __fmul_rn(f, f);
    float q = __fmaf_rn(s, 1.0f / 11.0f, 1.0f / 9.0f);
    q = __fmaf_rn(s, q, 1.0f / 7.0f);
    q = __fmaf_rn(s, q, 1.0f / 5.0f);
    q = __fmaf_rn(s, q, 1.0f / 3.0f);
    const float two_f = __fmul_rn(2.0f, f);
    const float ln_m = __fmaf_rn(__fmul_rn(two_f, s), q, two_f);
    const float ln2_hi = 0.693145752f;     // 16 significant bits: e * ln2_hi is exact
    const float ln2_lo = 1.42860677e-06f;
    const float fe = float(e);
    return __fmaf_rn(fe, ln2_hi, __fmaf_rn(fe, ln2_lo, ln_m));
}

__device__ __forceinline__ void sincos_2pi_f32(uint32_t k, float* s_out, float* c_out) {
    const uint32_t q = (k >> 22) & 3u;
    uint32_t r = k & 0x3fffffu;
    const bool folded = r > 0x200000u;
    if (folded) r = 0x400000u - r;
    const float x = __fmul_rn(float(r), 3.74507028e-07f);   // r * pi / 2^23
    const float z = __fmul_rn(x, x);
    float ps = __fmaf_rn(z, 1.0f / 362880.0f, -1.0f / 5040.0f);
    ps = __fmaf_rn(z, ps, 1.0f / 120.0f);
    ps = __fmaf_rn(z, ps, -1.0f / 6.0f);
    const float sin_x = __fmaf_rn(__fmul_rn(x, z), ps, x);
    float pc = __fmaf_rn(z, -1.0f / 3628800.0f, 1.0f / 40320.0f);
    pc = __fmaf_rn(z, pc, -1.0f / 720.0f);
    pc = __fmaf_rn(z, pc, 1.0f / 24.0f);
    pc = __fmaf_rn(z, pc, -0.5f);
    const float cos_x = __fmaf_rn(z, pc, 1.0f);
    const float sa = folded ? cos_x : sin_x;
    const float ca = folded ? sin_x : cos_x;
    float s, c;
    switch (q) {
        case 0: s = sa; c = ca; break;
        case 1: s = ca; c = -sa; break;
        case 2: s = -sa; c = -ca; break;
        default: s = -ca; c = sa; break;
    }
    *s_out = s;
    *c_out = c;
}

// Four N(0,1) draws of particle `id` at walk step `step`.
__device__ __forceinline__ float4 normals4(uint64_t seed, uint32_t id, uint64_t step) {
    const uint4 w = philox4x32_10(make_uint4(id, uint32_t(step), uint32_t(step >> 32), 0u),
                                  make_uint2(uint32_t(seed), uint32_t(seed >> 32)));
    float out[4];
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int pair = 0; pair < 2; ++pair) {
        const uint32_t ka = (words[2 * pair] >> 8) + 1u;
        const uint32_t kb = (words[2 * pair + 1] >> 8) + 1u;
        const float ua = __fmul_rn(float(ka), 5.9604644775390625e-08f);   // exact
        const float radius = __fsqrt_rn(__fmul_rn(-2.0f, log_f32(ua)));
        float sn, cs;
        sincos_2pi_f32(kb, &sn, &cs);
        out[2 * pair] = __fmul_rn(radius, cs);
        out[2 * pair + 1] = __fmul_rn(radius, sn);
    }
    return make_float4(out[0], out[1], out[2], out[3]);
}

}  // namespace mtpt
