// expneg.cuh -- K = exp(-a d2) in binary64 for the pair kernel (Eq. 4 with
// a = 1 / (2 h^2)).
//
// Table-driven method of P. T. P. Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2),
// 1989, arranged so that only the parts that set the accuracy use binary64
// (GB300 runs binary64 at about 1/70 of the binary32 rate):
//
//   t = a d2 = k ln2/256 + a r,   k = round(t 256 / ln 2),
//   exp(-t) = 2^-(k >> 8) * 2^(-(k & 255)/256) * exp(-a r).
//
// * k comes from the binary32 head of d2 (bit truncation, no binary64
//   instruction) times a 256 / ln 2 in binary32: it is within 0.53 of
//   t 256 / ln 2 for t <= 400, so |a r| <= 0.53 ln2 / 256 < 1.44e-3.  Any k
//   gives a correct reduction; only the bound on r depends on it.
// * r = d2 - k c with c = ln 2 / (256 a) held as c_hi + c_lo, c_hi with 32
//   significant bits so k c_hi is exact for k < 2^21; two fma.
// * exp(-a r) is its Taylor series through (a r)^4 with a folded into the
//   coefficients p_m = (-a)^m / m! (four fma on r; the first omitted term is
//   below 5e-17 relative), so no binary64 multiply forms a r or t.
// * 2^(-j/256) is a 256-entry host table; 2^-(k >> 8) goes into the exponent
//   field with an integer subtraction.
//
// Cost: 7 binary64 operations (2 + 4 fma, 1 mul) and integer/binary32 work.
// Valid for 0 <= a d2 <= 400.1 (lambda <= 20 with the band margin: the
// result stays normal) and a <= 5e34: the binary32 scale and p_4 stay finite,
// and a d2 whose head underflows binary32 (d2 < 2^-126, so k = 0) has
// a d2 < 6e-4, inside the polynomial's range.  The host rejects parameters
// outside.  Error: within 1.5 ulp of exp(-a d2) for the binary64 a and d2.
#pragma once
#include <cstdint>

namespace mtpt {

constexpr int kExpTable = 256;

struct ExpNegConsts {
    float k_scale;      // a * 256 / ln 2 in binary32
    double c_hi, c_lo;  // ln 2 / (256 a) = c_hi + c_lo
    double p1, p2, p3, p4;   // (-a)^m / m!
};

// Head of a binary64 x >= 0 with x < 2^128 as binary32, truncated (integer
// operations only); 0 below 2^-126.
__device__ __forceinline__ float head_f32(double x) {
    const uint32_t whi = uint32_t(__double2hiint(x));
    const uint32_t wlo = uint32_t(__double2loint(x));
    const int e = int(whi >> 20);
    const uint32_t bits = (uint32_t(e - 896) << 23) | ((whi & 0xfffffu) << 3) | (wlo >> 29);
    return e < 897 ? 0.0f : __uint_as_float(bits);
}

// Exact binary64 image of 0 <= k < 2^31 from integer operations.
__device__ __forceinline__ double small_uint_to_f64(uint32_t k) {
    const int m = 31 - __clz(int(k | 1u));
    const uint64_t mant = (uint64_t(k) << (52 - m)) & 0xfffffffffffffull;
    const double v = __longlong_as_double((long long)((uint64_t(1023 + m) << 52) | mant));
    return k == 0u ? 0.0 : v;
}

__device__ __forceinline__ double gauss_exp(double d2, const double* __restrict__ table,
                                            const ExpNegConsts& c) {
    const float yk = __fmaf_rn(head_f32(d2), c.k_scale, 12582912.0f);   // + 1.5 * 2^23
    const uint32_t k = uint32_t(__float_as_int(yk) - 0x4b400000);
    const double kd = small_uint_to_f64(k);
    double r = __fma_rn(-kd, c.c_hi, d2);
    r = __fma_rn(-kd, c.c_lo, r);
    double p = __fma_rn(c.p4, r, c.p3);
    p = __fma_rn(p, r, c.p2);
    p = __fma_rn(p, r, c.p1);
    p = __fma_rn(p, r, 1.0);
    const double v = __dmul_rn(table[k & (kExpTable - 1)], p);
    const long long scaled = __double_as_longlong(v) - (static_cast<long long>(k >> 8) << 52);
    return __longlong_as_double(scaled);
}

}  // namespace mtpt
