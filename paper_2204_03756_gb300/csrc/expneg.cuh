// expneg.cuh -- exp(-t) in binary64 for the pair kernel K = exp(-|dx|^2 / (2 h^2)).
//
// Table-driven method of P. T. P. Tang, "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2),
// 1989: write t = (64 q + j) ln2/64 + r with |r| <= ln2/128, j in [0, 64),
// so exp(-t) = 2^-q * 2^(-j/64) * exp(-r).  2^(-j/64) comes from a 64-entry
// table computed on the host, exp(-r) from its Taylor series through r^5
// (the first omitted term is below 4e-17 relative), and 2^-q is applied to
// the exponent field.  r is formed with ln2/64 split in two parts and fused
// multiply-adds, so its absolute error stays below 1e-18.  Valid for
// 0 <= t <= 700 (the result stays a normal number); the pair kernel only
// evaluates t <= lambda^2 (1 + 1e-4).
//
// Cost: 10 binary64 operations (1 mul, 2 add, 7 fma/mul) against the ~2x
// longer general-purpose exp; on GB300 every binary64 operation costs about
// 70 binary32 ones, so this is the pair loop's dominant arithmetic.
#pragma once
#include <cstdint>

namespace mtpt {

struct ExpNegConsts {
    double inv_step;   // 64 / ln 2
    double step_hi;    // ln 2 / 64, leading part
    double step_lo;    // ln 2 / 64 - step_hi
};

__device__ __forceinline__ double exp_neg(double t, const double* __restrict__ table,
                                          const ExpNegConsts& c) {
    constexpr double kRound = 6755399441055744.0;   // 1.5 * 2^52: adding it rounds to an integer
    const double y = __dadd_rn(__dmul_rn(t, c.inv_step), kRound);
    const int k = __double2loint(y);                 // round(t * 64 / ln 2), >= 0
    const double kd = __dsub_rn(y, kRound);
    double r = __fma_rn(-kd, c.step_hi, t);
    r = __fma_rn(-kd, c.step_lo, r);
    const double s = -r;
    double p = __fma_rn(s, 1.0 / 120.0, 1.0 / 24.0);
    p = __fma_rn(s, p, 1.0 / 6.0);
    p = __fma_rn(s, p, 0.5);
    p = __fma_rn(s, p, 1.0);
    p = __fma_rn(s, p, 1.0);
    const double v = __dmul_rn(table[k & 63], p);
    const long long scaled = __double_as_longlong(v) - (static_cast<long long>(k >> 6) << 52);
    return __longlong_as_double(scaled);
}

}  // namespace mtpt
