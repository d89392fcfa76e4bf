// exp64.cuh -- exp(-t) for t >= 0 in FP64, table-driven in the manner of
// P. T. P. Tang, "Table-driven implementation of the exponential function in
// IEEE floating-point arithmetic", ACM TOMS 15(2), 1989:
//
//   x = -t;  n = nearest integer to x * 64 / ln 2;  r = x - n (ln 2 / 64)
//   (ln 2 / 64 split in a short high part and a low part, so n * high is
//   exact);  n = 64 m + j with 0 <= j < 64;
//   exp(x) = 2^m * 2^(j/64) * exp(r),  |r| <= ln 2 / 128,
//   exp(r) by its degree-5 Taylor polynomial (truncation error
//   r^6 / 720 < 4e-17 relative).
//
// The 64 values 2^(j/64) and the split constants are computed on the host
// (make_exp_consts) and passed to kernels by value; kernels copy the table to
// shared memory. The scale by 2^m is an integer add on the exponent field.
// Results below 2^-1021 (t > 707) are returned as 0.
//
// Cost on the FP64 pipe: 9 FMA/ADD + 1 MUL (the FMA rounding trick replaces a
// float-to-int conversion).
#pragma once

#include <cstdint>

namespace rbf {

struct ExpConsts {
    double inv_l;     // 64 / ln 2
    double l_hi;      // high part of ln 2 / 64 (n * l_hi exact for |n| < 2^21)
    double l_lo;      // ln 2 / 64 - l_hi
    double tab[64];   // 2^(j/64)
};

// Host: fill the constants in extended precision (long double).
ExpConsts make_exp_consts();

// exp(-t), t >= 0; tab points at a (shared-memory) copy of c_exp.tab.
__device__ __forceinline__ double exp_neg(double t, const double* __restrict__ tab, double inv_l, double l_hi,
                                          double l_lo)
{
    const double kMagic = 6755399441055744.0;   // 1.5 * 2^52: adding it rounds to an integer
    double x = -t;
    double y = fma(x, inv_l, kMagic);
    int n = (int)__double2loint(y);              // low word of y holds n (two's complement)
    double nd = y - kMagic;                      // exact
    double r = fma(nd, -l_hi, x);
    r = fma(nd, -l_lo, r);
    double p = 1.0 / 120.0;
    p = fma(p, r, 1.0 / 24.0);
    p = fma(p, r, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    int j = n & 63;
    int m = n >> 6;                              // floor(n / 64)
    double v = tab[j] * p;                       // in [0.99, 2)
    long long bits = __double_as_longlong(v) + (long long)m * (1LL << 52);
    return (t < 707.0) ? __longlong_as_double(bits) : 0.0;
}

}  // namespace rbf
