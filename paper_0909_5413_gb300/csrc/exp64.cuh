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
// Host: tab[j] = 2^(-j/2048), j < 2048, and the cubic's coefficients c[0..2] = c1, c2, c3.
void make_exp2048(double* tab, double* c);

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

// The same method with 2048 table entries, in binary units, for a kernel
// value given by a squared distance: returns exp(-r2 s) = 2^(-u / 2048) with
// u = r2 K, K = 2048 s / ln 2. n = nearest integer to u (the FMA r2 K + 1.5 2^52
// rounds it), r = r2 K - n in [-1/2, 1/2] from a second FMA (one rounding),
// n = 2048 m + j, 2^(-u/2048) = 2^(-m) * tab2048[j] * 2^(-r/2048) with
// tab2048[j] = 2^(-j/2048). With z = -r ln 2 / 2048 (|z| <= 1.7e-4),
// 2^(-r/2048) = 1 + z + z^2/2 + z^3/6 + O(z^4 / 24 < 4e-17), written as a
// cubic in r with coefficients c1 = -ln2/2048, c2 = c1^2/2, c3 = c1^3/6.
// Cost on the FP64 pipe: 2 FMA + 1 ADD + 3 FMA + 1 MUL. Results below
// 2^-976 (u >= 2e6, t > 676) are returned as 0.
constexpr int kExpTab2048 = 2048;

__device__ __forceinline__ double exp_neg_r2(double r2, double K, const double* __restrict__ tab2048, double c1,
                                             double c2, double c3)
{
    const double kMagic = 6755399441055744.0;
    double y = fma(r2, K, kMagic);
    int n = (int)__double2loint(y);
    bool small = ((unsigned)__double2hiint(y) < 0x43400000u) && n < 2000000;   // u < 2e6 (and < 2^51)
    n = small ? n : 0;
    double nd = y - kMagic;
    double r = fma(r2, K, -nd);
    double p = fma(fma(fma(c3, r, c2), r, c1), r, 1.0);
    int j = n & (kExpTab2048 - 1);
    int m = n >> 11;
    double v = tab2048[j] * p;                   // in (0.4999, 1.0002]
    int hi = __double2hiint(v) - (m << 20);
    v = __hiloint2double(hi, __double2loint(v));
    return small ? v : 0.0;
}

}  // namespace rbf
