// fixexp.cuh -- Gaussian kernel value exp(-s r2) of a point pair evaluated in
// 64-bit fixed point on the integer pipes (one FP64 instruction per pair is
// then only the caller's accumulate).
//
// Coordinates are scaled by 2^S (S = 62 - e, |x| < 2^e) and rounded to int64;
// every FP64 coordinate with |x| >= 2^(e-10) is a multiple of 2^-S, so the
// pair offsets dx, dy are exact integers, as exact as the FP64 differences the
// index-list definition uses. With u = |dx| 2^sh (u < 2^63 inside the cutoff),
//   q  = hi64(u_x^2) + hi64(u_y^2)            (r2 to 2^-62 relative)
//   z  = hi64(q M) = r2 s log2(e) 2^F          (F fractional bits, F ~ 55)
// and exp(-s r2) = 2^-z = 2^-n T1[i1] T2[i2] 2^-rho with n = z >> F, two
// 10-bit table indices below it (T1[i] = 2^(-i/1024), T2[j] = 2^(-j/2^20),
// stored in Q1.63) and the remainder rho < 2^-20, for which
// 2^-rho = e^-x, x = rho ln 2 < 6.7e-7, is 1 - x + x^2/2 to 2^-64.
// The product m in Q1.63 is turned into an FP64 bit pattern with exponent
// -n (rounded to nearest on the dropped bits). This is the table-driven
// method of Tang (ACM TOMS 15, 1989) carried out in integer arithmetic.
#pragma once

#include <cstdint>

namespace rbf {

constexpr int kFxTab = 1024;   // entries of each table

// 2^-x in Q1.63 for the two tables (host; long double).
void make_fx_tables(unsigned long long* t1, unsigned long long* t2);

// Fixed-point constants of a problem: scale 2^S, shift sh, multiplier M and
// fraction bits F from the coordinate magnitude, r_c and s. False if the
// cutoff is too small or too large next to the coordinates for 64-bit fixed
// point (r_c < 2^-32 max|x|, or r_c / sigma beyond ~1000).
bool make_fx_constants(double amax, double rc, double s, double* scale, int* sh, int* F, unsigned long long* M);

__device__ __forceinline__ double kernel_fx(long long dx, long long dy, int sh, int F, unsigned long long M,
                                            const unsigned long long* __restrict__ T1,
                                            const unsigned long long* __restrict__ T2)
{
    const unsigned long long ux = (unsigned long long)(dx < 0 ? -dx : dx) << sh;   // < 2^63 (1 + 2^-50)
    const unsigned long long uy = (unsigned long long)(dy < 0 ? -dy : dy) << sh;
    const unsigned long long q = __umul64hi(ux, ux) + __umul64hi(uy, uy) + 1ull;   // +1: centre the truncations
    const unsigned long long z = __umul64hi(q, M);
    const unsigned int n = (unsigned int)(z >> F);
    const unsigned int i1 = (unsigned int)(z >> (F - 10)) & (kFxTab - 1);
    const unsigned int i2 = (unsigned int)(z >> (F - 20)) & (kFxTab - 1);
    const unsigned long long rho = z << (84 - F);                 // rho 2^20 in [0, 1), units 2^-64
    const unsigned long long x = __umul64hi(rho, 12193974156573ull);   // rho ln 2, units 2^-64 (ln 2 2^44)
    const unsigned long long onem = x - (__umul64hi(x, x) >> 1);          // 1 - e^-x
    unsigned long long m = __umul64hi(T1[i1], T2[i2]) << 1;               // Q1.63
    m -= __umul64hi(m, onem);
    const int lz = __clzll((long long)m);
    const unsigned long long mn = m << lz;                                // [2^63, 2^64)
    const unsigned long long bits =
        ((unsigned long long)(1022 - lz - (int)n) << 52) + (mn >> 11) + ((mn >> 10) & 1ull);
    return n < 1000u ? __longlong_as_double((long long)bits) : 0.0;
}

}  // namespace rbf
