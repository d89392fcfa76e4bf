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

// High 64 bits of a 64 x 64-bit product from three 32 x 32-bit products (the
// low x low one is dropped): in [exact - 3, exact].
__device__ __forceinline__ unsigned long long hi64a(unsigned long long a, unsigned long long b)
{
    const unsigned int ah = (unsigned int)(a >> 32), al = (unsigned int)a;
    const unsigned int bh = (unsigned int)(b >> 32), bl = (unsigned int)b;
    return (unsigned long long)ah * bh + __umulhi(ah, bl) + __umulhi(al, bh);
}

// High 64 bits of u^2: in [exact - 2, exact].
__device__ __forceinline__ unsigned long long sqhi(unsigned long long u)
{
    const unsigned int uh = (unsigned int)(u >> 32), ul = (unsigned int)u;
    return (unsigned long long)uh * uh + 2ull * __umulhi(uh, ul);
}

// Fixed-point coordinate pre-shifted by sh (wrapping: differences of two such
// values are the exact shifted offsets, which lie inside (-2^63, 2^63) for
// pairs inside the cutoff).
__device__ __forceinline__ long long fx_coord(double x, double scale, int sh)
{
    return (long long)((unsigned long long)__double2ll_rn(x * scale) << sh);
}

// exp(-s r2) from the shifted offsets du = (x_i - x_j) 2^(S+sh), dv likewise.
__device__ __forceinline__ double kernel_fx(long long du, long long dv, int F, unsigned long long M,
                                            const unsigned long long* __restrict__ T1,
                                            const unsigned long long* __restrict__ T2)
{
    const unsigned long long ux = (unsigned long long)(du < 0 ? -du : du);   // < 2^63 (1 + 2^-50)
    const unsigned long long uy = (unsigned long long)(dv < 0 ? -dv : dv);
    const unsigned long long q = sqhi(ux) + sqhi(uy) + 2ull;   // +2 centres the truncations
    const unsigned long long z = hi64a(q, M) + 1ull;
    const unsigned int n = (unsigned int)(z >> F);
    const unsigned int i1 = (unsigned int)(z >> (F - 10)) & (kFxTab - 1);
    const unsigned int i2 = (unsigned int)(z >> (F - 20)) & (kFxTab - 1);
    const unsigned long long rho = z << (84 - F);                   // rho 2^20 in [0, 1), units 2^-64
    const unsigned long long x = hi64a(rho, 12193974156573ull);       // rho ln 2, units 2^-64 (ln 2 2^44)
    const unsigned int xh = (unsigned int)(x >> 12);                 // x < 2^43.5: 32 bits suffice for x^2
    const unsigned long long onem = x - (((unsigned long long)xh * xh) >> 41);   // 1 - e^-x = x - x^2/2
    unsigned long long m = hi64a(T1[i1], T2[i2]) << 1;                // Q1.63, in (2^62, 2^63]
    m -= hi64a(m, onem);
    // m / 2^63 in (1/2, 1]: cap 1.0 at 1 - 2^-63 (which rounds back to 1.0), round
    // the 10 dropped bits to nearest, and let the implicit bit carry into the
    // exponent field: 2^-n m / 2^63 = (m / 2^62) 2^(-1-n).
    m = m - (m >> 63) + 512ull;
    const unsigned long long bits = ((unsigned long long)(1021 - (int)n) << 52) + (m >> 10);
    return n < 1000u ? __longlong_as_double((long long)bits) : 0.0;
}

// The same value for problems whose multiplier was scaled to F = 52 fraction
// bits (every r_c up to about 37 sigma on coordinates of moderate spread): z's
// high word then holds n (top 12 bits), i1 and i2, and its low word the
// remainder, so every extraction is a 32-bit operation; the squares use the
// signed split d = a 2^32 + b with b in [-2^31, 2^31), d^2 / 2^64 ~ a^2 + 2 a b /
// 2^32 (no absolute values); n < 1000 is guaranteed by the binning.
__device__ __forceinline__ unsigned long long sqhi_s(long long d)
{
    const int b = (int)(unsigned int)d;
    const int a = (int)(d >> 32) - (b >> 31);
    return (unsigned long long)((long long)a * a) + 2ull * (unsigned long long)(long long)__mulhi(a, b);
}

__device__ __forceinline__ double kernel_fx52(long long du, long long dv, unsigned long long M,
                                              const unsigned long long* __restrict__ T1,
                                              const unsigned long long* __restrict__ T2)
{
    const unsigned long long q = sqhi_s(du) + sqhi_s(dv) + 2ull;
    const unsigned long long z = __umul64hi(q, M);   // exact floor: 52 fraction bits leave no room for more
    const unsigned int zh = (unsigned int)(z >> 32), zl = (unsigned int)z;
    const unsigned int n = zh >> 20;
    const unsigned int i1 = (zh >> 10) & (kFxTab - 1), i2 = zh & (kFxTab - 1);
    // x = rho ln 2 in units 2^-64 with rho 2^20 = zl 2^-32: (zl * ln 2 2^44) >> 32
    constexpr unsigned long long kC = 12193974156573ull;   // ln 2 2^44
    const unsigned long long x =
        (unsigned long long)zl * (unsigned int)(kC >> 32) + __umulhi(zl, (unsigned int)kC);
    const unsigned int xh = (unsigned int)(x >> 12);
    const unsigned long long onem = x - (((unsigned long long)xh * xh) >> 41);
    unsigned long long m = hi64a(T1[i1], T2[i2]) << 1;
    m -= hi64a(m, onem);
    m = m - (m >> 63) + 512ull;
    const unsigned int lo = (unsigned int)(m >> 10);
    const unsigned int hi = (unsigned int)(m >> 42) + ((1021u - n) << 20);
    return __hiloint2double((int)hi, (int)lo);
}

}  // namespace rbf
