// vecops.cuh -- device helpers shared by the GMRES drivers: double-float
// accumulation of FP32 data and a block-wide FP64 sum.
#pragma once

#include <vector>

#include "common.cuh"

namespace rbf {

// Records the true relative residual of a restart; true when it is above 90 %
// of the value three restarts earlier (stagnation of restarted GMRES).
inline bool stagnating(std::vector<double>& hist, double relres)
{
    hist.push_back(relres);
    const size_t k = hist.size();
    return k >= 4 && relres > 0.9 * hist[k - 4];
}

constexpr int kDotThreads = 256;

namespace {

// flag = 1 if some x[i] is not +-0 (NaN included): the solvers' zero initial
// guess test (r0 = f without a product when w0 = 0).
__global__ void k_any_nonzero(const double* __restrict__ x, int64_t n, int* __restrict__ flag)
{
    bool nz = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        nz |= !(x[i] == 0.0);
    if (__syncthreads_or(nz) && threadIdx.x == 0) *flag = 1;
}

}  // namespace

// Double-float accumulator for FP32 data (Ogita, Rump and Oishi, "Accurate sum
// and dot product", SIAM J. Sci. Comput. 26(6), 2005: TwoProduct by FMA,
// TwoSum, and the Dot2 recurrence): a sum of exact FP32 products carried as an
// unevaluated hi + lo pair, as accurate as accumulating in twice the FP32
// precision. On GB300 this keeps FP64-class dot products on the FP32 pipe.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void df_add(DF& s, float h, float r)
{
    float p = s.hi + h;                 // TwoSum(s.hi, h) = (p, q)
    float z = p - s.hi;
    float q = (s.hi - (p - z)) + (h - z);
    s.hi = p;
    s.lo = s.lo + (q + r);
}

__device__ __forceinline__ void df_add_prod(DF& s, float a, float b)
{
    float h = a * b;                    // TwoProduct(a, b) = (h, r)
    float r = fmaf(a, b, -h);
    df_add(s, h, r);
}

// a += b for two double-float values: TwoSum of the high parts, low parts and
// the rounding error added (the sum keeps about 2 x 24 bits).
__device__ __forceinline__ void df_merge(DF& a, float bh, float bl)
{
    df_add(a, bh, bl);
}

// Block sum of one double-float value per thread, carried in double-float on
// the FP32 pipe through the shuffle tree and across warps (fixed order), and
// converted to FP64 once, by thread 0 (the only thread that gets the result).
__device__ __forceinline__ double block_sum_df(DF s, DF* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = 16; d > 0; d >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, s.hi, d), ol = __shfl_xor_sync(0xffffffffu, s.lo, d);
        df_merge(s, oh, ol);
    }
    if (lane == 0) red[warp] = s;
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0) {
        DF t = red[0];
        for (int w = 1; w < kDotThreads / 32; ++w) df_merge(t, red[w].hi, red[w].lo);
        out = (double)t.hi + (double)t.lo;
    }
    return out;
}

// Sum of one value per thread over a block of kDotThreads threads, returned
// to thread 0 (fixed order: shuffle tree within warps, warps in order).
__device__ __forceinline__ double block_sum(double a, double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
    if (lane == 0) red[warp] = a;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kDotThreads / 32; ++w) s += red[w];
    return s;
}

}  // namespace rbf
