// apply.cuh -- one subdomain of the restricted Schwarz apply of Eq. rasm,
// z_core = W_i r_ov (W_i = the core rows of A_i^{-1}, column-major), by one
// warp with a shared gather buffer rg of kMaxSub entries. Shared by the apply
// kernel and the fused Arnoldi step.
#pragma once

#include "common.cuh"

namespace rbf {

// active (optional): per-problem mask, read through pid_sub; a masked
// subdomain writes nothing.
template <class TW, class TV>
__device__ __forceinline__ void rasm_apply_one(int64_t sub, int lane, TV* __restrict__ rg,
                                               const int32_t* __restrict__ ov_ptr, const int32_t* __restrict__ ov_idx,
                                               const int32_t* __restrict__ core_ptr,
                                               const int32_t* __restrict__ core_idx, const int64_t* __restrict__ w_off,
                                               const TW* __restrict__ W, const int32_t* __restrict__ pid_sub,
                                               const int32_t* __restrict__ active, const TV* __restrict__ r,
                                               TV* __restrict__ z)
{
    // the problem's mask is read here but tested only once the first loads of W
    // and of the overlap list are in flight (its latency then overlaps theirs)
    const int32_t* mask = active ? active + pid_sub[sub] : nullptr;
    const int b = ov_ptr[sub];
    const int n = ov_ptr[sub + 1] - b;
    const int cb = core_ptr[sub];
    const int nc = core_ptr[sub + 1] - cb;
    const TW* Ws = W + w_off[sub];
    // G lanes cooperate on one core row; each lane sums its columns a = part,
    // part + G, ... in order, U loads of W issued together (FP32: 20, so that
    // a 4 x 4-core subdomain's whole W_i, 18 columns per lane, is in flight
    // before the gather; 16 measured 12 % slower at 51M points, 24 5 %).
    int G = 1;
    while (G < 32 && nc * G * 2 <= 32) G *= 2;
    const int rows_per_pass = 32 / G;
    const int part = lane % G;
    constexpr int U = sizeof(TW) == 4 ? 20 : 8;
    TW wv[U];
    {   // the first batch of W does not depend on r: issue it before the gather
        const int c = lane / G;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int a = part + u * G;
            wv[u] = (c < nc && a < n) ? Ws[(int64_t)a * nc + c] : (TW)0;
        }
    }
    {   // gather: all overlap indices first, then the values
        constexpr int kG = kMaxSub / 32;
        int ia[kG];
#pragma unroll
        for (int t = 0; t < kG; ++t) ia[t] = lane + 32 * t < n ? ov_idx[b + lane + 32 * t] : -1;
        if (mask && !*mask) return;   // masked problem (warp-uniform); nothing has been written
        TV rv[kG];
#pragma unroll
        for (int t = 0; t < kG; ++t) rv[t] = ia[t] >= 0 ? r[ia[t]] : (TV)0;
#pragma unroll
        for (int t = 0; t < kG; ++t)
            if (ia[t] >= 0) rg[lane + 32 * t] = rv[t];
    }
    __syncwarp();
    for (int c0 = 0; c0 < nc; c0 += rows_per_pass) {
        const int c = c0 + lane / G;
        TV acc = 0;
        if (c < nc) {
            for (int a0 = part; a0 < n; a0 += U * G) {
                if (c0 > 0 || a0 > part) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int a = a0 + u * G;
                        wv[u] = a < n ? Ws[(int64_t)a * nc + c] : (TW)0;
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int a = a0 + u * G;
                    if (a < n) acc += (TV)wv[u] * rg[a];
                }
            }
        }
        for (int d = G >> 1; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d, G);
        if (c < nc && part == 0) z[core_idx[cb + c]] = acc;
    }
}


}  // namespace rbf
