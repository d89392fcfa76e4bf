// ortho.cuh -- per-chunk device code of the classical Gram-Schmidt passes (with
// one reorthogonalisation for FP64 bases) used by the Arnoldi process of GMRES (Sec. 2.2),
// shared by the single-problem and the batched solvers so that both sum in
// the same order.
//
// A chunk is a range [b, e) of at most kOrthoChunk elements, one block of
// kDotThreads threads; thread t owns elements b + t + u * kDotThreads,
// u < kOrthoPer, and keeps them in registers for the whole pass. Per element
// the basis vectors are applied in index order (x -= c_k V_k, k = 0, 1, ...);
// per thread the products of a dot are summed over u in order, then over the
// block by a fixed shuffle tree and the warps in order. The loads of G basis
// vectors are issued together, so that one memory latency covers G vectors.
#pragma once

#include "vecops.cuh"

namespace rbf {

constexpr int kOrthoPer = 16;                            // elements per thread
constexpr int kOrthoChunk = kDotThreads * kOrthoPer;    // elements per chunk
constexpr int kOrthoWarps = kDotThreads / 32;

// FP32 vectors carry the update in double-float; FP64 vectors in FP64.
template <class T>
struct OrthoAcc {
    using type = double;
};
template <>
struct OrthoAcc<float> {
    using type = DF;
};

// Update coefficients of one pass, staged in shared memory: the FP64 value and
// its split into a float pair (FP32 vectors).
struct OrthoCoef {
    double c[kMaxRestart + 1];
    float hi[kMaxRestart + 1], lo[kMaxRestart + 1];
};

__device__ __forceinline__ void ortho_coef_set(OrthoCoef& cf, int k, double v)
{
    cf.c[k] = v;
    const float h = (float)v;
    cf.hi[k] = h;
    cf.lo[k] = (float)(v - (double)h);
}

// Shared scratch of the per-vector block sums.
struct OrthoRed {
    double d[(kMaxRestart + 1) * kOrthoWarps];
    DF f[(kMaxRestart + 1) * kOrthoWarps];
};

template <class T>
__device__ __forceinline__ void ortho_load_x(typename OrthoAcc<T>::type (&xl)[kOrthoPer], const T* __restrict__ x,
                                             int64_t b, int64_t e)
{
#pragma unroll
    for (int u = 0; u < kOrthoPer; ++u) {
        const int64_t i = b + threadIdx.x + (int64_t)u * kDotThreads;
        if constexpr (sizeof(T) == 4) {
            xl[u].hi = i < e ? x[i] : 0.f;
            xl[u].lo = 0.f;
        } else {
            xl[u] = i < e ? (double)x[i] : 0.0;
        }
    }
}

// One element of x -= c V_k.
__device__ __forceinline__ void ortho_axpy(DF& xl, float ch, float cl, float vi)
{
    const float h = ch * vi;
    const float r = fmaf(ch, vi, -h);
    df_add(xl, -h, fmaf(-cl, vi, -r));
}
__device__ __forceinline__ void ortho_axpy(double& xl, double c, double vi) { xl = fma(-c, vi, xl); }

// x -= sum_{k < nv} c_k V_k over the thread's elements, G vectors per load batch.
template <class T, int G>
__device__ __forceinline__ void ortho_apply(typename OrthoAcc<T>::type (&xl)[kOrthoPer], const T* __restrict__ V,
                                            int64_t ldv, int nv, const OrthoCoef& cf, int64_t b, int64_t e)
{
    const int64_t i0 = b + threadIdx.x;
    int k = 0;
    for (; k + G <= nv; k += G) {
        T vv[G][kOrthoPer];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const T* v = V + (int64_t)(k + g) * ldv;
#pragma unroll
            for (int u = 0; u < kOrthoPer; ++u) {
                const int64_t i = i0 + (int64_t)u * kDotThreads;
                vv[g][u] = i < e ? v[i] : (T)0;
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
#pragma unroll
            for (int u = 0; u < kOrthoPer; ++u) {
                const int64_t i = i0 + (int64_t)u * kDotThreads;
                if (i < e) {
                    if constexpr (sizeof(T) == 4) ortho_axpy(xl[u], cf.hi[k + g], cf.lo[k + g], vv[g][u]);
                    else ortho_axpy(xl[u], cf.c[k + g], vv[g][u]);
                }
            }
        }
    }
    for (; k < nv; ++k) {
        const T* v = V + (int64_t)k * ldv;
        T vv[kOrthoPer];
#pragma unroll
        for (int u = 0; u < kOrthoPer; ++u) {
            const int64_t i = i0 + (int64_t)u * kDotThreads;
            vv[u] = i < e ? v[i] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < kOrthoPer; ++u) {
            const int64_t i = i0 + (int64_t)u * kDotThreads;
            if (i < e) {
                if constexpr (sizeof(T) == 4) ortho_axpy(xl[u], cf.hi[k], cf.lo[k], vv[u]);
                else ortho_axpy(xl[u], cf.c[k], vv[u]);
            }
        }
    }
}

// Rounds the updated elements to T, stores them, keeps the rounded values in xs.
template <class T>
__device__ __forceinline__ void ortho_store_x(const typename OrthoAcc<T>::type (&xl)[kOrthoPer], T (&xs)[kOrthoPer],
                                              T* __restrict__ x, int64_t b, int64_t e)
{
#pragma unroll
    for (int u = 0; u < kOrthoPer; ++u) {
        const int64_t i = b + threadIdx.x + (int64_t)u * kDotThreads;
        if constexpr (sizeof(T) == 4) xs[u] = xl[u].hi + xl[u].lo;
        else xs[u] = xl[u];
        if (i < e) x[i] = xs[u];
    }
}

// Per-thread dot of the thread's elements (FP32: Dot2; FP64: FMA chain).
template <class T>
__device__ __forceinline__ typename OrthoAcc<T>::type ortho_thread_dot(const T (&a)[kOrthoPer],
                                                                       const T (&xs)[kOrthoPer], int64_t b, int64_t e)
{
    const int64_t i0 = b + threadIdx.x;
    if constexpr (sizeof(T) == 4) {
        DF s{0.f, 0.f};
#pragma unroll
        for (int u = 0; u < kOrthoPer; ++u)
            if (i0 + (int64_t)u * kDotThreads < e) df_add_prod(s, a[u], xs[u]);
        return s;
    } else {
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < kOrthoPer; ++u)
            if (i0 + (int64_t)u * kDotThreads < e) s = fma(a[u], xs[u], s);
        return s;
    }
}

// Warp stage of the block sum of slot k: shuffle tree, lane 0 stores the
// warp's value. (The order is that of block_sum / block_sum_df.)
__device__ __forceinline__ void ortho_warp_sum(DF s, OrthoRed& red, int k)
{
    for (int d = 16; d > 0; d >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, s.hi, d), ol = __shfl_xor_sync(0xffffffffu, s.lo, d);
        df_merge(s, oh, ol);
    }
    if ((threadIdx.x & 31) == 0) red.f[k * kOrthoWarps + (threadIdx.x >> 5)] = s;
}
__device__ __forceinline__ void ortho_warp_sum(double a, OrthoRed& red, int k)
{
    for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
    if ((threadIdx.x & 31) == 0) red.d[k * kOrthoWarps + (threadIdx.x >> 5)] = a;
}

// Block stage (after a barrier): the warps of slot k in order, as FP64.
template <class T>
__device__ __forceinline__ double ortho_block_total(const OrthoRed& red, int k)
{
    if constexpr (sizeof(T) == 4) {
        DF t = red.f[k * kOrthoWarps];
        for (int w = 1; w < kOrthoWarps; ++w) df_merge(t, red.f[k * kOrthoWarps + w].hi, red.f[k * kOrthoWarps + w].lo);
        return (double)t.hi + (double)t.lo;
    } else {
        double s = 0.0;
        for (int w = 0; w < kOrthoWarps; ++w) s += red.d[k * kOrthoWarps + w];
        return s;
    }
}

// out[k] = V_k . xs over the chunk for k < nv (block sums, written by threads
// k < nv), G vectors per load batch. Ends with a barrier.
template <class T, int G>
__device__ __forceinline__ void ortho_dots(const T* __restrict__ V, int64_t ldv, int nv, const T (&xs)[kOrthoPer],
                                           int64_t b, int64_t e, OrthoRed& red, double* __restrict__ out)
{
    const int64_t i0 = b + threadIdx.x;
    int k = 0;
    for (; k + G <= nv; k += G) {
        T vv[G][kOrthoPer];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const T* v = V + (int64_t)(k + g) * ldv;
#pragma unroll
            for (int u = 0; u < kOrthoPer; ++u) {
                const int64_t i = i0 + (int64_t)u * kDotThreads;
                vv[g][u] = i < e ? v[i] : (T)0;
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) ortho_warp_sum(ortho_thread_dot<T>(vv[g], xs, b, e), red, k + g);
    }
    for (; k < nv; ++k) {
        const T* v = V + (int64_t)k * ldv;
        T vv[kOrthoPer];
#pragma unroll
        for (int u = 0; u < kOrthoPer; ++u) {
            const int64_t i = i0 + (int64_t)u * kDotThreads;
            vv[u] = i < e ? v[i] : (T)0;
        }
        ortho_warp_sum(ortho_thread_dot<T>(vv, xs, b, e), red, k);
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)nv) out[threadIdx.x] = ortho_block_total<T>(red, (int)threadIdx.x);
    __syncthreads();
}

// *out = v . x over the chunk (one block per chunk and basis vector; the
// order of ortho_dots).
template <class T>
__device__ __forceinline__ void ortho_dot_one(const T* __restrict__ v, const T* __restrict__ x, int64_t b, int64_t e,
                                              OrthoRed& red, double* __restrict__ out)
{
    T a[kOrthoPer], xs[kOrthoPer];
#pragma unroll
    for (int u = 0; u < kOrthoPer; ++u) {
        const int64_t i = b + threadIdx.x + (int64_t)u * kDotThreads;
        a[u] = i < e ? v[i] : (T)0;
        xs[u] = i < e ? x[i] : (T)0;
    }
    ortho_warp_sum(ortho_thread_dot<T>(a, xs, b, e), red, 0);
    __syncthreads();
    if (threadIdx.x == 0) *out = ortho_block_total<T>(red, 0);
}

// Gram-Schmidt passes per Arnoldi step: FP64 bases (the outer solves, to
// 1e-13) are orthogonalised twice (CGS2); FP32 bases (the inner solves of
// the mixed form, to about 1e-5) once, classical Gram-Schmidt without
// refinement.
template <class T>
constexpr int gs_passes()
{
    return sizeof(T) == 4 ? 1 : 2;
}

// Arnoldi step j for one problem, run by one warp (j < kMaxRestart): column j
// of the Hessenberg matrix from the Gram-Schmidt coefficients (the sum of
// both passes when there are two) and |w|, the
// earlier Givens rotations applied to it, the new rotation, the rotated
// right-hand side g and the residual estimate |g_{j+1}| / |f|. The rotation
// chain runs in lane 0 on shared copies (one block per problem).
// The same with the warp's shared scratch passed in (hc: kMaxRestart + 1
// entries, cs and sn: kMaxRestart), for several warps of a block at once.
__device__ __forceinline__ void arnoldi_column_s(GmresDev* __restrict__ g, int j, int passes, double* hc, double* cs,
                                                 double* sn)
{
    const int lane = threadIdx.x & 31;
    const int M = kMaxRestart;
    for (int q = lane; q <= j; q += 32) hc[q] = passes == 2 ? g->h1[q] + g->h2[q] : g->h1[q];
    for (int q = lane; q < j; q += 32) {
        cs[q] = g->cs[q];
        sn[q] = g->sn[q];
    }
    __syncwarp();
    if (lane == 0) {
        const double hn = sqrt(fmax(g->nrm2, 0.0));
        double a = hc[0];
        for (int q = 0; q < j; ++q) {
            const double b = hc[q + 1];
            hc[q] = cs[q] * a + sn[q] * b;
            a = -sn[q] * a + cs[q] * b;
        }
        const double b = hn;
        double c, s;
        if (b == 0.0) { c = 1.0; s = 0.0; }
        else if (fabs(b) > fabs(a)) { double t = a / b; s = 1.0 / sqrt(1.0 + t * t); c = s * t; }
        else { double t = b / a; c = 1.0 / sqrt(1.0 + t * t); s = c * t; }
        g->cs[j] = c;
        g->sn[j] = s;
        hc[j] = c * a + s * b;
        hc[j + 1] = 0.0;
        const double gj = g->g[j];
        g->g[j + 1] = -s * gj;
        g->g[j] = c * gj;
        g->inv_h = hn > 0.0 ? 1.0 / hn : 0.0;
        g->breakdown = (hn == 0.0) ? 1 : 0;
        g->est = fabs(-s * gj) / sqrt(g->fnorm2);
    }
    __syncwarp();
    for (int q = lane; q <= j + 1; q += 32) g->H[q * M + j] = hc[q];
}

__device__ __forceinline__ void arnoldi_column(GmresDev* __restrict__ g, int j, int passes)
{
    __shared__ double hc[kMaxRestart + 1], cs[kMaxRestart], sn[kMaxRestart];
    arnoldi_column_s(g, j, passes, hc, cs, sn);
}

// Load-batch width per precision (registers: G x kOrthoPer values of T).
template <class T>
constexpr int ortho_group()
{
    return sizeof(T) == 4 ? 4 : 2;
}

}  // namespace rbf
