// batch.cuh -- the chunk table of the batched solver and the per-problem
// reduction of chunk partial sums, shared by the batched solver's kernels and
// the fused Arnoldi step.
#pragma once

#include "common.cuh"

namespace rbf {

enum BField { F_H1 = 0, F_H2 = 1, F_NRM2 = 2, F_BETA2 = 3, F_FNORM2 = 4 };


__device__ __forceinline__ double* field_ptr(GmresDev& g, int field)
{
    switch (field) {
    case F_H1: return g.h1;
    case F_H2: return g.h2;
    case F_NRM2: return &g.nrm2;
    case F_BETA2: return &g.beta2;
    default: return &g.fnorm2;
    }
}

struct Chunks {
    const int32_t* beg;   // first element of chunk
    const int32_t* end;   // one past the last
    const int32_t* pid;   // problem of the chunk
    const int32_t* cptr;  // chunks of problem b: [cptr[b], cptr[b+1])
    int64_t nc;
};

// Segments of a problem's chunk partials, summed one per warp and then in
// segment order: one for up to 2047 chunks, up to kRedSeg for large problems
// (a function of the problem's own chunk count only, so that every kernel
// that reduces a problem's partials sums them in the same order).
constexpr int kRedSeg = 8;

__host__ __device__ __forceinline__ int breduce_segments(int nch)
{
    const int s = nch / 1024;
    return s < 1 ? 1 : (s > kRedSeg ? kRedSeg : s);
}

// Sum of partial[c * 32 + k] over segment s of S of problem pb's chunks (one
// warp; the lanes take every 32nd chunk, 8 loads issued together and added in
// order, then a fixed shuffle tree); every lane returns the total.
__device__ __forceinline__ double breduce_seg(const double* __restrict__ partial, const Chunks& C, int pb, int k,
                                              int lane, int s, int S)
{
    const int p0 = C.cptr[pb], nch = C.cptr[pb + 1] - p0;
    const int c_beg = p0 + (int)((int64_t)nch * s / S), c1 = p0 + (int)((int64_t)nch * (s + 1) / S);
    double a = 0.0;
    constexpr int U = 8;
    for (int c0 = c_beg + lane; c0 < c1; c0 += 32 * U) {
        double p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + 32 * u;
            p[u] = c < c1 ? partial[(int64_t)c * 32 + k] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (c0 + 32 * u < c1) a += p[u];
    }
    for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
    return a;
}

// The problem's total by one warp: its segments in order (what k_breduce
// computes with a warp per segment).
__device__ __forceinline__ double breduce_one(const double* __restrict__ partial, const Chunks& C, int pb, int k,
                                              int lane)
{
    const int S = breduce_segments(C.cptr[pb + 1] - C.cptr[pb]);
    double t = 0.0;
    for (int s = 0; s < S; ++s) t += breduce_seg(partial, C, pb, k, lane, s, S);
    return t;
}

}  // namespace rbf
