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

// Sum over problem pb's chunks, in chunk order, of partial[c * 32 + k] (one
// warp; the lanes take every 32nd chunk, 8 loads issued together and added in
// order, then a fixed shuffle tree); every lane returns the total.
__device__ __forceinline__ double breduce_one(const double* __restrict__ partial, const Chunks& C, int pb, int k,
                                              int lane)
{
    double a = 0.0;
    constexpr int U = 8;
    const int c1 = C.cptr[pb + 1];
    for (int c0 = C.cptr[pb] + lane; c0 < c1; c0 += 32 * U) {
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

}  // namespace rbf
