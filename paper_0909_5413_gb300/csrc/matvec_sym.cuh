// matvec_sym.cuh -- pieces of the truncated Gaussian matvec (Sec. 2.3) shared
// by the matvec kernels and the fused Arnoldi step: the kernels' parameter
// block, packed FP32 helpers, and the per-warp body of the symmetric FP32
// matvec on the inner grid.
#pragma once

#include "common.cuh"

namespace rbf {

struct MvParams {
    const double* xy;          // cell-ordered source coordinates (x, y)
    const float* loc;          // FP32 scaled offsets from the point's cell corner (x, y)
    const int32_t* cell_s;     // global cell id of each cell-ordered point
    const int32_t* cell_start;
    const int32_t* work;       // (cell, first target) per block
    // targets (the sources themselves for A~ w; other points for s(x))
    const double* txy;
    const float* tloc;
    const int32_t* tcell_start;
    const unsigned long long* fxtab;   // T1, T2 of fixexp.cuh
    const Prob* prob;          // per-problem grid and kernel constants
    const int32_t* pid_cell;   // problem of each cell
    const int32_t* active;     // per-problem mask (null: every problem)
    int stage;                 // sources staged per pass (a multiple of 32)
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Packed FP32 pairs (two lanes of work per instruction on sm_100-class SMs).
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b)
{
    unsigned long long d, A = *reinterpret_cast<unsigned long long*>(&a), B = *reinterpret_cast<unsigned long long*>(&b);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(A), "l"(B));
    return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ float2 f2_add(float2 a, float2 b)
{
    unsigned long long d, A = *reinterpret_cast<unsigned long long*>(&a), B = *reinterpret_cast<unsigned long long*>(&b);
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(A), "l"(B));
    return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ float2 f2_mul(float2 a, float2 b)
{
    unsigned long long d, A = *reinterpret_cast<unsigned long long*>(&a), B = *reinterpret_cast<unsigned long long*>(&b);
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(A), "l"(B));
    return *reinterpret_cast<float2*>(&d);
}

__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c)
{
    unsigned long long d, A = *reinterpret_cast<unsigned long long*>(&a), B = *reinterpret_cast<unsigned long long*>(&b),
                          Cc = *reinterpret_cast<unsigned long long*>(&c);
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(A), "l"(B), "l"(Cc));
    return *reinterpret_cast<float2*>(&d);
}

// Symmetric FP32 matvec on the inner grid: every unordered pair of
// neighbouring cells is visited once. One warp per cell C (at most
// kSymMaxCell points, up to four targets per lane) takes C itself (row sums
// only: all pairs inside C) and its four forward neighbours D = C + d,
// d in {(1,0), (-1,1), (0,1), (1,1)}: each kernel value k_ij (i in C, j in D)
// feeds the row sum of i (registers) and the column sum of j, which is
// reduced over the warp's targets through a shared transpose (lane j adds the
// 32 rows in order) and written to point j's slot for direction d; the warp
// also writes zeros into its own points' slots of the directions whose source
// cell is missing (off the grid or empty). The gather then adds, per point,
// its row slot and the four column slots in a fixed order: deterministic,
// with half the exp2 evaluations of the stencil sweep. Sources are staged as FP32
// offsets from C's corner (scaled so that the kernel is exp2(-|dX|^2)), in
// chunks of 32 padded with far, zero-weight sources.
constexpr int kSymWarps = 4;
constexpr int kSymMaxCell = 128;
constexpr int kSymStage = kSymMaxCell + 32;
constexpr int kSymTld = 36;   // row stride of the transpose buffer (16-byte rows, conflict-free columns)

struct SymWarp {
    float sx[kSymStage], sy[kSymStage], sw[kSymStage];
    float T[32 * kSymTld];
};

template <int TPL, bool COL>
__device__ __forceinline__ void sym_pass(SymWarp& S, int lane, const float2 (&tx)[TPL], const float2 (&ty)[TPL],
                                         const float (&wt)[TPL], float2 (&acc)[TPL], float2 (&acc2)[TPL], int dn,
                                         float* __restrict__ colout, float knorm)
{
    const int dnp = (dn + 31) & ~31;
    float4* row = reinterpret_cast<float4*>(&S.T[lane * kSymTld]);
    for (int c0 = 0; c0 < dnp; c0 += 32) {
        // steps of four sources up to the last real one (the padding sources
        // would add exact zeros; the transpose's columns past dn are not stored)
        const int smax = dn - c0;
#pragma unroll
        for (int s = 0; s < 32; s += 4) {
            if (s >= smax) break;
            const float4 X = *reinterpret_cast<const float4*>(&S.sx[c0 + s]);
            const float4 Y = *reinterpret_cast<const float4*>(&S.sy[c0 + s]);
            const float4 Wv = *reinterpret_cast<const float4*>(&S.sw[c0 + s]);
            // this lane's column terms of sources s..s+3, summed over its targets
            // in order; stored to its row of the transpose as soon as complete
            float2 c01 = make_float2(0.f, 0.f), c23 = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < TPL; ++t) {
                const float2 dx0 = f2_sub(tx[t], make_float2(X.x, X.y)), dy0 = f2_sub(ty[t], make_float2(Y.x, Y.y));
                const float2 dx1 = f2_sub(tx[t], make_float2(X.z, X.w)), dy1 = f2_sub(ty[t], make_float2(Y.z, Y.w));
                const float2 r0 = f2_fma(dy0, dy0, f2_mul(dx0, dx0));
                const float2 r1 = f2_fma(dy1, dy1, f2_mul(dx1, dx1));
                const float2 e0 = make_float2(ex2_approx(-r0.x), ex2_approx(-r0.y));
                const float2 e1 = make_float2(ex2_approx(-r1.x), ex2_approx(-r1.y));
                acc[t] = f2_fma(e0, make_float2(Wv.x, Wv.y), acc[t]);
                acc2[t] = f2_fma(e1, make_float2(Wv.z, Wv.w), acc2[t]);
                if (COL) {
                    const float2 w2 = make_float2(wt[t], wt[t]);
                    c01 = f2_fma(e0, w2, c01);
                    c23 = f2_fma(e1, w2, c23);
                }
            }
            if (COL) row[s >> 2] = make_float4(c01.x, c01.y, c23.x, c23.y);
        }
        if (COL) {
            // column sums of the transpose: lane (g, q) = (lane % 8, lane / 8)
            // adds rows 8q .. 8q + 7 of columns 4g .. 4g + 3 in order (packed
            // pairs), then the four row groups are added by a fixed shuffle
            // tree; lane (g, q) stores column 4g + q
            __syncwarp();
            const int g = lane & 7, q = lane >> 3;
            float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 v = *reinterpret_cast<const float4*>(&S.T[(8 * q + i) * kSymTld + 4 * g]);
                a01 = f2_add(a01, make_float2(v.x, v.y));
                a23 = f2_add(a23, make_float2(v.z, v.w));
            }
#pragma unroll
            for (int d = 8; d <= 16; d <<= 1) {
                a01.x += __shfl_xor_sync(0xffffffffu, a01.x, d);
                a01.y += __shfl_xor_sync(0xffffffffu, a01.y, d);
                a23.x += __shfl_xor_sync(0xffffffffu, a23.x, d);
                a23.y += __shfl_xor_sync(0xffffffffu, a23.y, d);
            }
            __syncwarp();
            const float sum = q == 0 ? a01.x : (q == 1 ? a01.y : (q == 2 ? a23.x : a23.y));
            const int col = c0 + 4 * g + q;
            if (col < dn) colout[col] = sum * knorm;
        }
    }
}

template <int TPL>
__device__ __forceinline__ void sym_cell(const MvParams& P, SymWarp& S, int lane, int cell, int cb, int cnt,
                                         const Prob& pr, const float* __restrict__ w, float* __restrict__ rowslot,
                                         float* __restrict__ colslot, int64_t n)
{
    const int ncx = (int)pr.ncx, ncy = (int)pr.ncy, cbase = (int)pr.cellbase;
    const float ca = pr.ca, knorm = (float)pr.knorm;
    const int cx = (cell - cbase) % ncx, cy = (cell - cbase) / ncx;
    float2 tx[TPL], ty[TPL], acc[TPL], acc2[TPL];
    float wt[TPL];
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int q = lane + 32 * t;
        const bool ok = q < cnt;
        const float2 l = ok ? reinterpret_cast<const float2*>(P.loc)[cb + q] : make_float2(-1.0e4f, -1.0e4f);
        tx[t] = make_float2(l.x, l.x);
        ty[t] = make_float2(l.y, l.y);
        wt[t] = ok ? w[cb + q] : 0.f;
        acc[t] = make_float2(0.f, 0.f);
        acc2[t] = make_float2(0.f, 0.f);
    }
    // slots of the backward directions whose source cell is missing (off the
    // grid or empty) get zeros, so that the gather is a plain fixed-order sum
    {
        const int bx[4] = {cx - 1, cx + 1, cx, cx - 1}, by[4] = {cy, cy - 1, cy - 1, cy - 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bool missing = bx[q] < 0 || bx[q] >= ncx || by[q] < 0;
            if (!missing) {
                const int c = cbase + by[q] * ncx + bx[q];
                missing = P.cell_start[c + 1] == P.cell_start[c];
            }
            if (missing)
                for (int t = lane; t < cnt; t += 32) colslot[(int64_t)q * n + cb + t] = 0.f;
        }
    }
#pragma unroll 1
    for (int pass = 0; pass < 5; ++pass) {
        const int dx = (pass == 1 || pass == 4) ? 1 : (pass == 2 ? -1 : 0);
        const int dy = pass >= 2 ? 1 : 0;
        const int nx = cx + dx, ny = cy + dy;
        if (nx < 0 || nx >= ncx || ny >= ncy) continue;
        const int dcell = cbase + ny * ncx + nx;
        const int db = P.cell_start[dcell], dn = P.cell_start[dcell + 1] - db;
        if (dn == 0) continue;
        const int dnp = (dn + 31) & ~31;
        for (int s = lane; s < dnp; s += 32) {
            if (s < dn) {
                const float2 l = reinterpret_cast<const float2*>(P.loc)[db + s];
                S.sx[s] = l.x + (float)dx * ca;
                S.sy[s] = l.y + (float)dy * ca;
                S.sw[s] = w[db + s];
            } else {
                S.sx[s] = 1.0e4f;
                S.sy[s] = 1.0e4f;
                S.sw[s] = 0.f;
            }
        }
        __syncwarp();
        if (pass == 0) sym_pass<TPL, false>(S, lane, tx, ty, wt, acc, acc2, dn, nullptr, knorm);
        else sym_pass<TPL, true>(S, lane, tx, ty, wt, acc, acc2, dn, colslot + (int64_t)(pass - 1) * n + db, knorm);
        __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int q = lane + 32 * t;
        if (q < cnt) rowslot[cb + q] = ((acc[t].x + acc[t].y) + (acc2[t].x + acc2[t].y)) * knorm;
    }
}

// The symmetric FP32 kernel's parameters on the inner grid and its cell list
// (every size class, the batch's compacted list when one is in use); false
// when the inner grid is off or the kernel does not apply.
bool inner_sym_params(rbf_ctx* ctx, MvParams* P, const int32_t** cells, int64_t* ncells);

}  // namespace rbf
