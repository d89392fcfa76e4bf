// rasm_tc.cu -- FP32 subdomain inverses for the mixed form on the tensor cores.
//
// The restricted Schwarz preconditioner of Eq. rasm needs, per subdomain, the
// rows of A_i^{-1} that belong to the core (W_i = ~R_i A_i^{-1} R_i^T). In the
// mixed form these serve only the FP32 inner solves, so they are computed in
// FP32 here, with the dense work on the tensor pipe:
//
//   * A_i is formed over the overlap list in FP32: offsets from the list's
//     first point scaled so that the kernel is exp2(-|d|^2), the pair test
//     |d|^2 <= r_c^2 in those units, exp2 on the SFU (the entries carry a few
//     FP32 roundings, below the FP32 inverse's own error, which the
//     conditioning of A_i sets), and padded with an identity block to
//     Np = 8 ceil(n / 8) <= 48;
//   * A_i^{-1} comes from the block sweep (Gauss-Jordan elimination without
//     pivoting, which is stable on SPD matrices: its pivots are the Schur
//     complements): for each 8 x 8 diagonal block K in turn,
//         D = A_KK^{-1}                 (a scalar sweep of the 8 x 8 block, CUDA cores)
//         U = A_:K D                    (one MMA per 16 rows)
//         A_ij -= U_i A_jK^T, i, j not in K  (the rank-8 update, MMAs over the matrix)
//         A_:K = U, A_K: = U^T, A_KK = -D,
//     after which the matrix holds -A_i^{-1};
//   * every product is a warp-level mma.sync m16n8k8 on TF32 operands with
//     FP32 accumulation, each FP32 operand split into a TF32 high part and a
//     TF32 remainder (3 MMAs per product: lo x hi, hi x lo, hi x hi), which
//     keeps FP32 accuracy (Henry, Tang and Heinecke's three-term split,
//     "Leveraging the bfloat16 artificial intelligence datatype for
//     higher-precision computations", ARITH 2019, applied to TF32).
//
// One warp per subdomain, the matrix in shared memory (rows of 52 floats: the
// fragment loads of the MMA operands then touch 32 distinct banks). A
// subdomain with more than 48 overlap points, or whose FP32 pivot is not
// positive, is appended to a list and recomputed by the FP64 kernel.
#include <cmath>

#include "common.cuh"

namespace rbf {
namespace {

constexpr int kTcMax = 48;      // largest overlap list of the tensor-core path
constexpr int kTcLd = 52;       // row stride of the shared matrix (floats)
constexpr int kTcUld = 12;      // row stride of the panel U
constexpr int kTcWarps = 4;     // warps (subdomains) per block

// Per-warp shared layout (floats unless noted).
struct TcWarp {
    float A[kTcMax * kTcLd];
    float U[kTcMax * kTcUld];
    float P[64];                 // the 8 x 8 pivot block, swept in place
    float fx[kTcMax], fy[kTcMax];   // scaled offsets from the list's first point
    int cpos[kTcMax];
};

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo with both parts TF32.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo)
{
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// d += a b in FP32 accuracy from TF32 parts (small terms first).
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                           const uint32_t (&bh)[2], const uint32_t (&bl)[2])
{
    mma_tf32(d, al, bh);
    mma_tf32(d, ah, bl);
    mma_tf32(d, ah, bh);
}

// Operand A (16 x 8, row-major, stride ld) of m16n8k8: lane (g = lane / 4,
// t = lane % 4) holds (g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4).
__device__ __forceinline__ void load_a(const float* __restrict__ M, int ld, int lane, uint32_t (&hi)[4],
                                       uint32_t (&lo)[4])
{
    const int g = lane >> 2, t = lane & 3;
    split_tf32(M[g * ld + t], hi[0], lo[0]);
    split_tf32(M[(g + 8) * ld + t], hi[1], lo[1]);
    split_tf32(M[g * ld + t + 4], hi[2], lo[2]);
    split_tf32(M[(g + 8) * ld + t + 4], hi[3], lo[3]);
}

// Operand B (8 x 8, k x n) given as B[k][n] = S[n * ld + k] (the transpose of
// a row-major block S): lane holds (k = t, n = g) and (k = t + 4, n = g).
__device__ __forceinline__ void load_bt(const float* __restrict__ S, int ld, int lane, uint32_t (&hi)[2],
                                        uint32_t (&lo)[2])
{
    const int g = lane >> 2, t = lane & 3;
    split_tf32(S[g * ld + t], hi[0], lo[0]);
    split_tf32(S[g * ld + t + 4], hi[1], lo[1]);
}

// Accumulator (16 x 8, row-major, stride ld): (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1).
__device__ __forceinline__ void load_c(const float* __restrict__ M, int ld, int lane, float (&c)[4])
{
    const int g = lane >> 2, t = lane & 3;
    c[0] = M[g * ld + 2 * t];
    c[1] = M[g * ld + 2 * t + 1];
    c[2] = M[(g + 8) * ld + 2 * t];
    c[3] = M[(g + 8) * ld + 2 * t + 1];
}

__device__ __forceinline__ void store_c(float* __restrict__ M, int ld, int lane, const float (&c)[4])
{
    const int g = lane >> 2, t = lane & 3;
    M[g * ld + 2 * t] = c[0];
    M[g * ld + 2 * t + 1] = c[1];
    M[(g + 8) * ld + 2 * t] = c[2];
    M[(g + 8) * ld + 2 * t + 1] = c[3];
}

__global__ void __launch_bounds__(kTcWarps * 32)
    k_rasm_setup_tc(const double* __restrict__ xy_s, const int32_t* __restrict__ ov_ptr,
                    const int32_t* __restrict__ ov_idx, const int32_t* __restrict__ core_of,
                    const int32_t* __restrict__ core_ptr, const int64_t* __restrict__ w_off, int64_t nsub,
                    const Prob* __restrict__ prob, const int32_t* __restrict__ pid_sub, int full,
                    float* __restrict__ W32,
                    int32_t* __restrict__ fb_list, unsigned int* __restrict__ fb_count)
{
    extern __shared__ __align__(16) unsigned char tc_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t sub = (int64_t)blockIdx.x * kTcWarps + warp;
    if (sub >= nsub) return;
    TcWarp& S = reinterpret_cast<TcWarp*>(tc_smem)[warp];
    const int b = ov_ptr[sub];
    const int n = ov_ptr[sub + 1] - b;
    if (n == 0) return;
    if (n > kTcMax) {   // beyond the shared matrix: the FP64 kernel takes it
        if (lane == 0) fb_list[atomicAdd(fb_count, 1u)] = (int32_t)sub;
        return;
    }
    const Prob& pr = prob[pid_sub[sub]];
    const double al = (double)pr.a_loc;
    const float rc2s = (float)(pr.rc2 * al * al), knorm = (float)pr.knorm;
    const int np = (n + 7) & ~7;   // padded order
    const int nb = np >> 3;
    {
        const int p0 = ov_idx[b];
        const double x0 = xy_s[2 * (int64_t)p0], y0 = xy_s[2 * (int64_t)p0 + 1];
        for (int a = lane; a < n; a += 32) {
            const int p = ov_idx[b + a];
            S.fx[a] = (float)((xy_s[2 * (int64_t)p] - x0) * al);
            S.fy[a] = (float)((xy_s[2 * (int64_t)p + 1] - y0) * al);
        }
    }
    // kept rows (ascending positions in the overlap list)
    int nkept = 0;
    for (int a0 = 0; a0 < n; a0 += 32) {
        const int a = a0 + lane;
        const bool keep = a < n && (full || core_of[ov_idx[b + a]] == (int32_t)sub);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) S.cpos[nkept + __popc(m & ((1u << lane) - 1u))] = a;
        nkept += __popc(m);
    }
    // the matrix: zero rows beyond np (read by the last 16-row tile), identity padding
    for (int e = lane; e < kTcMax * kTcLd; e += 32) {
        const int r = e / kTcLd, c = e - r * kTcLd;
        S.A[e] = (r >= n && r == c) ? 1.0f : 0.0f;
    }
    __syncwarp();
    // A_i: lower triangle by packed index over the lanes, mirrored (FP32 pair
    // test and kernel value in the scaled units)
    {
        const int total = n * (n + 1) / 2;
        int i = 0, j = lane;
        while (j > i) { j -= i + 1; ++i; }
        for (int t = lane; t < total; t += 32) {
            const float dx = S.fx[i] - S.fx[j], dy = S.fy[i] - S.fy[j];
            const float r2 = fmaf(dy, dy, dx * dx);
            float v = 0.f;
            if (r2 <= rc2s) {
                float e;
                asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-r2));
                v = e * knorm;
            }
            S.A[i * kTcLd + j] = v;
            S.A[j * kTcLd + i] = v;
            j += 32;
            while (j > i) { j -= i + 1; ++i; }
        }
    }
    __syncwarp();
    const int mtiles = (np + 15) >> 4;
    const float piv_min = (float)(1e-9 * knorm);
    bool ok = true;
    for (int kb = 0; kb < nb && ok; ++kb) {
        const int k0 = kb * 8;
        // (1) scalar sweep of the pivot block: P = -A_KK^{-1}; lane owns entries lane, lane + 32
        for (int e = lane; e < 64; e += 32) S.P[e] = S.A[(k0 + (e >> 3)) * kTcLd + k0 + (e & 7)];
        __syncwarp();
        for (int p = 0; p < 8; ++p) {
            const float piv = S.P[p * 8 + p];
            if (!(piv > piv_min)) { ok = false; break; }   // warp-uniform
            const float d = 1.0f / piv;
            float nv[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int e = lane + 32 * h, r = e >> 3, c = e & 7;
                const float v = S.P[e];
                if (r == p && c == p) nv[h] = -d;
                else if (r == p || c == p) nv[h] = v * d;
                else nv[h] = v - S.P[r * 8 + p] * S.P[p * 8 + c] * d;
            }
            __syncwarp();
            S.P[lane] = nv[0];
            S.P[lane + 32] = nv[1];
            __syncwarp();
        }
        if (!ok) break;
        // (2) U' = A_:K P = -A_:K D, 16 rows per MMA tile
        {
            uint32_t bh[2], bl[2];
            {   // B[k][n] = P[k][n]: P is symmetric, so the transposed load reads the same values
                load_bt(S.P, 8, lane, bh, bl);
            }
            for (int mt = 0; mt < mtiles; ++mt) {
                uint32_t ah[4], al[4];
                load_a(S.A + (mt * 16) * kTcLd + k0, kTcLd, lane, ah, al);
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma_3xtf32(c, ah, al, bh, bl);
                store_c(S.U + (mt * 16) * kTcUld, kTcUld, lane, c);
            }
        }
        __syncwarp();
        // (3) A_ij += U'_i A_jK^T for column blocks j != K (rows of block K are overwritten next)
        for (int mt = 0; mt < mtiles; ++mt) {
            uint32_t ah[4], al[4];
            load_a(S.U + (mt * 16) * kTcUld, kTcUld, lane, ah, al);
            for (int nt = 0; nt < nb; ++nt) {
                if (nt == kb) continue;
                uint32_t bh[2], bl[2];
                load_bt(S.A + (nt * 8) * kTcLd + k0, kTcLd, lane, bh, bl);
                float c[4];
                load_c(S.A + (mt * 16) * kTcLd + nt * 8, kTcLd, lane, c);
                mma_3xtf32(c, ah, al, bh, bl);
                store_c(S.A + (mt * 16) * kTcLd + nt * 8, kTcLd, lane, c);
            }
        }
        __syncwarp();
        // (4) A_:K = U = -U', A_K: = U^T, A_KK = P (= -D)
        for (int e = lane; e < np * 8; e += 32) {
            const int i = e >> 3, c = e & 7;
            if (i >= k0 && i < k0 + 8) continue;
            const float u = -S.U[i * kTcUld + c];
            S.A[i * kTcLd + k0 + c] = u;
            S.A[(k0 + c) * kTcLd + i] = u;
        }
        for (int e = lane; e < 64; e += 32) S.A[(k0 + (e >> 3)) * kTcLd + k0 + (e & 7)] = S.P[e];
        __syncwarp();
    }
    if (!ok) {   // a pivot that FP32 cannot resolve: the FP64 kernel takes the subdomain
        if (lane == 0) fb_list[atomicAdd(fb_count, 1u)] = (int32_t)sub;
        return;
    }
    // W_i[a][c] = (A_i^{-1})[cpos[c]][a] = -A[cpos[c]][a], column-major over a (coalesced)
    const int nc = full ? n : nkept;
    const int64_t off = w_off[sub];
    for (int e = lane; e < n * nc; e += 32) {
        const int a = e / nc, c = e - a * nc;
        W32[off + e] = -S.A[S.cpos[c] * kTcLd + a];
    }
}

}  // namespace

// FP32 inverses of every subdomain on the tensor cores; the subdomains it
// leaves (over 48 points, or a failing FP32 pivot) are listed in fb_list and
// counted in *fb_host.
rbf_status rasm_factor_tc(rbf_ctx* ctx, int32_t* fb_list, unsigned int* fb_count_dev, int64_t* fb_host,
                          cudaStream_t st)
{
    const int64_t nsub = ctx->nsub;
    const size_t smem = sizeof(TcWarp) * kTcWarps;
    RBF_CUDA(ctx, cudaFuncSetAttribute(k_rasm_setup_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBF_CUDA(ctx, cudaMemsetAsync(fb_count_dev, 0, sizeof(unsigned int), st));
    RBF_LAUNCH(ctx, k_rasm_setup_tc, blocks_for(nsub, kTcWarps), kTcWarps * 32, smem, st, ctx->xy_s.p, ctx->ov_ptr.p,
               ctx->ov_idx.p, ctx->core_of.p, ctx->core_ptr.p, ctx->w_off.p, nsub, ctx->prob.p, ctx->pid_sub.p,
               ctx->rasm_additive ? 1 : 0, ctx->W32.p, fb_list, fb_count_dev);
    unsigned int cnt = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&cnt, fb_count_dev, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    *fb_host = cnt;
    return RBF_OK;
}

}  // namespace rbf
