// rasm.cu -- the restricted additive Schwarz preconditioner of Eq. rasm:
//     z = M^{-1} r = sum_i ~R_i^T A_i^{-1} R_i r,   A_i = R_i A~ R_i^T.
//
// Setup (one warp per subdomain): form A_i over the overlap list (Sec. 2.4:
// only the small A_i are formed), Cholesky-factor it in shared memory, and
// keep only what the restricted prolongation ~R_i^T needs: the rows of
// A_i^{-1} that belong to the core ~Omega_i,
//     W_i = ~R_i A_i^{-1} R_i^T   (n_core x n_overlap, stored column-major),
// so that the apply is one small dense GEMV per subdomain, z_core = W_i r_ov,
// with no triangular-solve dependency chain. Each point is in exactly one
// core, so every z entry is written once (no atomics, deterministic).
#include <cmath>

#include "common.cuh"

namespace rbf {
namespace {

constexpr int kSetupWarps = 4;

// Per-warp shared layout (doubles): A[n*n] | X[nc*n] | xs[n] | ys[n].
__global__ void __launch_bounds__(kSetupWarps * 32)
    k_rasm_setup(const double* __restrict__ xy_s, const int32_t* __restrict__ ov_ptr,
                 const int32_t* __restrict__ ov_idx, const int32_t* __restrict__ core_of,
                 const int32_t* __restrict__ core_ptr, const int64_t* __restrict__ w_off, int64_t nsub, int nmax,
                 int ncmax, int wpb, const Prob* __restrict__ prob, const int32_t* __restrict__ pid_sub,
                 double* __restrict__ W64, float* __restrict__ W32, int* __restrict__ status)
{
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t sub = (int64_t)blockIdx.x * wpb + warp;
    if (warp >= wpb || sub >= nsub) return;
    const Prob& pr = prob[pid_sub[sub]];
    const double rc2 = pr.rc2, s = pr.s, knorm = pr.knorm;
    const size_t per = (size_t)nmax * nmax + (size_t)ncmax * nmax + 2 * (size_t)nmax;
    double* A = sm + per * warp;
    double* X = A + (size_t)nmax * nmax;
    double* xs = X + (size_t)ncmax * nmax;
    double* ys = xs + nmax;
    __shared__ int cpos_all[kSetupWarps][kMaxSub];
    int* cpos = cpos_all[warp];

    const int b = ov_ptr[sub];
    const int n = ov_ptr[sub + 1] - b;
    const int nc = core_ptr[sub + 1] - core_ptr[sub];
    if (n == 0) return;
    for (int a = lane; a < n; a += 32) {
        int p = ov_idx[b + a];
        xs[a] = xy_s[2 * (int64_t)p];
        ys[a] = xy_s[2 * (int64_t)p + 1];
    }
    // positions of the core entries inside the overlap list (ascending)
    if (lane == 0) {
        int q = 0;
        for (int a = 0; a < n; ++a)
            if (core_of[ov_idx[b + a]] == (int32_t)sub) cpos[q++] = a;
    }
    __syncwarp();
    // A_i (lower triangle and diagonal), truncated exactly like A~
    for (int t = lane; t < n * n; t += 32) {
        int i = t / n, j = t % n;
        if (j > i) continue;
        double dx = __dsub_rn(xs[i], xs[j]), dy = __dsub_rn(ys[i], ys[j]);
        double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        A[i * n + j] = (r2 <= rc2) ? exp(-r2 * s) * knorm : 0.0;
    }
    __syncwarp();
    // right-looking Cholesky, lower triangle in place; a pivot below 1e-14 of
    // the diagonal k(0) counts as not positive definite (numerically singular,
    // e.g. two coincident points)
    bool ok = true;
    const double pivot_min = 1e-14 * knorm;
    for (int j = 0; j < n; ++j) {
        double d = A[j * n + j];
        if (!(d > pivot_min)) { ok = false; d = 1.0; }
        double ljj = sqrt(d);
        __syncwarp();
        for (int i = j + 1 + lane; i < n; i += 32) A[i * n + j] = A[i * n + j] / ljj;
        if (lane == 0) A[j * n + j] = ljj;
        __syncwarp();
        for (int i = j + 1 + lane; i < n; i += 32) {
            double lij = A[i * n + j];
            for (int kk = j + 1; kk <= i; ++kk) A[i * n + kk] -= lij * A[kk * n + j];
        }
        __syncwarp();
    }
    if (!ok) {
        if (lane == 0) atomicExch(status, RBF_ERR_NOT_SPD);
        return;
    }
    // X[c][:] = A_i^{-1} e_{cpos[c]} (= row cpos[c] of A_i^{-1}, A_i symmetric);
    // one right-hand side per lane, L read by all lanes in lockstep
    for (int c0 = 0; c0 < nc; c0 += 32) {
        int c = c0 + lane;
        bool act = c < nc;
        int cp = act ? cpos[c] : 0;
        double* x = X + (size_t)(act ? c : 0) * n;
        for (int i = 0; i < n; ++i) {                 // L y = e_cp
            double v = (i == cp) ? 1.0 : 0.0;
            for (int kk = 0; kk < i; ++kk) v -= A[i * n + kk] * (act ? x[kk] : 0.0);
            if (act) x[i] = v / A[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {            // L^T x = y
            double v = act ? x[i] : 0.0;
            for (int kk = i + 1; kk < n; ++kk) v -= A[kk * n + i] * (act ? x[kk] : 0.0);
            if (act) x[i] = v / A[i * n + i];
        }
        __syncwarp();
    }
    // W_i column-major: W[off + a * nc + c] = X[c][a]
    const int64_t off = w_off[sub];
    for (int t = lane; t < n * nc; t += 32) {
        int a = t / nc, c = t % nc;
        double v = X[(size_t)c * n + a];
        if (W64) W64[off + t] = v;
        if (W32) W32[off + t] = (float)v;
    }
}

template <class TW, class TV>
__global__ void __launch_bounds__(256)
    k_rasm_apply(const int32_t* __restrict__ ov_ptr, const int32_t* __restrict__ ov_idx,
                 const int32_t* __restrict__ core_ptr, const int32_t* __restrict__ core_idx,
                 const int64_t* __restrict__ w_off, const TW* __restrict__ W, int64_t nsub,
                 const int32_t* __restrict__ pid_sub, const int32_t* __restrict__ active, const TV* __restrict__ r,
                 TV* __restrict__ z)
{
    __shared__ TV rg_all[8][kMaxSub];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t sub = (int64_t)blockIdx.x * 8 + warp;
    if (sub >= nsub) return;
    if (active && !active[pid_sub[sub]]) return;   // masked problem (warp-uniform)
    TV* rg = rg_all[warp];
    const int b = ov_ptr[sub];
    const int n = ov_ptr[sub + 1] - b;
    const int cb = core_ptr[sub];
    const int nc = core_ptr[sub + 1] - cb;
    for (int a = lane; a < n; a += 32) rg[a] = r[ov_idx[b + a]];
    __syncwarp();
    const TW* Ws = W + w_off[sub];
    // G lanes cooperate on one core row
    int G = 1;
    while (G < 32 && nc * G * 2 <= 32) G *= 2;
    const int rows_per_pass = 32 / G;
    const int part = lane % G;
    for (int c0 = 0; c0 < nc; c0 += rows_per_pass) {
        int c = c0 + lane / G;
        TV acc = 0;
        if (c < nc)
            for (int a = part; a < n; a += G) acc += (TV)Ws[(int64_t)a * nc + c] * rg[a];
        for (int d = G >> 1; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d, G);
        if (c < nc && part == 0) z[core_idx[cb + c]] = acc;
    }
}

__global__ void k_sizes(const int32_t* __restrict__ ov_ptr, const int32_t* __restrict__ core_ptr, int64_t nsub,
                        int64_t* __restrict__ sizes)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsub) sizes[s] = (int64_t)(ov_ptr[s + 1] - ov_ptr[s]) * (core_ptr[s + 1] - core_ptr[s]);
}

}  // namespace

rbf_status rasm_factor(rbf_ctx* ctx, cudaStream_t st)
{
    const int64_t nsub = ctx->nsub;
    RBF_CHECK(ensure(ctx, ctx->w_off, nsub + 1));
    RBF_CHECK(ensure(ctx, ctx->w_size, nsub + 1));
    RBF_LAUNCH(ctx, k_sizes, blocks_for(nsub, 256), 256, 0, st, ctx->ov_ptr.p, ctx->core_ptr.p, nsub, ctx->w_size.p);
    RBF_CHECK(exclusive_scan_i64(ctx, ctx->w_size.p, ctx->w_off.p, nsub, st));
    int64_t total = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&total, ctx->w_off.p + nsub, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RBF_CHECK(ensure(ctx, ctx->status_dev, 1));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->status_dev.p, 0, sizeof(int), st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    double* W64 = nullptr;
    float* W32 = nullptr;
    if (ctx->rasm_precision == RBF_FP64) {
        RBF_CHECK(ensure(ctx, ctx->W64, (size_t)total));
        W64 = ctx->W64.p;
    } else {
        RBF_CHECK(ensure(ctx, ctx->W32, (size_t)total));
        W32 = ctx->W32.p;
    }
    const int nmax = ctx->max_ov, ncmax = ctx->max_core;
    if (nmax == 0) return RBF_OK;
    size_t per = ((size_t)nmax * nmax + (size_t)ncmax * nmax + 2 * (size_t)nmax) * sizeof(double);
    if (per > 200u * 1024u)
        return fail(ctx, RBF_ERR_SUBDOMAIN_TOO_LARGE,
                    "rbf_rasm_setup: a %d-point overlap list with %d core points needs %zu KB of shared memory", nmax,
                    ncmax, per / 1024);
    // as many warps per block as fit in 200 KB of shared memory (at most kSetupWarps)
    int wpb = (int)std::min<size_t>(kSetupWarps, std::max<size_t>(1, (200u * 1024u) / per));
    size_t smem = per * wpb;
    RBF_CUDA(ctx, cudaFuncSetAttribute(k_rasm_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBF_CHECK(prof_begin(ctx, RBF_PROF_RASM_SETUP, st));
    RBF_LAUNCH(ctx, k_rasm_setup, blocks_for(nsub, wpb), kSetupWarps * 32, smem, st, ctx->xy_s.p, ctx->ov_ptr.p,
               ctx->ov_idx.p, ctx->core_of.p, ctx->core_ptr.p, ctx->w_off.p, nsub, nmax, ncmax, wpb, ctx->prob.p,
               ctx->pid_sub.p, W64, W32, ctx->status_dev.p);
    RBF_CHECK(prof_end(ctx, RBF_PROF_RASM_SETUP, st));
    int status = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&status, ctx->status_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    if (status == RBF_ERR_NOT_SPD)
        return fail(ctx, RBF_ERR_NOT_SPD, "rbf_rasm_setup: a subdomain matrix is not positive definite");
    return RBF_OK;
}

rbf_status rasm_apply_sorted(rbf_ctx* ctx, const double* r, double* z, cudaStream_t st)
{
    RBF_CHECK(prof_begin(ctx, RBF_PROF_RASM_APPLY, st));
    if (ctx->rasm_precision == RBF_FP64)
        RBF_LAUNCH(ctx, (k_rasm_apply<double, double>), blocks_for(ctx->nsub, 8), 256, 0, st, ctx->ov_ptr.p,
                   ctx->ov_idx.p, ctx->core_ptr.p, ctx->core_idx.p, ctx->w_off.p, ctx->W64.p, ctx->nsub,
                   ctx->pid_sub.p, ctx->active_mask, r, z);
    else
        RBF_LAUNCH(ctx, (k_rasm_apply<float, double>), blocks_for(ctx->nsub, 8), 256, 0, st, ctx->ov_ptr.p,
                   ctx->ov_idx.p, ctx->core_ptr.p, ctx->core_idx.p, ctx->w_off.p, ctx->W32.p, ctx->nsub,
                   ctx->pid_sub.p, ctx->active_mask, r, z);
    return prof_end(ctx, RBF_PROF_RASM_APPLY, st);
}

rbf_status rasm_apply_sorted_f32(rbf_ctx* ctx, const float* r, float* z, cudaStream_t st)
{
    RBF_CHECK(prof_begin(ctx, RBF_PROF_RASM_APPLY, st));
    RBF_LAUNCH(ctx, (k_rasm_apply<float, float>), blocks_for(ctx->nsub, 8), 256, 0, st, ctx->ov_ptr.p, ctx->ov_idx.p,
               ctx->core_ptr.p, ctx->core_idx.p, ctx->w_off.p, ctx->W32.p, ctx->nsub, ctx->pid_sub.p,
               ctx->active_mask, r, z);
    return prof_end(ctx, RBF_PROF_RASM_APPLY, st);
}

}  // namespace rbf
