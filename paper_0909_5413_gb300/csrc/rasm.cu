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
//
// The plain additive Schwarz method of Eq. asm (kept for the comparison the
// paper makes between the two) stores the full A_i^{-1} (n x n) and adds
// every overlap entry back: the per-subdomain GEMV writes u_i = A_i^{-1} r_i
// to a scratch copy of the overlap lists, and a gather sums, for each point,
// its entries in subdomain order (deterministic, no atomics).
#include <cmath>

#include "common.cuh"
#include "apply.cuh"

namespace rbf {
namespace {

constexpr int kSetupWarps = 4;

// Packed lower triangle: row i starts at i (i + 1) / 2.
__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Shared layout per warp (8-byte words): L[nmax (nmax + 1) / 2] | X[32 * xs] | px | py | pxf | pyf |
// dinv (nmax each), xs = nmax rounded up to odd (conflict-free column buffers, one per lane).
__host__ __device__ inline size_t setup_doubles(int nmax)
{
    const size_t xs = (size_t)(nmax | 1);
    return (size_t)nmax * (nmax + 1) / 2 + 32 * xs + 5 * (size_t)nmax;
}

constexpr size_t kSetupSmemMax = 216u * 1024u;   // per warp (the block also holds cpos and the driver's 1 KB)

__global__ void __launch_bounds__(kSetupWarps * 32)
    k_rasm_setup(const double* __restrict__ xy_s, const int32_t* __restrict__ ov_ptr,
                 const int32_t* __restrict__ ov_idx, const int32_t* __restrict__ core_of,
                 const int32_t* __restrict__ core_ptr, const int64_t* __restrict__ w_off, int64_t nsub, int nmax,
                 int wpb, const Prob* __restrict__ prob, const int32_t* __restrict__ pid_sub, int full,
                 const unsigned long long* __restrict__ fxtab, double* __restrict__ W64, float* __restrict__ W32,
                 int* __restrict__ status, const int32_t* __restrict__ sub_list)
{
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t idx = (int64_t)blockIdx.x * wpb + warp;
    if (warp >= wpb || idx >= nsub) return;
    const int64_t sub = sub_list ? (int64_t)sub_list[idx] : idx;   // sub_list: the subdomains to factor
    const Prob& pr = prob[pid_sub[sub]];
    const double rc2 = pr.rc2, s = pr.s, knorm = pr.knorm;
    const int xstride = nmax | 1;
    double* A = sm + setup_doubles(nmax) * warp;
    double* X = A + (size_t)nmax * (nmax + 1) / 2;
    double* px = X + 32 * (size_t)xstride;
    double* py = px + nmax;
    long long* pxf = (long long*)(py + nmax);
    long long* pyf = pxf + nmax;
    double* dinv = (double*)(pyf + nmax);
    const double fxs = pr.fx_scale;
    const int sh = pr.fx_sh, F = pr.fx_F;
    const unsigned long long M = pr.fx_M;
    __shared__ int cpos_all[kSetupWarps][kMaxSub];
    int* cpos = cpos_all[warp];

    const int b = ov_ptr[sub];
    const int n = ov_ptr[sub + 1] - b;
    const int nc = full ? n : core_ptr[sub + 1] - core_ptr[sub];   // full: every overlap row
    if (n == 0) return;
    for (int a = lane; a < n; a += 32) {
        int p = ov_idx[b + a];
        px[a] = xy_s[2 * (int64_t)p];
        py[a] = xy_s[2 * (int64_t)p + 1];
        pxf[a] = fx_coord(px[a], fxs, sh);
        pyf[a] = fx_coord(py[a], fxs, sh);
    }
    // positions of the kept rows inside the overlap list (ascending): flags,
    // then a ballot prefix count per group of 32
    int nkept = 0;
    for (int a0 = 0; a0 < n; a0 += 32) {
        const int a = a0 + lane;
        const bool keep = a < n && (full || core_of[ov_idx[b + a]] == (int32_t)sub);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) cpos[nkept + __popc(m & ((1u << lane) - 1u))] = a;
        nkept += __popc(m);
    }
    __syncwarp();
    // A_i (lower triangle and diagonal): the entries of A~ itself, truncated by
    // the same FP64 pair test and valued by the same fixed-point evaluation as
    // the FP64 matvec, so A_i = R_i A~ R_i^T holds for the operator the GPU
    // applies. The packed index t = i (i + 1) / 2 + j runs over the lanes.
    (void)s;
    {
        const int total = n * (n + 1) / 2;
        int i = 0, j = lane;
        while (j > i) { j -= i + 1; ++i; }
        for (int t = lane; t < total; t += 32) {
            double dx = __dsub_rn(px[i], px[j]), dy = __dsub_rn(py[i], py[j]);
            double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            double v = 0.0;
            if (r2 <= rc2) {
                const long long du = (long long)((unsigned long long)pxf[i] - (unsigned long long)pxf[j]);
                const long long dv = (long long)((unsigned long long)pyf[i] - (unsigned long long)pyf[j]);
                v = (F == 52 ? kernel_fx52(du, dv, M, fxtab, fxtab + kFxTab)
                             : kernel_fx(du, dv, F, M, fxtab, fxtab + kFxTab)) * knorm;
            }
            A[t] = v;
            j += 32;
            while (j > i) { j -= i + 1; ++i; }
        }
    }
    __syncwarp();
    // right-looking Cholesky, lower triangle in place; a pivot below 1e-14 of
    // the diagonal k(0) counts as not positive definite (numerically singular,
    // e.g. two coincident points). The trailing update of step j runs over
    // the packed pairs (i, k), j < k <= i, spread over the lanes.
    bool ok = true;
    const double pivot_min = 1e-14 * knorm;
    for (int j = 0; j < n; ++j) {
        double d = A[tri(j, j)];
        if (!(d > pivot_min)) { ok = false; d = 1.0; }
        const double inv = rsqrt(d), ljj = d * inv;
        __syncwarp();
        for (int i = j + 1 + lane; i < n; i += 32) A[tri(i, j)] = A[tri(i, j)] * inv;
        if (lane == 0) {
            A[tri(j, j)] = ljj;
            dinv[j] = inv;
        }
        __syncwarp();
        const int m = n - 1 - j, total = m * (m + 1) / 2;
        int ii = 0, kk = lane;
        while (kk > ii) { kk -= ii + 1; ++ii; }
        for (int t = lane; t < total; t += 32) {
            const int i = j + 1 + ii, k = j + 1 + kk;
            A[tri(i, k)] -= A[tri(i, j)] * A[tri(k, j)];
            kk += 32;
            while (kk > ii) { kk -= ii + 1; ++ii; }
        }
        __syncwarp();
    }
    if (!ok) {
        if (lane == 0) atomicExch(status, RBF_ERR_NOT_SPD);
        return;
    }
    // Kept rows of A_i^{-1}: column c solves L L^T x = e_{cpos[c]} (= row
    // cpos[c] of A_i^{-1}, A_i symmetric) in its own column buffer, L read by
    // all lanes in lockstep. With at most 16 kept rows per pass, two lanes
    // share a column (even / odd terms of each row sum, combined by a
    // shuffle; both lanes write every entry, so each reads its own writes);
    // the forward solve starts at the pass's first unit position (the
    // entries above it are zero). The warp then writes the pass to W_i,
    // stored column-major (W[off + a * nc + c] = x_c[a]).
    const int64_t off = w_off[sub];
    const int Lc = nc <= 16 ? 2 : 1;
    const int per_pass = 32 / Lc;
    const int h = lane % Lc;
    double* x = X + (size_t)(lane / Lc) * xstride;
    for (int c0 = 0; c0 < nc; c0 += per_pass) {
        const int c = c0 + lane / Lc;
        const bool act = c < nc;
        const int cp = act ? cpos[c] : n;
        const int cpmin = __reduce_min_sync(0xffffffffu, cp);
        for (int i = 0; i < cpmin; ++i) x[i] = 0.0;
        for (int i = cpmin; i < n; ++i) {            // L y = e_cp
            double sum = 0.0;
            for (int k = cpmin + h; k < i; k += Lc) sum = fma(A[tri(i, k)], x[k], sum);
            if (Lc == 2) sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            x[i] = ((i == cp ? 1.0 : 0.0) - sum) * dinv[i];
        }
        for (int i = n - 1; i >= 0; --i) {           // L^T x = y
            double sum = 0.0;
            for (int k = i + 1 + h; k < n; k += Lc) sum = fma(A[tri(k, i)], x[k], sum);
            if (Lc == 2) sum += __shfl_xor_sync(0xffffffffu, sum, 1);
            x[i] = (x[i] - sum) * dinv[i];
        }
        if (act)
            for (int a = h; a < n; a += Lc) {
                const double v = x[a];
                if (W64) W64[off + (int64_t)a * nc + c] = v;
                if (W32) W32[off + (int64_t)a * nc + c] = (float)v;
            }
        __syncwarp();
    }
}

template <class TW, class TV>
__global__ void __launch_bounds__(256)
    k_rasm_apply(const int32_t* __restrict__ ov_ptr, const int32_t* __restrict__ ov_idx,
                 const int32_t* __restrict__ core_ptr, const int32_t* __restrict__ core_idx,
                 const int64_t* __restrict__ w_off, const TW* __restrict__ W, int64_t nsub,
                 const int32_t* __restrict__ sub_list, const int32_t* __restrict__ pid_sub,
                 const int32_t* __restrict__ active, const TV* __restrict__ r, TV* __restrict__ z)
{
    __shared__ TV rg_all[8][kMaxSub];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t idx = (int64_t)blockIdx.x * 8 + warp;
    if (idx >= nsub) return;
    const int64_t sub = sub_list ? (int64_t)sub_list[idx] : idx;   // sub_list: the active problems' subdomains
    rasm_apply_one<TW, TV>(sub, lane, rg_all[warp], ov_ptr, ov_idx, core_ptr, core_idx, w_off, W, pid_sub, active, r,
                           z);
}

__global__ void k_sizes(const int32_t* __restrict__ ov_ptr, const int32_t* __restrict__ core_ptr, int64_t nsub,
                        int full, int64_t* __restrict__ sizes)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsub) return;
    const int64_t n = ov_ptr[s + 1] - ov_ptr[s];
    sizes[s] = n * (full ? n : (int64_t)(core_ptr[s + 1] - core_ptr[s]));
}

// Eq. asm: overlap entries of each point (CSR over points, entries ascending).
__global__ void k_asm_count(const int32_t* __restrict__ ov_idx, int64_t tot, int32_t* __restrict__ cnt,
                            int32_t* __restrict__ iota)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tot) return;
    iota[e] = (int32_t)e;
    atomicAdd(&cnt[ov_idx[e]], 1);
}

__global__ void k_asm_fill(const int32_t* __restrict__ ov_idx, int64_t tot, const int32_t* __restrict__ tptr,
                           int32_t* __restrict__ fill, int32_t* __restrict__ tidx)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tot) return;
    const int32_t p = ov_idx[e];
    tidx[tptr[p] + atomicAdd(&fill[p], 1)] = (int32_t)e;
}

__global__ void k_asm_sort(const int32_t* __restrict__ tptr, int64_t n, int32_t* __restrict__ tidx)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t* row = tidx + tptr[p];
    const int32_t len = tptr[p + 1] - tptr[p];
    for (int32_t a = 1; a < len; ++a) {
        int32_t v = row[a], b = a - 1;
        while (b >= 0 && row[b] > v) { row[b + 1] = row[b]; --b; }
        row[b + 1] = v;
    }
}

// z_p = sum of the subdomain results u_e of p's overlap entries, in entry order.
template <class T>
__global__ void k_asm_gather(const int32_t* __restrict__ tptr, const int32_t* __restrict__ tidx,
                             const T* __restrict__ u, int64_t n, const int32_t* __restrict__ pid,
                             const int32_t* __restrict__ active, T* __restrict__ z)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    if (active && !active[pid[p]]) return;
    T acc = 0;
    for (int32_t q = tptr[p]; q < tptr[p + 1]; ++q) acc += u[tidx[q]];
    z[p] = acc;
}

}  // namespace

rbf_status asm_lists(rbf_ctx* ctx, cudaStream_t st)
{
    const int64_t n = ctx->n, nsub = ctx->nsub;
    int32_t tot32 = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&tot32, ctx->ov_ptr.p + nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    const int64_t tot = tot32;
    RBF_CHECK(ensure(ctx, ctx->asm_fill, n + 1));
    RBF_CHECK(ensure(ctx, ctx->asm_tptr, n + 1));
    RBF_CHECK(ensure(ctx, ctx->asm_tidx, tot));
    RBF_CHECK(ensure(ctx, ctx->asm_iota, tot));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->asm_fill.p, 0, sizeof(int32_t) * (n + 1), st));
    RBF_LAUNCH(ctx, k_asm_count, blocks_for(tot, 256), 256, 0, st, ctx->ov_idx.p, tot, ctx->asm_fill.p,
               ctx->asm_iota.p);
    RBF_CHECK(exclusive_scan_i32(ctx, ctx->asm_fill.p, ctx->asm_tptr.p, n, st));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->asm_fill.p, 0, sizeof(int32_t) * (n + 1), st));
    RBF_LAUNCH(ctx, k_asm_fill, blocks_for(tot, 256), 256, 0, st, ctx->ov_idx.p, tot, ctx->asm_tptr.p,
               ctx->asm_fill.p, ctx->asm_tidx.p);
    RBF_LAUNCH(ctx, k_asm_sort, blocks_for(n, 256), 256, 0, st, ctx->asm_tptr.p, n, ctx->asm_tidx.p);
    RBF_CHECK(ensure(ctx, ctx->asm_u64, tot));
    if (ctx->rasm_precision != RBF_FP64) RBF_CHECK(ensure(ctx, ctx->asm_u32, tot));
    return RBF_OK;
}

rbf_status rasm_factor(rbf_ctx* ctx, cudaStream_t st)
{
    const int64_t nsub = ctx->nsub;
    RBF_CHECK(ensure(ctx, ctx->w_off, nsub + 1));
    RBF_CHECK(ensure(ctx, ctx->w_size, nsub + 1));
    const int full = ctx->rasm_additive ? 1 : 0;
    RBF_LAUNCH(ctx, k_sizes, blocks_for(nsub, 256), 256, 0, st, ctx->ov_ptr.p, ctx->core_ptr.p, nsub, full,
               ctx->w_size.p);
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
    const int nmax = ctx->max_ov;
    ctx->factor_tc = 0;
    ctx->factor_fp64 = 0;
    if (nmax == 0) return RBF_OK;
    const size_t per = setup_doubles(nmax) * sizeof(double);
    // as many warps per block as fit in kSetupSmemMax of shared memory (at most kSetupWarps)
    const int wpb = (int)std::min<size_t>(kSetupWarps, std::max<size_t>(1, kSetupSmemMax / per));
    const size_t smem = per * wpb;
    const bool fits = per <= kSetupSmemMax;
    if (fits)
        RBF_CUDA(ctx, cudaFuncSetAttribute(k_rasm_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RBF_CHECK(prof_begin(ctx, RBF_PROF_RASM_SETUP, st));
    if (ctx->rasm_precision == RBF_FP32) {
        // FP32 inverses on the tensor cores; the subdomains they leave are factored in FP64
        RBF_CHECK(ensure(ctx, ctx->tc_fb, (size_t)nsub + 1));
        int64_t nfb = 0;
        RBF_CHECK(rasm_factor_tc(ctx, ctx->tc_fb.p + 1, (unsigned int*)ctx->tc_fb.p, &nfb, st));
        ctx->factor_tc = nsub - nfb;
        ctx->factor_fp64 = nfb;
        if (nfb > 0) {
            if (!fits)
                return fail(ctx, RBF_ERR_SUBDOMAIN_TOO_LARGE,
                            "rbf_rasm_setup: a %d-point overlap list needs %zu KB of shared memory", nmax, per / 1024);
            RBF_LAUNCH(ctx, k_rasm_setup, blocks_for(nfb, wpb), kSetupWarps * 32, smem, st, ctx->xy_s.p,
                       ctx->ov_ptr.p, ctx->ov_idx.p, ctx->core_of.p, ctx->core_ptr.p, ctx->w_off.p, nfb, nmax, wpb,
                       ctx->prob.p, ctx->pid_sub.p, full, ctx->fxtab.p, (double*)nullptr, W32, ctx->status_dev.p,
                       (const int32_t*)(ctx->tc_fb.p + 1));
        }
    } else {
        if (!fits)
            return fail(ctx, RBF_ERR_SUBDOMAIN_TOO_LARGE,
                        "rbf_rasm_setup: a %d-point overlap list needs %zu KB of shared memory", nmax, per / 1024);
        ctx->factor_fp64 = nsub;
        RBF_LAUNCH(ctx, k_rasm_setup, blocks_for(nsub, wpb), kSetupWarps * 32, smem, st, ctx->xy_s.p, ctx->ov_ptr.p,
                   ctx->ov_idx.p, ctx->core_of.p, ctx->core_ptr.p, ctx->w_off.p, nsub, nmax, wpb, ctx->prob.p,
                   ctx->pid_sub.p, full, ctx->fxtab.p, W64, W32, ctx->status_dev.p, (const int32_t*)nullptr);
    }
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
    const int64_t nsub = ctx->al.on ? ctx->al.nsub : ctx->nsub;
    const int32_t* sub_list = ctx->al.on ? ctx->al.sub.p : nullptr;
    // Eq. asm: the GEMV writes every overlap row to the scratch list, then a gather
    const bool add = ctx->rasm_additive;
    const int32_t* rows_ptr = add ? ctx->ov_ptr.p : ctx->core_ptr.p;
    const int32_t* rows_idx = add ? ctx->asm_iota.p : ctx->core_idx.p;
    if (ctx->rasm_precision == RBF_FP64) {
        double* out = add ? ctx->asm_u64.p : z;
        RBF_LAUNCH(ctx, (k_rasm_apply<double, double>), blocks_for(nsub, 8), 256, 0, st, ctx->ov_ptr.p,
                   ctx->ov_idx.p, rows_ptr, rows_idx, ctx->w_off.p, ctx->W64.p, nsub, sub_list, ctx->pid_sub.p,
                   ctx->active_mask, r, out);
        if (add)
            RBF_LAUNCH(ctx, k_asm_gather<double>, blocks_for(ctx->n, 256), 256, 0, st, ctx->asm_tptr.p,
                       ctx->asm_tidx.p, (const double*)out, ctx->n, ctx->pid.p, ctx->active_mask, z);
    } else {
        double* out = add ? ctx->asm_u64.p : z;
        RBF_LAUNCH(ctx, (k_rasm_apply<float, double>), blocks_for(nsub, 8), 256, 0, st, ctx->ov_ptr.p,
                   ctx->ov_idx.p, rows_ptr, rows_idx, ctx->w_off.p, ctx->W32.p, nsub, sub_list, ctx->pid_sub.p,
                   ctx->active_mask, r, out);
        if (add)
            RBF_LAUNCH(ctx, k_asm_gather<double>, blocks_for(ctx->n, 256), 256, 0, st, ctx->asm_tptr.p,
                       ctx->asm_tidx.p, (const double*)out, ctx->n, ctx->pid.p, ctx->active_mask, z);
    }
    return prof_end(ctx, RBF_PROF_RASM_APPLY, st);
}

rbf_status rasm_apply_sorted_f32(rbf_ctx* ctx, const float* r, float* z, cudaStream_t st)
{
    RBF_CHECK(prof_begin(ctx, RBF_PROF_RASM_APPLY, st));
    const int64_t nsub = ctx->al.on ? ctx->al.nsub : ctx->nsub;
    const int32_t* sub_list = ctx->al.on ? ctx->al.sub.p : nullptr;
    if (ctx->inner_on) {   // vectors in the inner grid's order: the lists re-indexed into it
        RBF_LAUNCH(ctx, (k_rasm_apply<float, float>), blocks_for(nsub, 8), 256, 0, st, ctx->ov_ptr.p,
                   ctx->in.ov_idx.p, ctx->core_ptr.p, ctx->in.core_idx.p, ctx->w_off.p, ctx->W32.p, nsub, sub_list,
                   ctx->pid_sub.p, ctx->active_mask, r, z);
        return prof_end(ctx, RBF_PROF_RASM_APPLY, st);
    }
    const bool add = ctx->rasm_additive;
    float* out = add ? ctx->asm_u32.p : z;
    RBF_LAUNCH(ctx, (k_rasm_apply<float, float>), blocks_for(nsub, 8), 256, 0, st, ctx->ov_ptr.p, ctx->ov_idx.p,
               add ? ctx->ov_ptr.p : ctx->core_ptr.p, add ? ctx->asm_iota.p : ctx->core_idx.p, ctx->w_off.p,
               ctx->W32.p, nsub, sub_list, ctx->pid_sub.p, ctx->active_mask, r, out);
    if (add)
        RBF_LAUNCH(ctx, k_asm_gather<float>, blocks_for(ctx->n, 256), 256, 0, st, ctx->asm_tptr.p, ctx->asm_tidx.p,
                   (const float*)out, ctx->n, ctx->pid.p, ctx->active_mask, z);
    return prof_end(ctx, RBF_PROF_RASM_APPLY, st);
}

}  // namespace rbf
