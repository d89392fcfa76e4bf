// subdomain.cu -- core and overlap index lists of the RASM boxes (Sec. 2.2:
// overlapping subdomains Omega_i and non-overlapping ~Omega_i; Sec. 2.3: a
// separate index list for the non-overlapping part).
//
// Box (bx, by) has core [x0 + bx B, x0 + (bx+1) B) x [...] (box index
// floor((x - x0) / B) clamped to the box grid) and overlap box widened by
// delta on each side, half-open; a point always lies in the overlap of its own
// core box. Lists hold cell-order positions, ordered by ascending user index.
#include "common.cuh"

namespace rbf {
namespace {

__device__ __forceinline__ int64_t box_axis(double v, double lo, double B, int64_t nb)
{
    double q = floor(__ddiv_rn(__dsub_rn(v, lo), B));
    int64_t k = (q < 0.0) ? -1 : (q > (double)nb ? nb : (int64_t)q);
    return k < 0 ? 0 : (k > nb - 1 ? nb - 1 : k);
}

__device__ __forceinline__ bool in_overlap(double v, int64_t k, int64_t kc, double o, double B, double delta)
{
    if (k == kc) return true;
    if (k < kc) return v < __dadd_rn(__dadd_rn(o, __dmul_rn((double)(k + 1), B)), delta);
    return v >= __dsub_rn(__dadd_rn(o, __dmul_rn((double)k, B)), delta);
}

// mode 0: count core / overlap members; mode 1: place them (unordered slots).
// Box grid and subdomain numbering of each point's problem from prob[pid[p]].
__global__ void k_boxes(const double* __restrict__ xy_s, int64_t n, const Prob* __restrict__ prob,
                        const int32_t* __restrict__ pid, int32_t* __restrict__ core_of, int32_t* __restrict__ ccnt,
                        int32_t* __restrict__ ocnt, const int32_t* __restrict__ cptr, const int32_t* __restrict__ optr,
                        int32_t* __restrict__ cidx, int32_t* __restrict__ oidx, int mode)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const Prob& bx = prob[pid[p]];
    double x = xy_s[2 * p], y = xy_s[2 * p + 1];
    int64_t cx = box_axis(x, bx.x0, bx.B, bx.nbx);
    int64_t cy = box_axis(y, bx.y0, bx.B, bx.nby);
    int64_t sc = bx.subbase + cy * bx.nbx + cx;
    if (mode == 0) {
        core_of[p] = (int32_t)sc;
        atomicAdd(&ccnt[sc], 1);
    } else {
        int32_t slot = atomicAdd(&ccnt[sc], 1);
        cidx[cptr[sc] + slot] = (int32_t)p;
    }
    int64_t ky0 = cy - bx.reach < 0 ? 0 : cy - bx.reach;
    int64_t ky1 = cy + bx.reach > bx.nby - 1 ? bx.nby - 1 : cy + bx.reach;
    int64_t kx0 = cx - bx.reach < 0 ? 0 : cx - bx.reach;
    int64_t kx1 = cx + bx.reach > bx.nbx - 1 ? bx.nbx - 1 : cx + bx.reach;
    for (int64_t ky = ky0; ky <= ky1; ++ky) {
        if (!in_overlap(y, ky, cy, bx.y0, bx.B, bx.delta)) continue;
        for (int64_t kx = kx0; kx <= kx1; ++kx) {
            if (!in_overlap(x, kx, cx, bx.x0, bx.B, bx.delta)) continue;
            int64_t s = bx.subbase + ky * bx.nbx + kx;
            if (mode == 0) {
                atomicAdd(&ocnt[s], 1);
            } else {
                int32_t slot = atomicAdd(&ocnt[s], 1);
                oidx[optr[s] + slot] = (int32_t)p;
            }
        }
    }
}

__global__ void k_pid_subs(const Prob* __restrict__ prob, int nprob, int64_t nsub, int32_t* __restrict__ pid_sub)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsub) return;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prob[mid].subbase <= s) lo = mid; else hi = mid - 1;
    }
    pid_sub[s] = lo;
}

// One warp per list: order the entries by the user index perm[entry] (rank sort).
__global__ void k_sort_lists(const int32_t* __restrict__ ptr, int64_t nlist, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ in, int32_t* __restrict__ out)
{
    int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (s >= nlist) return;
    int32_t b = ptr[s], e = ptr[s + 1];
    for (int32_t a = b + lane; a < e; a += 32) {
        int32_t v = in[a];
        int32_t key = perm[v];
        int32_t r = 0;
        for (int32_t q = b; q < e; ++q) r += (perm[in[q]] < key);
        out[b + r] = v;
    }
}

__global__ void k_export(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ perm,
                         int32_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = perm[in[i]];
}

}  // namespace

rbf_status build_subdomains(rbf_ctx* ctx, cudaStream_t st)
{
    const int64_t n = ctx->n, nsub = ctx->nsub;
    const int nprob = (int)ctx->nprob;
    RBF_CHECK(ensure(ctx, ctx->core_of, n));
    RBF_CHECK(ensure(ctx, ctx->core_ptr, nsub + 1));
    RBF_CHECK(ensure(ctx, ctx->ov_ptr, nsub + 1));
    RBF_CHECK(ensure(ctx, ctx->sub_cnt, 2 * (nsub + 1)));
    int32_t* ccnt = ctx->sub_cnt.p;
    int32_t* ocnt = ctx->sub_cnt.p + (nsub + 1);
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->sub_cnt.p, 0, sizeof(int32_t) * 2 * (nsub + 1), st));
    RBF_CHECK(ensure(ctx, ctx->pid_sub, nsub));
    RBF_LAUNCH(ctx, k_pid_subs, blocks_for(nsub, 256), 256, 0, st, ctx->prob.p, nprob, nsub, ctx->pid_sub.p);
    RBF_LAUNCH(ctx, k_boxes, blocks_for(n, 256), 256, 0, st, ctx->xy_s.p, n, ctx->prob.p, ctx->pid.p, ctx->core_of.p,
               ccnt, ocnt, (const int32_t*)nullptr, (const int32_t*)nullptr, (int32_t*)nullptr, (int32_t*)nullptr, 0);
    int32_t mx = 0;
    RBF_CHECK(reduce_max_i32(ctx, ocnt, nsub, &mx, st));
    ctx->max_ov = mx;
    RBF_CHECK(reduce_max_i32(ctx, ccnt, nsub, &mx, st));
    ctx->max_core = mx;
    if (ctx->max_ov > kMaxSub) return RBF_OK;   // caller reports SUBDOMAIN_TOO_LARGE
    RBF_CHECK(exclusive_scan_i32(ctx, ccnt, ctx->core_ptr.p, nsub, st));
    RBF_CHECK(exclusive_scan_i32(ctx, ocnt, ctx->ov_ptr.p, nsub, st));
    int32_t tot[2];
    RBF_CUDA(ctx, cudaMemcpyAsync(&tot[0], ctx->core_ptr.p + nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(&tot[1], ctx->ov_ptr.p + nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    if (tot[0] != n) return fail(ctx, RBF_ERR_CUDA, "internal: core lists hold %d of %lld points", tot[0], (long long)n);
    RBF_CHECK(ensure(ctx, ctx->core_idx, (size_t)tot[0]));
    RBF_CHECK(ensure(ctx, ctx->ov_idx, (size_t)tot[1]));
    RBF_CHECK(ensure(ctx, ctx->tmp_i32, std::max<int64_t>(std::max<int64_t>(tot[0], tot[1]), 2 * kNumSMs + 1)));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->sub_cnt.p, 0, sizeof(int32_t) * 2 * (nsub + 1), st));
    // place overlap members into tmp, core members directly (sorted below)
    RBF_CHECK(ensure(ctx, ctx->sub_fill, (size_t)tot[0]));
    RBF_LAUNCH(ctx, k_boxes, blocks_for(n, 256), 256, 0, st, ctx->xy_s.p, n, ctx->prob.p, ctx->pid.p, ctx->core_of.p,
               ccnt, ocnt, ctx->core_ptr.p, ctx->ov_ptr.p, ctx->sub_fill.p, ctx->tmp_i32.p, 1);
    RBF_LAUNCH(ctx, k_sort_lists, blocks_for(nsub * 32, 256), 256, 0, st, ctx->core_ptr.p, nsub, ctx->perm.p,
               ctx->sub_fill.p, ctx->core_idx.p);
    RBF_LAUNCH(ctx, k_sort_lists, blocks_for(nsub * 32, 256), 256, 0, st, ctx->ov_ptr.p, nsub, ctx->perm.p,
               ctx->tmp_i32.p, ctx->ov_idx.p);
    return RBF_OK;
}

rbf_status export_subdomains(rbf_ctx* ctx, int32_t* core_ptr, int32_t* core_idx, int32_t* ov_ptr, int32_t* ov_idx,
                             cudaStream_t st)
{
    const int64_t nsub = ctx->nsub;
    int32_t tot[2];
    RBF_CUDA(ctx, cudaMemcpyAsync(&tot[0], ctx->core_ptr.p + nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(&tot[1], ctx->ov_ptr.p + nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    RBF_CUDA(ctx, cudaMemcpyAsync(core_ptr, ctx->core_ptr.p, sizeof(int32_t) * (nsub + 1), cudaMemcpyDeviceToDevice, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(ov_ptr, ctx->ov_ptr.p, sizeof(int32_t) * (nsub + 1), cudaMemcpyDeviceToDevice, st));
    RBF_LAUNCH(ctx, k_export, blocks_for(tot[0], 256), 256, 0, st, ctx->core_idx.p, (int64_t)tot[0], ctx->perm.p,
               core_idx);
    RBF_LAUNCH(ctx, k_export, blocks_for(tot[1], 256), 256, 0, st, ctx->ov_idx.p, (int64_t)tot[1], ctx->perm.p,
               ov_idx);
    return RBF_OK;
}

}  // namespace rbf
