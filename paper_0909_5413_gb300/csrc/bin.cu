// bin.cu -- cell-list binning of the points (the data structure of the
// matrix-free truncated matvec), user <-> cell-order permutations, and the
// neighbour-list export used for parity checks.
//
// Binning: bounding box; cell (cx, cy) = floor((x - xmin) / c) clamped to the
// grid, ncx = floor((xmax - xmin) / c) + 1; stable sort by cy*ncx + cx with
// ties in user order. Every floating-point step uses explicit round-to-nearest
// intrinsics (no contraction), so the cell of each point is the IEEE result
// of that expression.
#include <cfloat>
#include <cmath>

#include "common.cuh"

namespace rbf {
namespace {

__device__ __forceinline__ int64_t cell_axis(double v, double lo, double c, int64_t nc)
{
    double q = floor(__ddiv_rn(__dsub_rn(v, lo), c));
    int64_t k = (q < 0.0) ? -1 : (q > (double)nc ? nc : (int64_t)q);
    return k < 0 ? 0 : (k > nc - 1 ? nc - 1 : k);
}

__device__ __forceinline__ double pair_r2(double xi, double yi, double xj, double yj)
{
    double dx = __dsub_rn(xi, xj), dy = __dsub_rn(yi, yj);
    return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Per-block min/max of x and y: part[4*b + {0,1,2,3}] = {xmin, ymin, xmax, ymax}.
__global__ void k_bbox(const double* __restrict__ xy, int64_t n, double* __restrict__ part)
{
    double x0 = DBL_MAX, y0 = DBL_MAX, x1 = -DBL_MAX, y1 = -DBL_MAX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        x0 = fmin(x0, x); x1 = fmax(x1, x);
        y0 = fmin(y0, y); y1 = fmax(y1, y);
    }
    for (int d = 16; d > 0; d >>= 1) {
        x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, d));
        y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, d));
        x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, d));
        y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, d));
    }
    __shared__ double sm[4][32];
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sm[0][w] = x0; sm[1][w] = y0; sm[2][w] = x1; sm[3][w] = y1; }
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        x0 = l < nw ? sm[0][l] : DBL_MAX;  y0 = l < nw ? sm[1][l] : DBL_MAX;
        x1 = l < nw ? sm[2][l] : -DBL_MAX; y1 = l < nw ? sm[3][l] : -DBL_MAX;
        for (int d = 16; d > 0; d >>= 1) {
            x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, d));
            y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, d));
            x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, d));
            y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, d));
        }
        if (l == 0) {
            part[4 * blockIdx.x + 0] = x0; part[4 * blockIdx.x + 1] = y0;
            part[4 * blockIdx.x + 2] = x1; part[4 * blockIdx.x + 3] = y1;
        }
    }
}

__global__ void k_bbox_final(const double* __restrict__ part, int nb, double* __restrict__ out)
{
    if (threadIdx.x != 0) return;
    double x0 = DBL_MAX, y0 = DBL_MAX, x1 = -DBL_MAX, y1 = -DBL_MAX;
    for (int b = 0; b < nb; ++b) {
        x0 = fmin(x0, part[4 * b]); y0 = fmin(y0, part[4 * b + 1]);
        x1 = fmax(x1, part[4 * b + 2]); y1 = fmax(y1, part[4 * b + 3]);
    }
    out[0] = x0; out[1] = y0; out[2] = x1; out[3] = y1;
}

// Cell id of every point (user order) and per-cell counts.
__global__ void k_cell_count(const double* __restrict__ xy, int64_t n, double xmin, double ymin, double c,
                             int64_t ncx, int64_t ncy, int32_t* __restrict__ cell_u, int32_t* __restrict__ counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t cx = cell_axis(xy[2 * i], xmin, c, ncx);
    int64_t cy = cell_axis(xy[2 * i + 1], ymin, c, ncy);
    int32_t cell = (int32_t)(cy * ncx + cx);
    cell_u[i] = cell;
    atomicAdd(&counts[cell], 1);
}

// Unordered placement into each cell's range (slot order is arbitrary here;
// k_cell_rank restores user order within the cell).
__global__ void k_cell_scatter(const int32_t* __restrict__ cell_u, int64_t n, const int32_t* __restrict__ cell_start,
                               int32_t* __restrict__ fill, int32_t* __restrict__ tmp)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = cell_u[i];
    int32_t slot = atomicAdd(&fill[c], 1);
    tmp[cell_start[c] + slot] = (int32_t)i;
}

// One warp per cell: each element's final position in the cell is the number
// of elements of the same cell with a smaller user index (all distinct).
__global__ void k_cell_rank(const int32_t* __restrict__ cell_start, int64_t ncell, const int32_t* __restrict__ tmp,
                            int32_t* __restrict__ perm)
{
    int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (c >= ncell) return;
    int32_t b = cell_start[c], e = cell_start[c + 1];
    for (int32_t p = b + lane; p < e; p += 32) {
        int32_t v = tmp[p];
        int32_t r = 0;
        for (int32_t q = b; q < e; ++q) r += (tmp[q] < v);
        perm[b + r] = v;
    }
}

__global__ void k_gather_sorted(const double* __restrict__ xy, int64_t n, const int32_t* __restrict__ perm,
                                const int32_t* __restrict__ cell_u, double* __restrict__ xy_s,
                                int32_t* __restrict__ iperm, int32_t* __restrict__ cell_s)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int32_t i = perm[p];
    xy_s[2 * p] = xy[2 * (int64_t)i];
    xy_s[2 * p + 1] = xy[2 * (int64_t)i + 1];
    iperm[i] = (int32_t)p;
    cell_s[p] = cell_u[i];
}

// FP32 offsets of each point from its cell's lower corner, scaled by a with
// a^2 = log2(e) / (2 sigma^2): the FP32 kernel value is exp2(-|dX|^2).
__global__ void k_local_coords(const double* __restrict__ xy_s, const int32_t* __restrict__ cell_s, int64_t n,
                               int64_t ncx, double xmin, double ymin, double c, double a, float* __restrict__ loc)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t cc = cell_s[p];
    int64_t cx = cc % ncx, cy = cc / ncx;
    double ox = xmin + (double)cx * c, oy = ymin + (double)cy * c;
    loc[2 * p] = (float)((xy_s[2 * p] - ox) * a);
    loc[2 * p + 1] = (float)((xy_s[2 * p + 1] - oy) * a);
}

// Matvec work items: cell c with m points gives ceil(m / 128) items (c, 128 q).
__global__ void k_work_count(const int32_t* __restrict__ cell_start, int64_t ncell, int32_t* __restrict__ cnt)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) cnt[c] = (cell_start[c + 1] - cell_start[c] + 127) / 128;
}

__global__ void k_work_fill(const int32_t* __restrict__ cnt, const int32_t* __restrict__ off, int64_t ncell,
                            int32_t* __restrict__ work)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    for (int q = 0; q < cnt[c]; ++q) {
        work[2 * (off[c] + q)] = (int32_t)c;
        work[2 * (off[c] + q) + 1] = 128 * q;
    }
}

__global__ void k_permute_to_sorted(const double* __restrict__ user, const int32_t* __restrict__ perm, int64_t n,
                                    double* __restrict__ sorted)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) sorted[p] = user[perm[p]];
}

__global__ void k_permute_to_user(const double* __restrict__ sorted, const int32_t* __restrict__ perm, int64_t n,
                                  double* __restrict__ user)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) user[perm[p]] = sorted[p];
}

// Neighbour counts (mode 0) or lists (mode 1) for targets in user order; rows
// are filled from the cell stencil, then put in ascending user order.
__global__ void k_neighbors(const double* __restrict__ xy_s, const int32_t* __restrict__ perm,
                            const int32_t* __restrict__ iperm, const int32_t* __restrict__ cell_s,
                            const int32_t* __restrict__ cell_start, int64_t n, int64_t ncx, int64_t ncy, int k,
                            double rc2, const int64_t* __restrict__ ptr, int32_t* __restrict__ cnt,
                            int32_t* __restrict__ idx, int mode)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = iperm[i];
    double xi = xy_s[2 * (int64_t)p], yi = xy_s[2 * (int64_t)p + 1];
    int64_t c = cell_s[p];
    int64_t cx = c % ncx, cy = c / ncx;
    int64_t ylo = cy - k < 0 ? 0 : cy - k, yhi = cy + k > ncy - 1 ? ncy - 1 : cy + k;
    int64_t xlo = cx - k < 0 ? 0 : cx - k, xhi = cx + k > ncx - 1 ? ncx - 1 : cx + k;
    int64_t w = (mode == 1) ? ptr[i] : 0;
    int32_t count = 0;
    for (int64_t yy = ylo; yy <= yhi; ++yy) {
        int32_t b = cell_start[yy * ncx + xlo], e = cell_start[yy * ncx + xhi + 1];
        for (int32_t q = b; q < e; ++q) {
            double r2 = pair_r2(xi, yi, xy_s[2 * (int64_t)q], xy_s[2 * (int64_t)q + 1]);
            if (r2 <= rc2) {
                if (mode == 1) idx[w + count] = perm[q];
                ++count;
            }
        }
    }
    if (mode == 0) {
        cnt[i] = count;
    } else {
        // insertion sort of the row (rows are a few hundred entries)
        int32_t* row = idx + w;
        for (int32_t a = 1; a < count; ++a) {
            int32_t v = row[a];
            int32_t b = a - 1;
            while (b >= 0 && row[b] > v) { row[b + 1] = row[b]; --b; }
            row[b + 1] = v;
        }
    }
}

__global__ void k_widen_i32_i64(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

}  // namespace

rbf_status bin_points(rbf_ctx* ctx, const double* xy, cudaStream_t st)
{
    const int64_t n = ctx->n;
    const int nb = 2 * kNumSMs;
    RBF_CHECK(ensure(ctx, ctx->bbox_part, 4 * nb));
    RBF_CHECK(ensure(ctx, ctx->bbox_dev, 4));
    RBF_LAUNCH(ctx, k_bbox, nb, 256, 0, st, xy, n, ctx->bbox_part.p);
    RBF_LAUNCH(ctx, k_bbox_final, 1, 32, 0, st, ctx->bbox_part.p, nb, ctx->bbox_dev.p);
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->bbox, ctx->bbox_dev.p, sizeof(ctx->bbox), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    for (double v : ctx->bbox)
        if (!std::isfinite(v)) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: non-finite coordinate");
    double fx = std::floor((ctx->bbox[2] - ctx->bbox[0]) / ctx->cell);
    double fy = std::floor((ctx->bbox[3] - ctx->bbox[1]) / ctx->cell);
    if (!(fx < 1.0e9) || !(fy < 1.0e9)) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: grid too large");
    ctx->ncx = (int64_t)fx + 1;
    ctx->ncy = (int64_t)fy + 1;
    const int64_t ncell = ctx->ncx * ctx->ncy;
    if (ncell > ((int64_t)1 << 28))
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: %lld cells exceed 2^28 (cell_size too small)", (long long)ncell);

    RBF_CHECK(ensure(ctx, ctx->counts, ncell + 1));
    RBF_CHECK(ensure(ctx, ctx->cell_start, ncell + 1));
    RBF_CHECK(ensure(ctx, ctx->cell_u, n));
    RBF_CHECK(ensure(ctx, ctx->cell_s, n));
    RBF_CHECK(ensure(ctx, ctx->perm, n));
    RBF_CHECK(ensure(ctx, ctx->iperm, n));
    RBF_CHECK(ensure(ctx, ctx->tmp_i32, std::max<int64_t>(n, 2 * kNumSMs + 1)));
    RBF_CHECK(ensure(ctx, ctx->xy_s, 2 * n));

    RBF_CHECK(prof_begin(ctx, RBF_PROF_BIN, st));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_cell_count, blocks_for(n, 256), 256, 0, st, xy, n, ctx->bbox[0], ctx->bbox[1], ctx->cell,
               ctx->ncx, ctx->ncy, ctx->cell_u.p, ctx->counts.p);
    RBF_CHECK(exclusive_scan_i32(ctx, ctx->counts.p, ctx->cell_start.p, ncell, st));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_cell_scatter, blocks_for(n, 256), 256, 0, st, ctx->cell_u.p, n, ctx->cell_start.p,
               ctx->counts.p, ctx->tmp_i32.p);
    RBF_LAUNCH(ctx, k_cell_rank, blocks_for(ncell * 32, 256), 256, 0, st, ctx->cell_start.p, ncell, ctx->tmp_i32.p,
               ctx->perm.p);
    RBF_LAUNCH(ctx, k_gather_sorted, blocks_for(n, 256), 256, 0, st, xy, n, ctx->perm.p, ctx->cell_u.p, ctx->xy_s.p,
               ctx->iperm.p, ctx->cell_s.p);
    RBF_CHECK(ensure(ctx, ctx->loc32, 2 * n));
    RBF_LAUNCH(ctx, k_local_coords, blocks_for(n, 256), 256, 0, st, ctx->xy_s.p, ctx->cell_s.p, n, ctx->ncx,
               ctx->bbox[0], ctx->bbox[1], ctx->cell, std::sqrt(M_LOG2E * ctx->s), ctx->loc32.p);
    RBF_CHECK(ensure(ctx, ctx->mv_wcnt, ncell + 1));
    RBF_CHECK(ensure(ctx, ctx->mv_woff, ncell + 1));
    RBF_LAUNCH(ctx, k_work_count, blocks_for(ncell, 256), 256, 0, st, ctx->cell_start.p, ncell, ctx->mv_wcnt.p);
    RBF_CHECK(exclusive_scan_i32(ctx, ctx->mv_wcnt.p, ctx->mv_woff.p, ncell, st));
    int32_t nwork = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&nwork, ctx->mv_woff.p + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    ctx->n_work = nwork;
    RBF_CHECK(ensure(ctx, ctx->mv_work, 2 * (size_t)std::max<int32_t>(nwork, 1)));
    RBF_LAUNCH(ctx, k_work_fill, blocks_for(ncell, 256), 256, 0, st, ctx->mv_wcnt.p, ctx->mv_woff.p, ncell,
               ctx->mv_work.p);
    return prof_end(ctx, RBF_PROF_BIN, st);
}

rbf_status permute_to_sorted(rbf_ctx* ctx, const double* user, double* sorted, cudaStream_t st)
{
    RBF_LAUNCH(ctx, k_permute_to_sorted, blocks_for(ctx->n, 256), 256, 0, st, user, ctx->perm.p, ctx->n, sorted);
    return RBF_OK;
}

rbf_status permute_to_user(rbf_ctx* ctx, const double* sorted, double* user, cudaStream_t st)
{
    RBF_LAUNCH(ctx, k_permute_to_user, blocks_for(ctx->n, 256), 256, 0, st, sorted, ctx->perm.p, ctx->n, user);
    return RBF_OK;
}

rbf_status neighbor_lists(rbf_ctx* ctx, int64_t* ptr, int32_t* idx, int64_t capacity, int64_t* total,
                          cudaStream_t st)
{
    const int64_t n = ctx->n;
    RBF_CHECK(ensure(ctx, ctx->nbr_cnt, n));
    RBF_CHECK(ensure(ctx, ctx->nbr_ptr_tmp, 2 * (n + 1)));
    RBF_LAUNCH(ctx, k_neighbors, blocks_for(n, 128), 128, 0, st, ctx->xy_s.p, ctx->perm.p, ctx->iperm.p,
               ctx->cell_s.p, ctx->cell_start.p, n, ctx->ncx, ctx->ncy, ctx->kst, ctx->rc2, (const int64_t*)nullptr,
               ctx->nbr_cnt.p, (int32_t*)nullptr, 0);
    int64_t* cnt64 = ctx->nbr_ptr_tmp.p;
    int64_t* p64 = ctx->nbr_ptr_tmp.p + (n + 1);
    RBF_LAUNCH(ctx, k_widen_i32_i64, blocks_for(n, 256), 256, 0, st, ctx->nbr_cnt.p, n, cnt64);
    RBF_CHECK(exclusive_scan_i64(ctx, cnt64, p64, n, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(total, p64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    if (!ptr) return RBF_OK;
    if (*total > capacity)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_get_neighbors: capacity %lld < %lld pairs", (long long)capacity,
                    (long long)*total);
    RBF_CUDA(ctx, cudaMemcpyAsync(ptr, p64, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, st));
    RBF_LAUNCH(ctx, k_neighbors, blocks_for(n, 128), 128, 0, st, ctx->xy_s.p, ctx->perm.p, ctx->iperm.p,
               ctx->cell_s.p, ctx->cell_start.p, n, ctx->ncx, ctx->ncy, ctx->kst, ctx->rc2, (const int64_t*)p64,
               ctx->nbr_cnt.p, idx, 1);
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    return RBF_OK;
}

}  // namespace rbf
