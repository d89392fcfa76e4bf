// bin.cu -- cell-list binning of the points (the data structure of the
// matrix-free truncated matvec), user <-> cell-order permutations, and the
// neighbour-list export used for parity checks.
//
// Binning of each problem: bounding box; cell (cx, cy) = floor((x - xmin) / c)
// clamped to the problem's grid, ncx = floor((xmax - xmin) / c) + 1; global
// cell id = cellbase + cy*ncx + cx; stable sort of all points by global cell
// id with ties in user order. Problems of a batch get consecutive cell ranges,
// so each problem's points stay a contiguous range in cell order. Every
// floating-point step uses explicit round-to-nearest intrinsics (no
// contraction), so the cell of each point is the IEEE result of that
// expression.
#include <algorithm>
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

// Index b with base[b] <= v < base[b+1] (base ascending, n entries + sentinel).
__device__ __forceinline__ int find_segment(const int64_t* __restrict__ base, int n, int64_t v)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Order-preserving map of doubles to unsigned keys (for atomic min / max).
__device__ __forceinline__ unsigned long long okey(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double okey_inv(unsigned long long k)
{
    unsigned long long b = (k & 0x8000000000000000ull) ? (k & ~0x8000000000000000ull) : ~k;
    return __longlong_as_double((long long)b);
}

__global__ void k_pid(const int64_t* __restrict__ pbeg, int nprob, int64_t n, int32_t* __restrict__ pid)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pid[i] = find_segment(pbeg, nprob, i);
}

__global__ void k_pid_cells(const Prob* __restrict__ prob, int nprob, int64_t ncell, int32_t* __restrict__ pid_cell)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prob[mid].cellbase <= c) lo = mid; else hi = mid - 1;
    }
    pid_cell[c] = lo;
}

constexpr int kBoxTile = 4096;

// Per-problem bounding boxes as ordered keys: keys[4 b + {0..3}] = min x, min y,
// -max x, -max y (all taken with atomicMin). A tile of one problem is reduced
// in the block first; tiles that straddle problems use per-thread atomics.
__global__ void k_bbox(const double* __restrict__ xy, int64_t n, const int32_t* __restrict__ pid,
                       unsigned long long* __restrict__ keys)
{
    __shared__ unsigned long long red[4][8];
    const int64_t t0 = (int64_t)blockIdx.x * kBoxTile;
    const int64_t t1 = min(t0 + kBoxTile, n);
    const int p0 = pid[t0], p1 = pid[t1 - 1];
    unsigned long long k[4] = {~0ull, ~0ull, ~0ull, ~0ull};
    int cur = -1;
    for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
        int b = pid[i];
        if (p0 != p1 && b != cur && cur >= 0) {
            for (int q = 0; q < 4; ++q) atomicMin(&keys[4 * cur + q], k[q]);
            k[0] = k[1] = k[2] = k[3] = ~0ull;
        }
        cur = b;
        double x = xy[2 * i], y = xy[2 * i + 1];
        // A NaN (whose sign arithmetic may not keep) would slip through the
        // ordered-key minima; key 0, which no finite or infinite value maps
        // to, makes the problem's x_min NaN instead, and the host rejects it.
        if (!(isfinite(x) && isfinite(y))) k[0] = 0ull;
        k[0] = min(k[0], okey(x));
        k[1] = min(k[1], okey(y));
        k[2] = min(k[2], okey(-x));
        k[3] = min(k[3], okey(-y));
    }
    if (p0 != p1) {
        if (cur >= 0)
            for (int q = 0; q < 4; ++q) atomicMin(&keys[4 * cur + q], k[q]);
        return;
    }
    for (int q = 0; q < 4; ++q)
        for (int d = 16; d > 0; d >>= 1) k[q] = min(k[q], __shfl_xor_sync(0xffffffffu, k[q], d));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int q = 0; q < 4; ++q) red[q][w] = k[q];
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long m = ~0ull;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) m = min(m, red[threadIdx.x][ww]);
        atomicMin(&keys[4 * p0 + threadIdx.x], m);
    }
}

__global__ void k_bbox_final(const unsigned long long* __restrict__ keys, int nprob, double* __restrict__ out)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nprob) return;
    out[4 * b + 0] = okey_inv(keys[4 * b + 0]);
    out[4 * b + 1] = okey_inv(keys[4 * b + 1]);
    out[4 * b + 2] = -okey_inv(keys[4 * b + 2]);
    out[4 * b + 3] = -okey_inv(keys[4 * b + 3]);
}

// Cell id of every point (user order) and per-cell counts.
__global__ void k_cell_count(const double* __restrict__ xy, int64_t n, const Prob* __restrict__ prob,
                             const int32_t* __restrict__ pid, int32_t* __restrict__ cell_u, int32_t* __restrict__ counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Prob& P = prob[pid[i]];
    int64_t cx = cell_axis(xy[2 * i], P.xmin, P.c, P.ncx);
    int64_t cy = cell_axis(xy[2 * i + 1], P.ymin, P.c, P.ncy);
    int32_t cell = (int32_t)(P.cellbase + cy * P.ncx + cx);
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
                               const Prob* __restrict__ prob, const int32_t* __restrict__ pid, float* __restrict__ loc)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const Prob& P = prob[pid[p]];
    int64_t cc = cell_s[p] - P.cellbase;
    int64_t cx = cc % P.ncx, cy = cc / P.ncx;
    double ox = P.xmin + (double)cx * P.c, oy = P.ymin + (double)cy * P.c;
    loc[2 * p] = (float)((xy_s[2 * p] - ox) * (double)P.a_loc);
    loc[2 * p + 1] = (float)((xy_s[2 * p + 1] - oy) * (double)P.a_loc);
}

// Matvec work items: cell c with m points gives ceil(m / T) items (c, T q).
__global__ void k_work_count(const int32_t* __restrict__ cell_start, int64_t ncell, int tile,
                             int32_t* __restrict__ cnt)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell) cnt[c] = (cell_start[c + 1] - cell_start[c] + tile - 1) / tile;
}

__global__ void k_work_fill(const int32_t* __restrict__ cnt, const int32_t* __restrict__ off, int64_t ncell,
                            int tile, int32_t* __restrict__ work)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    for (int q = 0; q < cnt[c]; ++q) {
        work[2 * (off[c] + q)] = (int32_t)c;
        work[2 * (off[c] + q) + 1] = tile * q;
    }
}

// Sources in the (2k+1)^2 stencil of each cell (what the matvec stages for it).
__global__ void k_stencil_count(const int32_t* __restrict__ cell_start, const Prob* __restrict__ prob,
                                const int32_t* __restrict__ pid_cell, int64_t ncell, int32_t* __restrict__ out)
{
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const Prob& P = prob[pid_cell[c]];
    const int64_t lc = c - P.cellbase, cx = lc % P.ncx, cy = lc / P.ncx;
    const int64_t x0 = max(cx - P.k, (int64_t)0), x1 = min(cx + P.k, P.ncx - 1);
    const int64_t y0 = max(cy - P.k, (int64_t)0), y1 = min(cy + P.k, P.ncy - 1);
    int64_t s = 0;
    for (int64_t yy = y0; yy <= y1; ++yy)
        s += cell_start[P.cellbase + yy * P.ncx + x1 + 1] - cell_start[P.cellbase + yy * P.ncx + x0];
    out[c] = (int32_t)min(s, (int64_t)0x7fffffff);
}

// Candidate pairs of a cell grid: each cell's points times the points of its
// (2k+1)^2 stencil, summed over the cells (64-bit, one atomic per warp).
__global__ void k_candidate_count(const int32_t* __restrict__ cell_start, const Prob* __restrict__ prob,
                                  const int32_t* __restrict__ pid_cell, int64_t ncell,
                                  unsigned long long* __restrict__ total)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (c < ncell) {
        const Prob& P = prob[pid_cell[c]];
        const int64_t lc = c - P.cellbase, cx = lc % P.ncx, cy = lc / P.ncx;
        const int64_t x0 = max(cx - P.k, (int64_t)0), x1 = min(cx + P.k, P.ncx - 1);
        const int64_t y0 = max(cy - P.k, (int64_t)0), y1 = min(cy + P.k, P.ncy - 1);
        int64_t s = 0;
        for (int64_t yy = y0; yy <= y1; ++yy)
            s += cell_start[P.cellbase + yy * P.ncx + x1 + 1] - cell_start[P.cellbase + yy * P.ncx + x0];
        v = (unsigned long long)((int64_t)(cell_start[c + 1] - cell_start[c]) * s);
    }
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// Size class t (ceil(points / 32) == t) flags of the cells, and the scatter of
// the flagged cells as (cell, 0) items.
__global__ void k_flag_class(const int32_t* __restrict__ cell_start, int64_t ncell, int t,
                             const int32_t* __restrict__ pid_cell, const int32_t* __restrict__ prob_ok,
                             const int32_t* __restrict__ min_cls, int32_t* __restrict__ flag)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int cnt = cell_start[c + 1] - cell_start[c];
    const int pb = pid_cell[c];
    const int cls = max((cnt + 31) / 32, min_cls ? min_cls[pb] : 1);
    flag[c] = (cnt > 0 && cls == t && (!prob_ok || prob_ok[pb])) ? 1 : 0;
}

// Largest cell of each problem (atomic max per problem).
__global__ void k_prob_max_cell(const int32_t* __restrict__ cell_start, int64_t ncell,
                                const int32_t* __restrict__ pid_cell, int32_t* __restrict__ pmax)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int cnt = cell_start[c + 1] - cell_start[c];
    if (cnt > 0) atomicMax(&pmax[pid_cell[c]], cnt);
}

__global__ void k_scatter_cells(int64_t ncell, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                int32_t* __restrict__ out)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncell && flag[c]) {
        out[2 * (int64_t)pos[c]] = (int32_t)c;
        out[2 * (int64_t)pos[c] + 1] = 0;
    }
}


// Pairs (i, j), i = j included, of a cell grid with r2_ij <= R^2 by the FP64
// pair test (R = r_c on the main grid, the cell side on the inner grid, whose
// cells are as wide as its cutoff), summed as 64-bit (one atomic per warp).
__global__ void k_pair_count(const double* __restrict__ xy_s, const int32_t* __restrict__ cell_s,
                             const int32_t* __restrict__ cell_start, int64_t n, const Prob* __restrict__ prob,
                             const int32_t* __restrict__ pid, int inner, unsigned long long* __restrict__ total)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (p < n) {
        const Prob& P = prob[pid[p]];
        const double R2 = inner ? P.c * P.c : P.rc2;
        const int64_t lc = cell_s[p] - P.cellbase, cx = lc % P.ncx, cy = lc / P.ncx;
        const int64_t x0 = max(cx - P.k, (int64_t)0), x1 = min(cx + P.k, P.ncx - 1);
        const int64_t y0 = max(cy - P.k, (int64_t)0), y1 = min(cy + P.k, P.ncy - 1);
        const double xi = xy_s[2 * p], yi = xy_s[2 * p + 1];
        for (int64_t yy = y0; yy <= y1; ++yy) {
            const int32_t b = cell_start[P.cellbase + yy * P.ncx + x0], e = cell_start[P.cellbase + yy * P.ncx + x1 + 1];
            for (int32_t q = b; q < e; ++q)
                v += pair_r2(xi, yi, xy_s[2 * (int64_t)q], xy_s[2 * (int64_t)q + 1]) <= R2 ? 1u : 0u;
        }
    }
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// Order-preserving selection of matvec work items (cell, first target) and
// subdomains whose problem is active: flags, an exclusive scan, a scatter.
__global__ void k_flag_work(const int32_t* __restrict__ work, int64_t nwork, const int32_t* __restrict__ pid_cell,
                            const int32_t* __restrict__ active, int32_t* __restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nwork) flag[i] = active[pid_cell[work[2 * i]]] ? 1 : 0;
}

__global__ void k_scatter_work(const int32_t* __restrict__ work, int64_t nwork, const int32_t* __restrict__ flag,
                               const int32_t* __restrict__ pos, int32_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nwork && flag[i]) {
        out[2 * (int64_t)pos[i]] = work[2 * i];
        out[2 * (int64_t)pos[i] + 1] = work[2 * i + 1];
    }
}

__global__ void k_flag_sub(const int32_t* __restrict__ pid_sub, int64_t nsub, const int32_t* __restrict__ active,
                           int32_t* __restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsub) flag[i] = active[pid_sub[i]] ? 1 : 0;
}

__global__ void k_scatter_sub(int64_t nsub, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                              int32_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsub && flag[i]) out[pos[i]] = (int32_t)i;
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
                            const int32_t* __restrict__ cell_start, int64_t n, const Prob* __restrict__ prob,
                            const int32_t* __restrict__ pid, const int64_t* __restrict__ ptr,
                            int32_t* __restrict__ cnt, int32_t* __restrict__ idx, int mode)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t p = iperm[i];
    const Prob& P = prob[pid[p]];
    const int64_t ncx = P.ncx, ncy = P.ncy, k = P.k;
    double xi = xy_s[2 * (int64_t)p], yi = xy_s[2 * (int64_t)p + 1];
    int64_t c = cell_s[p] - P.cellbase;
    int64_t cx = c % ncx, cy = c / ncx;
    int64_t ylo = cy - k < 0 ? 0 : cy - k, yhi = cy + k > ncy - 1 ? ncy - 1 : cy + k;
    int64_t xlo = cx - k < 0 ? 0 : cx - k, xhi = cx + k > ncx - 1 ? ncx - 1 : cx + k;
    int64_t w = (mode == 1) ? ptr[i] : 0;
    int32_t count = 0;
    for (int64_t yy = ylo; yy <= yhi; ++yy) {
        int32_t b = cell_start[P.cellbase + yy * ncx + xlo], e = cell_start[P.cellbase + yy * ncx + xhi + 1];
        for (int32_t q = b; q < e; ++q) {
            double r2 = pair_r2(xi, yi, xy_s[2 * (int64_t)q], xy_s[2 * (int64_t)q + 1]);
            if (r2 <= P.rc2) {
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

// Cell of each evaluation point in problem 0's grid (clamped to the edge
// cells, so the (2k+1)^2 stencil still covers every source within r_c of a
// point outside the bounding box); flags a non-finite coordinate.
__global__ void k_target_count(const double* __restrict__ xe, int64_t m, const Prob* __restrict__ prob,
                               int32_t* __restrict__ cell_u, int32_t* __restrict__ counts, int* __restrict__ bad)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const Prob& P = prob[0];
    const double x = xe[2 * i], y = xe[2 * i + 1];
    int32_t cell = 0;
    if (isfinite(x) && isfinite(y)) {
        int64_t cx = cell_axis(x, P.xmin, P.c, P.ncx);
        int64_t cy = cell_axis(y, P.ymin, P.c, P.ncy);
        cell = (int32_t)(cy * P.ncx + cx);
    } else {
        *bad = 1;
    }
    cell_u[i] = cell;
    atomicAdd(&counts[cell], 1);
}

__global__ void k_remap(const int32_t* __restrict__ idx, int64_t cnt, const int32_t* __restrict__ map,
                        int32_t* __restrict__ out)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < cnt) out[e] = map[idx[e]];
}

// out[q] = r[perm[q]] * scale (inner order from main order, FP32)
__global__ void k_inner_gather_scaled(const double* __restrict__ r, const int32_t* __restrict__ perm, int64_t n,
                                      const double* __restrict__ scale, float* __restrict__ out)
{
    const double f = *scale;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        out[q] = (float)(r[perm[q]] * f);
}

// Inner order <-> main cell order without scaling (diagnostics of the inner operator).
__global__ void k_inner_from_main(const double* __restrict__ r, const int32_t* __restrict__ perm, int64_t n,
                                  float* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[q] = (float)r[perm[q]];
}

__global__ void k_main_from_inner(const float* __restrict__ v, const int32_t* __restrict__ perm, int64_t n,
                                  double* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) out[perm[q]] = (double)v[q];
}

__global__ void k_widen_i32_i64(const int32_t* __restrict__ in, int64_t n, int64_t* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

}  // namespace

// Work items (cell, first target) of tile T over cells with the given starts.
rbf_status build_work(rbf_ctx* ctx, const int32_t* cell_start, int64_t ncell, int tile, DevArray<int32_t>& work,
                      int64_t* nwork_out, cudaStream_t st)
{
    RBF_LAUNCH(ctx, k_work_count, blocks_for(ncell, 256), 256, 0, st, cell_start, ncell, tile, ctx->mv_wcnt.p);
    RBF_CHECK(exclusive_scan_i32(ctx, ctx->mv_wcnt.p, ctx->mv_woff.p, ncell, st));
    int32_t nwork = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&nwork, ctx->mv_woff.p + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    *nwork_out = nwork;
    RBF_CHECK(ensure(ctx, work, 2 * (size_t)std::max<int32_t>(nwork, 1)));
    RBF_LAUNCH(ctx, k_work_fill, blocks_for(ncell, 256), 256, 0, st, ctx->mv_wcnt.p, ctx->mv_woff.p, ncell, tile,
               work.p);
    return RBF_OK;
}

static rbf_status build_class_lists(rbf_ctx* ctx, const int32_t* cell_start, int64_t ncell, int max_tpl,
                                    const int32_t* pid_cell, const int32_t* prob_ok, const int32_t* min_cls,
                                    DevArray<int32_t>& lists, int64_t* off, int32_t* flag, int32_t* pos,
                                    cudaStream_t st);
namespace {
rbf_status select_work_into(rbf_ctx* ctx, const int32_t* work, int64_t nwork, const int32_t* pid_cell,
                            const int32_t* active, int32_t* out, int64_t* nout, cudaStream_t st);
}  // namespace

// Bins all problems of ctx->prob_h (kernel parameters and point ranges filled
// in; grids are set here from the bounding boxes).
rbf_status bin_points(rbf_ctx* ctx, const double* xy, cudaStream_t st)
{
    ctx->f64s.valid = false;   // the kept pair values belong to the previous binning
    ctx->f64s.tried = false;
    const int64_t n = ctx->n;
    const int nprob = (int)ctx->nprob;
    std::vector<Prob>& P = ctx->prob_h;
    // problem of every point
    std::vector<int64_t> pbeg(nprob + 1);
    for (int b = 0; b < nprob; ++b) pbeg[b] = P[b].pbeg;
    pbeg[nprob] = n;
    RBF_CHECK(ensure(ctx, ctx->pbeg_dev, nprob + 1));
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->pbeg_dev.p, pbeg.data(), sizeof(int64_t) * (nprob + 1), cudaMemcpyHostToDevice,
                                  st));
    RBF_CHECK(ensure(ctx, ctx->pid, n));
    RBF_LAUNCH(ctx, k_pid, blocks_for(n, 256), 256, 0, st, ctx->pbeg_dev.p, nprob, n, ctx->pid.p);
    // bounding boxes
    const int64_t ntile = (n + kBoxTile - 1) / kBoxTile;
    RBF_CHECK(ensure(ctx, ctx->bbox_part, 4 * (size_t)nprob));   // keys, reinterpreted
    RBF_CHECK(ensure(ctx, ctx->bbox_dev, 4 * (size_t)nprob));
    unsigned long long* keys = (unsigned long long*)ctx->bbox_part.p;
    RBF_CUDA(ctx, cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * 4 * nprob, st));
    RBF_LAUNCH(ctx, k_bbox, (unsigned)ntile, 256, 0, st, xy, n, ctx->pid.p, keys);
    RBF_LAUNCH(ctx, k_bbox_final, blocks_for(nprob, 128), 128, 0, st, keys, nprob, ctx->bbox_dev.p);
    std::vector<double> bb(4 * (size_t)nprob);
    RBF_CUDA(ctx, cudaMemcpyAsync(bb.data(), ctx->bbox_dev.p, sizeof(double) * 4 * nprob, cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    int64_t ncell = 0;
    for (int b = 0; b < nprob; ++b) {
        Prob& q = P[b];
        q.xmin = bb[4 * b]; q.ymin = bb[4 * b + 1]; q.xmax = bb[4 * b + 2]; q.ymax = bb[4 * b + 3];
        if (!std::isfinite(q.xmin) || !std::isfinite(q.ymin) || !std::isfinite(q.xmax) || !std::isfinite(q.ymax))
            return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: non-finite coordinate in problem %d", b);
        double fx = std::floor((q.xmax - q.xmin) / q.c), fy = std::floor((q.ymax - q.ymin) / q.c);
        if (!(fx < 1.0e9) || !(fy < 1.0e9)) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: grid too large");
        q.ncx = (int64_t)fx + 1;
        q.ncy = (int64_t)fy + 1;
        q.cellbase = ncell;
        const double amax = std::max(std::max(std::fabs(q.xmin), std::fabs(q.xmax)),
                                     std::max(std::fabs(q.ymin), std::fabs(q.ymax)));
        if (!make_fx_constants(amax, q.rc, q.s, &q.fx_scale, &q.fx_sh, &q.fx_F, &q.fx_M))
            return fail(ctx, RBF_ERR_INVALID_ARG,
                        "rbf_bin: cutoff %g out of range for the coordinates (max |x| %g) or for sigma (problem %d)",
                        q.rc, amax, b);
        ncell += q.ncx * q.ncy;
        if (ncell > ((int64_t)1 << 28))
            return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: %lld cells exceed 2^28 (cell_size too small)",
                        (long long)ncell);
    }
    ctx->ncell_total = ncell;
    if (nprob == 1) {
        ctx->bbox[0] = P[0].xmin; ctx->bbox[1] = P[0].ymin; ctx->bbox[2] = P[0].xmax; ctx->bbox[3] = P[0].ymax;
        ctx->ncx = P[0].ncx;
        ctx->ncy = P[0].ncy;
    }
    RBF_CHECK(ensure(ctx, ctx->prob, nprob));
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->prob.p, P.data(), sizeof(Prob) * nprob, cudaMemcpyHostToDevice, st));

    RBF_CHECK(ensure(ctx, ctx->counts, ncell + 1));
    RBF_CHECK(ensure(ctx, ctx->cell_start, ncell + 1));
    RBF_CHECK(ensure(ctx, ctx->cell_u, n));
    RBF_CHECK(ensure(ctx, ctx->cell_s, n));
    RBF_CHECK(ensure(ctx, ctx->perm, n));
    RBF_CHECK(ensure(ctx, ctx->iperm, n));
    RBF_CHECK(ensure(ctx, ctx->tmp_i32, std::max<int64_t>(n, 2 * kNumSMs + 1)));
    RBF_CHECK(ensure(ctx, ctx->xy_s, 2 * n));
    RBF_CHECK(ensure(ctx, ctx->pid_cell, ncell));

    RBF_CHECK(prof_begin(ctx, RBF_PROF_BIN, st));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_cell_count, blocks_for(n, 256), 256, 0, st, xy, n, ctx->prob.p, ctx->pid.p, ctx->cell_u.p,
               ctx->counts.p);
    RBF_CHECK(exclusive_scan_i32(ctx, ctx->counts.p, ctx->cell_start.p, ncell, st));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_cell_scatter, blocks_for(n, 256), 256, 0, st, ctx->cell_u.p, n, ctx->cell_start.p,
               ctx->counts.p, ctx->tmp_i32.p);
    RBF_LAUNCH(ctx, k_cell_rank, blocks_for(ncell * 32, 256), 256, 0, st, ctx->cell_start.p, ncell, ctx->tmp_i32.p,
               ctx->perm.p);
    RBF_LAUNCH(ctx, k_gather_sorted, blocks_for(n, 256), 256, 0, st, xy, n, ctx->perm.p, ctx->cell_u.p, ctx->xy_s.p,
               ctx->iperm.p, ctx->cell_s.p);
    RBF_LAUNCH(ctx, k_pid_cells, blocks_for(ncell, 256), 256, 0, st, ctx->prob.p, nprob, ncell, ctx->pid_cell.p);
    RBF_CHECK(ensure(ctx, ctx->loc32, 2 * n));
    RBF_LAUNCH(ctx, k_local_coords, blocks_for(n, 256), 256, 0, st, ctx->xy_s.p, ctx->cell_s.p, n, ctx->prob.p,
               ctx->pid.p, ctx->loc32.p);
    RBF_CHECK(ensure(ctx, ctx->mv_wcnt, ncell + 1));
    RBF_CHECK(ensure(ctx, ctx->mv_woff, ncell + 1));
    RBF_CHECK(build_work(ctx, ctx->cell_start.p, ncell, ctx->tile64, ctx->mv_work, &ctx->n_work, st));
    RBF_CHECK(build_work(ctx, ctx->cell_start.p, ncell, ctx->tile32, ctx->mv_work32, &ctx->n_work32, st));
    // the largest stencil any cell stages
    RBF_LAUNCH(ctx, k_stencil_count, blocks_for(ncell, 256), 256, 0, st, ctx->cell_start.p, ctx->prob.p,
               ctx->pid_cell.p, ncell, ctx->mv_wcnt.p);
    int32_t smax = 0;
    RBF_CHECK(reduce_max_i32(ctx, ctx->mv_wcnt.p, ncell, &smax, st));
    ctx->stage_max = smax;
    // When enabled, the symmetric FP64 matvec serves each problem whose
    // stencil is 3 x 3 (cells as wide as r_c) and whose cells hold at most 160
    // points; the stencil kernel serves the others. The choice depends on the
    // problem alone, so a problem sums in the same order alone and in any
    // batch. The class lists, the other problems' work list and the slots are
    // made here, outside any graph capture.
    ctx->sym64 = ctx->sym64_all = false;
    if (ctx->sym64_mode == 0) {
        RBF_CHECK(ensure(ctx, ctx->sym64_prob, 2 * (size_t)nprob));
        int32_t* pmax = ctx->sym64_prob.p + nprob;
        RBF_CUDA(ctx, cudaMemsetAsync(pmax, 0, sizeof(int32_t) * nprob, st));
        RBF_LAUNCH(ctx, k_prob_max_cell, blocks_for(ncell, 256), 256, 0, st, ctx->cell_start.p, ncell,
                   ctx->pid_cell.p, pmax);
        std::vector<int32_t> hmax(nprob), ok(2 * (size_t)nprob);
        RBF_CUDA(ctx, cudaMemcpyAsync(hmax.data(), pmax, sizeof(int32_t) * nprob, cudaMemcpyDeviceToHost, st));
        RBF_CUDA(ctx, cudaStreamSynchronize(st));
        int64_t nsym = 0;
        for (int b = 0; b < nprob; ++b) {
            ok[b] = (P[b].k == 1 && hmax[b] <= 160) ? 1 : 0;
            ok[nprob + b] = 1 - ok[b];
            nsym += ok[b];
        }
        ctx->sym64 = nsym > 0;
        ctx->sym64_all = nsym == nprob;
        // [0, nprob): symmetric kernel; [nprob, 2 nprob): stencil kernel
        RBF_CUDA(ctx, cudaMemcpyAsync(ctx->sym64_prob.p, ok.data(), sizeof(int32_t) * 2 * nprob, cudaMemcpyHostToDevice,
                                      st));
        if (ctx->sym64) {
            RBF_CHECK(ensure(ctx, ctx->tmp_i32, std::max<int64_t>(2 * (ncell + 1), n)));
            RBF_CHECK(build_class_lists(ctx, ctx->cell_start.p, ncell, 5, ctx->pid_cell.p, ctx->sym64_prob.p, nullptr,
                                        ctx->sym64w, ctx->sym64off, ctx->tmp_i32.p, ctx->tmp_i32.p + (ncell + 1),
                                        st));
            RBF_CHECK(ensure(ctx, ctx->sym64_slots, (size_t)(5 * n)));
            RBF_CHECK(ensure(ctx, ctx->mv_work_ns, 2 * (size_t)std::max<int64_t>(ctx->n_work, 1)));
            RBF_CHECK(select_work_into(ctx, ctx->mv_work.p, ctx->n_work, ctx->pid_cell.p, ctx->sym64_prob.p + nprob,
                                       ctx->mv_work_ns.p, &ctx->n_work_ns, st));
        }
    }
    RBF_CHECK(matvec_prepare(ctx));
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
               ctx->cell_s.p, ctx->cell_start.p, n, ctx->prob.p, ctx->pid.p, (const int64_t*)nullptr, ctx->nbr_cnt.p,
               (int32_t*)nullptr, 0);
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
               ctx->cell_s.p, ctx->cell_start.p, n, ctx->prob.p, ctx->pid.p, (const int64_t*)p64, ctx->nbr_cnt.p, idx,
               1);
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    return RBF_OK;
}

// Bins m evaluation points (user order, device) into the grid of problem 0:
// cell-sorted coordinates, FP32 offsets, per-cell ranges and work items for
// the matvec kernel, in ctx->ev. INVALID_ARG for a non-finite coordinate.
rbf_status bin_targets(rbf_ctx* ctx, const double* xe, int64_t m, cudaStream_t st)
{
    EvalBins& E = ctx->ev;
    const int64_t ncell = ctx->ncell_total;
    RBF_CHECK(ensure(ctx, E.pid, m));
    RBF_CHECK(ensure(ctx, E.cell_u, m));
    RBF_CHECK(ensure(ctx, E.cell_s, m));
    RBF_CHECK(ensure(ctx, E.perm, m));
    RBF_CHECK(ensure(ctx, E.iperm, m));
    RBF_CHECK(ensure(ctx, E.tmp, std::max<int64_t>(m, 2 * kNumSMs + 1)));
    RBF_CHECK(ensure(ctx, E.counts, ncell + 1));
    RBF_CHECK(ensure(ctx, E.cell_start, ncell + 1));
    RBF_CHECK(ensure(ctx, E.wcnt, ncell + 1));
    RBF_CHECK(ensure(ctx, E.woff, ncell + 1));
    RBF_CHECK(ensure(ctx, E.xy_s, 2 * m));
    RBF_CHECK(ensure(ctx, E.loc, 2 * m));
    RBF_CHECK(ensure(ctx, E.flag, 1));
    RBF_CUDA(ctx, cudaMemsetAsync(E.pid.p, 0, sizeof(int32_t) * m, st));
    RBF_CUDA(ctx, cudaMemsetAsync(E.flag.p, 0, sizeof(int), st));
    RBF_CUDA(ctx, cudaMemsetAsync(E.counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_target_count, blocks_for(m, 256), 256, 0, st, xe, m, ctx->prob.p, E.cell_u.p, E.counts.p,
               E.flag.p);
    RBF_CHECK(exclusive_scan_i32(ctx, E.counts.p, E.cell_start.p, ncell, st));
    RBF_CUDA(ctx, cudaMemsetAsync(E.counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_cell_scatter, blocks_for(m, 256), 256, 0, st, E.cell_u.p, m, E.cell_start.p, E.counts.p,
               E.tmp.p);
    RBF_LAUNCH(ctx, k_cell_rank, blocks_for(ncell * 32, 256), 256, 0, st, E.cell_start.p, ncell, E.tmp.p, E.perm.p);
    RBF_LAUNCH(ctx, k_gather_sorted, blocks_for(m, 256), 256, 0, st, xe, m, E.perm.p, E.cell_u.p, E.xy_s.p,
               E.iperm.p, E.cell_s.p);
    RBF_LAUNCH(ctx, k_local_coords, blocks_for(m, 256), 256, 0, st, E.xy_s.p, E.cell_s.p, m, ctx->prob.p, E.pid.p,
               E.loc.p);
    RBF_LAUNCH(ctx, k_work_count, blocks_for(ncell, 256), 256, 0, st, E.cell_start.p, ncell, ctx->tile64, E.wcnt.p);
    RBF_CHECK(exclusive_scan_i32(ctx, E.wcnt.p, E.woff.p, ncell, st));
    int32_t hv[2] = {0, 0};
    RBF_CUDA(ctx, cudaMemcpyAsync(&hv[0], E.woff.p + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(&hv[1], E.flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    if (hv[1]) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_eval: non-finite evaluation point");
    E.m = m;
    E.nwork = hv[0];
    RBF_CHECK(ensure(ctx, E.work, 2 * (size_t)std::max<int32_t>(hv[0], 1)));
    RBF_LAUNCH(ctx, k_work_fill, blocks_for(ncell, 256), 256, 0, st, E.wcnt.p, E.woff.p, ncell, ctx->tile64,
               E.work.p);
    return RBF_OK;
}

rbf_status targets_to_user(rbf_ctx* ctx, const double* sorted, double* user, cudaStream_t st)
{
    RBF_LAUNCH(ctx, k_permute_to_user, blocks_for(ctx->ev.m, 256), 256, 0, st, sorted, ctx->ev.perm.p, ctx->ev.m,
               user);
    return RBF_OK;
}

// Cell lists by size class for the symmetric matvecs: non-empty cells of
// class t = max(ceil(points / 32), min_cls of their problem), t = 1..max_tpl,
// of the problems prob_ok marks (all when it is null; min_cls null: 1), as
// (cell, 0) items in `lists` (class t holds [off[t-1], off[t])), order kept
// within a class. flag and pos are scratch of ncell + 1 entries each.
static rbf_status build_class_lists(rbf_ctx* ctx, const int32_t* cell_start, int64_t ncell, int max_tpl,
                                    const int32_t* pid_cell, const int32_t* prob_ok, const int32_t* min_cls,
                                    DevArray<int32_t>& lists, int64_t* off, int32_t* flag, int32_t* pos,
                                    cudaStream_t st)
{
    RBF_CHECK(ensure(ctx, lists, 2 * (size_t)std::max<int64_t>(ncell, 1)));
    off[0] = 0;
    for (int t = 1; t <= max_tpl; ++t) {
        RBF_LAUNCH(ctx, k_flag_class, blocks_for(ncell, 256), 256, 0, st, cell_start, ncell, t, pid_cell, prob_ok,
                   min_cls, flag);
        RBF_CHECK(exclusive_scan_i32(ctx, flag, pos, ncell, st));
        RBF_LAUNCH(ctx, k_scatter_cells, blocks_for(ncell, 256), 256, 0, st, ncell, flag, pos, lists.p + 2 * off[t - 1]);
        int32_t cnt = 0;
        RBF_CUDA(ctx, cudaMemcpyAsync(&cnt, pos + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RBF_CUDA(ctx, cudaStreamSynchronize(st));
        off[t] = off[t - 1] + cnt;
    }
    return RBF_OK;
}

rbf_status bin_inner(rbf_ctx* ctx, double ri_sigmas, cudaStream_t st)
{
    InnerGrid& G = ctx->in;
    const int64_t n = ctx->n;
    const int nprob = (int)ctx->nprob;
    std::vector<Prob> P = ctx->prob_h;   // the main tables with the grid replaced
    int64_t ncell = 0;
    for (int b = 0; b < nprob; ++b) {
        Prob& q = P[b];
        q.c = std::min(ri_sigmas * q.sigma, q.rc);
        const double fx = std::floor((q.xmax - q.xmin) / q.c), fy = std::floor((q.ymax - q.ymin) / q.c);
        if (!(fx < 1.0e9) || !(fy < 1.0e9)) return fail(ctx, RBF_ERR_INVALID_ARG, "inner grid too large");
        q.ncx = (int64_t)fx + 1;
        q.ncy = (int64_t)fy + 1;
        q.k = 1;
        q.ca = (float)(q.c * (double)q.a_loc);
        q.cellbase = ncell;
        ncell += q.ncx * q.ncy;
        if (ncell > ((int64_t)1 << 28)) return fail(ctx, RBF_ERR_INVALID_ARG, "inner grid: too many cells");
    }
    G.ready = false;
    G.ncell = ncell;
    RBF_CHECK(ensure(ctx, G.prob, nprob));
    RBF_CUDA(ctx, cudaMemcpyAsync(G.prob.p, P.data(), sizeof(Prob) * nprob, cudaMemcpyHostToDevice, st));
    RBF_CHECK(ensure(ctx, G.cell_u, n));
    RBF_CHECK(ensure(ctx, G.cell_s, n));
    RBF_CHECK(ensure(ctx, G.perm, n));
    RBF_CHECK(ensure(ctx, G.iperm, n));
    RBF_CHECK(ensure(ctx, G.tmp, std::max<int64_t>(n, 2 * kNumSMs + 1)));
    RBF_CHECK(ensure(ctx, G.counts, ncell + 1));
    RBF_CHECK(ensure(ctx, G.cell_start, ncell + 1));
    RBF_CHECK(ensure(ctx, G.pid_cell, ncell));
    RBF_CHECK(ensure(ctx, G.wcnt, ncell + 1));
    RBF_CHECK(ensure(ctx, G.woff, ncell + 1));
    RBF_CHECK(ensure(ctx, G.xy_s, 2 * n));
    RBF_CHECK(ensure(ctx, G.loc, 2 * n));
    // counting sort of the main cell-ordered points by inner cell (ties: main position)
    RBF_CUDA(ctx, cudaMemsetAsync(G.counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_cell_count, blocks_for(n, 256), 256, 0, st, ctx->xy_s.p, n, G.prob.p, ctx->pid.p, G.cell_u.p,
               G.counts.p);
    RBF_CHECK(exclusive_scan_i32(ctx, G.counts.p, G.cell_start.p, ncell, st));
    RBF_CUDA(ctx, cudaMemsetAsync(G.counts.p, 0, sizeof(int32_t) * (ncell + 1), st));
    RBF_LAUNCH(ctx, k_cell_scatter, blocks_for(n, 256), 256, 0, st, G.cell_u.p, n, G.cell_start.p, G.counts.p,
               G.tmp.p);
    RBF_LAUNCH(ctx, k_cell_rank, blocks_for(ncell * 32, 256), 256, 0, st, G.cell_start.p, ncell, G.tmp.p, G.perm.p);
    RBF_LAUNCH(ctx, k_gather_sorted, blocks_for(n, 256), 256, 0, st, ctx->xy_s.p, n, G.perm.p, G.cell_u.p, G.xy_s.p,
               G.iperm.p, G.cell_s.p);
    RBF_LAUNCH(ctx, k_pid_cells, blocks_for(ncell, 256), 256, 0, st, G.prob.p, nprob, ncell, G.pid_cell.p);
    RBF_LAUNCH(ctx, k_local_coords, blocks_for(n, 256), 256, 0, st, G.xy_s.p, G.cell_s.p, n, G.prob.p, ctx->pid.p,
               G.loc.p);
    // work items of the FP32 kernel and the largest stencil
    RBF_LAUNCH(ctx, k_work_count, blocks_for(ncell, 256), 256, 0, st, G.cell_start.p, ncell, G.tile, G.wcnt.p);
    RBF_CHECK(exclusive_scan_i32(ctx, G.wcnt.p, G.woff.p, ncell, st));
    int32_t nwork = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&nwork, G.woff.p + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    G.n_work = nwork;
    RBF_CHECK(ensure(ctx, G.work, 2 * (size_t)std::max<int32_t>(nwork, 1)));
    RBF_LAUNCH(ctx, k_work_fill, blocks_for(ncell, 256), 256, 0, st, G.wcnt.p, G.woff.p, ncell, G.tile, G.work.p);
    RBF_LAUNCH(ctx, k_stencil_count, blocks_for(ncell, 256), 256, 0, st, G.cell_start.p, G.prob.p, G.pid_cell.p,
               ncell, G.wcnt.p);
    int32_t smax = 0;
    RBF_CHECK(reduce_max_i32(ctx, G.wcnt.p, ncell, &smax, st));
    G.stage_max = smax;
    // the symmetric FP32 kernel serves each problem whose inner cells hold at
    // most 128 points (four targets per lane), the stencil kernel the others:
    // a choice made per problem, so that it sums alike alone and in a batch
    {
        RBF_CHECK(ensure(ctx, G.sym_prob, 3 * (size_t)nprob));
        int32_t* pmax = G.sym_prob.p + nprob;
        RBF_CUDA(ctx, cudaMemsetAsync(pmax, 0, sizeof(int32_t) * nprob, st));
        RBF_LAUNCH(ctx, k_prob_max_cell, blocks_for(ncell, 256), 256, 0, st, G.cell_start.p, ncell, G.pid_cell.p, pmax);
        std::vector<int32_t> hmax(nprob), ok(3 * (size_t)nprob);
        RBF_CUDA(ctx, cudaMemcpyAsync(hmax.data(), pmax, sizeof(int32_t) * nprob, cudaMemcpyDeviceToHost, st));
        RBF_CUDA(ctx, cudaStreamSynchronize(st));
        int64_t nsym = 0;
        for (int b = 0; b < nprob; ++b) {
            ok[b] = hmax[b] <= 128 ? 1 : 0;
            ok[nprob + b] = 1 - ok[b];
            // a problem with cells of more than 32 points takes its smaller
            // (edge) cells in the two-target class too: one launch less, the
            // same sums (the second target of such a lane is empty)
            ok[2 * nprob + b] = hmax[b] > 32 ? 2 : 1;
            nsym += ok[b];
        }
        G.sym = nsym > 0;
        G.sym_all = nsym == nprob;
        RBF_CUDA(ctx, cudaMemcpyAsync(G.sym_prob.p, ok.data(), sizeof(int32_t) * 3 * nprob, cudaMemcpyHostToDevice, st));
    }
    if (G.sym) {
        // its slots are allocated here, outside the solver's graph capture
        RBF_CHECK(ensure(ctx, ctx->sym_slots, (size_t)(5 * n)));
        // its cell lists by size class (order kept within a class)
        RBF_CHECK(ensure(ctx, G.tmp, std::max<int64_t>(2 * (ncell + 1), 2 * kNumSMs + 1)));
        RBF_CHECK(build_class_lists(ctx, G.cell_start.p, ncell, 4, G.pid_cell.p, G.sym_prob.p, G.sym_prob.p + 2 * nprob,
                                    G.symw, G.symoff,
                                    G.tmp.p, G.tmp.p + (ncell + 1), st));
        RBF_CHECK(ensure(ctx, G.work_ns, 2 * (size_t)std::max<int64_t>(G.n_work, 1)));
        RBF_CHECK(select_work_into(ctx, G.work.p, G.n_work, G.pid_cell.p, G.sym_prob.p + nprob, G.work_ns.p,
                                   &G.n_work_ns, st));
    }
    // subdomain lists in inner positions
    if (ctx->rasm_ready) {
        int32_t tot[2] = {0, 0};
        RBF_CUDA(ctx, cudaMemcpyAsync(&tot[0], ctx->core_ptr.p + ctx->nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RBF_CUDA(ctx, cudaMemcpyAsync(&tot[1], ctx->ov_ptr.p + ctx->nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RBF_CUDA(ctx, cudaStreamSynchronize(st));
        RBF_CHECK(ensure(ctx, G.core_idx, std::max<int32_t>(tot[0], 1)));
        RBF_CHECK(ensure(ctx, G.ov_idx, std::max<int32_t>(tot[1], 1)));
        RBF_LAUNCH(ctx, k_remap, blocks_for(tot[0], 256), 256, 0, st, ctx->core_idx.p, (int64_t)tot[0], G.iperm.p,
                   G.core_idx.p);
        RBF_LAUNCH(ctx, k_remap, blocks_for(tot[1], 256), 256, 0, st, ctx->ov_idx.p, (int64_t)tot[1], G.iperm.p,
                   G.ov_idx.p);
    }
    G.ri_sigmas = ri_sigmas;
    G.ready = true;
    return RBF_OK;
}

rbf_status inner_gather_scaled(rbf_ctx* ctx, const double* r_main, const double* scale_dev, float* out_inner,
                               cudaStream_t st)
{
    RBF_LAUNCH(ctx, k_inner_gather_scaled, blocks_for(std::min<int64_t>(ctx->n, 16 * kNumSMs * 256), 256), 256, 0, st,
               r_main, ctx->in.perm.p, ctx->n, scale_dev, out_inner);
    return RBF_OK;
}

rbf_status inner_matvec_debug(rbf_ctx* ctx, double ri_sigmas, const double* w_main, double* y_main, int variant,
                              cudaStream_t st)
{
    if (!ctx->in.ready || ctx->in.ri_sigmas != ri_sigmas) RBF_CHECK(bin_inner(ctx, ri_sigmas, st));
    if (variant == 0 && !ctx->in.sym)
        return fail(ctx, RBF_ERR_STATE, "rbf_debug_inner_matvec: an inner cell holds more than 128 points");
    const int64_t n = ctx->n;
    RBF_CHECK(ensure(ctx, ctx->vec_c, (size_t)n));   // two FP32 vectors
    float* wf = (float*)ctx->vec_c.p;
    float* yf = wf + n;
    RBF_LAUNCH(ctx, k_inner_from_main, blocks_for(n, 256), 256, 0, st, w_main, ctx->in.perm.p, n, wf);
    const bool on = ctx->inner_on;
    const int mode = ctx->sym_mode;
    ctx->inner_on = true;
    ctx->sym_mode = variant;
    const rbf_status s = matvec_f32_raw(ctx, nullptr, wf, yf, st);
    ctx->inner_on = on;
    ctx->sym_mode = mode;
    RBF_CHECK(s);
    RBF_LAUNCH(ctx, k_main_from_inner, blocks_for(n, 256), 256, 0, st, yf, ctx->in.perm.p, n, y_main);
    return RBF_OK;
}

rbf_status count_candidates(rbf_ctx* ctx, int grid, int64_t* total, cudaStream_t st)
{
    const int32_t* cs;
    const Prob* pr;
    const int32_t* pc;
    int64_t ncell;
    if (grid == 0) {
        cs = ctx->cell_start.p;
        pr = ctx->prob.p;
        pc = ctx->pid_cell.p;
        ncell = ctx->ncell_total;
    } else {
        const InnerGrid& G = ctx->in;
        cs = G.cell_start.p;
        pr = G.prob.p;
        pc = G.pid_cell.p;
        ncell = G.ncell;
    }
    RBF_CHECK(ensure(ctx, ctx->count_u64, 1));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->count_u64.p, 0, sizeof(unsigned long long), st));
    if (ncell > 0)
        RBF_LAUNCH(ctx, k_candidate_count, blocks_for(ncell, 256), 256, 0, st, cs, pr, pc, ncell, ctx->count_u64.p);
    unsigned long long h = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&h, ctx->count_u64.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    *total = (int64_t)h;
    return RBF_OK;
}

rbf_status count_pairs(rbf_ctx* ctx, int grid, int64_t* total, cudaStream_t st)
{
    const bool inner = grid == 1;
    const InnerGrid& G = ctx->in;
    RBF_CHECK(ensure(ctx, ctx->count_u64, 1));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->count_u64.p, 0, sizeof(unsigned long long), st));
    RBF_LAUNCH(ctx, k_pair_count, blocks_for(ctx->n, 128), 128, 0, st, inner ? G.xy_s.p : ctx->xy_s.p,
               inner ? G.cell_s.p : ctx->cell_s.p, inner ? G.cell_start.p : ctx->cell_start.p, ctx->n,
               inner ? G.prob.p : ctx->prob.p, ctx->pid.p, inner ? 1 : 0, ctx->count_u64.p);
    unsigned long long h = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&h, ctx->count_u64.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    *total = (int64_t)h;
    return RBF_OK;
}

namespace {

// The items of `work` whose problem is active, in order, written to out (room for nwork items).
rbf_status select_work_into(rbf_ctx* ctx, const int32_t* work, int64_t nwork, const int32_t* pid_cell,
                            const int32_t* active, int32_t* out, int64_t* nout, cudaStream_t st)
{
    RBF_CHECK(ensure(ctx, ctx->al.flag, std::max<int64_t>(nwork, 1)));
    RBF_CHECK(ensure(ctx, ctx->al.pos, std::max<int64_t>(nwork, 1) + 1));
    if (nwork == 0) {
        *nout = 0;
        return RBF_OK;
    }
    RBF_LAUNCH(ctx, k_flag_work, blocks_for(nwork, 256), 256, 0, st, work, nwork, pid_cell, active, ctx->al.flag.p);
    RBF_CHECK(exclusive_scan_i32(ctx, ctx->al.flag.p, ctx->al.pos.p, nwork, st));
    RBF_LAUNCH(ctx, k_scatter_work, blocks_for(nwork, 256), 256, 0, st, work, nwork, ctx->al.flag.p, ctx->al.pos.p,
               out);
    int32_t cnt = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&cnt, ctx->al.pos.p + nwork, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    *nout = cnt;
    return RBF_OK;
}

rbf_status select_work(rbf_ctx* ctx, const int32_t* work, int64_t nwork, const int32_t* pid_cell,
                       const int32_t* active, DevArray<int32_t>& out, int64_t* nout, cudaStream_t st)
{
    RBF_CHECK(ensure(ctx, ctx->al.flag, std::max<int64_t>(nwork, 1)));
    RBF_CHECK(ensure(ctx, ctx->al.pos, std::max<int64_t>(nwork, 1) + 1));
    RBF_CHECK(ensure(ctx, out, 2 * std::max<int64_t>(nwork, 1)));
    if (nwork == 0) {
        *nout = 0;
        return RBF_OK;
    }
    RBF_LAUNCH(ctx, k_flag_work, blocks_for(nwork, 256), 256, 0, st, work, nwork, pid_cell, active, ctx->al.flag.p);
    RBF_CHECK(exclusive_scan_i32(ctx, ctx->al.flag.p, ctx->al.pos.p, nwork, st));
    RBF_LAUNCH(ctx, k_scatter_work, blocks_for(nwork, 256), 256, 0, st, work, nwork, ctx->al.flag.p, ctx->al.pos.p,
               out.p);
    int32_t cnt = 0;
    RBF_CUDA(ctx, cudaMemcpyAsync(&cnt, ctx->al.pos.p + nwork, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    *nout = cnt;
    return RBF_OK;
}

}  // namespace

rbf_status build_active_lists(rbf_ctx* ctx, const int32_t* active, cudaStream_t st)
{
    ctx->al.on = false;
    RBF_CHECK(select_work(ctx, ctx->mv_work.p, ctx->n_work, ctx->pid_cell.p, active, ctx->al.w64, &ctx->al.n64, st));
    if (ctx->sym64) {   // the symmetric FP64 kernel's class lists and the other problems' stencil items
        RBF_CHECK(ensure(ctx, ctx->al.sym64w, 2 * (size_t)std::max<int64_t>(ctx->sym64off[5], 1)));
        ctx->al.sym64off[0] = 0;
        for (int t = 1; t <= 5; ++t) {
            int64_t got = 0;
            RBF_CHECK(select_work_into(ctx, ctx->sym64w.p + 2 * ctx->sym64off[t - 1],
                                       ctx->sym64off[t] - ctx->sym64off[t - 1], ctx->pid_cell.p, active,
                                       ctx->al.sym64w.p + 2 * ctx->al.sym64off[t - 1], &got, st));
            ctx->al.sym64off[t] = ctx->al.sym64off[t - 1] + got;
        }
        RBF_CHECK(ensure(ctx, ctx->al.w64ns, 2 * (size_t)std::max<int64_t>(ctx->n_work_ns, 1)));
        RBF_CHECK(select_work_into(ctx, ctx->mv_work_ns.p, ctx->n_work_ns, ctx->pid_cell.p, active, ctx->al.w64ns.p,
                                   &ctx->al.n64ns, st));
    }
    if (ctx->inner_on)
        RBF_CHECK(select_work(ctx, ctx->in.work.p, ctx->in.n_work, ctx->in.pid_cell.p, active, ctx->al.w32,
                              &ctx->al.n32, st));
    else
        RBF_CHECK(select_work(ctx, ctx->mv_work32.p, ctx->n_work32, ctx->pid_cell.p, active, ctx->al.w32,
                              &ctx->al.n32, st));
    if (ctx->inner_on && ctx->in.sym) {   // the symmetric kernel's class lists, each filtered in order
        const InnerGrid& G = ctx->in;
        RBF_CHECK(ensure(ctx, ctx->al.symw, 2 * (size_t)std::max<int64_t>(G.symoff[4], 1)));
        ctx->al.symoff[0] = 0;
        for (int t = 1; t <= 4; ++t) {
            int64_t got = 0;
            RBF_CHECK(select_work_into(ctx, G.symw.p + 2 * G.symoff[t - 1], G.symoff[t] - G.symoff[t - 1],
                                       G.pid_cell.p, active, ctx->al.symw.p + 2 * ctx->al.symoff[t - 1], &got, st));
            ctx->al.symoff[t] = ctx->al.symoff[t - 1] + got;
        }
        RBF_CHECK(ensure(ctx, ctx->al.w32ns, 2 * (size_t)std::max<int64_t>(G.n_work_ns, 1)));
        RBF_CHECK(select_work_into(ctx, G.work_ns.p, G.n_work_ns, G.pid_cell.p, active, ctx->al.w32ns.p,
                                   &ctx->al.n32ns, st));
    }
    const int64_t nsub = ctx->nsub;
    RBF_CHECK(ensure(ctx, ctx->al.flag, std::max<int64_t>(nsub, 1)));
    RBF_CHECK(ensure(ctx, ctx->al.pos, std::max<int64_t>(nsub, 1) + 1));
    RBF_CHECK(ensure(ctx, ctx->al.sub, std::max<int64_t>(nsub, 1)));
    int32_t cnt = 0;
    if (nsub > 0) {
        RBF_LAUNCH(ctx, k_flag_sub, blocks_for(nsub, 256), 256, 0, st, ctx->pid_sub.p, nsub, active, ctx->al.flag.p);
        RBF_CHECK(exclusive_scan_i32(ctx, ctx->al.flag.p, ctx->al.pos.p, nsub, st));
        RBF_LAUNCH(ctx, k_scatter_sub, blocks_for(nsub, 256), 256, 0, st, nsub, ctx->al.flag.p, ctx->al.pos.p,
                   ctx->al.sub.p);
        RBF_CUDA(ctx, cudaMemcpyAsync(&cnt, ctx->al.pos.p + nsub, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RBF_CUDA(ctx, cudaStreamSynchronize(st));
    }
    ctx->al.nsub = cnt;
    ctx->al.on = true;
    return RBF_OK;
}

}  // namespace rbf
