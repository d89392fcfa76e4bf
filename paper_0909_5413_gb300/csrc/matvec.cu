// matvec.cu -- the truncated Gaussian matvec y = A~ w of Sec. 2.3, matrix-free:
// for each target i (cell order), sum over the sources j of the
// (2k+1) x (2k+1) neighbour cells with r2_ij <= r_c^2 of
// exp(-r2_ij / (2 sigma^2)) w_j. Each stencil row is one contiguous range of
// cell-ordered sources, read directly from HBM/L2 (there is no ghost exchange
// on one GPU).
#include <cmath>

#include "common.cuh"

namespace rbf {
namespace {

// FP64: one thread per target; sources of a warp's targets largely coincide,
// so their loads are served from L1.
__global__ void __launch_bounds__(128) k_matvec_f64(const double2* __restrict__ xy, const int32_t* __restrict__ cell_s,
                                                    const int32_t* __restrict__ cell_start, int64_t n, int ncx, int ncy,
                                                    int k, double rc2, double s, double knorm, ExpConsts ec,
                                                    const double* __restrict__ w, double* __restrict__ y)
{
    __shared__ double tab[64];
    if (threadIdx.x < 64) tab[threadIdx.x] = ec.tab[threadIdx.x];
    __syncthreads();
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double2 xi = xy[p];
    int c = cell_s[p];
    int cx = c % ncx, cy = c / ncx;
    int y0 = max(cy - k, 0), y1 = min(cy + k, ncy - 1);
    int x0 = max(cx - k, 0), x1 = min(cx + k, ncx - 1);
    double acc = 0.0;
    for (int yy = y0; yy <= y1; ++yy) {
        int b = cell_start[yy * ncx + x0], e = cell_start[yy * ncx + x1 + 1];
        for (int q = b; q < e; ++q) {
            double2 xj = xy[q];
            double dx = xi.x - xj.x, dy = xi.y - xj.y;
            double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
            if (r2 <= rc2) acc = fma(exp_neg(r2 * s, tab, ec.inv_l, ec.l_hi, ec.l_lo), w[q], acc);
        }
    }
    y[p] = acc * knorm;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// FP32 on cell-local scaled coordinates: loc[p] = (x_p - cell origin) * a with
// a^2 = log2(e) / (2 sigma^2), so the kernel is exp2(-|dX|^2); the cell shift
// between target and source cell is added as an integer multiple of c * a.
__global__ void __launch_bounds__(128) k_matvec_f32(const float2* __restrict__ loc, const int32_t* __restrict__ cell_s,
                                                    const int32_t* __restrict__ cell_start, int64_t n, int ncx, int ncy,
                                                    int k, float ca, float rc2s, float knorm,
                                                    const float* __restrict__ w, float* __restrict__ y)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float2 xi = loc[p];
    int c = cell_s[p];
    int cx = c % ncx, cy = c / ncx;
    int y0 = max(cy - k, 0), y1 = min(cy + k, ncy - 1);
    int x0 = max(cx - k, 0), x1 = min(cx + k, ncx - 1);
    float acc = 0.0f;
    for (int yy = y0; yy <= y1; ++yy) {
        float ty = xi.y - (float)(yy - cy) * ca;
        for (int xx = x0; xx <= x1; ++xx) {
            float tx = xi.x - (float)(xx - cx) * ca;
            int cc = yy * ncx + xx;
            int b = cell_start[cc], e = cell_start[cc + 1];
            for (int q = b; q < e; ++q) {
                float2 xj = loc[q];
                float dx = tx - xj.x, dy = ty - xj.y;
                float r2 = fmaf(dy, dy, dx * dx);
                float ev = ex2_approx(-r2);
                acc = (r2 <= rc2s) ? fmaf(ev, w[q], acc) : acc;
            }
        }
    }
    y[p] = acc * knorm;
}

__global__ void k_local_coords(const double* __restrict__ xy_s, const int32_t* __restrict__ cell_s, int64_t n,
                               int ncx, double xmin, double ymin, double c, double a, float2* __restrict__ loc)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int cc = cell_s[p];
    int cx = cc % ncx, cy = cc / ncx;
    double ox = xmin + (double)cx * c, oy = ymin + (double)cy * c;
    loc[p] = make_float2((float)((xy_s[2 * p] - ox) * a), (float)((xy_s[2 * p + 1] - oy) * a));
}

__global__ void k_to_f32(const double* __restrict__ in, int64_t n, float* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

__global__ void k_to_f64(const float* __restrict__ in, int64_t n, double* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

}  // namespace

rbf_status matvec_sorted_f64(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st)
{
    RBF_CHECK(prof_begin(ctx, RBF_PROF_MATVEC_F64, st));
    RBF_LAUNCH(ctx, k_matvec_f64, blocks_for(ctx->n, 128), 128, 0, st, (const double2*)ctx->xy_s.p, ctx->cell_s.p,
               ctx->cell_start.p, ctx->n, (int)ctx->ncx, (int)ctx->ncy, ctx->kst, ctx->rc2, ctx->s, ctx->knorm,
               ctx->expc, w, y);
    return prof_end(ctx, RBF_PROF_MATVEC_F64, st);
}

rbf_status matvec_sorted_f64_plain(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st)
{
    RBF_LAUNCH(ctx, k_matvec_f64, blocks_for(ctx->n, 128), 128, 0, st, (const double2*)ctx->xy_s.p, ctx->cell_s.p,
               ctx->cell_start.p, ctx->n, (int)ctx->ncx, (int)ctx->ncy, ctx->kst, ctx->rc2, ctx->s, ctx->knorm,
               ctx->expc, w, y);
    return RBF_OK;
}

// Scale of the FP32 local coordinates: a^2 = log2(e) / (2 sigma^2).
static double local_scale(const rbf_ctx* ctx) { return std::sqrt(M_LOG2E * ctx->s); }

rbf_status ensure_local_coords(rbf_ctx* ctx, float2** loc, cudaStream_t st)
{
    // stored after the FP32 work vectors in vec_c (2 floats per point = 1 double)
    RBF_CHECK(ensure(ctx, ctx->vec_c, (size_t)ctx->n * 2));
    *loc = (float2*)ctx->vec_c.p;
    RBF_LAUNCH(ctx, k_local_coords, blocks_for(ctx->n, 256), 256, 0, st, ctx->xy_s.p, ctx->cell_s.p, ctx->n,
               (int)ctx->ncx, ctx->bbox[0], ctx->bbox[1], ctx->cell, local_scale(ctx), *loc);
    return RBF_OK;
}

rbf_status matvec_f32_raw(rbf_ctx* ctx, const float2* loc, const float* w, float* y, cudaStream_t st)
{
    double a = local_scale(ctx);
    RBF_CHECK(prof_begin(ctx, RBF_PROF_MATVEC_F32, st));
    RBF_LAUNCH(ctx, k_matvec_f32, blocks_for(ctx->n, 128), 128, 0, st, loc, ctx->cell_s.p, ctx->cell_start.p, ctx->n,
               (int)ctx->ncx, (int)ctx->ncy, ctx->kst, (float)(ctx->cell * a), (float)(ctx->rc2 * a * a),
               (float)ctx->knorm, w, y);
    return prof_end(ctx, RBF_PROF_MATVEC_F32, st);
}

rbf_status matvec_sorted_f32(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st)
{
    float2* loc = nullptr;
    RBF_CHECK(ensure_local_coords(ctx, &loc, st));
    float* wf = (float*)(ctx->vec_c.p + ctx->n);   // second half of vec_c
    float* yf = wf + ctx->n;
    RBF_LAUNCH(ctx, k_to_f32, blocks_for(ctx->n, 256), 256, 0, st, w, ctx->n, wf);
    RBF_CHECK(matvec_f32_raw(ctx, loc, wf, yf, st));
    RBF_LAUNCH(ctx, k_to_f64, blocks_for(ctx->n, 256), 256, 0, st, yf, ctx->n, y);
    return RBF_OK;
}

}  // namespace rbf
