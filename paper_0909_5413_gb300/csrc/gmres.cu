// gmres.cu -- restarted GMRES(m) with right preconditioning (Sec. 2.2: GMRES
// with the RASM preconditioner; Sec. 3.1: relative tolerance 1e-13), all on
// the device:
//   * Arnoldi vectors V (m+1) x N in cell order;
//   * classical Gram-Schmidt applied twice, in three fused passes over V:
//       h1 = V^T v;  v -= V h1 and h2 = V^T v (same pass);  v -= V h2 and |v|^2;
//   * block partial sums reduced in a fixed order (deterministic);
//   * the Hessenberg column, the Givens rotations, the residual estimate
//     |g_{j+1}| and the stop flag are updated by a single-thread kernel; the
//     host reads the small status once per Arnoldi step.
// Mixed form: the same cycle runs on FP32 vectors with the FP32 matvec and
// FP32 subdomain inverses, while its dot products, Hessenberg and Givens stay
// FP64; each inner solve corrects w by FP64 iterative refinement on the true
// FP64 residual.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "common.cuh"
#include "ortho.cuh"
#include "vecops.cuh"

namespace rbf {

rbf_status rasm_apply_sorted_f32(rbf_ctx* ctx, const float* r, float* z, cudaStream_t st);
rbf_status ensure_local_coords(rbf_ctx* ctx, float2** loc, cudaStream_t st);
rbf_status matvec_f32_raw(rbf_ctx* ctx, const float2* loc, const float* w, float* y, cudaStream_t st);

namespace {

constexpr int kDotBlocksMax = 8 * kNumSMs;

// Vector passes are cut into chunks of kChunk elements (one block each);
// block partial sums go to partial[chunk * 32 + k] and are reduced over
// chunks in a fixed order.
constexpr int kChunkPerThread = kOrthoPer;
constexpr int kChunk = kOrthoChunk;

// The vector passes of one Gram-Schmidt step (kernels over chunks; the
// per-chunk code is shared with the batched solver). Block partial sums go
// to partial[chunk * 32 + k] and are reduced over chunks in a fixed order.

// MODE 0: partial_k = V_k . x over the chunk, one block per (chunk, k), k
// fastest so that the blocks reading one chunk of x run together and find it
// in L2.
template <class T>
__global__ void __launch_bounds__(kDotThreads)
    k_ortho_dots(const T* __restrict__ V, int64_t ldv, int nv, const T* __restrict__ x, int64_t n,
                 double* __restrict__ partial)
{
    __shared__ OrthoRed red;
    const int k = (int)(blockIdx.x % (unsigned)nv);
    const int64_t chunk = blockIdx.x / (unsigned)nv;
    ortho_dot_one<T>(V + k * ldv, x, chunk * kOrthoChunk, n, red, partial + chunk * 32 + k);
}

// MODE 1: x -= V coef (x rounded to T), then partial_k = V_k . x (the chunk
// of V is read twice, the second time from L2).
// MODE 2: x -= V coef, partial_0 = |x|^2.
template <class T, int MODE>
__global__ void __launch_bounds__(kDotThreads, 2)
    k_ortho_update(const T* __restrict__ V, int64_t ldv, int nv, const double* __restrict__ coef,
                   T* __restrict__ x, int64_t n, double* __restrict__ partial)
{
    __shared__ OrthoCoef cf;
    __shared__ OrthoRed red;
    if (threadIdx.x < (unsigned)nv) ortho_coef_set(cf, (int)threadIdx.x, coef[threadIdx.x]);
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * kOrthoChunk;
    typename OrthoAcc<T>::type xl[kOrthoPer];
    ortho_load_x<T>(xl, x, b, n);
    ortho_apply<T, ortho_group<T>()>(xl, V, ldv, nv, cf, b, n);
    T xs[kOrthoPer];
    ortho_store_x<T>(xl, xs, x, b, n);
    double* out = partial + (int64_t)blockIdx.x * 32;
    if (MODE == 1) {
        ortho_dots<T, ortho_group<T>()>(V, ldv, nv, xs, b, n, red, out);
    } else {
        ortho_warp_sum(ortho_thread_dot<T>(xs, xs, b, n), red, 0);
        __syncthreads();
        if (threadIdx.x == 0) out[0] = ortho_block_total<T>(red, 0);
    }
}

// out[k] = sum over blocks of partial[b*32 + k], k < nv: one warp per k, fixed order.
__global__ void k_reduce(const double* __restrict__ partial, int nblocks, int nv, double* __restrict__ out)
{
    int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= nv) return;
    double a = 0.0;
    constexpr int U = 8;   // loads issued together, added in order
    for (int b0 = lane; b0 < nblocks; b0 += 32 * U) {
        double p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = b0 + 32 * u;
            p[u] = b < nblocks ? partial[(int64_t)b * 32 + k] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (b0 + 32 * u < nblocks) a += p[u];
    }
    for (int d = 16; d > 0; d >>= 1) a += __shfl_xor_sync(0xffffffffu, a, d);
    if (lane == 0) out[k] = a;
}

// r = f - t (FP64); partial sums of |r|^2 per chunk (the chunks and the
// order of the vector passes, so that a problem solved alone and in a batch
// sums in the same order).
__global__ void __launch_bounds__(kDotThreads)
    k_residual(const double* __restrict__ f, const double* __restrict__ t, double* __restrict__ r, int64_t n,
               double* __restrict__ partial)
{
    __shared__ double red[kDotThreads / 32];
    const int64_t chunk = blockIdx.x;
    const int64_t base = chunk * kChunk + threadIdx.x;
    double a = 0.0;
#pragma unroll
    for (int u = 0; u < kChunkPerThread; ++u) {
        const int64_t i = base + (int64_t)u * kDotThreads;
        if (i < n) {
            const double v = t ? f[i] - t[i] : f[i];   // t null: A w with w = 0
            r[i] = v;
            a = fma(v, v, a);
        }
    }
    const double s = block_sum(a, red);
    if (threadIdx.x == 0) partial[chunk * 32] = s;
}

// Start of a cycle: beta = |r|, g = beta e_1, estimate beta / |f|. For an
// inner solve of the mixed form (inner = 1) the reference norm is |r| itself.
__global__ void k_cycle_init(GmresDev* g, int m, int inner)
{
    if (inner == 1) g->fnorm2 = g->beta2;
    if (inner == 2) g->fnorm2 = 1.0;   // inner solve on a right-hand side of norm 1
    double beta = sqrt(g->beta2);
    double fn = sqrt(g->fnorm2);
    for (int q = 0; q <= m; ++q) g->g[q] = 0.0;
    g->g[0] = beta;
    g->inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
    g->est = fn > 0.0 ? beta / fn : 0.0;
    g->done = (g->est <= g->rtol) ? 1 : 0;
    g->breakdown = 0;
    g->j = -1;
}

// Arnoldi step j (one warp): Hessenberg column, rotations, g, estimate.
__global__ void k_arnoldi(GmresDev* g, int j, int passes)
{
    arnoldi_column(g, j, passes);
    if (threadIdx.x == 0) {
        g->done = (g->est <= g->rtol || g->breakdown) ? 1 : 0;
        g->j = j;
    }
}

// y = H(0:k, 0:k)^{-1} g(0:k), upper triangular.
__global__ void k_solve_y(GmresDev* g, int k)
{
    const int M = kMaxRestart;
    for (int q = k - 1; q >= 0; --q) {
        double v = g->g[q];
        for (int p = q + 1; p < k; ++p) v -= g->H[q * M + p] * g->y[p];
        g->y[q] = v / g->H[q * M + q];
    }
}

// x *= factor (an FP32 vector is scaled in FP32: it is rounded to FP32 anyway)
template <class T>
__global__ void k_scale(T* __restrict__ x, int64_t n, const double* __restrict__ factor)
{
    const T f = (T)*factor;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = x[i] * f;
}

// t = sum_{q<k} y_q V_q (double-float for FP32 vectors)
template <class T>
__global__ void k_combine(const T* __restrict__ V, int64_t ldv, int k, const double* __restrict__ y,
                          T* __restrict__ t, int64_t n)
{
    __shared__ double ys[kMaxRestart];
    __shared__ float yh[kMaxRestart], yl[kMaxRestart];
    if (threadIdx.x < (unsigned)k) {
        double c = y[threadIdx.x];
        ys[threadIdx.x] = c;
        yh[threadIdx.x] = (float)c;
        yl[threadIdx.x] = (float)(c - (double)(float)c);
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(T) == 4) {
            DF a{0.f, 0.f};
            for (int q = 0; q < k; ++q) {
                float vi = V[q * ldv + i];
                float h = yh[q] * vi;
                df_add(a, h, fmaf(yl[q], vi, fmaf(yh[q], vi, -h)));
            }
            t[i] = a.hi + a.lo;
        } else {
            double a = 0.0;
            for (int q = 0; q < k; ++q) a = fma(ys[q], (double)V[q * ldv + i], a);
            t[i] = (T)a;
        }
    }
}

// w += u (u in T, w FP64)
template <class T>
__global__ void k_axpy(double* __restrict__ w, const T* __restrict__ u, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] += (double)u[i];
}

template <class T>
__global__ void k_axpy_same(T* __restrict__ w, const T* __restrict__ u, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] += u[i];
}

// w += a * d (FP64 w, FP32 d): the refinement update of the mixed form.
__global__ void k_axpy_scaled(double* __restrict__ w, const float* __restrict__ d, double a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] = fma(a, (double)d[i], w[i]);
}

// Inner residual of the mixed form: r = b - t (FP32); Dot2 partial sums of |r|^2.
__global__ void __launch_bounds__(kDotThreads)
    k_inner_residual(const float* __restrict__ b, const float* __restrict__ t, float* __restrict__ r, int64_t n,
                     double* __restrict__ partial)
{
    __shared__ DF red[kDotThreads / 32];
    DF s{0.f, 0.f};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v = b[i] - t[i];
        r[i] = v;
        df_add_prod(s, v, v);
    }
    double tot = block_sum_df(s, red);
    if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * 32] = tot;
}

// w[perm[q]] += a d[q]: the correction of an inner solve run in the inner grid's order.
__global__ void k_axpy_scaled_perm(double* __restrict__ w, const float* __restrict__ d, double a,
                                   const int32_t* __restrict__ perm, int64_t n)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
        w[perm[q]] = fma(a, (double)d[q], w[perm[q]]);
}

// FP32 copy of an FP64 vector scaled by a device factor: out = in * (*factor)
__global__ void k_to_f32_scaled(const double* __restrict__ in, int64_t n, const double* __restrict__ factor,
                                float* __restrict__ out)
{
    double f = *factor;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(in[i] * f);
}

__global__ void k_w64_to_w32(const double* __restrict__ in, int64_t n, float* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

unsigned dot_blocks(int64_t n)
{
    int64_t b = (n + kDotThreads - 1) / kDotThreads;
    if (b > kDotBlocksMax) b = kDotBlocksMax;
    return (unsigned)(b < 1 ? 1 : b);
}

unsigned stream_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 16 * kNumSMs) b = 16 * kNumSMs;
    return (unsigned)(b < 1 ? 1 : b);
}

int64_t num_chunks(int64_t n) { return std::max<int64_t>(1, (n + kChunk - 1) / kChunk); }

// MODE 0: out_k = V_k . x                      (one pass)
// MODE 1: x -= V coef, then out_k = V_k . x    (two passes)
// MODE 2: x -= V coef, out_0 = |x|^2           (one pass)
template <int MODE, class T>
rbf_status launch_mdot(rbf_ctx* ctx, const T* V, int64_t ldv, int nv, T* x, int64_t n, const double* coef,
                       double* out, cudaStream_t st)
{
    const int64_t nc = num_chunks(n);
    if (MODE == 0)
        RBF_LAUNCH(ctx, (k_ortho_dots<T>), (unsigned)(nc * nv), kDotThreads, 0, st, V, ldv, nv, (const T*)x, n,
                   ctx->partial.p);
    else
        RBF_LAUNCH(ctx, (k_ortho_update<T, MODE>), (unsigned)nc, kDotThreads, 0, st, V, ldv, nv, coef, x, n,
                   ctx->partial.p);
    const int nout = MODE == 2 ? 1 : nv;
    RBF_LAUNCH(ctx, k_reduce, 1, 32 * nout, 0, st, ctx->partial.p, (int)nc, nout, out);
    return RBF_OK;
}

struct StepStatus {
    double est;
    int done;
};

rbf_status read_status(rbf_ctx* ctx, cudaStream_t st, StepStatus* s)
{
    const size_t off = offsetof(GmresDev, est);
    const size_t len = offsetof(GmresDev, budget) - off;
    RBF_CUDA(ctx, cudaMemcpyAsync((char*)ctx->gm_host + off, (char*)ctx->gm.p + off, len, cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    s->est = ctx->gm_host->est;
    s->done = ctx->gm_host->done;
    return RBF_OK;
}

// Operators of one GMRES flavour on vectors of type T.
struct OpsF64 {
    static rbf_status amul(rbf_ctx* c, const double* x, double* y, cudaStream_t st, const float2*)
    {
        return matvec_sorted_f64(c, x, y, st);
    }
    static rbf_status minv(rbf_ctx* c, const double* x, double* y, cudaStream_t st)
    {
        return rasm_apply_sorted(c, x, y, st);
    }
};

struct OpsF32 {
    static rbf_status amul(rbf_ctx* c, const float* x, float* y, cudaStream_t st, const float2* loc)
    {
        return matvec_f32_raw(c, loc, x, y, st);
    }
    static rbf_status minv(rbf_ctx* c, const float* x, float* y, cudaStream_t st)
    {
        return rasm_apply_sorted_f32(c, x, y, st);
    }
};

// One GMRES cycle on vectors of type T starting from V_0 = r / |r| (V_0 holds
// r on entry and beta2 is in g->beta2). Accumulates the correction
// M^{-1} V y into w (FP64) or, if wT is given, into wT. Returns the number of
// Arnoldi steps.
template <class T, class Ops>
rbf_status gmres_cycle(rbf_ctx* ctx, T* V, int64_t ldv, int m, int max_steps, T* tmp_u, T* tmp_t, double* w,
                       T* wT, const float2* loc, bool scale_v0, cudaStream_t st, int* steps, double* est,
                       int* applies)
{
    const int64_t n = ctx->n;
    GmresDev* g = ctx->gm.p;
    int k = 0;
    StepStatus ss{0.0, 0};
    if (scale_v0) RBF_LAUNCH(ctx, (k_scale<T>), stream_blocks(n), 256, 0, st, V, n, &g->inv_beta);
    for (int j = 0; j < m && j < max_steps; ++j) {
        T* vj = V + (int64_t)j * ldv;
        T* vn = V + (int64_t)(j + 1) * ldv;
        RBF_CHECK(Ops::minv(ctx, vj, tmp_u, st));
        ++*applies;
        RBF_CHECK(Ops::amul(ctx, tmp_u, vn, st, loc));
        RBF_CHECK(prof_begin(ctx, RBF_PROF_ORTHO, st));
        RBF_CHECK((launch_mdot<0, T>(ctx, V, ldv, j + 1, vn, n, nullptr, g->h1, st)));
        if (gs_passes<T>() == 2) {
            RBF_CHECK((launch_mdot<1, T>(ctx, V, ldv, j + 1, vn, n, g->h1, g->h2, st)));
            RBF_CHECK((launch_mdot<2, T>(ctx, V, ldv, j + 1, vn, n, g->h2, &g->nrm2, st)));
        } else {
            RBF_CHECK((launch_mdot<2, T>(ctx, V, ldv, j + 1, vn, n, g->h1, &g->nrm2, st)));
        }
        RBF_CHECK(prof_end(ctx, RBF_PROF_ORTHO, st));
        RBF_LAUNCH(ctx, k_arnoldi, 1, 32, 0, st, g, j, gs_passes<T>());
        RBF_LAUNCH(ctx, (k_scale<T>), stream_blocks(n), 256, 0, st, vn, n, &g->inv_h);
        k = j + 1;
        RBF_CHECK(read_status(ctx, st, &ss));
        if (ss.done) break;
    }
    RBF_LAUNCH(ctx, k_solve_y, 1, 1, 0, st, g, k);
    RBF_LAUNCH(ctx, (k_combine<T>), stream_blocks(n), 256, 0, st, V, ldv, k, g->y, tmp_t, n);
    RBF_CHECK(Ops::minv(ctx, tmp_t, tmp_u, st));
    ++*applies;
    if (wT)
        RBF_LAUNCH(ctx, (k_axpy_same<T>), stream_blocks(n), 256, 0, st, wT, tmp_u, n);
    else
        RBF_LAUNCH(ctx, (k_axpy<T>), stream_blocks(n), 256, 0, st, w, tmp_u, n);
    *steps = k;
    *est = ss.est;
    return RBF_OK;
}

// True FP64 residual r = f - A w into r64, |r|^2 into g->beta2; returns |r| / |f|.
rbf_status true_residual(rbf_ctx* ctx, const double* f, const double* w, bool w_zero, double* t, double* r64,
                         cudaStream_t st,
                         double fnorm, double* relres)
{
    GmresDev* g = ctx->gm.p;
    if (!w_zero) RBF_CHECK(matvec_sorted_f64(ctx, w, t, st));   // w = 0: r = f exactly, no product
    const int64_t nc = num_chunks(ctx->n);
    RBF_LAUNCH(ctx, k_residual, (unsigned)nc, kDotThreads, 0, st, f, w_zero ? nullptr : t, r64, ctx->n,
               ctx->partial.p);
    RBF_LAUNCH(ctx, k_reduce, 1, 32, 0, st, ctx->partial.p, (int)nc, 1, &g->beta2);
    RBF_CUDA(ctx, cudaMemcpyAsync(&ctx->gm_host->beta2, &g->beta2, sizeof(double), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    *relres = std::sqrt(ctx->gm_host->beta2) / fnorm;
    return RBF_OK;
}

}  // namespace

rbf_status gmres_solve(rbf_ctx* ctx, const double* f, double* w, const rbf_solve_params* p, rbf_solve_info* info,
                       cudaStream_t st)
{
    const int64_t n = ctx->n;
    const int m = p->restart > 0 ? p->restart : 30;
    const int max_iters = p->max_iters > 0 ? p->max_iters : 10000;
    const bool mixed = p->mixed != 0;
    RBF_CHECK(ensure(ctx, ctx->gm, 1));
    RBF_CHECK(ensure(ctx, ctx->partial, (size_t)std::max<int64_t>(kDotBlocksMax, num_chunks(n)) * 32));
    RBF_CHECK(ensure(ctx, ctx->vec_a, n));
    RBF_CHECK(ensure(ctx, ctx->vec_b, n));
    GmresDev* g = ctx->gm.p;

    // device state: zero, rtol
    std::memset(ctx->gm_host, 0, sizeof(GmresDev));
    ctx->gm_host->rtol = mixed ? (p->inner_rtol > 0.0 ? p->inner_rtol : 1e-5) : p->rtol;
    RBF_CUDA(ctx, cudaMemcpyAsync(g, ctx->gm_host, sizeof(GmresDev), cudaMemcpyHostToDevice, st));
    // |f|^2, and whether the initial guess is zero (then r0 = f without a product)
    RBF_CHECK((launch_mdot<0, double>(ctx, f, 0, 1, const_cast<double*>(f), n, nullptr, &g->fnorm2, st)));
    RBF_CHECK(ensure(ctx, ctx->flag_dev, 1));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->flag_dev.p, 0, sizeof(int), st));
    RBF_LAUNCH(ctx, k_any_nonzero, stream_blocks(n), 256, 0, st, w, n, ctx->flag_dev.p);
    int w_nonzero = 1;
    RBF_CUDA(ctx, cudaMemcpyAsync(&ctx->gm_host->fnorm2, &g->fnorm2, sizeof(double), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(&w_nonzero, ctx->flag_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    bool w_zero = w_nonzero == 0;
    const double fnorm = std::sqrt(ctx->gm_host->fnorm2);
    if (!std::isfinite(fnorm)) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_solve: f is not finite");
    if (fnorm == 0.0) {
        RBF_CUDA(ctx, cudaMemsetAsync(w, 0, sizeof(double) * n, st));
        info->relres = 0.0;
        return RBF_OK;
    }

    int it = 0, cycles = 0, refine = 0, matvecs = 0, applies = 0;
    std::vector<double> hist;   // true relative residual at each restart
    bool stagnated = false;
    double relres = 0.0, est = 0.0;
    rbf_status result = RBF_ERR_NOT_CONVERGED;

    if (!mixed) {
        RBF_CHECK(ensure(ctx, ctx->V, (size_t)(m + 1) * n));
        double* V = ctx->V.p;
        for (;;) {
            RBF_CHECK(true_residual(ctx, f, w, w_zero, ctx->vec_a.p, V, st, fnorm, &relres));
            if (!w_zero) ++matvecs;
            w_zero = false;
            if (!std::isfinite(relres)) return fail(ctx, RBF_ERR_NOT_CONVERGED, "rbf_solve: residual is not finite");
            if (relres <= p->rtol) { result = RBF_OK; break; }
            if (it >= max_iters) break;
            if (stagnating(hist, relres)) { stagnated = true; break; }
            RBF_LAUNCH(ctx, k_cycle_init, 1, 1, 0, st, g, m, 0);
            int steps = 0;
            RBF_CHECK((gmres_cycle<double, OpsF64>(ctx, V, n, m, max_iters - it, ctx->vec_b.p, ctx->vec_a.p, w,
                                                   (double*)nullptr, nullptr, true, st, &steps, &est, &applies)));
            it += steps;
            matvecs += steps;
            ++cycles;
        }
    } else {
        // FP32 inner GMRES inside FP64 iterative refinement:
        //   r = f - A w (FP64);  solve A d = r in FP32 to inner_rtol;  w += d.
        const int max_refine = p->max_refine > 0 ? p->max_refine : 40;
        if (ctx->rasm_precision == RBF_FP64 || !ctx->W32.p) {
            RBF_CHECK(ensure(ctx, ctx->W32, ctx->W64.count));
            RBF_LAUNCH(ctx, k_w64_to_w32, stream_blocks((int64_t)ctx->W64.count), 256, 0, st, ctx->W64.p,
                       (int64_t)ctx->W64.count, ctx->W32.p);
        }
        float2* loc = nullptr;
        RBF_CHECK(ensure_local_coords(ctx, &loc, st));
        // the inner grid (shorter cutoff, own order) for the FP32 inner solves
        const bool use_inner = p->inner_cutoff > 0.0 && !ctx->rasm_additive;
        if (use_inner && (!ctx->in.ready || ctx->in.ri_sigmas != p->inner_cutoff))
            RBF_CHECK(bin_inner(ctx, p->inner_cutoff, st));
        struct InnerOn {
            rbf_ctx* c;
            ~InnerOn() { c->inner_on = false; }
        } inner_guard{ctx};
        ctx->inner_on = use_inner;
        // FP32 Krylov basis and four FP32 work vectors (u, t, b, d), in V's storage
        const int64_t ldv = ((n + 63) / 64) * 64;
        RBF_CHECK(ensure(ctx, ctx->V, (size_t)((m + 5) * ldv + 1) / 2 + 1));
        float* Vf = (float*)ctx->V.p;
        float* uf = Vf + (int64_t)(m + 1) * ldv;
        float* tf = uf + ldv;
        float* bf = tf + ldv;   // inner right-hand side r / |r|
        float* df = bf + ldv;   // inner solution
        double* r64 = ctx->vec_b.p;
        const double inner_rtol = p->inner_rtol > 0.0 ? p->inner_rtol : 1e-5;
        // One inner cycle per refinement step: restarting the inner solve on the
        // FP32 residual b - A d stalls near 1e-3, because A d is formed from
        // entries much larger than the result (cancellation in FP32 once the
        // correction d is large on an ill-conditioned system). Every restart
        // therefore starts from the FP64 residual, which is the refinement step.
        constexpr int kMaxInnerCycles = 1;
        for (;;) {
            RBF_CHECK(true_residual(ctx, f, w, w_zero, ctx->vec_a.p, r64, st, fnorm, &relres));
            if (!w_zero) ++matvecs;
            w_zero = false;
            if (!std::isfinite(relres)) return fail(ctx, RBF_ERR_NOT_CONVERGED, "rbf_solve: residual is not finite");
            if (relres <= p->rtol) { result = RBF_OK; break; }
            if (it >= max_iters || refine >= max_refine) break;
            if (stagnating(hist, relres)) { stagnated = true; break; }
            const double rnorm = relres * fnorm;
            // inner solve of A d = b, b = r / |r| (norm 1), from d = 0, restarted on
            // the FP32 inner residual b - A d until inner_rtol or kMaxInnerCycles
            RBF_LAUNCH(ctx, k_cycle_init, 1, 1, 0, st, g, m, 1);   // inv_beta = 1 / |r|
            if (use_inner) RBF_CHECK(inner_gather_scaled(ctx, r64, &g->inv_beta, bf, st));
            else RBF_LAUNCH(ctx, k_to_f32_scaled, stream_blocks(n), 256, 0, st, r64, n, &g->inv_beta, bf);
            RBF_CUDA(ctx, cudaMemsetAsync(df, 0, sizeof(float) * n, st));
            for (int ic = 0; ic < kMaxInnerCycles && it < max_iters; ++ic) {
                if (ic == 0) {
                    RBF_CUDA(ctx, cudaMemcpyAsync(Vf, bf, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
                } else {
                    RBF_CHECK(OpsF32::amul(ctx, df, tf, st, loc));
                    ++matvecs;
                }
                if (ic > 0) {
                    unsigned nb = dot_blocks(n);
                    RBF_LAUNCH(ctx, k_inner_residual, nb, kDotThreads, 0, st, bf, tf, Vf, n, ctx->partial.p);
                    RBF_LAUNCH(ctx, k_reduce, 1, 32, 0, st, ctx->partial.p, (int)nb, 1, &g->beta2);
                } else {
                    RBF_CHECK((launch_mdot<0, float>(ctx, Vf, 0, 1, Vf, n, nullptr, &g->beta2, st)));
                }
                RBF_LAUNCH(ctx, k_cycle_init, 1, 1, 0, st, g, m, 2);
                StepStatus s0{0.0, 0};
                RBF_CHECK(read_status(ctx, st, &s0));
                if (ic > 0 && s0.est <= inner_rtol) break;
                int steps = 0;
                RBF_CHECK((gmres_cycle<float, OpsF32>(ctx, Vf, ldv, m, max_iters - it, uf, tf, nullptr, df, loc, true,
                                                      st, &steps, &est, &applies)));
                it += steps;
                matvecs += steps;
                ++cycles;
                if (est <= inner_rtol) break;
            }
            if (use_inner)
                RBF_LAUNCH(ctx, k_axpy_scaled_perm, stream_blocks(n), 256, 0, st, w, df, rnorm, ctx->in.perm.p, n);
            else
                RBF_LAUNCH(ctx, k_axpy_scaled, stream_blocks(n), 256, 0, st, w, df, rnorm, n);
            ++refine;
        }
    }
    info->iters = it;
    info->restarts = cycles;
    info->refinements = refine;
    info->relres = relres;
    info->relres_est = est;
    info->matvecs = matvecs;
    info->applies = applies;
    info->status = result;
    info->stagnated = stagnated ? 1 : 0;
    if (result != RBF_OK)
        fail(ctx, RBF_ERR_NOT_CONVERGED, "rbf_solve: relative residual %.3e after %d steps (rtol %.1e)", relres, it,
             p->rtol);
    return result;
}

}  // namespace rbf
