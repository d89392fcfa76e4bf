// gmres_batch.cu -- restarted right-preconditioned GMRES(m) for a batch of
// independent problems solved together: one launch of each kernel serves all
// problems, and every problem keeps its own Krylov basis segment, Gram-Schmidt
// coefficients, Hessenberg matrix, Givens rotations and stopping test.
//
// Vectors are the concatenation of the problems' cell-ordered vectors. They
// are cut into chunks of at most kBChunk elements that never cross a problem
// boundary; block partial sums of a chunk are reduced per problem in a fixed
// order (deterministic: a problem's result does not depend on the other
// problems of the batch). Converged problems are masked: their kernels return
// at once; within a cycle, a problem that meets its estimate (or its step
// budget) leaves the step mask, and the rest of the cycle's steps skip it. An
// Arnoldi cycle runs with no host synchronisation (each problem's stop flag
// lives on the device), so the cycle is captured once as a CUDA graph and
// replayed; the host reads the problems' residuals once per cycle. A single
// problem (rbf_solve) is a batch of one.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ortho.cuh"
#include "batch.cuh"
#include "bulk.cuh"
#include "vecops.cuh"

namespace rbf {

rbf_status rasm_apply_sorted_f32(rbf_ctx* ctx, const float* r, float* z, cudaStream_t st);
rbf_status matvec_f32_raw(rbf_ctx* ctx, const float2* loc, const float* w, float* y, cudaStream_t st);

namespace {

// Active problems from which the adaptive mode (RBF_OPT_FUSED_STEP = 2) runs
// the fused Arnoldi step: in the tail of a batch the separate kernels are
// short and their launches dominate; with many problems active they keep
// more warps resident than the persistent kernel and are faster.
constexpr int kFusedTail = 64;
// A single problem takes it up to this many points: below, its launches
// dominate the step (4,096 points: 12.2 against 13.6 ms per solve; 65,536:
// 15.9 against 17.5 ms); above, the separate kernels keep more warps resident
// (524,176 points: 43.0 against 34.7 ms).
constexpr int64_t kFusedSingleMax = 262144;

constexpr int kBPer = kOrthoPer;       // elements per thread (the single solver's chunking)
constexpr int kBChunk = kOrthoChunk;   // elements per chunk

// The Gram-Schmidt vector passes over one chunk (the single solver's per-chunk code;
// a chunk never spans two problems). Chunks of masked problems write zeros.
// MODE 0: partial_k = V_k . x, one block per (chunk, k), k fastest.
template <class T>
__global__ void __launch_bounds__(kDotThreads)
    k_bdots(const T* __restrict__ V, int64_t ldv, int nv, const T* __restrict__ x, Chunks C,
            const int32_t* __restrict__ active, double* __restrict__ partial)
{
    __shared__ OrthoRed red;
    const int k = (int)(blockIdx.x % (unsigned)nv);
    const int64_t c = blockIdx.x / (unsigned)nv;
    if (!active[C.pid[c]]) {
        if (threadIdx.x == 0) partial[c * 32 + k] = 0.0;
        return;
    }
    ortho_dot_one<T>(V + k * ldv, x, C.beg[c], C.end[c], red, partial + c * 32 + k);
}

// MODE 1: x -= V coef with the chunk's problem's coefficients (field h1 or h2
// of its state), then partial_k = V_k . x. MODE 2: x -= V coef, partial_0 = |x|^2.
template <class T, int MODE>
__global__ void __launch_bounds__(kDotThreads, 2)
    k_bupdate(const T* __restrict__ V, int64_t ldv, int nv, GmresDev* __restrict__ gm, int field, T* __restrict__ x,
              Chunks C, const int32_t* __restrict__ active, double* __restrict__ partial)
{
    __shared__ OrthoCoef cf;
    __shared__ OrthoRed red;
    const int64_t c = blockIdx.x;
    const int pb = C.pid[c];
    double* out = partial + c * 32;
    if (!active[pb]) {
        if (threadIdx.x < (unsigned)(MODE == 2 ? 1 : nv)) out[threadIdx.x] = 0.0;
        return;
    }
    if (threadIdx.x < (unsigned)nv) ortho_coef_set(cf, (int)threadIdx.x, field_ptr(gm[pb], field)[threadIdx.x]);
    __syncthreads();
    const int64_t b = C.beg[c], e = C.end[c];
    typename OrthoAcc<T>::type xl[kOrthoPer];
    ortho_load_x<T>(xl, x, b, e);
    ortho_apply<T, ortho_group<T>()>(xl, V, ldv, nv, cf, b, e);
    T xs[kOrthoPer];
    ortho_store_x<T>(xl, xs, x, b, e);
    if (MODE == 1) {
        ortho_dots<T, ortho_group<T>()>(V, ldv, nv, xs, b, e, red, out);
    } else {
        ortho_warp_sum(ortho_thread_dot<T>(xs, xs, b, e), red, 0);
        __syncthreads();
        if (threadIdx.x == 0) out[0] = ortho_block_total<T>(red, 0);
    }
}

// The FP32 passes with the basis streamed through shared memory: one block per
// chunk keeps its x elements in registers while a thread issues bulk copies
// of the chunk's segment of V_0, V_1, ... into kStreamStages stages (copies in
// flight: the stages, not registers), every thread taking its elements from
// the stage. Element for element the arithmetic and the summation order are
// those of k_bdots / k_bupdate (and of the fused step), so the results are
// the same bits. A stage holds the chunk widened to 16-byte boundaries
// (V is 16-byte aligned, ldv a multiple of 4). A copy that does not arrive
// within `spin` polls ends the pass: status = RBF_ERR_TIMEOUT, x and the
// partial sums are left alone once the copies in flight have landed (each
// waited for at most `spin` polls). check = 1: every wait is on a barrier that
// no copy completes and nothing is copied (the check of that path).
constexpr int kStreamStages = 4;
constexpr int kStreamLd = kOrthoChunk + 4;   // floats per stage
constexpr size_t kStreamSmem = sizeof(float) * kStreamStages * kStreamLd;

struct StreamChunk {
    int64_t b, e, b0;   // the chunk and its 16-byte aligned start
    int off;            // b - b0
    uint32_t bytes;     // of one copy
};

__device__ __forceinline__ StreamChunk stream_chunk(const Chunks& C, int64_t c)
{
    StreamChunk s;
    s.b = C.beg[c];
    s.e = C.end[c];
    s.b0 = s.b & ~3LL;
    s.off = (int)(s.b - s.b0);
    s.bytes = (uint32_t)((((s.e + 3) & ~3LL) - s.b0) * (int64_t)sizeof(float));
    return s;
}

// Issues the first copies; returns how many were issued (thread 0 only).
__device__ __forceinline__ int stream_start(float* stage, uint64_t* bar, const float* V, int64_t ldv, int nv,
                                            const StreamChunk& s, int check)
{
    if (threadIdx.x == 0) {
        for (int q = 0; q <= kStreamStages; ++q) mbar_init(&bar[q], 1);
        mbar_init_fence();
    }
    __syncthreads();
    const int npre = check ? 0 : min(nv, kStreamStages);
    if (threadIdx.x == 0)
        for (int k = 0; k < npre; ++k) bulk_load(stage + k * kStreamLd, V + (int64_t)k * ldv + s.b0, s.bytes, &bar[k]);
    return npre;
}

// After a failed wait at vector kf: record the timeout, then let the copies
// still in flight (vectors kf .. issued - 1) land before the block exits.
__device__ __forceinline__ void stream_abort(uint64_t* bar, int kf, int issued, int* status,
                                             unsigned long long spin)
{
    if (threadIdx.x != 0) return;
    atomicExch(status, (int)RBF_ERR_TIMEOUT);
    for (int k = kf; k < issued; ++k) mbar_wait(&bar[k % kStreamStages], (k / kStreamStages) & 1, spin);
}

// partial_k = V_k . x over the chunk, k < nv (k_bdots for all k of a chunk).
__global__ void __launch_bounds__(kDotThreads)
    k_bdots_stream(const float* __restrict__ V, int64_t ldv, int nv, const float* __restrict__ x, Chunks C,
                   const int32_t* __restrict__ active, double* __restrict__ partial, int* __restrict__ status,
                   unsigned long long spin, int check)
{
    extern __shared__ __align__(128) float stream_stage[];
    __shared__ __align__(8) uint64_t bar[kStreamStages + 1];
    __shared__ OrthoRed red;
    const int64_t c = blockIdx.x;
    double* out = partial + c * 32;
    if (!active[C.pid[c]]) {
        if (threadIdx.x < (unsigned)nv) out[threadIdx.x] = 0.0;
        return;
    }
    const StreamChunk s = stream_chunk(C, c);
    int issued = stream_start(stream_stage, bar, V, ldv, nv, s, check);
    float xs[kOrthoPer];
#pragma unroll
    for (int u = 0; u < kOrthoPer; ++u) {
        const int64_t i = s.b + threadIdx.x + (int64_t)u * kDotThreads;
        xs[u] = i < s.e ? x[i] : 0.f;
    }
    for (int k = 0; k < nv; ++k) {
        const int q = k % kStreamStages;
        const bool ok = mbar_wait(check ? &bar[kStreamStages] : &bar[q], (k / kStreamStages) & 1, spin);
        if (ok) {
            const float* v = stream_stage + q * kStreamLd + s.off;
            float a[kOrthoPer];
#pragma unroll
            for (int u = 0; u < kOrthoPer; ++u) a[u] = v[threadIdx.x + u * kDotThreads];
            ortho_warp_sum(ortho_thread_dot<float>(a, xs, s.b, s.e), red, k);
        }
        if (__syncthreads_or(!ok)) {
            stream_abort(bar, k, issued, status, spin);
            return;
        }
        if (threadIdx.x == 0 && k + kStreamStages < nv) {
            fence_async_smem();
            bulk_load(stream_stage + q * kStreamLd, V + (int64_t)(k + kStreamStages) * ldv + s.b0, s.bytes, &bar[q]);
            ++issued;
        }
    }
    if (threadIdx.x < (unsigned)nv) out[threadIdx.x] = ortho_block_total<float>(red, (int)threadIdx.x);
}

// x -= V coef (the chunk's problem's coefficients, field `field`), then
// partial_0 = |x|^2 (k_bupdate<float, 2>).
__global__ void __launch_bounds__(kDotThreads)
    k_bupdate_stream(const float* __restrict__ V, int64_t ldv, int nv, GmresDev* __restrict__ gm, int field,
                     float* __restrict__ x, Chunks C, const int32_t* __restrict__ active, double* __restrict__ partial,
                     int* __restrict__ status, unsigned long long spin, int check)
{
    extern __shared__ __align__(128) float stream_stage[];
    __shared__ __align__(8) uint64_t bar[kStreamStages + 1];
    __shared__ OrthoCoef cf;
    __shared__ OrthoRed red;
    const int64_t c = blockIdx.x;
    const int pb = C.pid[c];
    double* out = partial + c * 32;
    if (!active[pb]) {
        if (threadIdx.x == 0) out[0] = 0.0;
        return;
    }
    if (threadIdx.x < (unsigned)nv) ortho_coef_set(cf, (int)threadIdx.x, field_ptr(gm[pb], field)[threadIdx.x]);
    const StreamChunk s = stream_chunk(C, c);
    int issued = stream_start(stream_stage, bar, V, ldv, nv, s, check);   // its block barrier publishes cf
    DF xl[kOrthoPer];
    ortho_load_x<float>(xl, x, s.b, s.e);
    for (int k = 0; k < nv; ++k) {
        const int q = k % kStreamStages;
        const bool ok = mbar_wait(check ? &bar[kStreamStages] : &bar[q], (k / kStreamStages) & 1, spin);
        if (ok) {
            const float* v = stream_stage + q * kStreamLd + s.off;
            const float ch = cf.hi[k], cl = cf.lo[k];
#pragma unroll
            for (int u = 0; u < kOrthoPer; ++u)
                if (s.b + threadIdx.x + (int64_t)u * kDotThreads < s.e)
                    ortho_axpy(xl[u], ch, cl, v[threadIdx.x + u * kDotThreads]);
        }
        if (__syncthreads_or(!ok)) {
            stream_abort(bar, k, issued, status, spin);
            return;
        }
        if (threadIdx.x == 0 && k + kStreamStages < nv) {
            fence_async_smem();
            bulk_load(stream_stage + q * kStreamLd, V + (int64_t)(k + kStreamStages) * ldv + s.b0, s.bytes, &bar[q]);
            ++issued;
        }
    }
    float xs[kOrthoPer];
    ortho_store_x<float>(xl, xs, x, s.b, s.e);
    ortho_warp_sum(ortho_thread_dot<float>(xs, xs, s.b, s.e), red, 0);
    __syncthreads();
    if (threadIdx.x == 0) out[0] = ortho_block_total<float>(red, 0);
}

// r = f - t over one chunk (FP64) and |r|^2 partial sums.
__global__ void __launch_bounds__(kDotThreads)
    k_bresidual(const double* __restrict__ f, const double* __restrict__ t, double* __restrict__ r, Chunks C,
                const int32_t* __restrict__ active, double* __restrict__ partial)
{
    __shared__ double red[kDotThreads / 32];
    const int64_t c = blockIdx.x;
    if (!active[C.pid[c]]) {
        if (threadIdx.x == 0) partial[c * 32] = 0.0;
        return;
    }
    const int64_t b = C.beg[c], e = C.end[c];
    double a = 0.0;
    for (int u = 0; u < kBPer; ++u) {
        int64_t i = b + threadIdx.x + (int64_t)u * kDotThreads;
        if (i < e) {
            double v = t ? f[i] - t[i] : f[i];   // t null: A w with w = 0
            r[i] = v;
            a = fma(v, v, a);
        }
    }
    double s = block_sum(a, red);
    if (threadIdx.x == 0) partial[c * 32] = s;
}

// Per (problem, vector k) block: the problem's chunk partials of k summed in
// a fixed order (a warp per segment, then the segments in order; the value of
// breduce_one), written to the field of its state.
__global__ void k_breduce(const double* __restrict__ partial, Chunks C, int nprob, int nv, GmresDev* __restrict__ gm,
                          int field, const int32_t* __restrict__ active)
{
    __shared__ double seg[kRedSeg];
    const int pb = blockIdx.x / nv, k = blockIdx.x % nv;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (pb >= nprob || !active[pb]) return;   // block-uniform
    const int S = breduce_segments(C.cptr[pb + 1] - C.cptr[pb]);
    if (w < S) {
        const double a = breduce_seg(partial, C, pb, k, lane, w, S);
        if (lane == 0) seg[w] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int s = 0; s < S; ++s) t += seg[s];
        field_ptr(gm[pb], field)[k] = t;
    }
}

// Start of a cycle of every active problem (mode 1: reference norm = |r|).
// run[b] (the step mask of the Arnoldi kernels) starts as active and not done.
__global__ void k_bcycle_init(GmresDev* __restrict__ gm, int nprob, int m, int mode,
                              const int32_t* __restrict__ active, const int32_t* __restrict__ budget,
                              int32_t* __restrict__ run)
{
    int pb = blockIdx.x * blockDim.x + threadIdx.x;
    if (pb >= nprob) return;
    if (!active[pb]) {
        run[pb] = 0;
        return;
    }
    GmresDev& g = gm[pb];
    g.budget = budget[pb];   // steps left before max_iters (the cycle stops there, as the single solver's)
    if (mode == 1) g.fnorm2 = g.beta2;
    double beta = sqrt(g.beta2);
    double fn = sqrt(g.fnorm2);
    for (int q = 0; q <= m; ++q) g.g[q] = 0.0;
    g.g[0] = beta;
    g.inv_beta = beta > 0.0 ? 1.0 / beta : 0.0;
    g.est = fn > 0.0 ? beta / fn : 0.0;
    g.done = (g.est <= g.rtol || g.budget <= 0) ? 1 : 0;
    g.breakdown = 0;
    g.j = 0;       // steps taken in this cycle
    run[pb] = g.done ? 0 : 1;
}

__global__ void k_bsolve_y(GmresDev* __restrict__ gm, int nprob, const int32_t* __restrict__ active)
{
    int pb = blockIdx.x * blockDim.x + threadIdx.x;
    if (pb >= nprob || !active[pb]) return;
    GmresDev* g = &gm[pb];
    const int M = kMaxRestart, k = g->j;
    for (int q = k - 1; q >= 0; --q) {
        double v = g->g[q];
        for (int p = q + 1; p < k; ++p) v -= g->H[q * M + p] * g->y[p];
        g->y[q] = v / g->H[q * M + q];
    }
}

// x *= the problem's factor (inv_beta if which = 0, inv_h if which = 1).
// x *= inv_beta (which 0) or inv_h (which 1) of the chunk's problem, one block
// per chunk (chunks of stopped problems and of a broken-down step skipped).
template <class T>
__global__ void k_bscale(T* __restrict__ x, Chunks C, const GmresDev* __restrict__ gm, int which,
                         const int32_t* __restrict__ active)
{
    const int64_t c = blockIdx.x;
    const int pb = C.pid[c];
    if (!active[pb]) return;
    const GmresDev& g = gm[pb];
    if (which == 1 && g.done && g.breakdown) return;
    const double f = which == 0 ? g.inv_beta : g.inv_h;
    // FP32 bases are scaled in FP32 (the factor rounded once): the FP64 pipe of
    // GB300 would make a per-element FP64 product the cost of the pass
    const T fT = (T)f;
    for (int64_t i = C.beg[c] + threadIdx.x; i < C.end[c]; i += blockDim.x) x[i] = x[i] * fT;
}

// End of Arnoldi step j, one block per chunk: v_{j+1} /= |v_{j+1}| for the
// problems still running (1 / |v| from the norm of the last Gram-Schmidt pass,
// as the Arnoldi column computes it), and, in the block of each problem's
// first chunk, the Arnoldi column itself (Hessenberg column, rotations,
// estimate) and the stop test, which takes a stopped problem out of the step
// mask. A block of the same problem that already sees the problem stopped
// skips its scaling: v_{j+1} of a stopped problem is never used.
template <class T>
__global__ void __launch_bounds__(256)
    k_bscale_norm(T* __restrict__ x, Chunks C, GmresDev* __restrict__ gm, int nprob, int j, int32_t* __restrict__ run,
                  int passes)
{
    const int64_t c = blockIdx.x;
    const int pb = C.pid[c];
    if (!run[pb]) return;
    GmresDev* g = &gm[pb];
    const double hn = sqrt(fmax(g->nrm2, 0.0));
    const double f = hn > 0.0 ? 1.0 / hn : 0.0;
    if (c == C.cptr[pb] && threadIdx.x < 32) {
        arnoldi_column(g, j, passes);
        if (threadIdx.x == 0) {
            const int done = (g->est <= g->rtol || g->breakdown || j + 1 >= g->budget) ? 1 : 0;
            g->done = done;
            g->j = j + 1;
            if (done) run[pb] = 0;
        }
    }
    // FP32 bases are scaled in FP32 (the factor rounded once): the FP64 pipe of
    // GB300 would make a per-element FP64 product the cost of the pass
    const T fT = (T)f;
    for (int64_t i = C.beg[c] + threadIdx.x; i < C.end[c]; i += blockDim.x) x[i] = x[i] * fT;
}

// FP32 copy of r scaled by the problem's inv_beta (inner start of the mixed form).
// (with perm: out[q] = r[perm[q]] ..., the inner grid's order from the main one)
__global__ void k_bto_f32_scaled(const double* __restrict__ r, int64_t n, const int32_t* __restrict__ pid,
                                 const GmresDev* __restrict__ gm, const int32_t* __restrict__ active,
                                 const int32_t* __restrict__ perm, float* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int pb = pid[i];
        if (active[pb]) out[i] = (float)(r[perm ? perm[i] : i] * gm[pb].inv_beta);
    }
}

// t = sum_{q < k_b} y_q V_q with the problem's own step count and y, one
// block per chunk: the chunk's problem's coefficients are staged once in
// shared memory (with their float split for FP32 bases), and every element
// sums its q terms in order.
template <class T>
__global__ void __launch_bounds__(256)
    k_bcombine(const T* __restrict__ V, int64_t ldv, const GmresDev* __restrict__ gm, Chunks C,
               const int32_t* __restrict__ active, T* __restrict__ t)
{
    __shared__ double ys[kMaxRestart];
    __shared__ float yh[kMaxRestart], yl[kMaxRestart];
    const int64_t c = blockIdx.x;
    const int pb = C.pid[c];
    if (!active[pb]) return;
    const GmresDev& g = gm[pb];
    const int k = g.j;
    if (threadIdx.x < (unsigned)k) {
        const double v = g.y[threadIdx.x];
        ys[threadIdx.x] = v;
        yh[threadIdx.x] = (float)v;
        yl[threadIdx.x] = (float)(v - (double)(float)v);
    }
    __syncthreads();
    for (int64_t i = C.beg[c] + threadIdx.x; i < C.end[c]; i += blockDim.x) {
        if constexpr (sizeof(T) == 4) {
            DF a{0.f, 0.f};
            for (int q = 0; q < k; ++q) {
                const float vi = V[q * ldv + i];
                const float h = yh[q] * vi;
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

// w += u (with perm: w[perm[i]] += u[i], u in the inner grid's order)
template <class T>
__global__ void k_baxpy(double* __restrict__ w, const T* __restrict__ u, const int32_t* __restrict__ pid,
                        const int32_t* __restrict__ active, const int32_t* __restrict__ perm, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (active[pid[i]]) w[perm ? perm[i] : i] += (double)u[i];
}

__global__ void k_binit(GmresDev* __restrict__ gm, int nprob, double rtol)
{
    int pb = blockIdx.x * blockDim.x + threadIdx.x;
    if (pb >= nprob) return;
    gm[pb].rtol = rtol;
    gm[pb].done = 0;
    gm[pb].j = 0;
}

// Per-problem summary for the host: (|r|^2, |f|^2, steps of the last cycle, estimate).
__global__ void k_bpack(const GmresDev* __restrict__ gm, int nprob, double* __restrict__ out)
{
    int pb = blockIdx.x * blockDim.x + threadIdx.x;
    if (pb >= nprob) return;
    out[4 * pb + 0] = gm[pb].beta2;
    out[4 * pb + 1] = gm[pb].fnorm2;
    out[4 * pb + 2] = (double)gm[pb].j;
    out[4 * pb + 3] = gm[pb].est;
}

__global__ void k_w64_to_w32(const double* __restrict__ in, int64_t n, float* __restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void k_bzero_inactive_w(double* __restrict__ w, const int32_t* __restrict__ pid,
                                   const int32_t* __restrict__ zero, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (zero[pid[i]]) w[i] = 0.0;
}

unsigned bstream_blocks(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b > 16 * kNumSMs) b = 16 * kNumSMs;
    return (unsigned)(b < 1 ? 1 : b);
}

struct BatchWork {
    rbf_ctx* ctx;
    cudaStream_t st;
    Chunks C;
    int nprob;
    GmresDev* gm;
    const int32_t* active;   // problems of this cycle
    int32_t* run;            // problems still stepping in this cycle (the Arnoldi kernels' mask)
    double* partial;
    bool fused;              // FP32 cycle: one persistent launch per Arnoldi step (fused.cu)
    const int32_t* pid;
    int64_t n;
    int red_warps;           // warps of a k_breduce block: the most segments of any problem

    // The Gram-Schmidt passes of one step, over the problems still running.
    template <int MODE, class T>
    rbf_status mdot(const T* V, int64_t ldv, int nv, T* x, int field_in, int field_out, const int32_t* mask)
    {
        if constexpr (sizeof(T) == 4) {
            if (ctx->gs_stream && MODE != 1) {   // the basis streamed by bulk copies
                int* status = ctx->fused_sync.p + 5;
                const int check = ctx->stream_check;
                if (MODE == 0)
                    RBF_LAUNCH(ctx, k_bdots_stream, (unsigned)C.nc, kDotThreads, kStreamSmem, st, V, ldv, nv,
                               (const T*)x, C, mask, partial, status, ctx->fused_spin_limit, check);
                else
                    RBF_LAUNCH(ctx, k_bupdate_stream, (unsigned)C.nc, kDotThreads, kStreamSmem, st, V, ldv, nv, gm,
                               field_in, x, C, mask, partial, status, ctx->fused_spin_limit, check);
                const int nout = MODE == 2 ? 1 : nv;
                RBF_LAUNCH(ctx, k_breduce, (unsigned)(nprob * nout), 32 * red_warps, 0, st, partial, C, nprob, nout, gm,
                           field_out,
                           mask);
                return RBF_OK;
            }
        }
        if (MODE == 0)
            RBF_LAUNCH(ctx, (k_bdots<T>), (unsigned)(C.nc * nv), kDotThreads, 0, st, V, ldv, nv, (const T*)x, C,
                       mask, partial);
        else
            RBF_LAUNCH(ctx, (k_bupdate<T, MODE>), (unsigned)C.nc, kDotThreads, 0, st, V, ldv, nv, gm, field_in, x,
                       C, mask, partial);
        const int nout = MODE == 2 ? 1 : nv;
        RBF_LAUNCH(ctx, k_breduce, (unsigned)(nprob * nout), 32 * red_warps, 0, st, partial, C, nprob, nout, gm,
                   field_out, mask);
        return RBF_OK;
    }
};

template <class T>
struct BOps;

template <>
struct BOps<double> {
    static rbf_status amul(rbf_ctx* c, const double* x, double* y, cudaStream_t st)
    {
        return matvec_sorted_f64(c, x, y, st);
    }
    static rbf_status minv(rbf_ctx* c, const double* x, double* y, cudaStream_t st)
    {
        return rasm_apply_sorted(c, x, y, st);
    }
};

template <>
struct BOps<float> {
    static rbf_status amul(rbf_ctx* c, const float* x, float* y, cudaStream_t st)
    {
        return matvec_f32_raw(c, nullptr, x, y, st);
    }
    static rbf_status minv(rbf_ctx* c, const float* x, float* y, cudaStream_t st)
    {
        return rasm_apply_sorted_f32(c, x, y, st);
    }
};

// The launches of one Arnoldi cycle (m steps and the update of w), with no
// host synchronisation; V_0 holds the normalised start vector.
template <class T>
rbf_status batch_cycle(BatchWork& B, T* V, int64_t ldv, int m, T* u, T* t, double* w)
{
    rbf_ctx* ctx = B.ctx;
    cudaStream_t st = B.st;
    const int64_t n = B.n;
    const unsigned pb_blocks = blocks_for(B.nprob, 128);
    if constexpr (sizeof(T) == 4) {
        if (B.fused) {   // one persistent launch per Arnoldi step
            for (int j = 0; j < m; ++j)
                RBF_CHECK(fused_step(ctx, V, ldv, j, u, B.C, B.gm, B.nprob, B.run, B.partial, st));
        }
    }
    for (int j = 0; j < m && !B.fused; ++j) {
        T* vj = V + (int64_t)j * ldv;
        T* vn = V + (int64_t)(j + 1) * ldv;
        // the operators of the step skip the problems that have stopped in this cycle
        ctx->prof_step = j;
        ctx->active_mask = B.run;
        RBF_CHECK(BOps<T>::minv(ctx, vj, u, st));
        RBF_CHECK(BOps<T>::amul(ctx, u, vn, st));
        ctx->active_mask = B.active;
        RBF_CHECK(prof_begin(ctx, RBF_PROF_ORTHO, st));
        RBF_CHECK((B.mdot<0, T>(V, ldv, j + 1, vn, -1, F_H1, B.run)));
        if (gs_passes<T>() == 2) {
            RBF_CHECK((B.mdot<1, T>(V, ldv, j + 1, vn, F_H1, F_H2, B.run)));
            RBF_CHECK((B.mdot<2, T>(V, ldv, j + 1, vn, F_H2, F_NRM2, B.run)));
        } else {
            RBF_CHECK((B.mdot<2, T>(V, ldv, j + 1, vn, F_H1, F_NRM2, B.run)));
        }
        RBF_CHECK(prof_end(ctx, RBF_PROF_ORTHO, st));
        RBF_LAUNCH(ctx, (k_bscale_norm<T>), (unsigned)B.C.nc, 256, 0, st, vn, B.C, B.gm, B.nprob, j, B.run,
                   gs_passes<T>());
    }
    ctx->prof_step = -1;
    RBF_LAUNCH(ctx, k_bsolve_y, pb_blocks, 128, 0, st, B.gm, B.nprob, B.active);
    RBF_LAUNCH(ctx, (k_bcombine<T>), (unsigned)B.C.nc, 256, 0, st, V, ldv, B.gm, B.C, B.active, t);
    RBF_CHECK(BOps<T>::minv(ctx, t, u, st));
    RBF_LAUNCH(ctx, (k_baxpy<T>), bstream_blocks(n), 256, 0, st, w, u, B.pid, B.active,
               (sizeof(T) == 4 && ctx->inner_on) ? (const int32_t*)ctx->in.perm.p : nullptr, n);
    return RBF_OK;
}

// One cycle: captured into a CUDA graph on its first use in a solve and
// replayed afterwards (the kernel arguments of a cycle do not change within a
// solve; the per-problem masks and states they read live in device memory).
template <class T>
rbf_status run_cycle(BatchWork& B, T* V, int64_t ldv, int m, T* u, T* t, double* w)
{
    rbf_ctx* ctx = B.ctx;
    // profiled classes are recorded by event nodes inside the graph: a change of
    // the profiler's state takes a new capture
    const unsigned pmask = ctx->prof ? ctx->prof_mask : 0u;
    if (ctx->bgraph && pmask != ctx->bgraph_prof_mask) batch_graph_reset(ctx);
    if (ctx->bgraph_off) return batch_cycle<T>(B, V, ldv, m, u, t, w);   // launched directly (see below)
    if (!ctx->bgraph) {
        const uint64_t l0 = ctx->launches;
        ctx->capturing = true;
        ctx->bgraph_prof_mask = pmask;
        RBF_CUDA(ctx, cudaStreamBeginCapture(B.st, cudaStreamCaptureModeThreadLocal));
        rbf_status s = batch_cycle<T>(B, V, ldv, m, u, t, w);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(B.st, &g);
        ctx->capturing = false;
        ctx->prof_step = -1;
        if (s != RBF_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();   // a failed capture leaves its error behind for the next launch check
            if (B.fused) {
                // a runtime that cannot capture the cooperative launch: the fused
                // cycle is launched directly for the rest of the solve
                ctx->bgraph_off = true;
                return batch_cycle<T>(B, V, ldv, m, u, t, w);
            }
            if (s != RBF_OK) return s;
            return cuda_fail(ctx, e, "rbf_solve_batch: graph capture");
        }
        e = cudaGraphInstantiate(&ctx->bgraph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->bgraph = nullptr;
            return cuda_fail(ctx, e, "rbf_solve_batch: graph instantiation");
        }
        ctx->bgraph_launches = ctx->launches - l0;
        ctx->launches = l0;
    }
    RBF_CUDA(ctx, cudaGraphLaunch(ctx->bgraph, B.st));
    ctx->launches += ctx->bgraph_launches;
    return RBF_OK;
}

// Clears the matvec / apply mask, the inner-grid switch and the streamed
// passes' switch when the batched solve returns.
struct MaskGuard {
    rbf_ctx* ctx;
    ~MaskGuard()
    {
        ctx->active_mask = nullptr;
        ctx->inner_on = false;
        ctx->al.on = false;
        ctx->gs_stream = false;
    }
};

}  // namespace

void batch_graph_reset(rbf_ctx* ctx)
{
    if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
    ctx->bgraph = nullptr;
    ctx->bgraph_launches = 0;
    for (const rbf_graph_prof& g : ctx->bgraph_prof) {
        cudaEventDestroy(g.a);
        cudaEventDestroy(g.b);
    }
    ctx->bgraph_prof.clear();
    ctx->bgraph_prof_mask = 0;
}

rbf_status gmres_solve_batch(rbf_ctx* ctx, const double* f, double* w, const rbf_solve_params* p,
                             rbf_solve_info* infos, cudaStream_t user_st)
{
    // the solve runs on a stream of its own (capturable), ordered after user_st
    if (!ctx->bstream) {
        RBF_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->bstream, cudaStreamNonBlocking));
        RBF_CUDA(ctx, cudaEventCreateWithFlags(&ctx->bevent, cudaEventDisableTiming));
    }
    RBF_CUDA(ctx, cudaEventRecord(ctx->bevent, user_st));
    RBF_CUDA(ctx, cudaStreamWaitEvent(ctx->bstream, ctx->bevent, 0));
    cudaStream_t st = ctx->bstream;
    MaskGuard guard{ctx};
    const int64_t n = ctx->n;
    const int nprob = (int)ctx->nprob;
    const int m = p->restart > 0 ? p->restart : 30;
    const int max_iters = p->max_iters > 0 ? p->max_iters : 10000;
    const bool mixed = p->mixed != 0;
    const int max_refine = p->max_refine > 0 ? p->max_refine : 40;

    // chunk table
    std::vector<int32_t> cb, ce, cp, cptr(nprob + 1);
    for (int b = 0; b < nprob; ++b) {
        cptr[b] = (int32_t)cb.size();
        const Prob& q = ctx->prob_h[b];
        for (int64_t s = q.pbeg; s < q.pend; s += kBChunk) {
            cb.push_back((int32_t)s);
            ce.push_back((int32_t)std::min<int64_t>(s + kBChunk, q.pend));
            cp.push_back(b);
        }
    }
    cptr[nprob] = (int32_t)cb.size();
    const int64_t nc = (int64_t)cb.size();
    const size_t ctab = 3 * (size_t)nc + nprob + 1;   // one chunk table; the second half holds the compacted one
    RBF_CHECK(ensure(ctx, ctx->bch, 2 * ctab));
    int32_t* dch = ctx->bch.p;
    RBF_CUDA(ctx, cudaMemcpyAsync(dch, cb.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(dch + nc, ce.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(dch + 2 * nc, cp.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(dch + 3 * nc, cptr.data(), sizeof(int32_t) * (nprob + 1), cudaMemcpyHostToDevice,
                                  st));
    Chunks C{dch, dch + nc, dch + 2 * nc, dch + 3 * nc, nc};

    RBF_CHECK(ensure(ctx, ctx->gmb, nprob));
    RBF_CHECK(ensure(ctx, ctx->bactive, 4 * (size_t)nprob));
    RBF_CHECK(ensure(ctx, ctx->bstat, 4 * (size_t)nprob));
    RBF_CHECK(ensure(ctx, ctx->partial, (size_t)std::max<int64_t>(nc, 1) * 64));   // dots, and the fused step's norms
    RBF_CHECK(ensure(ctx, ctx->vec_a, n));
    RBF_CHECK(ensure(ctx, ctx->vec_b, n));
    GmresDev* gm = ctx->gmb.p;
    int32_t* active = ctx->bactive.p;
    int32_t* zero_mask = ctx->bactive.p + nprob;
    int32_t* budget = ctx->bactive.p + 2 * nprob;   // steps left per problem
    int32_t* run = ctx->bactive.p + 3 * nprob;      // problems still stepping in the current cycle
    RBF_CUDA(ctx, cudaMemsetAsync(gm, 0, sizeof(GmresDev) * nprob, st));
    const double rt = mixed ? (p->inner_rtol > 0.0 ? p->inner_rtol : 1e-5) : p->rtol;
    RBF_LAUNCH(ctx, k_binit, blocks_for(nprob, 128), 128, 0, st, gm, nprob, rt);
    std::vector<int32_t> act(nprob, 1), zmask(nprob, 0);
    RBF_CUDA(ctx, cudaMemcpyAsync(active, act.data(), sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st));

    // the FP64 products of this solve replay kept pair values when they fit:
    // an FP64 solve keeps them here, before any cycle (whose products they
    // serve) is captured; a mixed solve keeps them with its first outer
    // residual product, which they then form as well (outside the captured
    // inner cycles)
    if (!mixed) RBF_CHECK(f64_store_prepare(ctx, st));
    int max_chunks = 0;
    for (int b = 0; b < nprob; ++b) max_chunks = std::max(max_chunks, cptr[b + 1] - cptr[b]);
    BatchWork B{ctx, st, C, nprob, gm, active, run, ctx->partial.p, false, ctx->pid.p, n,
                breduce_segments(max_chunks)};
    // |f_b|^2
    RBF_CHECK((B.mdot<0, double>(f, 0, 1, const_cast<double*>(f), -1, F_FNORM2, active)));
    std::vector<double> stat(4 * (size_t)nprob);
    auto read_stat = [&]() -> rbf_status {
        RBF_LAUNCH(ctx, k_bpack, blocks_for(nprob, 128), 128, 0, st, gm, nprob, ctx->bstat.p);
        RBF_CUDA(ctx, cudaMemcpyAsync(stat.data(), ctx->bstat.p, sizeof(double) * 4 * nprob, cudaMemcpyDeviceToHost,
                                      st));
        RBF_CUDA(ctx, cudaStreamSynchronize(st));
        return RBF_OK;
    };
    RBF_CHECK(read_stat());
    std::vector<double> fnorm(nprob), relres(nprob, 0.0), est(nprob, 0.0);
    std::vector<int> iters(nprob, 0), cycles(nprob, 0), refines(nprob, 0), fmv(nprob, 0);
    bool any_zero = false;
    for (int b = 0; b < nprob; ++b) {
        fnorm[b] = std::sqrt(stat[4 * b + 1]);
        if (!std::isfinite(fnorm[b])) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_solve_batch: f of problem %d", b);
        if (fnorm[b] == 0.0) { act[b] = 0; zmask[b] = 1; any_zero = true; }
    }
    if (any_zero) {
        RBF_CUDA(ctx, cudaMemcpyAsync(zero_mask, zmask.data(), sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st));
        RBF_LAUNCH(ctx, k_bzero_inactive_w, bstream_blocks(n), 256, 0, st, w, ctx->pid.p, zero_mask, n);
        RBF_CUDA(ctx, cudaMemcpyAsync(active, act.data(), sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st));
    }

    // Krylov storage
    const int64_t ldv = ((n + 63) / 64) * 64;
    double* V64 = nullptr;
    float *Vf = nullptr, *uf = nullptr, *tf = nullptr;
    if (!mixed) {
        RBF_CHECK(ensure(ctx, ctx->V, (size_t)(m + 1) * ldv));
        V64 = ctx->V.p;
    } else {
        if (ctx->rasm_precision == RBF_FP64) {
            // FP64 subdomain inverses: the inner solves use an FP32 copy of them
            RBF_CHECK(ensure(ctx, ctx->W32, ctx->W64.count));
            RBF_LAUNCH(ctx, k_w64_to_w32, bstream_blocks((int64_t)ctx->W64.count), 256, 0, st, ctx->W64.p,
                       (int64_t)ctx->W64.count, ctx->W32.p);
            if (ctx->rasm_additive) RBF_CHECK(ensure(ctx, ctx->asm_u32, ctx->asm_u64.count));
        }
        RBF_CHECK(ensure(ctx, ctx->V, (size_t)((m + 3) * ldv + 1) / 2 + 1));
        Vf = (float*)ctx->V.p;
        // the inner grid (shorter cutoff, own order) for the FP32 inner solves
        if (p->inner_cutoff > 0.0 && !ctx->rasm_additive) {
            if (!ctx->in.ready || ctx->in.ri_sigmas != p->inner_cutoff) RBF_CHECK(bin_inner(ctx, p->inner_cutoff, st));
            ctx->inner_on = true;   // cleared with the mask when the solve returns
        }
        uf = Vf + (int64_t)(m + 1) * ldv;
        tf = uf + ldv;
    }
    double* r64 = mixed ? ctx->vec_b.p : V64;
    int total_steps = 0, rounds = 0;
    rbf_status result = RBF_ERR_NOT_CONVERGED;
    std::vector<std::vector<double>> hist(nprob);
    std::vector<int> stagnated(nprob, 0);
    std::vector<int32_t> left(nprob, 0);
    int compact_at = nprob / 2, compactions = 0;
    ctx->active_mask = active;   // converged problems are skipped by the matvec and the apply
    batch_graph_reset(ctx);      // buffers may have moved since the last solve
    ctx->bgraph_off = false;
    bool fused_ok = false;
    // the fused Arnoldi step: batches of the mixed form on the symmetric inner
    // matvec, unless a kernel class of the cycle is being profiled
    {
        constexpr unsigned kCycleClasses = (1u << RBF_PROF_MATVEC_F64) | (1u << RBF_PROF_MATVEC_F32) |
                                           (1u << RBF_PROF_RASM_APPLY) | (1u << RBF_PROF_ORTHO);
        const bool profiling = ctx->prof && (ctx->prof_mask & kCycleClasses);
        fused_ok = mixed && (nprob > 1 || ctx->fused_mode == 1 || n <= kFusedSingleMax) && !profiling &&
                   fused_step_applies(ctx);
        if (mixed) {   // the fused step's barrier state and the status words of the cycle's waits
            RBF_CHECK(ensure(ctx, ctx->fused_sync, 8));
            RBF_CUDA(ctx, cudaMemsetAsync(ctx->fused_sync.p, 0, 8 * sizeof(int), st));
        }
        ctx->gs_stream = mixed && ctx->gs_stream_mode != 0;
        if (ctx->gs_stream && !ctx->gs_stream_ready) {   // before any capture
            RBF_CUDA(ctx, cudaFuncSetAttribute(k_bdots_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kStreamSmem));
            RBF_CUDA(ctx, cudaFuncSetAttribute(k_bupdate_stream, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kStreamSmem));
            ctx->gs_stream_ready = true;
        }
        B.fused = fused_ok && (ctx->fused_mode == 1 || nprob <= kFusedTail);
    }
    // a zero initial guess (every problem) gives r0 = f without a product
    RBF_CHECK(ensure(ctx, ctx->flag_dev, 1));
    RBF_CUDA(ctx, cudaMemsetAsync(ctx->flag_dev.p, 0, sizeof(int), st));
    RBF_LAUNCH(ctx, k_any_nonzero, bstream_blocks(n), 256, 0, st, w, n, ctx->flag_dev.p);
    int w_nonzero = 1;
    RBF_CUDA(ctx, cudaMemcpyAsync(&w_nonzero, ctx->flag_dev.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    bool w_zero = w_nonzero == 0;
    for (;;) {
        // true FP64 residual of the active problems
        if (!w_zero) RBF_CHECK(matvec_sorted_f64_keep(ctx, w, ctx->vec_a.p, st));
        RBF_LAUNCH(ctx, k_bresidual, (unsigned)B.C.nc, kDotThreads, 0, st, f, w_zero ? nullptr : ctx->vec_a.p, r64,
                   B.C, active, B.partial);
        RBF_LAUNCH(ctx, k_breduce, (unsigned)nprob, 32 * B.red_warps, 0, st, B.partial, B.C, nprob, 1, gm, F_BETA2,
                   active);
        RBF_CHECK(read_stat());
        int nact = 0;
        for (int b = 0; b < nprob; ++b) {
            if (!act[b]) continue;
            if (!w_zero) ++fmv[b];
            relres[b] = std::sqrt(stat[4 * b + 0]) / fnorm[b];
            if (!std::isfinite(relres[b])) return fail(ctx, RBF_ERR_NOT_CONVERGED, "rbf_solve_batch: residual of "
                                                       "problem %d is not finite", b);
            if (relres[b] <= p->rtol || iters[b] >= max_iters || (mixed && refines[b] >= max_refine)) {
                act[b] = 0;
            } else if (stagnating(hist[b], relres[b])) {
                act[b] = 0;
                stagnated[b] = 1;
            } else {
                ++nact;
            }
        }
        RBF_CUDA(ctx, cudaMemcpyAsync(active, act.data(), sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st));
        w_zero = false;
        if (nact == 0) break;
        if (nact <= compact_at) {
            // Most problems have stopped: restrict the chunk table, the matvec
            // work lists and the subdomain list to the active problems (same
            // order within each problem) and capture the cycle again.
            std::vector<int32_t> kb, ke, kp, kptr(nprob + 1);
            for (int b = 0; b < nprob; ++b) {
                kptr[b] = (int32_t)kb.size();
                if (!act[b]) continue;
                for (int32_t c = cptr[b]; c < cptr[b + 1]; ++c) {
                    kb.push_back(cb[c]);
                    ke.push_back(ce[c]);
                    kp.push_back(cp[c]);
                }
            }
            kptr[nprob] = (int32_t)kb.size();
            const int64_t nk = (int64_t)kb.size();
            int32_t* dk = dch + ctab;
            RBF_CUDA(ctx, cudaMemcpyAsync(dk, kb.data(), sizeof(int32_t) * nk, cudaMemcpyHostToDevice, st));
            RBF_CUDA(ctx, cudaMemcpyAsync(dk + nk, ke.data(), sizeof(int32_t) * nk, cudaMemcpyHostToDevice, st));
            RBF_CUDA(ctx, cudaMemcpyAsync(dk + 2 * nk, kp.data(), sizeof(int32_t) * nk, cudaMemcpyHostToDevice, st));
            RBF_CUDA(ctx, cudaMemcpyAsync(dk + 3 * nk, kptr.data(), sizeof(int32_t) * (nprob + 1),
                                          cudaMemcpyHostToDevice, st));
            B.C = Chunks{dk, dk + nk, dk + 2 * nk, dk + 3 * nk, nk};
            RBF_CHECK(build_active_lists(ctx, active, st));
            batch_graph_reset(ctx);
            // few problems left: the fused step (one launch per Arnoldi step)
            B.fused = fused_ok && (ctx->fused_mode == 1 || nact <= kFusedTail);
            compact_at = nact / 2;
            ++compactions;
        }
        for (int b = 0; b < nprob; ++b) left[b] = std::max(0, max_iters - iters[b]);
        RBF_CUDA(ctx, cudaMemcpyAsync(budget, left.data(), sizeof(int32_t) * nprob, cudaMemcpyHostToDevice, st));
        // one cycle of every active problem
        RBF_LAUNCH(ctx, k_bcycle_init, blocks_for(nprob, 128), 128, 0, st, gm, nprob, m, mixed ? 1 : 0, active,
                   budget, run);
        if (!mixed) {
            RBF_LAUNCH(ctx, k_bscale<double>, (unsigned)B.C.nc, 256, 0, st, V64, B.C, gm, 0, active);
            RBF_CHECK(run_cycle<double>(B, V64, ldv, m, ctx->vec_b.p, ctx->vec_a.p, w));
        } else {
            RBF_LAUNCH(ctx, k_bto_f32_scaled, bstream_blocks(n), 256, 0, st, r64, n, ctx->pid.p, gm, active,
                       ctx->inner_on ? (const int32_t*)ctx->in.perm.p : nullptr, Vf);
            RBF_CHECK(run_cycle<float>(B, Vf, ldv, m, uf, tf, w));
        }
        int cycle_status[2] = {0, 0};   // the fused step's grid barriers; the bulk copies of the passes
        if (mixed)
            RBF_CUDA(ctx, cudaMemcpyAsync(cycle_status, ctx->fused_sync.p + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                          st));
        RBF_CHECK(read_stat());
        if (cycle_status[0] != 0)
            return fail(ctx, (rbf_status)cycle_status[0],
                        "rbf_solve_batch: a grid barrier of the fused Arnoldi step gave up waiting");
        if (cycle_status[1] != 0)
            return fail(ctx, (rbf_status)cycle_status[1],
                        "rbf_solve_batch: a bulk copy of a Gram-Schmidt pass did not arrive in time");
        if (!ctx->bgraph_prof.empty()) {
            int steps_run = 0;
            for (int b = 0; b < nprob; ++b)
                if (act[b]) steps_run = std::max(steps_run, (int)stat[4 * b + 2]);
            RBF_CHECK(prof_harvest_graph(ctx, steps_run));
        }
        for (int b = 0; b < nprob; ++b) {
            if (!act[b]) continue;
            iters[b] += (int)stat[4 * b + 2];
            est[b] = stat[4 * b + 3];
            ++cycles[b];
            if (mixed) ++refines[b];
        }
        total_steps += m;
        ++rounds;
    }
    result = RBF_OK;
    for (int b = 0; b < nprob; ++b)
        if (!(relres[b] <= p->rtol)) result = RBF_ERR_NOT_CONVERGED;
    if (infos) {
        for (int b = 0; b < nprob; ++b) {
            rbf_solve_info& I = infos[b];
            std::memset(&I, 0, sizeof(I));
            I.iters = iters[b];
            I.restarts = cycles[b];
            I.refinements = refines[b];
            I.relres = relres[b];
            I.relres_est = est[b] * (mixed ? relres[b] : 1.0);
            I.matvecs = fmv[b] + iters[b];
            I.applies = iters[b] + cycles[b];
            I.status = relres[b] <= p->rtol ? RBF_OK : RBF_ERR_NOT_CONVERGED;
            I.stagnated = stagnated[b];
        }
    }
    ctx->batch_rounds = rounds;
    ctx->batch_compactions = compactions;
    if (result != RBF_OK) fail(ctx, RBF_ERR_NOT_CONVERGED, "rbf_solve_batch: some problems missed rtol %.1e", p->rtol);
    return result;
}

}  // namespace rbf
