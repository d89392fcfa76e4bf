// fused.cu -- one persistent launch per Arnoldi step of the batched mixed
// solver (Sec. 2.3: many subdomains per process, here every subdomain and
// every problem of the batch on one GPU).
//
// The step's phases, for every problem still running in the cycle (the step
// mask `run`), separated by grid-wide barriers:
//   1. u = M^{-1} v_j            RASM apply, one warp per subdomain (Eq. rasm)
//   2. A_i u                     symmetric FP32 matvec, one warp per inner cell
//   3. v_{j+1}, V_k . v_{j+1}    v_{j+1} summed from the matvec's slots (stored by
//                                the chunk's k = 0 block), dots, one block per (chunk, k)
//   4. v_{j+1} -= V h, |v|^2     per chunk: h of its problem reduced over the
//                                problem's chunks, then the update pass
//   5. v_{j+1} /= |v_{j+1}|      per chunk: |v|^2 of its problem reduced, the
//                                scaling; the problem's first chunk also runs the
//                                Arnoldi column (Hessenberg, Givens, estimate, stop)
// run in one cooperative launch of a grid that is resident at once, with a
// grid-wide barrier between phases. Each phase uses the same per-warp and
// per-chunk code as the separate kernels of the step, in the same order, so
// a problem's result is the same bit for bit with and without the fused step.
//
// Every wait at a barrier is bounded: after `spin_limit` polls a block gives
// up, raises the abort flag and records RBF_ERR_TIMEOUT in the status word;
// every other block leaves at its next barrier, and the host reports the
// status after the cycle. No wait is unbounded and nothing traps.
#include <algorithm>

#include "apply.cuh"
#include "batch.cuh"
#include "common.cuh"
#include "matvec_sym.cuh"
#include "ortho.cuh"
#include "vecops.cuh"

namespace rbf {

// Barrier state of one launch (cleared before it) and the solve's status word.
struct FusedSync {
    unsigned int count;    // blocks arrived at the current barrier
    unsigned int gen;      // barriers completed
    int abort;             // a block gave up waiting
    int pad;
};

struct FusedArgs {
    // phase 1: the apply, over the inner grid's subdomain lists
    const int32_t *ov_ptr, *ov_idx, *core_ptr, *core_idx, *sub_list, *pid_sub;
    const int64_t* w_off;
    const float* W;
    int64_t nsub;
    // phases 2-3: the symmetric matvec and its gather
    MvParams P;
    const int32_t* cells;
    int64_t ncells;
    float *rowslot, *colslot;
    const int32_t* pid;
    int64_t n;
    // phases 4-8: the Krylov basis and the per-problem state
    float* V;
    int64_t ldv;
    int j;
    float* u;
    Chunks C;
    GmresDev* gm;
    int nprob;
    int32_t* run;
    double* partial;
    // the barrier
    FusedSync* sync;
    int* status;
    unsigned int nblocks;            // blocks that must arrive (the grid; one more only in the timeout check)
    unsigned long long spin_limit;   // polls before a wait gives up
};

namespace {

constexpr int kFusedThreads = kDotThreads;   // 256: the per-chunk code's block
constexpr int kFusedWarps = kFusedThreads / 32;

// Shared memory of the step: the largest phase (the matvec's per-warp stage
// and transpose) with the others overlaid.
struct FusedSmem {
    union {
        SymWarp sym[kFusedWarps];
        float rg[kFusedWarps][kMaxSub];
        struct {
            OrthoCoef cf;
            OrthoRed red;
        } o;
        struct {
            double hc[kFusedWarps][kMaxRestart + 1];
            double cs[kFusedWarps][kMaxRestart];
            double sn[kFusedWarps][kMaxRestart];
        } a;
    };
};

// Grid-wide barrier with a bounded wait. Returns false (in every thread of
// the block) when the step is to be abandoned: this block or another gave up.
__device__ bool fused_barrier(const FusedArgs& A)
{
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile FusedSync* s = A.sync;
        const unsigned int g = s->gen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&A.sync->count, 1u) + 1u;
        if (arrived == A.nblocks) {
            A.sync->count = 0u;
            __threadfence();
            atomicAdd(&A.sync->gen, 1u);
        } else {
            unsigned long long polls = 0;
            while (s->gen == g) {
                if (s->abort) {
                    ok = 0;
                    break;
                }
                if (++polls > A.spin_limit) {
                    atomicExch(&A.sync->abort, 1);
                    atomicExch(A.status, (int)RBF_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (s->abort) ok = 0;
    }
    return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(kFusedThreads, 2) k_fused_step(FusedArgs A)
{
    extern __shared__ __align__(16) unsigned char fused_raw[];
    FusedSmem& S = *reinterpret_cast<FusedSmem*>(fused_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t gwarp = (int64_t)blockIdx.x * kFusedWarps + warp;
    const int64_t nwarps = (int64_t)gridDim.x * kFusedWarps;
    float* vj = A.V + (int64_t)A.j * A.ldv;
    float* vn = A.V + (int64_t)(A.j + 1) * A.ldv;
    const int nv = A.j + 1;

    // 1. u = M^{-1} v_j
    for (int64_t idx = gwarp; idx < A.nsub; idx += nwarps) {
        const int64_t sub = A.sub_list ? (int64_t)A.sub_list[idx] : idx;
        rasm_apply_one<float, float>(sub, lane, S.rg[warp], A.ov_ptr, A.ov_idx, A.core_ptr, A.core_idx, A.w_off, A.W,
                                     A.pid_sub, A.run, vj, A.u);
    }
    if (!fused_barrier(A)) return;
    // 2. the symmetric matvec's cells
    for (int64_t it = gwarp; it < A.ncells; it += nwarps) {
        const int cell = A.cells[2 * it];
        const int pcell = A.P.pid_cell[cell];
        if (!A.run[pcell]) continue;
        const Prob& pr = A.P.prob[pcell];
        const int cb = A.P.cell_start[cell], cnt = A.P.cell_start[cell + 1] - cb;
        switch ((cnt + 31) >> 5) {
        case 1: sym_cell<1>(A.P, S.sym[warp], lane, cell, cb, cnt, pr, A.u, A.rowslot, A.colslot, A.n); break;
        case 2: sym_cell<2>(A.P, S.sym[warp], lane, cell, cb, cnt, pr, A.u, A.rowslot, A.colslot, A.n); break;
        case 3: sym_cell<3>(A.P, S.sym[warp], lane, cell, cb, cnt, pr, A.u, A.rowslot, A.colslot, A.n); break;
        default: sym_cell<4>(A.P, S.sym[warp], lane, cell, cb, cnt, pr, A.u, A.rowslot, A.colslot, A.n); break;
        }
    }
    if (!fused_barrier(A)) return;
    // 3. v_{j+1} from the matvec's slots (the gather's fixed order; the k = 0
    // block of a chunk stores it) and the dots V_k . v_{j+1}, one block per (chunk, k)
    const int64_t n = A.n;
    for (int64_t unit = blockIdx.x; unit < A.C.nc * nv; unit += gridDim.x) {
        const int k = (int)(unit % nv);
        const int64_t c = unit / nv;
        __syncthreads();   // the previous unit is done with the reduction scratch
        if (!A.run[A.C.pid[c]]) {
            if (tid == 0) A.partial[c * 32 + k] = 0.0;
            continue;
        }
        const int64_t b = A.C.beg[c], e = A.C.end[c];
        const float* vk = A.V + k * A.ldv;
        float a[kOrthoPer], xs[kOrthoPer];
#pragma unroll
        for (int q = 0; q < kOrthoPer; ++q) {
            const int64_t i = b + tid + (int64_t)q * kFusedThreads;
            a[q] = i < e ? vk[i] : 0.f;
            xs[q] = i < e ? (((A.rowslot[i] + A.colslot[i]) + A.colslot[n + i]) + A.colslot[2 * n + i]) +
                                A.colslot[3 * n + i]
                          : 0.f;
        }
        if (k == 0) {
#pragma unroll
            for (int q = 0; q < kOrthoPer; ++q) {
                const int64_t i = b + tid + (int64_t)q * kFusedThreads;
                if (i < e) vn[i] = xs[q];
            }
        }
        ortho_warp_sum(ortho_thread_dot<float>(a, xs, b, e), S.o.red, 0);
        __syncthreads();
        if (tid == 0) A.partial[c * 32 + k] = ortho_block_total<float>(S.o.red, 0);
    }
    if (!fused_barrier(A)) return;
    // 4. per chunk: h of its problem (reduced over the problem's chunks, the
    // per-problem order; the problem's first chunk also stores it), then
    // v_{j+1} -= V h and the chunk's |v_{j+1}|^2
    double* partial2 = A.partial + A.C.nc * 32;
    for (int64_t c = blockIdx.x; c < A.C.nc; c += gridDim.x) {
        const int pb = A.C.pid[c];
        double* out = partial2 + c * 32;
        __syncthreads();   // the previous chunk is done with cf and red
        if (!A.run[pb]) {
            if (tid == 0) out[0] = 0.0;
            continue;
        }
        const bool first = c == A.C.cptr[pb];
        for (int k = warp; k < nv; k += kFusedWarps) {
            const double hk = breduce_one(A.partial, A.C, pb, k, lane);
            if (lane == 0) {
                ortho_coef_set(S.o.cf, k, hk);
                if (first) A.gm[pb].h1[k] = hk;
            }
        }
        __syncthreads();
        const int64_t b = A.C.beg[c], e = A.C.end[c];
        DF xl[kOrthoPer];
        ortho_load_x<float>(xl, vn, b, e);
        ortho_apply<float, ortho_group<float>()>(xl, A.V, A.ldv, nv, S.o.cf, b, e);
        float xs[kOrthoPer];
        ortho_store_x<float>(xl, xs, vn, b, e);
        ortho_warp_sum(ortho_thread_dot<float>(xs, xs, b, e), S.o.red, 0);
        __syncthreads();
        if (tid == 0) out[0] = ortho_block_total<float>(S.o.red, 0);
    }
    if (!fused_barrier(A)) return;
    // 5. per chunk: |v_{j+1}|^2 of its problem, v_{j+1} /= |v_{j+1}|; the
    // problem's first chunk also takes the Arnoldi column and the stop test
    // (a chunk that already sees its problem stopped leaves v_{j+1} as it is:
    // it is not used)
    for (int64_t c = blockIdx.x; c < A.C.nc; c += gridDim.x) {
        const int pb = A.C.pid[c];
        __syncthreads();
        if (!A.run[pb]) continue;
        if (warp == 0) {
            const double nrm2 = breduce_one(partial2, A.C, pb, 0, lane);
            if (lane == 0) S.a.hc[1][0] = nrm2;
            if (c == A.C.cptr[pb]) {
                GmresDev* g = &A.gm[pb];
                if (lane == 0) g->nrm2 = nrm2;
                __syncwarp();
                arnoldi_column_s(g, A.j, 1, S.a.hc[0], S.a.cs[0], S.a.sn[0]);
                if (lane == 0) {
                    const int done = (g->est <= g->rtol || g->breakdown || A.j + 1 >= g->budget) ? 1 : 0;
                    g->done = done;
                    g->j = A.j + 1;
                    if (done) A.run[pb] = 0;
                }
            }
        }
        __syncthreads();
        const double hn = sqrt(fmax(S.a.hc[1][0], 0.0));
        const float f = (float)(hn > 0.0 ? 1.0 / hn : 0.0);
        for (int64_t i = A.C.beg[c] + tid; i < A.C.end[c]; i += kFusedThreads) vn[i] = vn[i] * f;
    }
}

}  // namespace

// Grid of the fused step: as many blocks as are resident at once (a
// cooperative launch requires it), computed once per context.
static rbf_status fused_grid(rbf_ctx* ctx, unsigned int* grid, size_t* smem)
{
    *smem = sizeof(FusedSmem);
    if (ctx->fused_grid == 0) {
        RBF_CUDA(ctx, cudaFuncSetAttribute(k_fused_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
        int per_sm = 0;
        RBF_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_step, kFusedThreads, *smem));
        int sms = 0;
        RBF_CUDA(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        if (per_sm < 1) return fail(ctx, RBF_ERR_CUDA, "fused Arnoldi step: no block fits on an SM");
        ctx->fused_grid = (unsigned int)(per_sm * sms);
    }
    *grid = ctx->fused_grid;
    return RBF_OK;
}

bool fused_step_applies(rbf_ctx* ctx)
{
    MvParams P;
    const int32_t* cells = nullptr;
    int64_t ncells = 0;
    return ctx->fused_mode != 0 && inner_sym_params(ctx, &P, &cells, &ncells);
}

rbf_status fused_step(rbf_ctx* ctx, float* V, int64_t ldv, int j, float* u, const Chunks& C, GmresDev* gm, int nprob,
                      int32_t* run, double* partial, cudaStream_t st)
{
    FusedArgs A;
    if (!inner_sym_params(ctx, &A.P, &A.cells, &A.ncells))
        return fail(ctx, RBF_ERR_STATE, "fused Arnoldi step: needs the symmetric FP32 matvec on the inner grid");
    A.P.active = run;
    A.ov_ptr = ctx->ov_ptr.p;
    A.ov_idx = ctx->in.ov_idx.p;
    A.core_ptr = ctx->core_ptr.p;
    A.core_idx = ctx->in.core_idx.p;
    A.sub_list = ctx->al.on ? ctx->al.sub.p : nullptr;
    A.nsub = ctx->al.on ? ctx->al.nsub : ctx->nsub;
    A.pid_sub = ctx->pid_sub.p;
    A.w_off = ctx->w_off.p;
    A.W = ctx->W32.p;
    A.rowslot = ctx->sym_slots.p;
    A.colslot = ctx->sym_slots.p + ctx->n;
    A.pid = ctx->pid.p;
    A.n = ctx->n;
    A.V = V;
    A.ldv = ldv;
    A.j = j;
    A.u = u;
    A.C = C;
    A.gm = gm;
    A.nprob = nprob;
    A.run = run;
    A.partial = partial;
    A.sync = reinterpret_cast<FusedSync*>(ctx->fused_sync.p);
    A.status = reinterpret_cast<int*>(ctx->fused_sync.p) + 4;
    unsigned int grid = 0;
    size_t smem = 0;
    RBF_CHECK(fused_grid(ctx, &grid, &smem));
    A.nblocks = grid + (ctx->fused_extra_block ? 1u : 0u);
    A.spin_limit = ctx->fused_spin_limit;
    RBF_CUDA(ctx, cudaMemsetAsync(A.sync, 0, sizeof(FusedSync), st));
    void* args[] = {&A};
    RBF_CUDA(ctx, cudaLaunchCooperativeKernel((const void*)k_fused_step, dim3(grid), dim3(kFusedThreads), args, smem,
                                              st));
    ctx->launches++;
    return RBF_OK;
}

}  // namespace rbf
