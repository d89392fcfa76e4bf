// noalloc.cu -- rbf_matvec_noalloc: the FP64 truncated matvec for callers that
// must not allocate device memory.
//
// rbf_matvec permutes w into cell order and the result back through two work
// vectors that the context allocates on first use. Some callers cannot let a
// library allocate: real-time loops that must not take the allocator's
// implicit device synchronisation, and applications whose device memory is
// owned by a pool of another framework with a fixed budget. This variant
// takes its two work vectors from one file-scope __device__ array of fixed
// size instead, so it calls no allocating routine.
//
// Limits and sharing:
//  * at most kNoAllocMaxPoints points (2 x 8 MiB of FP64 scratch, held by
//    every GPU that loads the library until the process exits);
//  * every call made in one CUDA context on a device (the runtime's primary
//    context, for ordinary callers) shares the one array; calls that overlap
//    on the GPU (different streams) race on it;
//  * the array keeps the previous call's contents; nothing here needs it to
//    start at zero (every entry used is written before it is read);
//  * the array's device address is looked up (cudaGetSymbolAddress) by the
//    first call made in each CUDA context, with that context current, and
//    cached per context: a context created later, or the primary context
//    recreated after cudaDeviceReset, gets its own lookup. Make that first
//    call in a context before any stream capture is begun in it.
#include <mutex>

#include "common.cuh"

namespace rbf {
namespace {

constexpr int64_t kNoAllocMaxPoints = 1 << 20;
constexpr int kNoAllocMaxContexts = 64;

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxPoints];

// cuCtxGetCurrent, fetched through the runtime (the library does not link the driver API).
typedef int (*CtxGetCurrentFn)(void**);

struct ScratchEntry {
    void* cu_ctx;
    double* addr;
};
ScratchEntry g_scratch[kNoAllocMaxContexts] = {};
int g_scratch_used = 0;
CtxGetCurrentFn g_ctx_get_current = nullptr;
std::mutex g_scratch_mu;

// Device address of the scratch array in the current CUDA context (whose device is current).
rbf_status scratch_address(rbf_ctx* ctx, double** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_ctx_get_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(ctx, RBF_ERR_CUDA, "rbf_matvec_noalloc: cuCtxGetCurrent is not available");
        g_ctx_get_current = (CtxGetCurrentFn)fn;
    }
    void* cu = nullptr;
    if (g_ctx_get_current(&cu) != 0 || !cu)
        return fail(ctx, RBF_ERR_CUDA, "rbf_matvec_noalloc: no current CUDA context");
    for (int i = 0; i < g_scratch_used; ++i) {
        if (g_scratch[i].cu_ctx == cu) {
            *out = g_scratch[i].addr;
            return RBF_OK;
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rbf_matvec_noalloc: cudaGetSymbolAddress");
    // a full table recycles the oldest entry (its context may have been destroyed)
    const int slot = g_scratch_used < kNoAllocMaxContexts ? g_scratch_used++ : 0;
    g_scratch[slot] = ScratchEntry{cu, (double*)p};
    *out = (double*)p;
    return RBF_OK;
}

}  // namespace
}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_matvec_noalloc(rbf_ctx* ctx, const double* w_dev, double* y_dev, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_matvec_noalloc: call rbf_bin first");
    if (ctx->al.on || ctx->active_mask)
        return fail(ctx, RBF_ERR_STATE, "rbf_matvec_noalloc: a batched solve is in progress on this context");
    if (!w_dev || !y_dev) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_matvec_noalloc: null vector");
    if (ctx->n > kNoAllocMaxPoints)
        return fail(ctx, RBF_ERR_INVALID_ARG,
                    "rbf_matvec_noalloc: n = %lld exceeds the static scratch capacity of %lld points",
                    (long long)ctx->n, (long long)kNoAllocMaxPoints);
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    double* scratch = nullptr;
    RBF_CHECK(scratch_address(ctx, &scratch));
    cudaStream_t st = (cudaStream_t)stream;
    double* w_sorted = scratch;
    double* y_sorted = scratch + kNoAllocMaxPoints;
    RBF_CHECK(permute_to_sorted(ctx, w_dev, w_sorted, st));
    RBF_CHECK(matvec_sorted_f64_plain(ctx, w_sorted, y_sorted, st));
    return permute_to_user(ctx, y_sorted, y_dev, st);
}
