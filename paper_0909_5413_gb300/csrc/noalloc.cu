// noalloc.cu -- rbf_matvec_noalloc: the FP64 truncated matvec for callers that
// must not allocate device memory.
//
// rbf_matvec permutes w into cell order and the result back through two work
// vectors that the context allocates on first use. Some callers cannot let a
// library allocate: code that runs while a CUDA graph is being captured (a
// cudaMalloc there fails or breaks the capture), real-time loops that must
// not take the allocator's implicit device synchronisation, and applications
// whose device memory is owned by a pool of another framework with a fixed
// budget. This variant takes its two work vectors from one file-scope
// __device__ array of fixed size instead, so it calls no allocating routine.
//
// Limits and sharing:
//  * at most kNoAllocMaxPoints points (2 x 8 MiB of FP64 scratch, held by
//    every GPU that loads the library until the process exits);
//  * every call on a device shares the one array; calls that overlap on the
//    GPU (different streams, or different contexts on one device) race on it;
//  * the array keeps the previous call's contents; nothing here needs it to
//    start at zero (every entry used is written before it is read);
//  * the first call on each device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture.
#include <mutex>

#include "common.cuh"

namespace rbf {
namespace {

constexpr int64_t kNoAllocMaxPoints = 1 << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxPoints];

double* g_scratch_addr[kNoAllocMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on `device` (which must be current).
rbf_status scratch_address(rbf_ctx* ctx, int device, double** out)
{
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rbf_matvec_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[device] = (double*)p;
    }
    *out = g_scratch_addr[device];
    return RBF_OK;
}

}  // namespace
}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_matvec_noalloc(rbf_ctx* ctx, const double* w_dev, double* y_dev, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_matvec_noalloc: call rbf_bin first");
    if (!w_dev || !y_dev) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_matvec_noalloc: null vector");
    if (ctx->n > kNoAllocMaxPoints)
        return fail(ctx, RBF_ERR_INVALID_ARG,
                    "rbf_matvec_noalloc: n = %lld exceeds the static scratch capacity of %lld points",
                    (long long)ctx->n, (long long)kNoAllocMaxPoints);
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_matvec_noalloc: device %d out of range", ctx->device);
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    double* scratch = nullptr;
    RBF_CHECK(scratch_address(ctx, ctx->device, &scratch));
    cudaStream_t st = (cudaStream_t)stream;
    double* w_sorted = scratch;
    double* y_sorted = scratch + kNoAllocMaxPoints;
    RBF_CHECK(permute_to_sorted(ctx, w_dev, w_sorted, st));
    RBF_CHECK(matvec_sorted_f64_plain(ctx, w_sorted, y_sorted, st));
    return permute_to_user(ctx, y_sorted, y_dev, st);
}
