// scan.cu -- multi-level exclusive prefix sums and a max-reduction over device arrays.
#include "common.cuh"

namespace rbf {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-local exclusive scan of one tile; writes the tile total to sums[block].
template <class Tin, class Tout>
__global__ void k_scan_tile(const Tin* in, Tout* out, int64_t n, int64_t* __restrict__ sums)
{
    __shared__ int64_t warp_tot[kScanThreads / 32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        int64_t x = (i < n) ? (int64_t)in[i] : 0;
        v[k] = run;
        run += x;
    }
    // inclusive scan of thread totals across the block
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t t = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t u = __shfl_up_sync(0xffffffffu, t, d);
        if (lane >= d) t += u;
    }
    if (lane == 31) warp_tot[warp] = t;
    __syncthreads();
    if (warp == 0) {
        int64_t w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += u;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = w;
    }
    __syncthreads();
    int64_t excl = t - run + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i < n) out[i] = (Tout)(v[k] + excl);
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = excl + run;
}

template <class Tout>
__global__ void k_scan_add(Tout* __restrict__ out, int64_t n, const int64_t* __restrict__ offs)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (Tout)((int64_t)out[i] + offs[i / kScanTile]);
}

template <class Tout>
__global__ void k_scan_total(Tout* __restrict__ out, int64_t n, const int64_t* __restrict__ total)
{
    out[n] = (Tout)total[0];
}

// Scan of int64 block sums in place (recursive), returns grand total in *total.
rbf_status scan_sums(rbf_ctx* ctx, int64_t* sums, int64_t nb, int64_t* total, int64_t* scratch, cudaStream_t st)
{
    int64_t nb2 = (nb + kScanTile - 1) / kScanTile;
    int64_t* sums2 = scratch;
    int64_t* rest = scratch + nb2;
    RBF_LAUNCH(ctx, (k_scan_tile<int64_t, int64_t>), blocks_for(nb, kScanTile), kScanThreads, 0, st, sums, sums, nb,
               sums2);
    if (nb2 > 1) {
        RBF_CHECK(scan_sums(ctx, sums2, nb2, total, rest, st));
        RBF_LAUNCH(ctx, k_scan_add<int64_t>, blocks_for(nb, 256), 256, 0, st, sums, nb, sums2);
    } else {
        RBF_CUDA(ctx, cudaMemcpyAsync(total, sums2, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    return RBF_OK;
}

template <class Tin, class Tout>
rbf_status exclusive_scan(rbf_ctx* ctx, const Tin* in, Tout* out, int64_t n, cudaStream_t st)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    // scratch: block sums, then space for the recursive levels, then the total
    int64_t need = nb + 2 * (nb / kScanTile + 2) + 64;
    RBF_CHECK(ensure(ctx, ctx->scan_tmp, (size_t)need + 1));
    int64_t* sums = ctx->scan_tmp.p;
    int64_t* total = ctx->scan_tmp.p + need;
    RBF_LAUNCH(ctx, (k_scan_tile<Tin, Tout>), (unsigned)nb, kScanThreads, 0, st, in, out, n, sums);
    if (nb > 1) {
        RBF_CHECK(scan_sums(ctx, sums, nb, total, sums + nb, st));
        RBF_LAUNCH(ctx, k_scan_add<Tout>, blocks_for(n, 256), 256, 0, st, out, n, sums);
    } else {
        RBF_CUDA(ctx, cudaMemcpyAsync(total, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    }
    RBF_LAUNCH(ctx, k_scan_total<Tout>, 1, 1, 0, st, out, n, total);
    return RBF_OK;
}

__global__ void k_max_partial(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ part)
{
    int32_t m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, in[i]);
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
    __shared__ int32_t sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        int32_t v = (threadIdx.x < blockDim.x / 32) ? sm[threadIdx.x] : 0;
        for (int d = 16; d > 0; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
        if (threadIdx.x == 0) part[blockIdx.x] = v;
    }
}

}  // namespace

rbf_status exclusive_scan_i32(rbf_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st)
{
    return exclusive_scan<int32_t, int32_t>(ctx, in, out, n, st);
}

rbf_status exclusive_scan_i64(rbf_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t st)
{
    return exclusive_scan<int64_t, int64_t>(ctx, in, out, n, st);
}

rbf_status reduce_max_i32(rbf_ctx* ctx, const int32_t* in, int64_t n, int32_t* out_host, cudaStream_t st)
{
    const int blocks = 2 * kNumSMs;
    RBF_CHECK(ensure(ctx, ctx->tmp_i32, blocks + 1));
    RBF_LAUNCH(ctx, k_max_partial, blocks, 256, 0, st, in, n, ctx->tmp_i32.p);
    RBF_LAUNCH(ctx, k_max_partial, 1, 256, 0, st, ctx->tmp_i32.p, (int64_t)blocks, ctx->tmp_i32.p + blocks);
    RBF_CUDA(ctx, cudaMemcpyAsync(out_host, ctx->tmp_i32.p + blocks, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    return RBF_OK;
}

}  // namespace rbf
