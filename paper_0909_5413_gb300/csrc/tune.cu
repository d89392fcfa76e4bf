// tune.cu -- autotuning of the cell-list cell size and the matvec tiles.
//
// For each candidate cell side (r_c, r_c/2, r_c/3, relative to the base cell
// side when one is given) the points are binned, and for each tile (32, 64,
// 128 targets per block) the FP64 and FP32 matvecs are timed with CUDA events
// on the caller's stream (one warm launch, then the best of three). The work
// of both kernels does not depend on the weights, so a zero vector serves.
// The candidate with the lowest w_f64 t_f64 + w_f32 t_f32 wins; the context
// is left binned with it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace rbf {
namespace {

constexpr int kTiles[3] = {32, 64, 128};

// Best of `reps` timed launches of fn() on st, after one untimed launch.
template <class Fn>
rbf_status time_best(rbf_ctx* ctx, cudaStream_t st, int reps, Fn fn, float* ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    RBF_CUDA(ctx, cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    if (err != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ctx, err, "rbf_tune: event");
    }
    rbf_status s = fn();
    float best = 3.0e38f;
    for (int r = 0; r < reps && s == RBF_OK; ++r) {
        cudaEventRecord(e0, st);
        s = fn();
        cudaEventRecord(e1, st);
        if (s != RBF_OK) break;
        err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) {
            s = cuda_fail(ctx, err, "rbf_tune: timing");
            break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return s;
}

}  // namespace
}  // namespace rbf

using namespace rbf;

extern "C" rbf_status rbf_tune(rbf_ctx* ctx, const double* xy_dev, int64_t n, const rbf_params* base, double w_f64,
                               double w_f32, rbf_params* best, double* score_ms, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!base || !best || !(w_f64 >= 0.0) || !(w_f32 >= 0.0) || !(w_f64 + w_f32 > 0.0))
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_tune: need parameters and non-negative weights, not both 0");
    cudaStream_t st = (cudaStream_t)stream;
    const double c0 = base->cell_size > 0.0 ? base->cell_size : base->cutoff;
    const double factors[3] = {1.0, 0.5, 1.0 / 3.0};
    double best_score = -1.0;
    rbf_params pick = *base;
    for (double f : factors) {
        rbf_params p = *base;
        p.cell_size = c0 * f;
        p.tile_f64 = p.tile_f32 = 128;
        if (std::ceil(p.cutoff / p.cell_size) > 64.0) continue;
        rbf_status s = rbf_bin(ctx, xy_dev, n, &p, stream);
        if (s == RBF_ERR_INVALID_ARG) continue;   // e.g. too many cells for this size
        RBF_CHECK(s);
        const int64_t ncell = ctx->ncell_total;
        RBF_CHECK(ensure(ctx, ctx->vec_a, (size_t)n));
        RBF_CHECK(ensure(ctx, ctx->vec_b, (size_t)n));
        RBF_CHECK(ensure(ctx, ctx->vec_c, (size_t)n));   // two FP32 vectors
        RBF_CUDA(ctx, cudaMemsetAsync(ctx->vec_a.p, 0, sizeof(double) * n, st));
        RBF_CUDA(ctx, cudaMemsetAsync(ctx->vec_c.p, 0, sizeof(double) * n, st));
        float* wf = (float*)ctx->vec_c.p;
        float* yf = wf + n;
        float t64 = 3.0e38f, t32 = 0.f;
        int tile64 = 128, tile32 = 128;
        for (int T : kTiles) {
            ctx->tile64 = T;
            RBF_CHECK(build_work(ctx, ctx->cell_start.p, ncell, T, ctx->mv_work, &ctx->n_work, st));
            float ms = 0.f;
            RBF_CHECK(time_best(ctx, st, 3, [&] { return matvec_sorted_f64_plain(ctx, ctx->vec_a.p, ctx->vec_b.p, st); },
                                &ms));
            if (ms < t64) {
                t64 = ms;
                tile64 = T;
            }
        }
        if (w_f32 > 0.0) {
            t32 = 3.0e38f;
            for (int T : kTiles) {
                ctx->tile32 = T;
                RBF_CHECK(build_work(ctx, ctx->cell_start.p, ncell, T, ctx->mv_work32, &ctx->n_work32, st));
                float ms = 0.f;
                RBF_CHECK(time_best(ctx, st, 3, [&] { return matvec_f32_raw(ctx, nullptr, wf, yf, st); }, &ms));
                if (ms < t32) {
                    t32 = ms;
                    tile32 = T;
                }
            }
        }
        const double score = w_f64 * t64 + w_f32 * t32;
        if (best_score < 0.0 || score < best_score) {
            best_score = score;
            pick = p;
            pick.tile_f64 = tile64;
            pick.tile_f32 = tile32;
        }
    }
    if (best_score < 0.0) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_tune: no candidate cell size could be binned");
    RBF_CHECK(rbf_bin(ctx, xy_dev, n, &pick, stream));
    *best = pick;
    if (score_ms) *score_ms = best_score;
    return RBF_OK;
}
