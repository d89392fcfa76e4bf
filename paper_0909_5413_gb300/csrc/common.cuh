// common.cuh -- internal declarations shared by the librbf.so translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/rbf.h"
#include "exp64.cuh"
#include "fixexp.cuh"

namespace rbf {

constexpr int kMaxRestart = 32;   // GMRES(m): m <= 32 (coefficients and partial sums use 32-wide slots)
constexpr int kMaxSub = 192;      // overlap list cap (subdomain matrix dimension)
constexpr int kNumSMs = 152;      // GB300

// Device-resident small state of one GMRES cycle (Hessenberg, Givens, g).
struct GmresDev {
    double H[(kMaxRestart + 1) * kMaxRestart];   // row-major (m+1) x m, stride kMaxRestart
    double cs[kMaxRestart], sn[kMaxRestart];
    double g[kMaxRestart + 1];
    double y[kMaxRestart];
    double h1[kMaxRestart + 1];   // first Gram-Schmidt pass coefficients
    double h2[kMaxRestart + 1];   // second pass coefficients
    double nrm2;                  // |v|^2 after the second pass
    double beta2;                 // |r|^2 of the cycle's starting residual
    double fnorm2;                // |f|^2
    double inv_h;                 // 1 / H[j+1][j] (0 on breakdown)
    double inv_beta;              // 1 / beta
    double est;                   // |g_{j+1}| / |f|
    double rtol;
    int j;                        // last completed step
    int done;                     // 1: cycle may stop (estimate met or breakdown)
    int breakdown;
    int budget;                   // batched solver: steps this problem may still take in the cycle
};

template <class T>
struct DevArray {
    T* p = nullptr;
    size_t count = 0;
};

// One interpolation problem of a context (a context holds one problem, or a
// batch of independent ones). Its points occupy [pbeg, pend) both in user
// order and in cell order; its cells are [cellbase, cellbase + ncx*ncy) and
// its subdomains [subbase, subbase + nbx*nby) of the context's global ids.
struct Prob {
    // kernel and cell grid
    double sigma, rc, rc2, s, knorm, K;   // K = 2048 s / ln 2 (FP64 matvec exp)
    double xmin, ymin, xmax, ymax, c;
    int64_t ncx, ncy, cellbase;
    int64_t pbeg, pend;
    int k;                                // stencil half-width ceil(rc / c)
    float a_loc;                          // FP32 offset scale sqrt(log2(e) s)
    float ca, rc2f_lo, rc2f_hi;           // c * a_loc; FP32 accept / exact-test band around rc2 a_loc^2
    // fixed-point kernel evaluation (fixexp.cuh)
    double fx_scale;                      // 2^S: coordinate -> int64
    unsigned long long fx_M;
    int fx_sh, fx_F;
    // subdomain boxes
    double x0, y0, B, delta;
    int64_t nbx, nby, subbase;
    int reach;
    int pad;
};

}  // namespace rbf

// The FP64 matvec's accept masks and kernel values of one binning, in the
// order its walk takes them (per work item of the full list).
struct F64Keep {
    bool valid = false;
    bool tried = false;   // did not fit for the current binning and settings: not tried again
    int tile = 0;
    int64_t bytes = 0;   // values and masks of the current binning
    rbf::DevArray<int64_t> cnt, nwords, val_off, mask_off;
    rbf::DevArray<double> val;
    rbf::DevArray<uint32_t> mask;
};

// The inner grid of the mixed form: the points binned again with cells of side
// r_i (a shorter cutoff for the FP32 inner matvec, stencil 3 x 3), their own
// order (inner position q holds main cell-ordered point perm[q]), and the
// subdomain lists re-indexed into that order.
struct InnerGrid {
    bool ready = false;
    // The symmetric FP32 kernel serves each problem whose inner cells hold at
    // most 128 points; the stencil kernel serves the others.
    bool sym = false;          // ... some problem
    bool sym_all = false;      // ... every problem
    rbf::DevArray<int32_t> sym_prob;   // per problem: 1 symmetric kernel; then 1 stencil kernel
    rbf::DevArray<int32_t> symw;   // its (cell, 0) items, non-empty cells by size class ceil(points / 32)
    int64_t symoff[5] = {0, 0, 0, 0, 0};   // class t holds items [symoff[t-1], symoff[t])
    rbf::DevArray<int32_t> work_ns;   // stencil kernel items of the other problems
    int64_t n_work_ns = 0;
    double ri_sigmas = 0.0;
    int tile = 64;
    int stage_max = 0;
    int64_t ncell = 0, n_work = 0;
    rbf::DevArray<int32_t> perm, iperm, cell_u, cell_s, counts, cell_start, tmp, work, pid_cell, wcnt, woff;
    rbf::DevArray<int32_t> ov_idx, core_idx;
    rbf::DevArray<double> xy_s;
    rbf::DevArray<float> loc;
    rbf::DevArray<rbf::Prob> prob;
};

// Evaluation points binned into a context's grid (rbf_eval).
struct EvalBins {
    int64_t m = 0, nwork = 0;
    rbf::DevArray<int32_t> pid, cell_u, cell_s, perm, iperm, tmp, counts, cell_start, wcnt, woff, work;
    rbf::DevArray<double> xy_s, w_s, s_s;   // sorted targets; w in cell order; s in target order
    rbf::DevArray<float> loc;
    rbf::DevArray<int> flag;
};

struct rbf_prof_slot {
    std::vector<cudaEvent_t> ev;   // pairs (start, stop)
    int64_t used = 0;
    double graph_ms = 0.0;         // launches inside replayed graphs, harvested after each replay
    int64_t graph_launches = 0;
};

// An event pair recorded by a captured Arnoldi cycle around one launch of a
// profiled class: `step` is the Arnoldi step of the launch (-1 after the steps).
struct rbf_graph_prof {
    int cls;
    int step;
    cudaEvent_t a, b;
};

struct rbf_ctx {
    int device = 0;
    bool prof = false;
    unsigned prof_mask = ~0u;     // classes recorded while prof is on (bit k: class k)
    rbf_prof_slot prof_slots[RBF_PROF_COUNT];
    rbf::ExpConsts expc;
    std::string err;
    uint64_t launches = 0;
    int64_t dev_bytes = 0;
    int64_t mem_limit = 0;        // rbf_set_memory_limit: cap on dev_bytes (0 = none)
    std::vector<std::pair<void*, size_t>> owned;   // every live allocation

    // ---- problems (one for rbf_bin, several for rbf_bin_batch)
    int64_t nprob = 0;
    std::vector<rbf::Prob> prob_h;
    rbf::DevArray<rbf::Prob> prob;
    rbf::DevArray<int32_t> pid;        // problem of each point (user order == cell order ranges)
    rbf::DevArray<int32_t> pid_cell;   // problem of each cell
    rbf::DevArray<int32_t> pid_sub;    // problem of each subdomain
    rbf::DevArray<int64_t> pbeg_dev;   // pbeg of each problem, plus the total

    // ---- binning (rbf_bin)
    bool binned = false;
    int64_t n = 0;
    double sigma = 0, rc = 0, rc2 = 0, cell = 0, s = 0, knorm = 1.0;
    int normalized = 0;
    int64_t ncx = 0, ncy = 0;      // grid of a single problem
    int64_t ncell_total = 0;       // cells of all problems
    int kst = 1;                   // stencil half-width ceil(rc / c)
    double bbox[4] = {0, 0, 0, 0};
    rbf::DevArray<int32_t> perm, iperm, cell_start, cell_s, counts, cell_u, tmp_i32;
    rbf::DevArray<double> xy_s;    // sorted coordinates, interleaved (x, y)
    rbf::DevArray<double> bbox_part, bbox_dev;
    rbf::DevArray<float> loc32;    // FP32 cell-local offsets scaled by sqrt(log2(e) s), interleaved
    rbf::DevArray<int32_t> mv_work, mv_wcnt, mv_woff;   // FP64 matvec work items (cell, first target), scan
    rbf::DevArray<int32_t> mv_work32;                    // FP32 matvec work items
    int64_t n_work = 0, n_work32 = 0;
    int tile64 = 128, tile32 = 128;   // targets per block of the FP64 / FP32 matvec
    int stage_max = 0;                // largest stencil source count of any cell (matvec staging)
    rbf::DevArray<double> exp2048; // 2^(-j/2048), j < 2048
    rbf::DevArray<unsigned long long> fxtab;   // T1 (1024) then T2 (1024), Q1.63
    EvalBins ev;                   // rbf_eval targets
    InnerGrid in;                  // mixed form: FP32 inner grid (built on demand by the solvers)
    bool inner_on = false;         // the FP32 operators and hand-offs use the inner grid
    int sym_mode = 0;              // inner FP32 operator: 0 symmetric kernel when the grid allows, 1 stencil kernel
    bool sym64 = false;            // the symmetric FP64 matvec serves some problem (3 x 3 stencil, cells <= 160 points)
    bool sym64_all = false;        // ... every problem
    rbf::DevArray<int32_t> sym64_prob;   // per problem: 1 symmetric kernel; then 1 stencil kernel
    rbf::DevArray<int32_t> mv_work_ns;   // stencil kernel items of the problems the symmetric one does not serve
    int64_t n_work_ns = 0;
    int sym64_mode = 1;            // FP64 matvec: 0 symmetric kernel where it applies (from the next binning), 1 stencil kernel
    rbf::DevArray<int32_t> sym64w;    // its (cell, 0) items by size class ceil(points / 32) = 1..5
    int64_t sym64off[6] = {0, 0, 0, 0, 0, 0};
    rbf::DevArray<double> sym64_slots;   // its row slot and four column slots per point
    rbf::DevArray<float> sym_slots;   // symmetric FP32 kernel: row slot and four column slots per point
    rbf::DevArray<unsigned long long> count_u64;   // one 64-bit counter (rbf_count_candidates)
    rbf::DevArray<int> flag_dev;                   // one flag (zero initial guess test of the solvers)
    double exp2048_c[3] = {0, 0, 0};

    // ---- subdomains (rbf_rasm_setup)
    bool rasm_ready = false;
    int rasm_precision = RBF_FP64;
    double x0 = 0, y0 = 0, B = 0, delta = 0;
    int64_t nbx = 0, nby = 0, nsub = 0;
    int max_ov = 0, max_core = 0;
    rbf::DevArray<int32_t> core_ptr, core_idx, ov_ptr, ov_idx, core_of, sub_cnt, sub_fill;
    rbf::DevArray<int64_t> w_off, w_size;
    rbf::DevArray<double> W64;
    rbf::DevArray<float> W32;
    bool rasm_additive = false;    // Eq. asm: W holds full inverses, applies gather through asm_t*
    rbf::DevArray<int32_t> asm_tptr, asm_tidx, asm_fill, asm_iota;   // overlap entries of each point
    rbf::DevArray<double> asm_u64;
    rbf::DevArray<float> asm_u32;
    rbf::DevArray<int> status_dev;
    rbf::DevArray<int32_t> tc_fb;   // tensor-core setup: [0] count, then the subdomains left to FP64
    int64_t factor_tc = 0, factor_fp64 = 0;   // subdomains factored by each path at the last setup

    // ---- solver workspace
    rbf::DevArray<double> V, vec_a, vec_b, vec_c, vec_d, vec_e, partial;
    rbf::DevArray<rbf::GmresDev> gm;
    rbf::GmresDev* gm_host = nullptr;   // pinned mirror for the per-step status read
    rbf::DevArray<int64_t> scan_tmp;
    rbf::DevArray<int32_t> nbr_cnt;
    rbf::DevArray<int64_t> nbr_ptr_tmp;

    // ---- batched solver workspace
    rbf::DevArray<int32_t> bch;        // chunk table
    rbf::DevArray<rbf::GmresDev> gmb;  // per-problem GMRES state
    rbf::DevArray<int32_t> bactive;    // per-problem active / zero masks
    rbf::DevArray<double> bstat;       // per-problem summary for the host
    int batch_rounds = 0;
    int batch_compactions = 0;              // work-list compactions of the last batched solve
    const int32_t* active_mask = nullptr;   // problems the matvec / apply skip when 0 (null: none)
    cudaStream_t bstream = nullptr;         // capturable stream of the batched solver
    cudaEvent_t bevent = nullptr;
    cudaGraphExec_t bgraph = nullptr;       // captured Arnoldi cycle of the batched solver
    uint64_t bgraph_launches = 0;           // kernels in that graph
    bool capturing = false;                 // launches are being captured into bgraph
    // fused Arnoldi step of the batched mixed solver (fused.cu)
    int fused_mode = 2;                     // fused Arnoldi step: 0 never, 1 always, 2 once few problems are active
    unsigned int fused_grid = 0;            // its resident grid (computed on first use)
    unsigned long long fused_spin_limit = 1ull << 23;   // polls of a barrier wait before it gives up
    int fused_extra_block = 0;              // check of the timeout path: barriers wait for one block too many
    bool bgraph_off = false;                // this solve launches its cycles directly (no capture)
    rbf::DevArray<double> host_xy, host_f, host_w;   // rbf_interpolate_host's device copies (kept between calls)
    F64Keep f64s;                  // the FP64 matvec's pair values, kept for replays (valid until the next binning)
    int store_mode = 1;            // keep them when they fit (1), never (0)
    rbf::DevArray<int> fused_sync;          // barrier state (4 ints), then status words: fused step, bulk copies
    int gs_stream_mode = 1;                 // FP32 Gram-Schmidt passes: 1 basis streamed by bulk copies, 0 registers
    bool gs_stream = false;                 // ... in the current solve
    bool gs_stream_ready = false;           // the kernels' shared-memory attribute is set
    int stream_check = 0;                   // 1: the bulk-copy waits wait on a barrier nothing completes
    int prof_step = -1;                     // Arnoldi step of the launches being issued (-1: none)
    unsigned bgraph_prof_mask = 0;          // profiler classes the captured graph records
    std::vector<rbf_graph_prof> bgraph_prof;   // its event pairs
    // Work lists of the batched solver restricted to the problems still active
    // (built when most problems have stopped; used by the matvecs and the apply
    // while `on`; cleared when the solve returns). Order-preserving subsets of
    // the full lists, so every problem's sums run in the same order.
    struct ActiveLists {
        bool on = false;
        rbf::DevArray<int32_t> w64, w32, sub, flag, pos, symw, sym64w, w64ns, w32ns;
        int64_t n64 = 0, n32 = 0, nsub = 0, n64ns = 0, n32ns = 0;
        int64_t symoff[5] = {0, 0, 0, 0, 0};
        int64_t sym64off[6] = {0, 0, 0, 0, 0, 0};
    } al;
};

namespace rbf {

rbf_status fail(rbf_ctx* ctx, rbf_status st, const char* fmt, ...);
rbf_status cuda_fail(rbf_ctx* ctx, cudaError_t e, const char* where);

template <class T>
rbf_status ensure(rbf_ctx* ctx, DevArray<T>& a, size_t count);
void release(rbf_ctx* ctx, void* p);

#define RBF_CUDA(ctx, call)                                                \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::rbf::cuda_fail((ctx), e_, #call);  \
    } while (0)

#define RBF_CHECK(call)                     \
    do {                                    \
        rbf_status s_ = (call);             \
        if (s_ != RBF_OK) return s_;        \
    } while (0)

// Launch a kernel, count it, and report a launch error.
#define RBF_LAUNCH(ctx, kernel, grid, block, smem, stream, ...)                       \
    do {                                                                              \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                   \
        (ctx)->launches++;                                                            \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess) return ::rbf::cuda_fail((ctx), e_, #kernel);           \
    } while (0)

inline unsigned blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 0x7fffffffLL) b = 0x7fffffffLL;
    return (unsigned)b;
}

// Profiler hooks: event pair around one launch (or launch sequence) of class id.
rbf_status prof_begin(rbf_ctx* ctx, int id, cudaStream_t st);
rbf_status prof_end(rbf_ctx* ctx, int id, cudaStream_t st);
// After a replay of the captured cycle has completed: add the durations of its
// recorded launches of steps < steps_run (and of those after the steps) to the
// profiler's totals; the launches of later steps found every problem stopped.
rbf_status prof_harvest_graph(rbf_ctx* ctx, int steps_run);

// ---- scan.cu
// out[0] = 0, out[i+1] = in[0] + ... + in[i] for i < n (int32 or int64 in, int64 or int32 out)
rbf_status exclusive_scan_i32(rbf_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);
rbf_status exclusive_scan_i64(rbf_ctx* ctx, const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
rbf_status reduce_max_i32(rbf_ctx* ctx, const int32_t* in, int64_t n, int32_t* out_host, cudaStream_t st);

// ---- bin.cu
rbf_status bin_points(rbf_ctx* ctx, const double* xy, cudaStream_t st);
rbf_status permute_to_sorted(rbf_ctx* ctx, const double* user, double* sorted, cudaStream_t st);
rbf_status permute_to_user(rbf_ctx* ctx, const double* sorted, double* user, cudaStream_t st);
rbf_status neighbor_lists(rbf_ctx* ctx, int64_t* ptr, int32_t* idx, int64_t capacity, int64_t* total,
                          cudaStream_t st);

rbf_status bin_targets(rbf_ctx* ctx, const double* xe, int64_t m, cudaStream_t st);
// Builds ctx->in for an inner cutoff of ri_sigmas sigma (after binning and RASM setup).
rbf_status bin_inner(rbf_ctx* ctx, double ri_sigmas, cudaStream_t st);
// Builds ctx->al from the per-problem mask `active` (device) and sets al.on.
rbf_status build_active_lists(rbf_ctx* ctx, const int32_t* active, cudaStream_t st);
// Sum over the cells of grid 0 (r_c cells) or 1 (inner grid) of points x stencil points.
rbf_status count_candidates(rbf_ctx* ctx, int grid, int64_t* total, cudaStream_t st);
// The FP32 inner operator on main cell-ordered FP64 vectors (variant 0: symmetric kernel, 1: stencil kernel).
rbf_status inner_matvec_debug(rbf_ctx* ctx, double ri_sigmas, const double* w_main, double* y_main, int variant,
                              cudaStream_t st);
// Pairs within the grid's cutoff (r_c on grid 0, the inner cutoff on grid 1), FP64 pair test.
rbf_status count_pairs(rbf_ctx* ctx, int grid, int64_t* total, cudaStream_t st);
// Main cell order <-> inner order for the FP32 hand-offs of the mixed form.
rbf_status inner_gather_scaled(rbf_ctx* ctx, const double* r_main, const double* scale_dev, float* out_inner,
                               cudaStream_t st);
rbf_status build_work(rbf_ctx* ctx, const int32_t* cell_start, int64_t ncell, int tile, DevArray<int32_t>& work,
                      int64_t* nwork_out, cudaStream_t st);
rbf_status matvec_f32_raw(rbf_ctx* ctx, const float2* loc, const float* w, float* y, cudaStream_t st);
rbf_status targets_to_user(rbf_ctx* ctx, const double* sorted, double* user, cudaStream_t st);

// ---- subdomain.cu
rbf_status build_subdomains(rbf_ctx* ctx, cudaStream_t st);
rbf_status export_subdomains(rbf_ctx* ctx, int32_t* core_ptr, int32_t* core_idx, int32_t* ov_ptr,
                             int32_t* ov_idx, cudaStream_t st);

// ---- matvec.cu  (vectors in cell order)
rbf_status matvec_sorted_f64(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st);
rbf_status matvec_sorted_f32(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st);
// The FP64 matvec launch alone (no profiler events), for the allocation-free entry point.
rbf_status matvec_sorted_f64_plain(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st);
// Computes and keeps the FP64 matvec's accept masks and pair values of the
// current binning when the store is enabled and they fit in free memory (the
// following FP64 products replay them, bit for bit); a no-op otherwise.
rbf_status f64_store_prepare(rbf_ctx* ctx, cudaStream_t st);   // keep the FP64 pair values (no product)
// y = A~ w (cell order), keeping the FP64 pair values in the same pass when
// they are not kept yet and may be (matvec_sorted_f64 otherwise)
rbf_status matvec_sorted_f64_keep(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st);
void f64_store_release(rbf_ctx* ctx);   // frees the kept values (the small per-item tables stay)
// The FP64 kernel for targets binned by bin_targets (cell-sorted; s in target order).
rbf_status eval_sorted_f64(rbf_ctx* ctx, const double* txy, const float* tloc, const int32_t* tcell_start,
                           const int32_t* twork, int64_t nwork, const double* w, double* s, cudaStream_t st);
// Function attributes of the matvec kernels (called once per binning, outside any capture).
rbf_status matvec_prepare(rbf_ctx* ctx);
// Drop the captured batched cycle (its kernels hold pointers into the context).
void batch_graph_reset(rbf_ctx* ctx);

// ---- rasm.cu  (vectors in cell order)
rbf_status rasm_factor(rbf_ctx* ctx, cudaStream_t st);
rbf_status asm_lists(rbf_ctx* ctx, cudaStream_t st);   // overlap entries per point (Eq. asm only)
rbf_status rasm_apply_sorted(rbf_ctx* ctx, const double* r, double* z, cudaStream_t st);
// ---- rasm_tc.cu: FP32 inverses on the tensor cores (RBF_FP32); the subdomains
// it cannot take are written to fb_list and counted in *fb_host
rbf_status rasm_factor_tc(rbf_ctx* ctx, int32_t* fb_list, unsigned int* fb_count_dev, int64_t* fb_host,
                          cudaStream_t st);

// ---- gmres.cu
rbf_status gmres_solve(rbf_ctx* ctx, const double* f_sorted, double* w_sorted, const rbf_solve_params* p,
                       rbf_solve_info* info, cudaStream_t st);

// ---- fused.cu: one persistent launch per Arnoldi step (batched mixed solve, inner grid)
struct Chunks;
bool fused_step_applies(rbf_ctx* ctx);
rbf_status fused_step(rbf_ctx* ctx, float* V, int64_t ldv, int j, float* u, const Chunks& C, GmresDev* gm, int nprob,
                      int32_t* run, double* partial, cudaStream_t st);

// ---- gmres_batch.cu
rbf_status gmres_solve_batch(rbf_ctx* ctx, const double* f_sorted, double* w_sorted, const rbf_solve_params* p,
                             rbf_solve_info* infos, cudaStream_t st);

}  // namespace rbf
