/*
 * rbf.h -- C ABI of the GB300 Gaussian RBF interpolation library (librbf.so).
 *
 * The library solves the interpolation system of Eq. rbf2 with a Gaussian
 * basis and no polynomial block (the Gaussian is positive definite, Sec. 2.1):
 *
 *     sum_j w_j k(|x_i - x_j|^2) = f_i,   k(r2) = exp(-r2 / (2 sigma^2))
 *
 * (optionally times 1/(2 pi sigma^2), the normalised form of Sec. 2.3), with
 * entries of pairs farther apart than the cutoff r_c dropped (Sec. 2.3), by
 * GMRES preconditioned with the restricted additive Schwarz method of
 * Eq. rasm over small overlapping box subdomains (Sec. 2.2 - 2.4).
 *
 * Conventions for every call:
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library reads or writes them only in stream order on `stream`.
 *    Pointers named *_host are host pointers owned by the caller.
 *  - Point arrays are AoS FP64 pairs (x0, y0, x1, y1, ...); vectors are FP64
 *    and indexed in the caller's point order ("user order") unless a call
 *    says otherwise.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *  - Every call returns an rbf_status; nothing aborts, traps or exits.
 *    rbf_last_error() gives a human-readable detail of the last failure.
 *  - The context owns every internal device buffer (sorted points, index
 *    lists, factors, Krylov basis) until rbf_destroy() or the next rbf_bin().
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef RBF_H
#define RBF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RBF_OK = 0,
    RBF_ERR_INVALID_ARG = 1,          /* bad pointer, size or parameter */
    RBF_ERR_OOM = 2,                  /* a device allocation failed */
    RBF_ERR_CUDA = 3,                 /* a CUDA runtime call failed (see rbf_last_error) */
    RBF_ERR_NOT_SPD = 4,              /* a subdomain matrix had a pivot <= 0 */
    RBF_ERR_SUBDOMAIN_TOO_LARGE = 5,  /* an overlap list exceeds max_sub_points */
    RBF_ERR_NOT_CONVERGED = 6,        /* tolerance not reached within max_iters */
    RBF_ERR_TIMEOUT = 7,              /* a bounded device wait gave up */
    RBF_ERR_STATE = 8                 /* call out of order (e.g. apply before setup) */
} rbf_status;

/* Precisions. For rbf_matvec: RBF_FP64 or RBF_FP32. For the subdomain
 * inverses of rbf_rasm_setup (rbf_rasm_params.precision):
 *   RBF_FP64           computed and stored in FP64 (Cholesky, Sec. 2.2);
 *   RBF_FP32           computed in FP32 on the tensor cores and stored in FP32,
 *                      for the inner solves of the mixed form: A_i formed in
 *                      FP32 (the pair test and exp2 on scaled offsets), then
 *                      the block sweep
 *                      (Gauss-Jordan without pivoting on the SPD A_i, 8 x 8
 *                      blocks) with every product a TF32 MMA split into three
 *                      (FP32 accuracy) and FP32 accumulation; a subdomain of
 *                      more than 48 overlap points, or with an FP32 pivot that
 *                      is not positive, is computed in FP64 instead;
 *   RBF_FP32_FROM_FP64 computed in FP64 (as RBF_FP64), stored in FP32. */
enum { RBF_FP64 = 0, RBF_FP32 = 1, RBF_FP32_FROM_FP64 = 2 };

typedef struct rbf_ctx rbf_ctx;
typedef void* rbf_stream;

/* Kernel and binning parameters (Sec. 2.3, Sec. 3.1). */
typedef struct {
    double sigma;      /* Gaussian width sigma > 0 */
    double cutoff;     /* r_c > 0; pairs with r2 > r_c^2 are dropped */
    double cell_size;  /* cell side c of the cell list; <= 0 selects c = r_c */
    int normalized;    /* 1: multiply the kernel by 1/(2 pi sigma^2) (Sec. 2.3) */
    int tile_f64;      /* targets per block of the FP64 matvec: 32, 64 or 128 (0 = 128) */
    int tile_f32;      /* targets per block of the FP32 matvec: 32, 64 or 128 (0 = 128) */
} rbf_params;

/* Subdomain boxes (Sec. 2.2, Sec. 3.1): core box (bx, by) covers
 * [x0 + bx B, x0 + (bx+1) B) x [y0 + by B, y0 + (by+1) B) (clamped at the
 * edges); its overlap box adds `overlap` on every side (half-open). */
typedef struct {
    double x0, y0;        /* box origin */
    double core_size;     /* B > 0 */
    double overlap;       /* delta >= 0 */
    int max_sub_points;   /* cap on an overlap list, 1..192 (0 = 192) */
    int precision;        /* subdomain inverses: RBF_FP64, RBF_FP32 (tensor cores) or RBF_FP32_FROM_FP64 */
    int additive;         /* 0: restricted (Eq. rasm, default); 1: plain additive Schwarz (Eq. asm), for
                           * comparison: every overlap entry of A_i^{-1} r_i is added back (full n x n
                           * inverses, about n_overlap / n_core times the memory) */
} rbf_rasm_params;

/* GMRES settings (Sec. 2.2, Sec. 3.1: GMRES with RASM, rtol 1e-13). */
typedef struct {
    double rtol;          /* stop when ||f - A w||_2 / ||f||_2 <= rtol (true residual) */
    int restart;          /* m of GMRES(m), 1..32 (0 = 30) */
    int max_iters;        /* total Arnoldi steps (inner steps summed) (0 = 10000) */
    int mixed;            /* 1: FP32 inner GMRES + FP64 iterative refinement */
    int max_refine;       /* mixed only: outer refinement steps (0 = 40) */
    double inner_rtol;    /* mixed only: relative tolerance of each inner solve (0 = 1e-5) */
    double inner_cutoff;  /* mixed only: > 0 runs the FP32 inner solves on a second grid with this shorter
                           * cutoff, in units of sigma (6.1: dropped entries below e^-18.6 = 8e-9, under
                           * FP32 rounding); the FP64 residual keeps r_c. 0 = the r_c grid. Not used with
                           * the additive Schwarz variant. The grid is built at the first such solve. */
} rbf_solve_params;

typedef struct {
    int iters;            /* Arnoldi steps taken (all cycles, all refinements) */
    int restarts;         /* GMRES cycles completed */
    int refinements;      /* outer FP64 refinement steps (mixed), 0 otherwise */
    double relres;        /* final true relative residual, FP64 matvec */
    double relres_est;    /* last GMRES residual estimate |g_{j+1}| / ||f|| */
    int matvecs;          /* FP64 matvecs + FP32 matvecs applied (none for r0 when w0 = 0) */
    int applies;          /* preconditioner applications */
    int status;           /* rbf_status of this solve / problem */
    int stagnated;        /* 1: stopped because the true residual stopped decreasing */
} rbf_solve_info;

/* Create a context on CUDA device `device` (makes it current). */
rbf_status rbf_create(rbf_ctx** out, int device);
/* Release every buffer the context owns. NULL is a no-op. */
void rbf_destroy(rbf_ctx* ctx);

/* Cell-list binning (the matrix-free matvec's data structure, Sec. 2.3):
 * bounding box; cell (cx, cy) = floor((x - xmin) / c), clamped to the grid,
 * with ncx = floor((xmax - xmin) / c) + 1; stable sort of the points by cell
 * id cy*ncx + cx (ties keep the user order). Copies xy_dev (n x 2 FP64) into
 * the context in cell order. Synchronises `stream` once (grid size).
 * Invalidates any previous RASM setup. Errors: INVALID_ARG for n < 1 or
 * sigma, cutoff <= 0, or a grid over 2^28 cells. */
rbf_status rbf_bin(rbf_ctx* ctx, const double* xy_dev, int64_t n, const rbf_params* params, rbf_stream stream);

/* y = A~ w (Sec. 2.3 truncated Gaussian matvec, matrix-free), vectors of n
 * FP64 in user order. precision RBF_FP64 evaluates every pair in FP64;
 * RBF_FP32 evaluates in FP32 on cell-local coordinates (inner solves of the
 * mixed form) and returns the result widened to FP64. Needs rbf_bin. */
rbf_status rbf_matvec(rbf_ctx* ctx, const double* w_dev, double* y_dev, int precision, rbf_stream stream);

/* RASM setup (Sec. 2.2, Eq. rasm; Sec. 2.4): builds core and overlap index
 * lists of every box, forms A_i = R_i A~ R_i^T over each overlap list and
 * factors it (Cholesky); stores the core rows of A_i^{-1}. Synchronises
 * `stream`. Errors: SUBDOMAIN_TOO_LARGE if an overlap list exceeds
 * max_sub_points, NOT_SPD on a pivot <= 0, STATE without rbf_bin. */
rbf_status rbf_rasm_setup(rbf_ctx* ctx, const rbf_rasm_params* params, rbf_stream stream);

/* Subdomains whose inverse the last rbf_rasm_setup computed on the tensor
 * cores (RBF_FP32) and in FP64 (every other one: all of them for RBF_FP64 and
 * RBF_FP32_FROM_FP64), host outputs (either may be NULL). STATE before setup. */
rbf_status rbf_rasm_factor_counts(rbf_ctx* ctx, int64_t* tensor_core, int64_t* fp64);

/* z = M^{-1} r = sum_i ~R_i^T A_i^{-1} R_i r (Eq. rasm), n FP64 in user
 * order. Errors: STATE without rbf_rasm_setup. */
rbf_status rbf_rasm_apply(rbf_ctx* ctx, const double* r_dev, double* z_dev, rbf_stream stream);

/* Solve A~ w = f by right-preconditioned restarted GMRES with RASM (Sec. 2.2,
 * Sec. 3.1). w_dev holds the initial guess on entry (zeros for none) and the
 * solution on return, so a later call continues from it. An all-zero guess
 * is detected and its residual taken as f itself (no product; the same bits
 * as forming A 0). info (host,
 * optional) is filled. Synchronises `stream`. Returns NOT_CONVERGED (with the
 * best w) if rtol is not met within max_iters, or as soon as the true
 * residual stagnates: less than 10 % reduction over three consecutive restart
 * cycles (info.stagnated = 1). Needs rbf_rasm_setup. */
rbf_status rbf_solve(rbf_ctx* ctx, const double* f_dev, double* w_dev, const rbf_solve_params* params,
                     rbf_solve_info* info, rbf_stream stream);

/* End-to-end call on host buffers: copies xy_host (n x 2) and f_host to the
 * device, runs rbf_bin, rbf_rasm_setup and rbf_solve from w = 0, and copies w
 * back into w_host. Host buffers should be pinned for full copy speed. The
 * device copies of xy, f and w (32 B per point) stay with the context for the
 * next call, so repeated calls of the same size allocate nothing; they are
 * freed by rbf_destroy. */
rbf_status rbf_interpolate_host(rbf_ctx* ctx, const double* xy_host, const double* f_host, double* w_host,
                                int64_t n, const rbf_params* params, const rbf_rasm_params* rasm,
                                const rbf_solve_params* solve, rbf_solve_info* info, rbf_stream stream);

/* Evaluate the interpolant s(x) = sum_j w_j phi(|x - x_j|) (Eq. rbf2 with the
 * truncated kernel of Sec. 2.3: terms with |x - x_j|^2 > r_c^2 dropped, the
 * same FP64 pair test as the system matrix) at m points x: the paper's target
 * use, interpolation from the scattered centres onto other points such as a
 * lattice (Sec. 3.2). xe_dev: m x 2 interleaved (x, y), device, any order;
 * w_dev: n weights in user order (from rbf_solve); s_dev: m outputs (device,
 * caller-owned). At the centres themselves s equals rbf_matvec's y (bit for
 * bit with the stencil FP64 kernel, to rounding with the symmetric one, which
 * sums in another order). Points farther than r_c from every centre get 0. Needs rbf_bin (one
 * problem: STATE for a batch); INVALID_ARG for a non-finite point. The
 * points are binned into the centres' grid on each call (clamped to the edge
 * cells). */
rbf_status rbf_eval(rbf_ctx* ctx, const double* xe_dev, int64_t m, const double* w_dev, double* s_dev,
                    rbf_stream stream);

/* y = A~ w in FP64, like rbf_matvec(..., RBF_FP64, ...), without allocating.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library allocate device memory -- real-time loops that must
 * avoid the allocator's implicit synchronisation, or applications whose device
 * memory belongs to another framework's pool with a fixed budget. Its two
 * cell-order work vectors live in one file-scope __device__ array sized for
 * n <= 1,048,576 points (16 MiB, held by every GPU that loads the library
 * until the process exits); it calls no cudaMalloc, cudaFree or other
 * allocating routine and records no profiler events. Errors: INVALID_ARG if
 * the binned point count exceeds 1,048,576, STATE without rbf_bin or while a
 * batched solve runs on the context. The first call in each CUDA context (the
 * runtime's primary context of the device, for ordinary callers) looks up the
 * array's device address with that context current: make it before any stream
 * capture. All calls in one context share the array, so calls that overlap on
 * the GPU (different streams) race; the array keeps the last call's contents
 * (nothing relies on it being zero). */
rbf_status rbf_matvec_noalloc(rbf_ctx* ctx, const double* w_dev, double* y_dev, rbf_stream stream);

/* ---- batches of independent problems in one context ----
 * The problems are solved together: one launch of each kernel serves every
 * problem (all subdomains of all problems are batched, as Sec. 2.3 batches many
 * subdomains per process). Problem b owns the points [ptr[b], ptr[b+1]) of the
 * concatenated arrays (user order), has its own kernel width, cutoff, cell grid
 * and subdomain boxes, and gets its own GMRES (its own Krylov basis segment,
 * reductions, Hessenberg and stopping test). rbf_matvec and rbf_rasm_apply act
 * on all problems at once (block-diagonal operators). */

/* Bin nprob problems: xy_dev holds ptr_host[nprob] points; ptr_host (nprob+1
 * entries, ptr[0] = 0, strictly increasing) and params_host (nprob entries)
 * are host arrays. Errors as rbf_bin, plus INVALID_ARG for an empty problem. */
rbf_status rbf_bin_batch(rbf_ctx* ctx, const double* xy_dev, const int64_t* ptr_host, int64_t nprob,
                         const rbf_params* params_host, rbf_stream stream);
/* Subdomain boxes of every problem (params_host: nprob entries; precision of
 * the first entry applies to all). Errors as rbf_rasm_setup. */
rbf_status rbf_rasm_setup_batch(rbf_ctx* ctx, const rbf_rasm_params* params_host, rbf_stream stream);
/* Solve every problem of the batch (f_dev, w_dev: concatenated, user order; w
 * holds the initial guesses). info_host (nprob entries, optional) receives each
 * problem's iterations, final true relative residual and status. A problem
 * stops on its own when it meets rtol, reaches max_iters, or stagnates (as in
 * rbf_solve); the others go on. Returns NOT_CONVERGED if any problem misses
 * rtol. The Arnoldi cycle is replayed as a CUDA graph on an internal stream
 * that is ordered after `stream` on entry; the call returns when the solve is
 * complete. */
rbf_status rbf_solve_batch(rbf_ctx* ctx, const double* f_dev, double* w_dev, const rbf_solve_params* params,
                           rbf_solve_info* info_host, rbf_stream stream);

/* ---- autotuning of the cell size and the matvec tiles ----
 *
 * No counterpart in the paper. Bins the points with each candidate cell side
 * c in {r_c, r_c/2, r_c/3} (times base->cell_size / r_c when that is set, as a
 * base) and times the FP64 and FP32 matvecs with each tile (32, 64, 128
 * targets per block) on the device (CUDA events, the best of 3 launches
 * each); the score of a candidate is w_f64 * t_f64 + w_f32 * t_f32 (for a
 * plain FP64 solve w_f32 = 0; for the mixed form about 1 FP64 matvec per 26
 * FP32 ones). Writes the fastest setting to *best (a copy of *base with
 * cell_size, tile_f64 and tile_f32 set) and its score in ms to *score_ms
 * (optional), and leaves the context binned with it. Results of the matvec do
 * not depend on the tile; they depend on the cell size only through the
 * summation order (within the matvec tolerance). Errors as rbf_bin. */
rbf_status rbf_tune(rbf_ctx* ctx, const double* xy_dev, int64_t n, const rbf_params* base, double w_f64,
                    double w_f32, rbf_params* best, double* score_ms, rbf_stream stream);

/* ---- serving: independent requests admitted while others run ----
 *
 * No counterpart in the paper (its runs solve one problem per job); this is the
 * serving form of the same solve. A server owns `slots` contexts, each with its
 * own non-blocking stream and resident device buffers (points, lists, factors,
 * Krylov basis) that are reused from request to request. A submitted request
 * waits in a FIFO queue until a slot is free and its estimated device
 * footprint fits in the memory budget together with what the other slots hold;
 * a later, smaller request may go ahead of a head that does not fit (at most
 * `slots` times in a row). Admitted requests run concurrently, each on its own
 * stream: bin, RASM setup and GMRES solve, exactly as rbf_interpolate_host, so
 * a request's result does not depend on the others in flight. */
typedef struct rbf_server rbf_server;

typedef struct {
    int device;
    int slots;            /* requests in flight at once, 1..64 */
    int64_t mem_budget;   /* device bytes all slots may hold together; 0 = 90% of the free memory */
} rbf_server_params;

typedef struct {
    const double* xy;     /* host, n x 2 interleaved (x, y), user order; read until the request completes */
    const double* f;      /* host, n */
    double* w;            /* host, n; written when the request completes */
    int64_t n;
    rbf_params kernel;
    rbf_rasm_params rasm;
    rbf_solve_params solve;
} rbf_request;

typedef struct {
    rbf_solve_info info;
    int status;           /* rbf_status of the request (NOT_CONVERGED keeps the last iterate in w) */
    int slot;             /* slot that ran it */
    double t_submit;      /* seconds on the server's clock (rbf_server_clock) */
    double t_admit;
    double t_done;
    int64_t footprint;    /* estimated device bytes charged at admission */
} rbf_request_result;

typedef struct {
    int64_t submitted, completed, queued, running;
    int64_t resident_bytes;   /* device bytes the slots hold now */
    int64_t mem_budget;
    int64_t peak_resident_bytes;
    int64_t trims;            /* idle slots that released their buffers to admit a request */
    int64_t launches;         /* kernels launched by completed requests */
} rbf_server_stats;

/* Create a server (contexts are created lazily, on first use of a slot).
 * INVALID_ARG for slots outside 1..64 or a negative budget. */
rbf_status rbf_server_create(rbf_server** out, const rbf_server_params* params);
/* Finish the admitted requests, fail the queued ones (status STATE), free everything. */
void rbf_server_destroy(rbf_server* server);
/* Queue a request (host call, returns at once) and give its ticket. The caller
 * keeps req->xy, f and w alive until rbf_server_wait returns for it. OOM when
 * the request alone exceeds the budget; INVALID_ARG for null buffers or n < 1. */
rbf_status rbf_server_submit(rbf_server* server, const rbf_request* req, int64_t* ticket);
/* Wait up to timeout_s seconds (< 0: no limit) for a ticket; TIMEOUT if it has
 * not completed, INVALID_ARG for an unknown ticket. On success the result is
 * copied out and the ticket is forgotten. */
rbf_status rbf_server_wait(rbf_server* server, int64_t ticket, double timeout_s, rbf_request_result* result);
rbf_status rbf_server_get_stats(rbf_server* server, rbf_server_stats* stats);
/* Seconds since the server was created (steady clock). */
double rbf_server_clock(rbf_server* server);
/* Estimated device bytes of a request (host only, no GPU): staging, sorted
 * points, lists, RASM factors of the requested precision and the Krylov basis
 * (FP64, or FP32 for the mixed form); reads req->xy for the bounding box. */
int64_t rbf_request_footprint(const rbf_request* req);

/* ---- parity / inspection getters (synchronous; device outputs caller-owned) ---- */

/* Grid after rbf_bin: cells per axis and bounding box {xmin, ymin, xmax, ymax} (host). */
rbf_status rbf_get_grid(rbf_ctx* ctx, int64_t* ncx, int64_t* ncy, double* bbox_host);
/* perm_dev[p] = user index of the p-th point in cell order (n int32);
 * cell_start_dev[c] = first position of cell c (ncx*ncy + 1 int32). */
rbf_status rbf_get_bins(rbf_ctx* ctx, int32_t* perm_dev, int32_t* cell_start_dev, rbf_stream stream);
/* Subdomain counts after rbf_rasm_setup (host outputs). */
rbf_status rbf_get_subdomain_sizes(rbf_ctx* ctx, int64_t* nbx, int64_t* nby, int64_t* core_total,
                                   int64_t* overlap_total);
/* Core and overlap lists, CSR over subdomains s = by*nbx + bx (ptr arrays of
 * nsub + 1 int32), entries are user indices ascending within each list. */
rbf_status rbf_get_subdomains(rbf_ctx* ctx, int32_t* core_ptr_dev, int32_t* core_idx_dev, int32_t* ov_ptr_dev,
                              int32_t* ov_idx_dev, rbf_stream stream);
/* Total number of (i, j) pairs with r2 <= r_c^2 (i = j included), host output. */
rbf_status rbf_count_neighbors(rbf_ctx* ctx, int64_t* total, rbf_stream stream);
/* Candidate pairs the FP32 matvec evaluates (the unmasked work of the
 * cell-list method, Sec. 3.1): the sum over cells of (points in the cell) x
 * (points in its 3 x 3 stencil), host output. grid 0: the cells of side r_c
 * built by rbf_bin / rbf_bin_batch; grid 1: the inner grid of the mixed form
 * (cells of side inner_cutoff * sigma), which exists after a mixed solve with
 * inner_cutoff > 0 and until the next binning or subdomain setup
 * (RBF_ERR_STATE otherwise). Synchronises `stream`. */
rbf_status rbf_count_candidates(rbf_ctx* ctx, int grid, int64_t* total, rbf_stream stream);
/* Pairs (i, j), i = j included, within a grid's cutoff by the FP64 pair test
 * of Sec. 2.3, host output: grid 0 counts r2 <= r_c^2 (the truncated matrix's
 * nonzeros, as rbf_count_neighbors); grid 1 counts r2 <= (inner_cutoff
 * sigma)^2, the entries the mixed form's FP32 inner operator keeps (STATE
 * without an inner grid, as rbf_count_candidates). Synchronises `stream`. */
rbf_status rbf_count_pairs(rbf_ctx* ctx, int grid, int64_t* total, rbf_stream stream);
/* Neighbour lists, CSR over targets in user order (ptr: n + 1 int64; idx:
 * `capacity` int32), each row the user indices j with r2_ij <= r_c^2,
 * ascending. INVALID_ARG if capacity is below the total. */
rbf_status rbf_get_neighbors(rbf_ctx* ctx, int64_t* ptr_dev, int32_t* idx_dev, int64_t capacity,
                             rbf_stream stream);

/* ---- profiling and diagnostics ---- */

/* Kernel classes timed by the built-in profiler. */
enum {
    RBF_PROF_MATVEC_F64 = 0,   /* FP64 truncated matvec launches */
    RBF_PROF_MATVEC_F32 = 1,   /* FP32 truncated matvec launches */
    RBF_PROF_RASM_APPLY = 2,   /* subdomain GEMV apply launches */
    RBF_PROF_ORTHO = 3,        /* one Arnoldi orthogonalisation (three passes over V + reductions) */
    RBF_PROF_RASM_SETUP = 4,   /* subdomain factor/inverse launch */
    RBF_PROF_BIN = 5,          /* the whole binning sequence */
    RBF_PROF_STORE_F64 = 6,    /* counting and keeping the FP64 pair values (RBF_OPT_STORE_F64), with the
                                  product a mixed solve's first outer residual needs formed in the same pass */
    RBF_PROF_COUNT = 7
};
/* enable != 0: record a CUDA event pair on the launching stream around every
 * launch of the classes above (a fixed cost of two event records each). */
rbf_status rbf_profile_enable(rbf_ctx* ctx, int enable);
/* Classes recorded while profiling is enabled: bit k selects class k
 * (default: all). A class left out costs no event records. */
rbf_status rbf_profile_classes(rbf_ctx* ctx, unsigned mask);
/* Synchronises the recorded events and returns, for kernel class `kernel`,
 * the number of recorded launches and their summed device time; clears that
 * class's record. */
rbf_status rbf_profile_read(rbf_ctx* ctx, int kernel, int64_t* launches, double* total_ms);
/* Kernel values exp(-|x_i - x_j|^2 / (2 sigma^2)) of n point pairs, pairs_dev
 * holding (x_i, y_i, x_j, y_j) per pair (device, FP64), computed by the FP64
 * matvec's fixed-point evaluation with the constants of the binned problem
 * (problem 0 of a batch); 0 for pairs beyond the cutoff (Sec. 2.3 kernel,
 * without the normalisation factor). STATE before rbf_bin. */
rbf_status rbf_debug_kernel_pairs(rbf_ctx* ctx, const double* pairs_dev, double* out_dev, int64_t n,
                                  rbf_stream stream);
/* The FP32 operator of the mixed form's inner solves, y = A_i w, on the grid
 * of the inner cutoff (inner_cutoff sigma; built if needed, as the solver
 * builds it): every pair of the 3 x 3 cell stencil, FP32 on cell-local
 * offsets, no cutoff mask. w_dev, y_dev: n FP64 in user order (rounded to FP32
 * on the way in). variant 0: the symmetric kernel the solver uses (each
 * neighbouring cell pair once, column sums gathered in a fixed order; STATE
 * if a cell holds more than 128 points); variant 1: the stencil kernel (every
 * target against its 3 x 3 cells). For accuracy checks of the two against
 * each other and against the FP64 truncated matvec. */
rbf_status rbf_debug_inner_matvec(rbf_ctx* ctx, double inner_cutoff, const double* w_dev, double* y_dev, int variant,
                                  rbf_stream stream);
/* out[i] = exp(-t[i]) for n FP64 values on the device: variant 0 is the
 * library's table-driven exp with 64 entries (subdomain setup), variant 2 the
 * 2048-entry one of the FP64 matvec, variant 1 CUDA's exp(); for accuracy
 * checks of the library's against CUDA's. */
rbf_status rbf_debug_exp(rbf_ctx* ctx, const double* t_dev, double* out_dev, int64_t n, int variant,
                         rbf_stream stream);

/* ---- diagnostics ---- */
const char* rbf_status_string(rbf_status status);
const char* rbf_last_error(rbf_ctx* ctx);
/* Number of kernels this context has launched so far. */
uint64_t rbf_launch_count(rbf_ctx* ctx);
/* Device bytes the context currently holds. */
int64_t rbf_device_bytes(rbf_ctx* ctx);
/* Bytes of the FP64 pair values and accept masks kept for the current
 * binning (RBF_OPT_STORE_F64; every FP64 product reads them once), 0 when
 * none are kept: before the first solve after a binning, when they did not
 * fit, or with the option off. */
int64_t rbf_store_f64_bytes(rbf_ctx* ctx);
/* Context options (no counterpart in the paper). */
enum {
    /* The fused Arnoldi step of a batched mixed solve on the inner grid: each
     * step as one persistent cooperative launch (apply, matvec, Gram-Schmidt,
     * Arnoldi column and scaling for every running problem, with grid-wide
     * barriers between the phases; the results are bit for bit those of the
     * separate kernels). 0: never (separate kernels); 1: always; 2 (default):
     * once at most 64 problems are still active, where the separate kernels'
     * launches dominate the step, and for a single problem of at most 262,144
     * points. Not used while a kernel class of the cycle is being profiled. */
    RBF_OPT_FUSED_STEP = 1,
    /* 1 (default): the inner FP32 matvec of the mixed form visits each pair of
     * neighbouring cells once (cells of at most 128 points); 0: every target
     * against its 3 x 3 cells. */
    RBF_OPT_SYMMETRIC_F32 = 2,
    /* 1: the FP64 matvec visits each pair of neighbouring cells once, for
     * each problem with cells as wide as r_c holding at most 160 points (kernel
     * values shared by both directions, column sums gathered in a fixed
     * order); 0 (default): every target against its 3 x 3 cells. Both give the
     * truncated product to rounding. Takes effect at the next rbf_bin or
     * rbf_bin_batch (which allocates its 5 N doubles of slots); setting 0
     * after binning returns to the stencil kernel at once. The default is the
     * faster form on GB300: the FP64 pipe, which carries one FMA per directed
     * pair in both, bounds the symmetric form. */
    RBF_OPT_SYMMETRIC_F64 = 5,
    /* Polls of a device-side wait before it gives up -- a grid barrier of the
     * fused step, or the arrival of a bulk copy in a Gram-Schmidt pass: the
     * kernel then ends (once its copies in flight have landed), and the solve
     * returns RBF_ERR_TIMEOUT (value >= 1; default 2^23, about a second). */
    RBF_OPT_BARRIER_SPIN_LIMIT = 3,
    /* Check of the timeout path: 1 makes every barrier of the fused step wait
     * for one block more than the grid has, so that every wait runs out. */
    RBF_OPT_BARRIER_EXTRA_BLOCK = 4,
    /* 1 (default): the FP32 Gram-Schmidt passes of the mixed form stream the
     * basis vectors through shared memory by bulk asynchronous copies (several
     * vectors in flight per chunk); 0: each thread loads them into registers.
     * The results are the same bits. */
    RBF_OPT_STREAM_GS = 6,
    /* Check of the timeout path: 1 makes every bulk-copy wait of those passes
     * wait on a barrier that no copy completes (and copy nothing), so that it
     * runs out and the solve returns RBF_ERR_TIMEOUT. */
    RBF_OPT_STREAM_WAIT_CHECK = 7,
    /* 1 (default): the FP64 matvec's accept masks and kernel values of the
     * current binning are computed once (at the start of an FP64 solve; with
     * the first outer residual product of a mixed solve, which that pass forms
     * as well) and kept in device memory (about 8.9 B per in-cutoff pair: 8 B values in slots
     * padded to the walk's warp steps, and the masks; 363 pairs per point at
     * h/sigma = 0.8), if they fit in the device's free memory less 8 GiB and in
     * the context's memory limit; the FP64 products then read them instead of
     * evaluating the kernel, with the same sums bit for bit. Recomputed in
     * the first solve after each binning; freed by rbf_destroy or by setting
     * 0. Not used by the symmetric FP64 kernel (RBF_OPT_SYMMETRIC_F64), by a
     * batched solve once some of its problems have stopped (their products
     * run on lists of the active problems' items), or by a solve under
     * stream capture; an allocation that fails leaves the solve matrix-free.
     * Values that did not fit are not tried again for the same binning until
     * this option or the memory limit is set again. 0: never (matrix-free). */
    RBF_OPT_STORE_F64 = 8
};
/* Set a context option. INVALID_ARG for an unknown option or value. */
rbf_status rbf_set_option(rbf_ctx* ctx, int option, int64_t value);

/* Cap on the device bytes the context may hold (0 = no cap, the default): an
 * allocation that would take rbf_device_bytes() above it fails with
 * RBF_ERR_OOM before cudaMalloc is called, as a real shortage would. For a
 * host that shares the GPU under a fixed budget, and for tests that drive
 * the library into its out-of-memory paths without exhausting the device.
 * INVALID_ARG for a negative value. */
rbf_status rbf_set_memory_limit(rbf_ctx* ctx, int64_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* RBF_H */
