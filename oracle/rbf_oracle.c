/*
 * rbf_oracle.c -- plain, slow, FP64 CPU oracle for the Gaussian RBF
 * interpolation solve (GMRES preconditioned by the restricted additive
 * Schwarz method over small overlapping subdomains).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg use it. It shares no code with the CUDA library.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 * -ffp-contract=off matters: every product below rounds separately, so the
 * pair test, the cell index and the box tests give the same bits as any
 * other IEEE implementation that evaluates the same expression in the same
 * order without fused multiply-adds.
 *
 * What follows the paper, and where:
 *   kernel        Sec. 2.3, the normalised 2-D Gaussian
 *                 A_ij = exp(-|x_i-x_j|^2 / (2 sigma^2)) / (2 pi sigma^2);
 *                 the factor is optional (flag), the bare exponential is the
 *                 default, Table 1's Gaussian with eps^2 = 1/(2 sigma^2).
 *   truncation    Sec. 2.3 / Sec. 3.1: entries of far pairs are dropped. The
 *                 cut is radial: the pair (i, j) is kept iff
 *                 r2 = dx*dx + dy*dy <= rc*rc (dx = x_i - x_j, dy = y_i - y_j).
 *   subdomains    Sec. 2.2 (Eq. rasm): overlapping boxes Omega_i and the
 *                 non-overlapping cores ~Omega_i; Sec. 2.3: the restriction
 *                 uses a separate index list for the core.
 *   A_i           Sec. 2.2: A_i = R_i A R_i^T (the truncated A restricted to
 *                 the overlap list), solved directly (Sec. 3.1 uses a dense
 *                 direct solve; A_i is SPD, so Cholesky).
 *   RASM          Eq. rasm: z = sum_i ~R_i^T A_i^{-1} R_i r.
 *   ASM           Eq. asm (for the comparison of Sec. 2.2): the same solves
 *                 with every overlap entry added back, z = sum_i R_i^T A_i^{-1} R_i r.
 *   evaluation    Eq. rbf2 at points other than the centres (the use of
 *                 Sec. 3.2: interpolation onto a lattice), same truncation.
 *   GMRES         Sec. 2.2 / Sec. 3.1: GMRES with the RASM preconditioner,
 *                 restarted, relative tolerance 1e-13. Right preconditioning,
 *                 classical Gram-Schmidt applied twice, Givens rotations.
 *   dense solve   Eq. rbf2 with the Gaussian (no polynomial block): the full,
 *                 untruncated A solved by Cholesky, for small N only.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_NOT_SPD 4
#define ORC_ERR_TOO_LARGE 5
#define ORC_ERR_NOT_CONVERGED 6

typedef struct {
    double sigma;      /* Gaussian width */
    double rc;         /* cutoff radius */
    int normalized;    /* 1: multiply by 1/(2 pi sigma^2) */
} orc_kernel_params;

/* ------------------------------------------------------------------ kernel */

/* k(r2): the Gaussian of Sec. 2.3 as a function of the squared distance. */
double orc_kernel(double r2, const orc_kernel_params* p)
{
    double two_s2 = 2.0 * p->sigma * p->sigma;
    double v = exp(-(r2 / two_s2));
    if (p->normalized) v = v / (M_PI * two_s2);
    return v;
}

/* Squared distance, rounded term by term (no FMA): dx*dx, dy*dy, then the sum. */
static double pair_r2(const double* xy, int64_t i, int64_t j)
{
    double dx = xy[2 * i] - xy[2 * j];
    double dy = xy[2 * i + 1] - xy[2 * j + 1];
    double a = dx * dx;
    double b = dy * dy;
    return a + b;
}

double orc_pair_r2(const double* xy, int64_t i, int64_t j) { return pair_r2(xy, i, j); }

/* ----------------------------------------------------------------- binning */

typedef struct {
    double xmin, ymin, xmax, ymax;
    double c;          /* cell side */
    int64_t ncx, ncy;  /* cells per axis */
} orc_grid;

/* Bounding box and cell counts: ncx = floor((xmax - xmin) / c) + 1. */
int orc_grid_dims(const double* xy, int64_t n, double c, orc_grid* g)
{
    if (n < 1 || !(c > 0.0)) return ORC_ERR_ARG;
    double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1];
    for (int64_t i = 1; i < n; ++i) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        if (x < xmin) xmin = x;
        if (x > xmax) xmax = x;
        if (y < ymin) ymin = y;
        if (y > ymax) ymax = y;
    }
    g->xmin = xmin; g->xmax = xmax; g->ymin = ymin; g->ymax = ymax; g->c = c;
    double fx = floor((xmax - xmin) / c), fy = floor((ymax - ymin) / c);
    if (!(fx < 1.0e9) || !(fy < 1.0e9)) return ORC_ERR_TOO_LARGE;
    g->ncx = (int64_t)fx + 1;
    g->ncy = (int64_t)fy + 1;
    if (g->ncx * g->ncy > ((int64_t)1 << 28)) return ORC_ERR_TOO_LARGE;
    return ORC_OK;
}

static int64_t clamp64(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Cell coordinate along one axis: floor((x - lo) / c), clamped to [0, nc-1]. */
static int64_t cell_axis(double x, double lo, double c, int64_t nc)
{
    double q = floor((x - lo) / c);
    int64_t k = (q < 0.0) ? -1 : (q > (double)nc ? nc : (int64_t)q);
    return clamp64(k, 0, nc - 1);
}

int64_t orc_cell_of(const double* xy, int64_t i, const orc_grid* g)
{
    int64_t cx = cell_axis(xy[2 * i], g->xmin, g->c, g->ncx);
    int64_t cy = cell_axis(xy[2 * i + 1], g->ymin, g->c, g->ncy);
    return cy * g->ncx + cx;
}

/* Stable counting sort of the points by cell id (ties keep the original
 * order). perm[p] = original index of the p-th point in cell order;
 * cell_start[c] .. cell_start[c+1] is the range of cell c (size ncx*ncy + 1). */
int orc_bin(const double* xy, int64_t n, const orc_grid* g, int32_t* perm, int32_t* cell_start)
{
    int64_t ncell = g->ncx * g->ncy;
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* next = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    if (!cell || !next) { free(cell); free(next); return ORC_ERR_OOM; }
    for (int64_t i = 0; i < n; ++i) {
        cell[i] = orc_cell_of(xy, i, g);
        next[cell[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c) next[c + 1] += next[c];
    for (int64_t c = 0; c <= ncell; ++c) cell_start[c] = (int32_t)next[c];
    for (int64_t i = 0; i < n; ++i) perm[next[cell[i]]++] = (int32_t)i;
    free(cell);
    free(next);
    return ORC_OK;
}

/* Stencil half-width in cells: every pair within rc lies in cells whose
 * coordinates differ by at most ceil(rc / c) per axis. */
int64_t orc_stencil(double rc, double c) { return (int64_t)ceil(rc / c); }

/* --------------------------------------------------- neighbours and matvec */

typedef struct {
    const double* xy;
    int64_t n;
    orc_grid g;
    const int32_t* perm;
    const int32_t* cell_start;
    int64_t k;       /* stencil half-width */
    double rc2;      /* rc * rc */
} orc_cells;

static void cells_init(orc_cells* s, const double* xy, int64_t n, const orc_grid* g,
                       const int32_t* perm, const int32_t* cell_start, double rc)
{
    s->xy = xy; s->n = n; s->g = *g; s->perm = perm; s->cell_start = cell_start;
    s->k = orc_stencil(rc, g->c);
    s->rc2 = rc * rc;
}

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Visit all j with r2(i, j) <= rc2 by scanning the cells around i. */
#define FOR_NEIGHBOURS(S, I, J, R2, BODY)                                            \
    do {                                                                             \
        const orc_cells* s_ = (S);                                                   \
        int64_t ci_ = orc_cell_of(s_->xy, (I), &s_->g);                              \
        int64_t cx_ = ci_ % s_->g.ncx, cy_ = ci_ / s_->g.ncx;                        \
        int64_t y0_ = clamp64(cy_ - s_->k, 0, s_->g.ncy - 1);                        \
        int64_t y1_ = clamp64(cy_ + s_->k, 0, s_->g.ncy - 1);                        \
        int64_t x0_ = clamp64(cx_ - s_->k, 0, s_->g.ncx - 1);                        \
        int64_t x1_ = clamp64(cx_ + s_->k, 0, s_->g.ncx - 1);                        \
        for (int64_t yy_ = y0_; yy_ <= y1_; ++yy_)                                   \
            for (int64_t xx_ = x0_; xx_ <= x1_; ++xx_) {                             \
                int64_t c_ = yy_ * s_->g.ncx + xx_;                                  \
                for (int64_t p_ = s_->cell_start[c_]; p_ < s_->cell_start[c_ + 1]; ++p_) { \
                    int64_t J = s_->perm[p_];                                        \
                    double R2 = pair_r2(s_->xy, (I), J);                             \
                    if (R2 <= s_->rc2) { BODY }                                      \
                }                                                                    \
            }                                                                        \
    } while (0)

/* Neighbour counts per target (original order). */
int orc_neighbor_counts(const double* xy, int64_t n, const orc_grid* g, const int32_t* perm,
                        const int32_t* cell_start, double rc, int64_t* counts)
{
    orc_cells s;
    cells_init(&s, xy, n, g, perm, cell_start, rc);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t cnt = 0;
        FOR_NEIGHBOURS(&s, i, j, r2, { (void)j; (void)r2; ++cnt; });
        counts[i] = cnt;
    }
    return ORC_OK;
}

/* Neighbour lists: CSR over targets in original order, each row ascending
 * by original source index (the target itself included, r2 = 0). */
int orc_neighbors(const double* xy, int64_t n, const orc_grid* g, const int32_t* perm,
                  const int32_t* cell_start, double rc, const int64_t* ptr, int32_t* idx)
{
    orc_cells s;
    cells_init(&s, xy, n, g, perm, cell_start, rc);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t w = ptr[i];
        FOR_NEIGHBOURS(&s, i, j, r2, { (void)r2; idx[w++] = (int32_t)j; });
        qsort(idx + ptr[i], (size_t)(ptr[i + 1] - ptr[i]), sizeof(int32_t), cmp_i32);
    }
    return ORC_OK;
}

/* Truncated matvec y = A~ w over the cell lists (Sec. 2.3): y_i = sum of
 * k(r2_ij) w_j over the j with r2_ij <= rc^2. Vectors in original order. */
int orc_matvec_cutoff(const double* xy, int64_t n, const orc_grid* g, const int32_t* perm,
                      const int32_t* cell_start, const orc_kernel_params* kp,
                      const double* w, double* y)
{
    orc_cells s;
    cells_init(&s, xy, n, g, perm, cell_start, kp->rc);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        FOR_NEIGHBOURS(&s, i, j, r2, { acc += orc_kernel(r2, kp) * w[j]; });
        y[i] = acc;
    }
    return ORC_OK;
}

/* Dense matvec with every pair (no truncation), O(N^2). */
int orc_matvec_dense(const double* xy, int64_t n, const orc_kernel_params* kp,
                     const double* w, double* y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) acc += orc_kernel(pair_r2(xy, i, j), kp) * w[j];
        y[i] = acc;
    }
    return ORC_OK;
}

/* Interpolant at other points (Eq. rbf2 evaluated off the centres, with the
 * truncation of Sec. 2.3): s_i = sum over all centres j, in index order, of
 * k(r2) w_j where r2 = |xe_i - x_j|^2 <= rc^2 (same rounding as pair_r2). */
int orc_eval(const double* xy, int64_t n, const orc_kernel_params* kp, const double* w,
             const double* xe, int64_t m, double* s)
{
    double rc2 = kp->rc * kp->rc;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double dx = xe[2 * i] - xy[2 * j];
            double dy = xe[2 * i + 1] - xy[2 * j + 1];
            double r2 = dx * dx + dy * dy;
            if (r2 <= rc2) acc += orc_kernel(r2, kp) * w[j];
        }
        s[i] = acc;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------- Cholesky */

/* Textbook Cholesky A = L L^T of an n x n row-major SPD matrix (row by row:
 * L_jj = sqrt(A_jj - sum_k L_jk^2), L_ij = (A_ij - sum_k L_ik L_jk) / L_jj).
 * L overwrites the lower triangle; returns ORC_ERR_NOT_SPD on a pivot <= 0. */
int orc_cholesky(double* a, int64_t n)
{
    for (int64_t j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int64_t k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
        if (!(d > 0.0)) return ORC_ERR_NOT_SPD;
        double ljj = sqrt(d);
        a[j * n + j] = ljj;
#pragma omp parallel for schedule(static) if (n > 512)
        for (int64_t i = j + 1; i < n; ++i) {
            double v = a[i * n + j];
            for (int64_t k = 0; k < j; ++k) v -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = v / ljj;
        }
    }
    return ORC_OK;
}

/* Solve L L^T x = b in place (b -> x), L in the lower triangle of row-major a. */
void orc_cholesky_solve(const double* a, int64_t n, double* b)
{
    for (int64_t i = 0; i < n; ++i) {            /* L y = b */
        double v = b[i];
        for (int64_t k = 0; k < i; ++k) v -= a[i * n + k] * b[k];
        b[i] = v / a[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {       /* L^T x = y */
        double v = b[i];
        for (int64_t k = i + 1; k < n; ++k) v -= a[k * n + i] * b[k];
        b[i] = v / a[i * n + i];
    }
}

/* Dense direct solve of the untruncated system A w = f (small N only). */
int orc_dense_solve(const double* xy, int64_t n, const orc_kernel_params* kp,
                    const double* f, double* w)
{
    double* a = (double*)malloc(sizeof(double) * (size_t)(n * n));
    if (!a) return ORC_ERR_OOM;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) a[i * n + j] = orc_kernel(pair_r2(xy, i, j), kp);
    int st = orc_cholesky(a, n);
    if (st == ORC_OK) {
        memcpy(w, f, sizeof(double) * (size_t)n);
        orc_cholesky_solve(a, n, w);
    }
    free(a);
    return st;
}

/* ------------------------------------------------------------- subdomains */

typedef struct {
    double x0, y0;     /* box origin */
    double B;          /* core box side */
    double delta;      /* overlap ring width */
    int64_t nbx, nby;  /* boxes per axis */
} orc_boxes;

/* nbx = floor((xmax - x0) / B) + 1 (at least 1). */
int orc_box_dims(const orc_grid* g, double x0, double y0, double B, double delta, orc_boxes* b)
{
    if (!(B > 0.0) || !(delta >= 0.0)) return ORC_ERR_ARG;
    b->x0 = x0; b->y0 = y0; b->B = B; b->delta = delta;
    double fx = floor((g->xmax - x0) / B), fy = floor((g->ymax - y0) / B);
    if (!(fx < 1.0e9) || !(fy < 1.0e9)) return ORC_ERR_TOO_LARGE;
    b->nbx = fx < 0.0 ? 1 : (int64_t)fx + 1;
    b->nby = fy < 0.0 ? 1 : (int64_t)fy + 1;
    if (b->nbx * b->nby > ((int64_t)1 << 30)) return ORC_ERR_TOO_LARGE;
    return ORC_OK;
}

/* Is coordinate v inside the overlap interval of box k, given its core box kc?
 * Box k spans [o + k*B, o + (k+1)*B); its overlap adds delta on both sides,
 * half-open. A point always belongs to the overlap of its own core box. */
static int in_overlap(double v, int64_t k, int64_t kc, double o, double B, double delta)
{
    if (k == kc) return 1;
    if (k < kc) return v < (o + (double)(k + 1) * B) + delta;
    return v >= (o + (double)k * B) - delta;
}

static int64_t box_reach(const orc_boxes* b) { return (int64_t)ceil(b->delta / b->B) + 1; }

/* Core and overlap index lists (CSR over subdomains s = by * nbx + bx, each
 * list ascending by original point index). Pass ptr arrays of size nsub + 1;
 * if idx arrays are NULL only the counts/pointers are produced. */
int orc_subdomains(const double* xy, int64_t n, const orc_boxes* b,
                   int64_t* core_ptr, int32_t* core_idx, int64_t* ov_ptr, int32_t* ov_idx)
{
    int64_t nsub = b->nbx * b->nby;
    int64_t K = box_reach(b);
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1 && (!core_idx || !ov_idx)) break;
        int64_t* cfill = NULL;
        int64_t* ofill = NULL;
        if (pass == 0) {
            memset(core_ptr, 0, sizeof(int64_t) * (size_t)(nsub + 1));
            memset(ov_ptr, 0, sizeof(int64_t) * (size_t)(nsub + 1));
        } else {
            cfill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nsub);
            ofill = (int64_t*)malloc(sizeof(int64_t) * (size_t)nsub);
            if (!cfill || !ofill) { free(cfill); free(ofill); return ORC_ERR_OOM; }
            memcpy(cfill, core_ptr, sizeof(int64_t) * (size_t)nsub);
            memcpy(ofill, ov_ptr, sizeof(int64_t) * (size_t)nsub);
        }
        for (int64_t i = 0; i < n; ++i) {
            double x = xy[2 * i], y = xy[2 * i + 1];
            int64_t bx = cell_axis(x, b->x0, b->B, b->nbx);
            int64_t by = cell_axis(y, b->y0, b->B, b->nby);
            int64_t sc = by * b->nbx + bx;
            if (pass == 0) core_ptr[sc + 1] += 1; else core_idx[cfill[sc]++] = (int32_t)i;
            for (int64_t ky = clamp64(by - K, 0, b->nby - 1); ky <= clamp64(by + K, 0, b->nby - 1); ++ky) {
                if (!in_overlap(y, ky, by, b->y0, b->B, b->delta)) continue;
                for (int64_t kx = clamp64(bx - K, 0, b->nbx - 1); kx <= clamp64(bx + K, 0, b->nbx - 1); ++kx) {
                    if (!in_overlap(x, kx, bx, b->x0, b->B, b->delta)) continue;
                    int64_t s = ky * b->nbx + kx;
                    if (pass == 0) ov_ptr[s + 1] += 1; else ov_idx[ofill[s]++] = (int32_t)i;
                }
            }
        }
        if (pass == 0) {
            for (int64_t s = 0; s < nsub; ++s) {
                core_ptr[s + 1] += core_ptr[s];
                ov_ptr[s + 1] += ov_ptr[s];
            }
        }
        free(cfill);
        free(ofill);
    }
    return ORC_OK;
}

/* --------------------------------------------------------------------- RASM */

typedef struct {
    int64_t n, nsub;
    const double* xy;
    orc_kernel_params kp;
    const int64_t* core_ptr; const int32_t* core_idx;
    const int64_t* ov_ptr;   const int32_t* ov_idx;
    int64_t* fac_ptr;        /* offsets of each n_i x n_i factor */
    double* fac;             /* Cholesky factors (lower triangles, row-major) */
    int32_t* core_of;        /* subdomain whose core holds each point */
    int additive;            /* 1: plain additive Schwarz, Eq. asm (no restriction) */
} orc_rasm;

/* Form A_i = R_i A~ R_i^T over each overlap list and factor it (Sec. 2.2). */
int orc_rasm_setup(orc_rasm* r, int64_t max_sub_points)
{
    double rc2 = r->kp.rc * r->kp.rc;
    r->fac_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(r->nsub + 1));
    r->core_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)r->n);
    if (!r->fac_ptr || !r->core_of) return ORC_ERR_OOM;
    r->fac_ptr[0] = 0;
    for (int64_t s = 0; s < r->nsub; ++s) {
        int64_t m = r->ov_ptr[s + 1] - r->ov_ptr[s];
        if (m > max_sub_points) return ORC_ERR_TOO_LARGE;
        r->fac_ptr[s + 1] = r->fac_ptr[s] + m * m;
        for (int64_t q = r->core_ptr[s]; q < r->core_ptr[s + 1]; ++q) r->core_of[r->core_idx[q]] = (int32_t)s;
    }
    r->fac = (double*)malloc(sizeof(double) * (size_t)(r->fac_ptr[r->nsub] > 0 ? r->fac_ptr[r->nsub] : 1));
    if (!r->fac) return ORC_ERR_OOM;
    int status = ORC_OK;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = 0; s < r->nsub; ++s) {
        const int32_t* ov = r->ov_idx + r->ov_ptr[s];
        int64_t m = r->ov_ptr[s + 1] - r->ov_ptr[s];
        double* a = r->fac + r->fac_ptr[s];
        for (int64_t p = 0; p < m; ++p)
            for (int64_t q = 0; q < m; ++q) {
                double r2 = pair_r2(r->xy, ov[p], ov[q]);
                a[p * m + q] = (r2 <= rc2) ? orc_kernel(r2, &r->kp) : 0.0;
            }
        if (orc_cholesky(a, m) != ORC_OK) {
#pragma omp critical
            status = ORC_ERR_NOT_SPD;
        }
    }
    return status;
}

/* Additive Schwarz, Eq. asm: z = sum_i R_i^T A_i^{-1} R_i v, every overlap
 * entry of every subdomain added back. The subdomain solves run in parallel
 * into a scratch copy of the overlap lists; the sums are then taken serially
 * in subdomain order (deterministic). */
static void asm_apply(const orc_rasm* r, const double* v, double* z)
{
    memset(z, 0, sizeof(double) * (size_t)r->n);
    int64_t tot = r->ov_ptr[r->nsub];
    double* u = (double*)malloc(sizeof(double) * (size_t)(tot > 0 ? tot : 1));
    if (!u) return;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = 0; s < r->nsub; ++s) {
        const int32_t* ov = r->ov_idx + r->ov_ptr[s];
        int64_t m = r->ov_ptr[s + 1] - r->ov_ptr[s];
        double* buf = u + r->ov_ptr[s];
        for (int64_t p = 0; p < m; ++p) buf[p] = v[ov[p]];
        orc_cholesky_solve(r->fac + r->fac_ptr[s], m, buf);
    }
    for (int64_t e = 0; e < tot; ++e) z[r->ov_idx[e]] += u[e];
    free(u);
}

/* z = sum_i ~R_i^T A_i^{-1} R_i v (Eq. rasm): restrict v to the overlap list,
 * solve with the factor, keep only the entries whose point is in the core
 * of the same subdomain. Vectors in original order. */
void orc_rasm_apply(const orc_rasm* r, const double* v, double* z)
{
    if (r->additive) {
        asm_apply(r, v, z);
        return;
    }
    memset(z, 0, sizeof(double) * (size_t)r->n);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t s = 0; s < r->nsub; ++s) {
        const int32_t* ov = r->ov_idx + r->ov_ptr[s];
        int64_t m = r->ov_ptr[s + 1] - r->ov_ptr[s];
        double b[1024];
        double* buf = m <= 1024 ? b : (double*)malloc(sizeof(double) * (size_t)m);
        for (int64_t p = 0; p < m; ++p) buf[p] = v[ov[p]];
        orc_cholesky_solve(r->fac + r->fac_ptr[s], m, buf);
        for (int64_t p = 0; p < m; ++p)
            if (r->core_of[ov[p]] == s) z[ov[p]] += buf[p];
        if (buf != b) free(buf);
    }
}

void orc_rasm_free(orc_rasm* r)
{
    free(r->fac_ptr); free(r->fac); free(r->core_of);
    r->fac_ptr = NULL; r->fac = NULL; r->core_of = NULL;
}

/* ------------------------------------------------------------------- GMRES */

typedef void (*orc_op)(void* ctx, const double* in, double* out);

static double dot(const double* a, const double* b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

typedef struct {
    int64_t iters;        /* Arnoldi steps taken */
    int64_t restarts;     /* completed cycles */
    double relres;        /* final true ||f - A w|| / ||f|| */
    int status;
} orc_gmres_info;

/* Restarted GMRES(m) with right preconditioning: solve A M^{-1} u = f,
 * w = w0 + M^{-1} V y. Each cycle: r = f - A w, V_0 = r / |r|; per step
 * v = A M^{-1} V_j, two classical Gram-Schmidt passes against V_0..V_j,
 * H_{j+1,j} = |v|; Givens rotations keep H upper triangular and |g_{j+1}|
 * equals the residual norm of the cycle. The cycle ends when
 * |g_{j+1}| <= rtol |f| or after m steps; w is updated and the true
 * residual is recomputed. Stops when the true relative residual <= rtol.
 * hist (optional, max_iters entries) receives |g_{j+1}| / |f| per step. */
int orc_gmres(int64_t n, orc_op amul, void* actx, orc_op minv, void* mctx,
              const double* f, double* w, int64_t m, double rtol, int64_t max_iters,
              double* hist, orc_gmres_info* info)
{
    double* V = (double*)malloc(sizeof(double) * (size_t)(n * (m + 1)));
    double* H = (double*)calloc((size_t)((m + 1) * m), sizeof(double));
    double* cs = (double*)malloc(sizeof(double) * (size_t)m);
    double* sn = (double*)malloc(sizeof(double) * (size_t)m);
    double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)m);
    double* t = (double*)malloc(sizeof(double) * (size_t)n);
    double* u = (double*)malloc(sizeof(double) * (size_t)n);
    double* hc = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    if (!V || !H || !cs || !sn || !g || !y || !t || !u || !hc) return ORC_ERR_OOM;

    double fnorm = sqrt(dot(f, f, n));
    int64_t it = 0, cycles = 0;
    int status = ORC_ERR_NOT_CONVERGED;
    double relres = 0.0;
    if (fnorm == 0.0) {
        memset(w, 0, sizeof(double) * (size_t)n);
        status = ORC_OK;
        goto done;
    }
    for (;;) {
        /* true residual r = f - A w */
        amul(actx, w, t);
        for (int64_t i = 0; i < n; ++i) V[i] = f[i] - t[i];
        double beta = sqrt(dot(V, V, n));
        relres = beta / fnorm;
        if (relres <= rtol) { status = ORC_OK; break; }
        if (it >= max_iters) break;
        for (int64_t i = 0; i < n; ++i) V[i] /= beta;
        memset(g, 0, sizeof(double) * (size_t)(m + 1));
        g[0] = beta;
        int64_t k = 0;   /* steps in this cycle */
        for (int64_t j = 0; j < m && it < max_iters; ++j) {
            double* vj = V + j * n;
            double* vn = V + (j + 1) * n;
            minv(mctx, vj, u);
            amul(actx, u, vn);
            for (int64_t q = 0; q <= j; ++q) H[q * m + j] = 0.0;
            for (int pass = 0; pass < 2; ++pass) {
                for (int64_t q = 0; q <= j; ++q) hc[q] = dot(V + q * n, vn, n);
                for (int64_t q = 0; q <= j; ++q) {
                    const double* vq = V + q * n;
                    for (int64_t i = 0; i < n; ++i) vn[i] -= hc[q] * vq[i];
                    H[q * m + j] += hc[q];
                }
            }
            double hn = sqrt(dot(vn, vn, n));
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int64_t i = 0; i < n; ++i) vn[i] /= hn;
            /* previous rotations on column j */
            for (int64_t q = 0; q < j; ++q) {
                double a = H[q * m + j], b = H[(q + 1) * m + j];
                H[q * m + j] = cs[q] * a + sn[q] * b;
                H[(q + 1) * m + j] = -sn[q] * a + cs[q] * b;
            }
            /* new rotation zeroing H[j+1][j] */
            double a = H[j * m + j], b = H[(j + 1) * m + j];
            double c, s;
            if (b == 0.0) { c = 1.0; s = 0.0; }
            else if (fabs(b) > fabs(a)) { double tau = a / b; s = 1.0 / sqrt(1.0 + tau * tau); c = s * tau; }
            else { double tau = b / a; c = 1.0 / sqrt(1.0 + tau * tau); s = c * tau; }
            cs[j] = c; sn[j] = s;
            H[j * m + j] = c * a + s * b;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -s * g[j];
            g[j] = c * g[j];
            ++it;
            k = j + 1;
            if (hist) hist[it - 1] = fabs(g[j + 1]) / fnorm;
            if (fabs(g[j + 1]) <= rtol * fnorm || hn == 0.0) break;
        }
        /* y = H^{-1} g (upper triangular, k x k) */
        for (int64_t q = k - 1; q >= 0; --q) {
            double v = g[q];
            for (int64_t p = q + 1; p < k; ++p) v -= H[q * m + p] * y[p];
            y[q] = v / H[q * m + q];
        }
        /* w += M^{-1} (V y) */
        memset(t, 0, sizeof(double) * (size_t)n);
        for (int64_t q = 0; q < k; ++q) {
            const double* vq = V + q * n;
            for (int64_t i = 0; i < n; ++i) t[i] += y[q] * vq[i];
        }
        minv(mctx, t, u);
        for (int64_t i = 0; i < n; ++i) w[i] += u[i];
        ++cycles;
    }
done:
    info->iters = it;
    info->restarts = cycles;
    info->relres = relres;
    info->status = status;
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(t); free(u); free(hc);
    return status;
}

/* ------------------------------------------------- end-to-end cutoff solve */

typedef struct {
    const double* xy;
    int64_t n;
    orc_grid g;
    int32_t* perm;
    int32_t* cell_start;
    orc_kernel_params kp;
    orc_rasm rasm;
    int64_t* core_ptr; int32_t* core_idx;
    int64_t* ov_ptr;   int32_t* ov_idx;
    orc_boxes boxes;
    int64_t matvecs, applies;
} orc_problem;

static void op_amul(void* ctx, const double* in, double* out)
{
    orc_problem* p = (orc_problem*)ctx;
    orc_matvec_cutoff(p->xy, p->n, &p->g, p->perm, p->cell_start, &p->kp, in, out);
    p->matvecs++;
}

static void op_minv(void* ctx, const double* in, double* out)
{
    orc_problem* p = (orc_problem*)ctx;
    orc_rasm_apply(&p->rasm, in, out);
    p->applies++;
}

static void op_identity(void* ctx, const double* in, double* out)
{
    orc_problem* p = (orc_problem*)ctx;
    memcpy(out, in, sizeof(double) * (size_t)p->n);
}

/* Set up binning, subdomains and factors for one problem. */
int orc_problem_create(orc_problem** out, const double* xy, int64_t n, double sigma, double rc,
                       int normalized, double cell_size, double x0, double y0, double B,
                       double delta, int64_t max_sub_points)
{
    orc_problem* p = (orc_problem*)calloc(1, sizeof(orc_problem));
    if (!p) return ORC_ERR_OOM;
    *out = p;
    p->xy = xy; p->n = n;
    p->kp.sigma = sigma; p->kp.rc = rc; p->kp.normalized = normalized;
    int st = orc_grid_dims(xy, n, cell_size > 0.0 ? cell_size : rc, &p->g);
    if (st) return st;
    int64_t ncell = p->g.ncx * p->g.ncy;
    p->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    p->cell_start = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    if (!p->perm || !p->cell_start) return ORC_ERR_OOM;
    st = orc_bin(xy, n, &p->g, p->perm, p->cell_start);
    if (st) return st;
    st = orc_box_dims(&p->g, x0, y0, B, delta, &p->boxes);
    if (st) return st;
    int64_t nsub = p->boxes.nbx * p->boxes.nby;
    p->core_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nsub + 1));
    p->ov_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nsub + 1));
    if (!p->core_ptr || !p->ov_ptr) return ORC_ERR_OOM;
    orc_subdomains(xy, n, &p->boxes, p->core_ptr, NULL, p->ov_ptr, NULL);
    p->core_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(p->core_ptr[nsub] + 1));
    p->ov_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(p->ov_ptr[nsub] + 1));
    if (!p->core_idx || !p->ov_idx) return ORC_ERR_OOM;
    orc_subdomains(xy, n, &p->boxes, p->core_ptr, p->core_idx, p->ov_ptr, p->ov_idx);
    p->rasm.n = n; p->rasm.nsub = nsub; p->rasm.xy = xy; p->rasm.kp = p->kp;
    p->rasm.core_ptr = p->core_ptr; p->rasm.core_idx = p->core_idx;
    p->rasm.ov_ptr = p->ov_ptr; p->rasm.ov_idx = p->ov_idx;
    return orc_rasm_setup(&p->rasm, max_sub_points);
}

void orc_problem_destroy(orc_problem* p)
{
    if (!p) return;
    orc_rasm_free(&p->rasm);
    free(p->perm); free(p->cell_start);
    free(p->core_ptr); free(p->core_idx); free(p->ov_ptr); free(p->ov_idx);
    free(p);
}

void orc_problem_grid(const orc_problem* p, orc_grid* g, orc_boxes* b)
{
    *g = p->g;
    *b = p->boxes;
}

const int32_t* orc_problem_perm(const orc_problem* p) { return p->perm; }
const int32_t* orc_problem_cell_start(const orc_problem* p) { return p->cell_start; }
const int64_t* orc_problem_core_ptr(const orc_problem* p) { return p->core_ptr; }
const int32_t* orc_problem_core_idx(const orc_problem* p) { return p->core_idx; }
const int64_t* orc_problem_ov_ptr(const orc_problem* p) { return p->ov_ptr; }
const int32_t* orc_problem_ov_idx(const orc_problem* p) { return p->ov_idx; }

/* Select the plain additive Schwarz preconditioner (Eq. asm) instead of RASM. */
void orc_problem_set_additive(orc_problem* p, int additive) { p->rasm.additive = additive; }

void orc_problem_matvec(orc_problem* p, const double* w, double* y) { op_amul(p, w, y); }
void orc_problem_rasm_apply(orc_problem* p, const double* v, double* z) { op_minv(p, v, z); }

/* GMRES(m) + RASM on the truncated system; w holds the initial guess on
 * entry. precondition = 0 runs unpreconditioned GMRES (for pins). */
int orc_problem_solve(orc_problem* p, const double* f, double* w, int64_t m, double rtol,
                      int64_t max_iters, int precondition, double* hist, orc_gmres_info* info)
{
    return orc_gmres(p->n, op_amul, p, precondition ? op_minv : op_identity, p, f, w, m, rtol,
                     max_iters, hist, info);
}

int64_t orc_problem_counts(const orc_problem* p, int64_t which)
{
    return which == 0 ? p->matvecs : p->applies;
}
