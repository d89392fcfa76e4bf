// capi.cu -- the extern "C" entry points declared in include/rbf.h, plus the
// context's allocation and error bookkeeping.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace rbf {

rbf_status fail(rbf_ctx* ctx, rbf_status st, const char* fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

rbf_status cuda_fail(rbf_ctx* ctx, cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ctx, RBF_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
    }
    return fail(ctx, RBF_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

void release(rbf_ctx* ctx, void* p)
{
    if (!p) return;
    for (size_t i = 0; i < ctx->owned.size(); ++i) {
        if (ctx->owned[i].first == p) {
            ctx->dev_bytes -= (int64_t)ctx->owned[i].second;
            ctx->owned.erase(ctx->owned.begin() + (long)i);
            break;
        }
    }
    cudaFree(p);
}

template <class T>
rbf_status ensure(rbf_ctx* ctx, DevArray<T>& a, size_t count)
{
    if (count == 0) count = 1;
    if (a.p && a.count >= count) return RBF_OK;
    if (ctx->capturing)   // a cudaMalloc would invalidate the solver's graph capture
        return fail(ctx, RBF_ERR_STATE, "device allocation requested while the solver captures its cycle");
    release(ctx, a.p);
    a.p = nullptr;
    a.count = 0;
    void* p = nullptr;
    size_t bytes = count * sizeof(T);
    if (ctx->mem_limit > 0 && ctx->dev_bytes + (int64_t)bytes > ctx->mem_limit)
        return fail(ctx, RBF_ERR_OOM, "allocation of %zu bytes exceeds the context's memory limit (%lld of %lld held)",
                    bytes, (long long)ctx->dev_bytes, (long long)ctx->mem_limit);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, RBF_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    ctx->owned.emplace_back(p, bytes);
    ctx->dev_bytes += (int64_t)bytes;
    a.p = (T*)p;
    a.count = count;
    return RBF_OK;
}

template rbf_status ensure<int32_t>(rbf_ctx*, DevArray<int32_t>&, size_t);
template rbf_status ensure<int64_t>(rbf_ctx*, DevArray<int64_t>&, size_t);
template rbf_status ensure<double>(rbf_ctx*, DevArray<double>&, size_t);
template rbf_status ensure<float>(rbf_ctx*, DevArray<float>&, size_t);
template rbf_status ensure<uint32_t>(rbf_ctx*, DevArray<uint32_t>&, size_t);
template rbf_status ensure<GmresDev>(rbf_ctx*, DevArray<GmresDev>&, size_t);
template rbf_status ensure<Prob>(rbf_ctx*, DevArray<Prob>&, size_t);
template rbf_status ensure<unsigned long long>(rbf_ctx*, DevArray<unsigned long long>&, size_t);

constexpr int64_t kMaxProfPairs = 1 << 16;

rbf_status prof_begin(rbf_ctx* ctx, int id, cudaStream_t st)
{
    if (!ctx->prof || !((ctx->prof_mask >> id) & 1u)) return RBF_OK;
    if (ctx->capturing) {   // an event record node of the captured cycle
        rbf_graph_prof g{id, ctx->prof_step, nullptr, nullptr};
        RBF_CUDA(ctx, cudaEventCreate(&g.a));
        cudaError_t e = cudaEventCreate(&g.b);
        if (e != cudaSuccess) {
            cudaEventDestroy(g.a);
            return cuda_fail(ctx, e, "cudaEventCreate");
        }
        ctx->bgraph_prof.push_back(g);
        RBF_CUDA(ctx, cudaEventRecordWithFlags(g.a, st, cudaEventRecordExternal));
        return RBF_OK;
    }
    rbf_prof_slot& s = ctx->prof_slots[id];
    if (s.used >= kMaxProfPairs) return RBF_OK;
    while ((int64_t)s.ev.size() < 2 * (s.used + 1)) {
        cudaEvent_t e;
        RBF_CUDA(ctx, cudaEventCreate(&e));
        s.ev.push_back(e);
    }
    RBF_CUDA(ctx, cudaEventRecord(s.ev[2 * s.used], st));
    return RBF_OK;
}

rbf_status prof_end(rbf_ctx* ctx, int id, cudaStream_t st)
{
    if (!ctx->prof || !((ctx->prof_mask >> id) & 1u)) return RBF_OK;
    if (ctx->capturing) {
        for (size_t i = ctx->bgraph_prof.size(); i-- > 0;)
            if (ctx->bgraph_prof[i].cls == id) {
                RBF_CUDA(ctx, cudaEventRecordWithFlags(ctx->bgraph_prof[i].b, st, cudaEventRecordExternal));
                return RBF_OK;
            }
        return fail(ctx, RBF_ERR_STATE, "profiler: end of a launch that was not begun");
    }
    rbf_prof_slot& s = ctx->prof_slots[id];
    if (s.used >= kMaxProfPairs) return RBF_OK;
    RBF_CUDA(ctx, cudaEventRecord(s.ev[2 * s.used + 1], st));
    s.used++;
    return RBF_OK;
}

rbf_status prof_harvest_graph(rbf_ctx* ctx, int steps_run)
{
    for (const rbf_graph_prof& g : ctx->bgraph_prof) {
        if (g.step >= steps_run) continue;   // every problem had stopped: the launch did no work
        float ms = 0.f;
        RBF_CUDA(ctx, cudaEventElapsedTime(&ms, g.a, g.b));
        ctx->prof_slots[g.cls].graph_ms += ms;
        ctx->prof_slots[g.cls].graph_launches += 1;
    }
    return RBF_OK;
}

// 2^(j/64), 64 / ln 2 and a two-part ln 2 / 64, evaluated in long double.
ExpConsts make_exp_consts()
{
    ExpConsts c;
    const long double ln2 = 0.693147180559945309417232121458176568L;
    c.inv_l = (double)(64.0L / ln2);
    double l = (double)(ln2 / 64.0L);
    uint64_t bits;
    std::memcpy(&bits, &l, sizeof(bits));
    bits &= ~((uint64_t(1) << 21) - 1);   // keep 32 significant bits
    std::memcpy(&c.l_hi, &bits, sizeof(bits));
    c.l_lo = (double)(ln2 / 64.0L - (long double)c.l_hi);
    for (int j = 0; j < 64; ++j) c.tab[j] = (double)exp2l((long double)j / 64.0L);
    return c;
}

void make_exp2048(double* tab, double* c)
{
    const long double ln2 = 0.693147180559945309417232121458176568L;
    for (int j = 0; j < kExpTab2048; ++j) tab[j] = (double)exp2l(-(long double)j / 2048.0L);
    long double c1 = -ln2 / 2048.0L;
    c[0] = (double)c1;
    c[1] = (double)(c1 * c1 / 2.0L);
    c[2] = (double)(c1 * c1 * c1 / 6.0L);
}

void make_fx_tables(unsigned long long* t1, unsigned long long* t2)
{
    for (int i = 0; i < kFxTab; ++i) {
        t1[i] = (unsigned long long)(exp2l(-(long double)i / 1024.0L) * 0x1p63L + 0.5L);
        t2[i] = (unsigned long long)(exp2l(-(long double)i / 1048576.0L) * 0x1p63L + 0.5L);
    }
}

bool make_fx_constants(double amax, double rc, double s, double* scale, int* sh, int* F, unsigned long long* M)
{
    const double a = std::max(amax, rc);
    if (!(a > 0.0) || !std::isfinite(a) || !(s > 0.0) || !std::isfinite(s)) return false;
    int e = 0;
    std::frexp(a, &e);                       // a < 2^e
    const int S = 62 - e;                    // |x| 2^S < 2^62
    if (S < -1000 || S > 1000) return false;
    int eR = 0;
    std::frexp(std::ldexp(rc, S), &eR);      // R = r_c 2^S < 2^eR
    if (eR < 31 || eR > 62) return false;    // r_c below 2^-32 max|x|: too few bits for the offsets
    const int shift = 63 - eR;               // |dx| 2^sh < 2^63 (1 + 2^-50) for r2 <= r_c^2
    const long double g = (long double)s * 1.442695040888963407359924681001892137L;   // s log2(e)
    int ge = 0;
    const long double gm = std::frexp(g, &ge);                  // g = gm 2^ge, gm in [0.5, 1)
    const int f = 2 * S + 2 * shift - 64 - ge;                  // makes M = gm 2^64 in [2^63, 2^64); z < 2^62
    if (f < 21 || f > 63) return false;
    unsigned long long m = (unsigned long long)std::ldexp(gm, 64);
    int fb = f;
    // the 32-bit layout of kernel_fx52 (M scaled down to exactly 52 fraction bits) when it
    // fits and the exponent n = floor(r2 s log2 e) stays below 1000 inside the cutoff
    // (r_c up to about 37 sigma); otherwise the general path
    if (f >= 52 && (long double)rc * rc * g < 999.0L) {
        m >>= (f - 52);
        fb = 52;
    }
    *scale = std::ldexp(1.0, S);
    *sh = shift;
    *F = fb;
    *M = m;
    return true;
}

namespace {

// Kernel values of point pairs (x_i, y_i, x_j, y_j) by the matvec's fixed-point
// evaluation with problem 0's constants; 0 beyond the cutoff.
__global__ void k_debug_kernel_pairs(const double* __restrict__ pr4, double* __restrict__ out, int64_t n,
                                     const Prob* __restrict__ prob, const unsigned long long* __restrict__ tab)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Prob& q = prob[0];
    const double xi = pr4[4 * i], yi = pr4[4 * i + 1], xj = pr4[4 * i + 2], yj = pr4[4 * i + 3];
    const double ex = __dsub_rn(xi, xj), ey = __dsub_rn(yi, yj);
    if (__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) > q.rc2) {
        out[i] = 0.0;
        return;
    }
    const long long du = (long long)((unsigned long long)fx_coord(xi, q.fx_scale, q.fx_sh) -
                                     (unsigned long long)fx_coord(xj, q.fx_scale, q.fx_sh));
    const long long dv = (long long)((unsigned long long)fx_coord(yi, q.fx_scale, q.fx_sh) -
                                     (unsigned long long)fx_coord(yj, q.fx_scale, q.fx_sh));
    out[i] = q.fx_F == 52 ? kernel_fx52(du, dv, q.fx_M, tab, tab + kFxTab)
                          : kernel_fx(du, dv, q.fx_F, q.fx_M, tab, tab + kFxTab);
}

__global__ void k_debug_exp(const double* __restrict__ t, double* __restrict__ out, int64_t n, int variant,
                            ExpConsts ec, const double* __restrict__ tab2048, double c1, double c2, double c3)
{
    __shared__ double tab[64];
    if (threadIdx.x < 64) tab[threadIdx.x] = ec.tab[threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (variant == 0)
        out[i] = exp_neg(t[i], tab, ec.inv_l, ec.l_hi, ec.l_lo);
    else if (variant == 1)
        out[i] = exp(-t[i]);
    else
        out[i] = exp_neg_r2(t[i], 2048.0 / M_LN2, tab2048, c1, c2, c3);
}

}  // namespace

}  // namespace rbf

using namespace rbf;

static cudaStream_t S(rbf_stream s) { return (cudaStream_t)s; }

extern "C" {

const char* rbf_status_string(rbf_status s)
{
    switch (s) {
    case RBF_OK: return "ok";
    case RBF_ERR_INVALID_ARG: return "invalid argument";
    case RBF_ERR_OOM: return "out of device memory";
    case RBF_ERR_CUDA: return "CUDA error";
    case RBF_ERR_NOT_SPD: return "subdomain matrix not positive definite";
    case RBF_ERR_SUBDOMAIN_TOO_LARGE: return "subdomain overlap list too large";
    case RBF_ERR_NOT_CONVERGED: return "not converged";
    case RBF_ERR_TIMEOUT: return "device wait timed out";
    case RBF_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* rbf_last_error(rbf_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

uint64_t rbf_launch_count(rbf_ctx* ctx) { return ctx ? ctx->launches : 0; }

int64_t rbf_device_bytes(rbf_ctx* ctx) { return ctx ? ctx->dev_bytes : 0; }

int64_t rbf_store_f64_bytes(rbf_ctx* ctx) { return ctx && ctx->f64s.valid ? ctx->f64s.bytes : 0; }

rbf_status rbf_set_option(rbf_ctx* ctx, int option, int64_t value)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    switch (option) {
    case RBF_OPT_FUSED_STEP:
        if (value < 0 || value > 2) break;
        ctx->fused_mode = (int)value;
        return RBF_OK;
    case RBF_OPT_SYMMETRIC_F32:
        if (value != 0 && value != 1) break;
        ctx->sym_mode = value ? 0 : 1;
        return RBF_OK;
    case RBF_OPT_SYMMETRIC_F64:
        if (value != 0 && value != 1) break;
        ctx->sym64_mode = value ? 0 : 1;
        return RBF_OK;
    case RBF_OPT_BARRIER_SPIN_LIMIT:
        if (value < 1) break;
        ctx->fused_spin_limit = (unsigned long long)value;
        return RBF_OK;
    case RBF_OPT_BARRIER_EXTRA_BLOCK:
        if (value != 0 && value != 1) break;
        ctx->fused_extra_block = (int)value;
        return RBF_OK;
    case RBF_OPT_STREAM_GS:
        if (value != 0 && value != 1) break;
        ctx->gs_stream_mode = (int)value;
        return RBF_OK;
    case RBF_OPT_STREAM_WAIT_CHECK:
        if (value != 0 && value != 1) break;
        ctx->stream_check = (int)value;
        return RBF_OK;
    case RBF_OPT_STORE_F64:
        if (value != 0 && value != 1) break;
        ctx->store_mode = (int)value;
        if (value == 0) f64_store_release(ctx);
        ctx->f64s.tried = false;
        return RBF_OK;
    default:
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_set_option: unknown option %d", option);
    }
    return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_set_option: value %lld out of range for option %d", (long long)value,
                option);
}

rbf_status rbf_set_memory_limit(rbf_ctx* ctx, int64_t bytes)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (bytes < 0) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_set_memory_limit: negative limit");
    ctx->mem_limit = bytes;
    ctx->f64s.tried = false;   // the kept FP64 values may fit now
    return RBF_OK;
}

rbf_status rbf_create(rbf_ctx** out, int device)
{
    if (!out) return RBF_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return RBF_ERR_INVALID_ARG;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return RBF_ERR_CUDA;
    rbf_ctx* ctx = new rbf_ctx();
    ctx->device = device;
    ctx->expc = make_exp_consts();
    e = cudaMallocHost(&ctx->gm_host, sizeof(GmresDev));
    if (e != cudaSuccess) {
        delete ctx;
        return RBF_ERR_OOM;
    }
    std::vector<double> tab(kExpTab2048);
    make_exp2048(tab.data(), ctx->exp2048_c);
    if (ensure(ctx, ctx->exp2048, kExpTab2048) != RBF_OK ||
        cudaMemcpy(ctx->exp2048.p, tab.data(), sizeof(double) * kExpTab2048, cudaMemcpyHostToDevice) != cudaSuccess) {
        rbf_destroy(ctx);
        return RBF_ERR_OOM;
    }
    std::vector<unsigned long long> fx(2 * kFxTab);
    make_fx_tables(fx.data(), fx.data() + kFxTab);
    if (ensure(ctx, ctx->fxtab, 2 * kFxTab) != RBF_OK ||
        cudaMemcpy(ctx->fxtab.p, fx.data(), sizeof(unsigned long long) * 2 * kFxTab, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        rbf_destroy(ctx);
        return RBF_ERR_OOM;
    }
    *out = ctx;
    return RBF_OK;
}

void rbf_destroy(rbf_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    batch_graph_reset(ctx);
    if (ctx->bstream) cudaStreamDestroy(ctx->bstream);
    if (ctx->bevent) cudaEventDestroy(ctx->bevent);
    for (auto& a : ctx->owned) cudaFree(a.first);
    ctx->owned.clear();
    for (auto& s : ctx->prof_slots)
        for (cudaEvent_t e : s.ev) cudaEventDestroy(e);
    if (ctx->gm_host) cudaFreeHost(ctx->gm_host);
    delete ctx;
}

// Kernel part of a problem from its parameters (Sec. 2.3); grid set by binning.
static rbf_status init_prob(rbf_ctx* ctx, Prob& q, const rbf_params* p, int64_t pbeg, int64_t pend)
{
    if (!(p->sigma > 0.0) || !(p->cutoff > 0.0) || !std::isfinite(p->sigma) || !std::isfinite(p->cutoff))
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: sigma and cutoff must be positive");
    std::memset(&q, 0, sizeof(q));
    q.sigma = p->sigma;
    q.rc = p->cutoff;
    q.rc2 = p->cutoff * p->cutoff;
    q.s = 1.0 / (2.0 * p->sigma * p->sigma);
    q.knorm = p->normalized ? 1.0 / (2.0 * M_PI * p->sigma * p->sigma) : 1.0;
    q.K = 2048.0 * q.s / M_LN2;
    q.c = (p->cell_size > 0.0) ? p->cell_size : p->cutoff;
    double k = std::ceil(q.rc / q.c);
    if (!(k >= 1.0) || k > 64.0)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: cutoff / cell_size = %g gives a stencil outside 1..64", k);
    q.k = (int)k;
    double a = std::sqrt(M_LOG2E * q.s);
    q.a_loc = (float)a;
    q.ca = (float)(q.c * (double)q.a_loc);
    double rc2f = q.rc2 * (double)q.a_loc * (double)q.a_loc;
    q.rc2f_lo = (float)(rc2f * (1.0 - 1e-4));
    q.rc2f_hi = (float)(rc2f * (1.0 + 1e-4));
    q.pbeg = pbeg;
    q.pend = pend;
    return RBF_OK;
}

static rbf_status bin_batch(rbf_ctx* ctx, const double* xy_dev, const int64_t* ptr, int64_t nprob,
                            const rbf_params* params, cudaStream_t st)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!xy_dev || !ptr || !params || nprob < 1 || nprob > (1 << 24))
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: need xy, point ranges, parameters and 1 <= nprob <= 2^24");
    const int64_t n = ptr[nprob];
    if (ptr[0] != 0 || n < 1 || n > (int64_t)0x7fffffff - 1)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: need ptr[0] = 0 and 1 <= n < 2^31 (n = %lld)", (long long)n);
    if (((uintptr_t)xy_dev) % 8 != 0) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: xy must be 8-byte aligned");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->binned = false;
    ctx->rasm_ready = false;
    ctx->in.ready = false;
    ctx->prob_h.assign((size_t)nprob, Prob{});
    for (int64_t b = 0; b < nprob; ++b) {
        if (ptr[b + 1] <= ptr[b])
            return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: problem %lld has no points", (long long)b);
        RBF_CHECK(init_prob(ctx, ctx->prob_h[b], &params[b], ptr[b], ptr[b + 1]));
    }
    for (int which = 0; which < 2; ++which) {
        const int t = which == 0 ? params[0].tile_f64 : params[0].tile_f32;
        if (t != 0 && t != 32 && t != 64 && t != 128)
            return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: tiles must be 0, 32, 64 or 128 (got %d)", t);
    }
    ctx->tile64 = params[0].tile_f64 > 0 ? params[0].tile_f64 : 128;
    ctx->tile32 = params[0].tile_f32 > 0 ? params[0].tile_f32 : 128;
    ctx->nprob = nprob;
    ctx->n = n;
    const Prob& q = ctx->prob_h[0];
    ctx->sigma = q.sigma;
    ctx->rc = q.rc;
    ctx->rc2 = q.rc2;
    ctx->cell = q.c;
    ctx->s = q.s;
    ctx->knorm = q.knorm;
    ctx->normalized = params[0].normalized ? 1 : 0;
    ctx->kst = q.k;
    RBF_CHECK(bin_points(ctx, xy_dev, st));
    ctx->binned = true;
    return RBF_OK;
}

rbf_status rbf_bin(rbf_ctx* ctx, const double* xy_dev, int64_t n, const rbf_params* p, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (n < 1 || n > (int64_t)0x7fffffff - 1)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_bin: need 1 <= n < 2^31 (n = %lld)", (long long)n);
    int64_t ptr[2] = {0, n};
    return bin_batch(ctx, xy_dev, ptr, 1, p, S(stream));
}

rbf_status rbf_bin_batch(rbf_ctx* ctx, const double* xy_dev, const int64_t* ptr_host, int64_t nprob,
                         const rbf_params* params_host, rbf_stream stream)
{
    return bin_batch(ctx, xy_dev, ptr_host, nprob, params_host, S(stream));
}

rbf_status rbf_matvec(rbf_ctx* ctx, const double* w_dev, double* y_dev, int precision, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_matvec: call rbf_bin first");
    if (!w_dev || !y_dev) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_matvec: null vector");
    if (precision != RBF_FP64 && precision != RBF_FP32)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_matvec: precision must be RBF_FP64 or RBF_FP32");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_CHECK(ensure(ctx, ctx->vec_a, ctx->n));
    RBF_CHECK(ensure(ctx, ctx->vec_b, ctx->n));
    RBF_CHECK(permute_to_sorted(ctx, w_dev, ctx->vec_a.p, S(stream)));
    if (precision == RBF_FP64)
        RBF_CHECK(matvec_sorted_f64(ctx, ctx->vec_a.p, ctx->vec_b.p, S(stream)));
    else
        RBF_CHECK(matvec_sorted_f32(ctx, ctx->vec_a.p, ctx->vec_b.p, S(stream)));
    return permute_to_user(ctx, ctx->vec_b.p, y_dev, S(stream));
}

static rbf_status rasm_setup_batch(rbf_ctx* ctx, const rbf_rasm_params* params, cudaStream_t st)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_rasm_setup: call rbf_bin first");
    if (!params) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_rasm_setup: null parameters");
    const int precision = params[0].precision;
    if (precision != RBF_FP64 && precision != RBF_FP32 && precision != RBF_FP32_FROM_FP64)
        return fail(ctx, RBF_ERR_INVALID_ARG,
                    "rbf_rasm_setup: precision must be RBF_FP64, RBF_FP32 or RBF_FP32_FROM_FP64");
    int cap = 0;
    int64_t nsub = 0;
    for (int64_t b = 0; b < ctx->nprob; ++b) {
        const rbf_rasm_params* p = &params[b];
        if (!(p->core_size > 0.0) || !(p->overlap >= 0.0) || !std::isfinite(p->x0) || !std::isfinite(p->y0) ||
            !std::isfinite(p->core_size) || !std::isfinite(p->overlap))
            return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_rasm_setup: need core_size > 0, overlap >= 0 (problem %lld)",
                        (long long)b);
        int c = p->max_sub_points > 0 ? p->max_sub_points : kMaxSub;
        if (c > kMaxSub) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_rasm_setup: max_sub_points > %d", kMaxSub);
        cap = (b == 0) ? c : std::min(cap, c);
        Prob& q = ctx->prob_h[b];
        q.x0 = p->x0;
        q.y0 = p->y0;
        q.B = p->core_size;
        q.delta = p->overlap;
        double fx = std::floor((q.xmax - q.x0) / q.B), fy = std::floor((q.ymax - q.y0) / q.B);
        double reach = std::ceil(q.delta / q.B) + 1.0;
        if (!(fx < 1.0e9) || !(fy < 1.0e9) || reach > 64.0)
            return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_rasm_setup: too many boxes or overlap / core_size too large");
        q.nbx = fx < 0.0 ? 1 : (int64_t)fx + 1;
        q.nby = fy < 0.0 ? 1 : (int64_t)fy + 1;
        q.reach = (int)reach;
        q.subbase = nsub;
        nsub += q.nbx * q.nby;
        if (nsub > ((int64_t)1 << 30)) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_rasm_setup: too many boxes");
    }
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    ctx->rasm_ready = false;
    ctx->in.ready = false;   // its re-indexed lists follow the subdomains
    ctx->rasm_precision = precision;
    ctx->rasm_additive = params[0].additive != 0;
    ctx->nsub = nsub;
    if (ctx->nprob == 1) {
        const Prob& q = ctx->prob_h[0];
        ctx->x0 = q.x0;
        ctx->y0 = q.y0;
        ctx->B = q.B;
        ctx->delta = q.delta;
        ctx->nbx = q.nbx;
        ctx->nby = q.nby;
    } else {   // a batch reports its total subdomain count as nbx x 1
        ctx->nbx = nsub;
        ctx->nby = 1;
    }
    RBF_CUDA(ctx, cudaMemcpyAsync(ctx->prob.p, ctx->prob_h.data(), sizeof(Prob) * ctx->nprob, cudaMemcpyHostToDevice,
                                  st));
    RBF_CHECK(build_subdomains(ctx, st));
    if (ctx->max_ov > cap)
        return fail(ctx, RBF_ERR_SUBDOMAIN_TOO_LARGE, "rbf_rasm_setup: an overlap list has %d points (cap %d)",
                    ctx->max_ov, cap);
    if (ctx->rasm_additive) RBF_CHECK(asm_lists(ctx, st));
    RBF_CHECK(rasm_factor(ctx, st));
    ctx->rasm_ready = true;
    return RBF_OK;
}

rbf_status rbf_rasm_setup(rbf_ctx* ctx, const rbf_rasm_params* p, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (ctx->binned && ctx->nprob != 1)
        return fail(ctx, RBF_ERR_STATE, "rbf_rasm_setup: the context holds a batch; use rbf_rasm_setup_batch");
    return rasm_setup_batch(ctx, p, S(stream));
}

rbf_status rbf_rasm_setup_batch(rbf_ctx* ctx, const rbf_rasm_params* params_host, rbf_stream stream)
{
    return rasm_setup_batch(ctx, params_host, S(stream));
}

rbf_status rbf_rasm_factor_counts(rbf_ctx* ctx, int64_t* tensor_core, int64_t* fp64)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->rasm_ready) return fail(ctx, RBF_ERR_STATE, "rbf_rasm_factor_counts: call rbf_rasm_setup first");
    if (tensor_core) *tensor_core = ctx->factor_tc;
    if (fp64) *fp64 = ctx->factor_fp64;
    return RBF_OK;
}

rbf_status rbf_rasm_apply(rbf_ctx* ctx, const double* r_dev, double* z_dev, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->rasm_ready) return fail(ctx, RBF_ERR_STATE, "rbf_rasm_apply: call rbf_rasm_setup first");
    if (!r_dev || !z_dev) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_rasm_apply: null vector");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_CHECK(ensure(ctx, ctx->vec_a, ctx->n));
    RBF_CHECK(ensure(ctx, ctx->vec_b, ctx->n));
    RBF_CHECK(permute_to_sorted(ctx, r_dev, ctx->vec_a.p, S(stream)));
    RBF_CHECK(rasm_apply_sorted(ctx, ctx->vec_a.p, ctx->vec_b.p, S(stream)));
    return permute_to_user(ctx, ctx->vec_b.p, z_dev, S(stream));
}

rbf_status rbf_solve(rbf_ctx* ctx, const double* f_dev, double* w_dev, const rbf_solve_params* p,
                     rbf_solve_info* info, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->rasm_ready) return fail(ctx, RBF_ERR_STATE, "rbf_solve: call rbf_rasm_setup first");
    if (ctx->nprob != 1)
        return fail(ctx, RBF_ERR_STATE, "rbf_solve: the context holds a batch; use rbf_solve_batch");
    if (!f_dev || !w_dev || !p) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_solve: null argument");
    if (!(p->rtol > 0.0) || p->restart < 0 || p->restart > kMaxRestart || p->max_iters < 0)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_solve: need rtol > 0, 0 <= restart <= %d", kMaxRestart);
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_CHECK(ensure(ctx, ctx->vec_d, ctx->n));
    RBF_CHECK(ensure(ctx, ctx->vec_e, ctx->n));
    RBF_CHECK(permute_to_sorted(ctx, f_dev, ctx->vec_d.p, S(stream)));
    RBF_CHECK(permute_to_sorted(ctx, w_dev, ctx->vec_e.p, S(stream)));
    rbf_solve_info local;
    std::memset(&local, 0, sizeof(local));
    rbf_status st = gmres_solve(ctx, ctx->vec_d.p, ctx->vec_e.p, p, &local, S(stream));
    if (info) *info = local;
    if (st != RBF_OK && st != RBF_ERR_NOT_CONVERGED) return st;
    rbf_status st2 = permute_to_user(ctx, ctx->vec_e.p, w_dev, S(stream));
    if (st2 != RBF_OK) return st2;
    RBF_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return st;
}

rbf_status rbf_solve_batch(rbf_ctx* ctx, const double* f_dev, double* w_dev, const rbf_solve_params* p,
                           rbf_solve_info* info_host, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->rasm_ready) return fail(ctx, RBF_ERR_STATE, "rbf_solve_batch: call rbf_rasm_setup_batch first");
    if (!f_dev || !w_dev || !p) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_solve_batch: null argument");
    if (!(p->rtol > 0.0) || p->restart < 0 || p->restart > kMaxRestart || p->max_iters < 0)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_solve_batch: need rtol > 0, 0 <= restart <= %d", kMaxRestart);
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_CHECK(ensure(ctx, ctx->vec_d, ctx->n));
    RBF_CHECK(ensure(ctx, ctx->vec_e, ctx->n));
    RBF_CHECK(permute_to_sorted(ctx, f_dev, ctx->vec_d.p, S(stream)));
    RBF_CHECK(permute_to_sorted(ctx, w_dev, ctx->vec_e.p, S(stream)));
    rbf_status st = gmres_solve_batch(ctx, ctx->vec_d.p, ctx->vec_e.p, p, info_host, S(stream));
    if (st != RBF_OK && st != RBF_ERR_NOT_CONVERGED) return st;
    rbf_status st2 = permute_to_user(ctx, ctx->vec_e.p, w_dev, S(stream));
    if (st2 != RBF_OK) return st2;
    RBF_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return st;
}

rbf_status rbf_interpolate_host(rbf_ctx* ctx, const double* xy_host, const double* f_host, double* w_host,
                                int64_t n, const rbf_params* params, const rbf_rasm_params* rasm,
                                const rbf_solve_params* solve, rbf_solve_info* info, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!xy_host || !f_host || !w_host || n < 1)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_interpolate_host: null buffer or n < 1");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    static_assert(sizeof(double) == 8, "double");
    // staging buffers held by the context between calls (no allocation when the size repeats)
    rbf::DevArray<double>& xy = ctx->host_xy;
    rbf::DevArray<double>& f = ctx->host_f;
    rbf::DevArray<double>& w = ctx->host_w;
    RBF_CHECK(ensure(ctx, xy, (size_t)(2 * n)));
    rbf_status st = ensure(ctx, f, (size_t)n);
    if (st == RBF_OK) st = ensure(ctx, w, (size_t)n);
    cudaStream_t s = S(stream);
    if (st == RBF_OK) {
        cudaError_t e = cudaMemcpyAsync(xy.p, xy_host, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(f.p, f_host, sizeof(double) * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.p, 0, sizeof(double) * n, s);
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "rbf_interpolate_host: copy in");
    }
    if (st == RBF_OK) st = rbf_bin(ctx, xy.p, n, params, stream);
    if (st == RBF_OK) st = rbf_rasm_setup(ctx, rasm, stream);
    if (st == RBF_OK || st == RBF_ERR_NOT_CONVERGED) {
        rbf_status ss = rbf_solve(ctx, f.p, w.p, solve, info, stream);
        if (ss == RBF_OK || ss == RBF_ERR_NOT_CONVERGED) {
            cudaError_t e = cudaMemcpyAsync(w_host, w.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) ss = cuda_fail(ctx, e, "rbf_interpolate_host: copy out");
        }
        st = ss;
    }
    return st;
}

rbf_status rbf_get_grid(rbf_ctx* ctx, int64_t* ncx, int64_t* ncy, double* bbox_host)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_get_grid: call rbf_bin first");
    if (ncx) *ncx = ctx->ncx;
    if (ncy) *ncy = ctx->ncy;
    if (bbox_host) std::memcpy(bbox_host, ctx->bbox, sizeof(ctx->bbox));
    return RBF_OK;
}

rbf_status rbf_get_bins(rbf_ctx* ctx, int32_t* perm_dev, int32_t* cell_start_dev, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_get_bins: call rbf_bin first");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = S(stream);
    if (perm_dev)
        RBF_CUDA(ctx, cudaMemcpyAsync(perm_dev, ctx->perm.p, sizeof(int32_t) * ctx->n, cudaMemcpyDeviceToDevice, s));
    if (cell_start_dev)
        RBF_CUDA(ctx, cudaMemcpyAsync(cell_start_dev, ctx->cell_start.p, sizeof(int32_t) * (ctx->ncx * ctx->ncy + 1),
                                      cudaMemcpyDeviceToDevice, s));
    RBF_CUDA(ctx, cudaStreamSynchronize(s));
    return RBF_OK;
}

rbf_status rbf_get_subdomain_sizes(rbf_ctx* ctx, int64_t* nbx, int64_t* nby, int64_t* core_total,
                                   int64_t* overlap_total)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->rasm_ready) return fail(ctx, RBF_ERR_STATE, "rbf_get_subdomain_sizes: call rbf_rasm_setup first");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    int32_t tot[2] = {0, 0};
    RBF_CUDA(ctx, cudaMemcpy(&tot[0], ctx->core_ptr.p + ctx->nsub, sizeof(int32_t), cudaMemcpyDeviceToHost));
    RBF_CUDA(ctx, cudaMemcpy(&tot[1], ctx->ov_ptr.p + ctx->nsub, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (nbx) *nbx = ctx->nbx;
    if (nby) *nby = ctx->nby;
    if (core_total) *core_total = tot[0];
    if (overlap_total) *overlap_total = tot[1];
    return RBF_OK;
}

rbf_status rbf_get_subdomains(rbf_ctx* ctx, int32_t* core_ptr_dev, int32_t* core_idx_dev, int32_t* ov_ptr_dev,
                              int32_t* ov_idx_dev, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->rasm_ready) return fail(ctx, RBF_ERR_STATE, "rbf_get_subdomains: call rbf_rasm_setup first");
    if (!core_ptr_dev || !core_idx_dev || !ov_ptr_dev || !ov_idx_dev)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_get_subdomains: null output");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_CHECK(export_subdomains(ctx, core_ptr_dev, core_idx_dev, ov_ptr_dev, ov_idx_dev, S(stream)));
    RBF_CUDA(ctx, cudaStreamSynchronize(S(stream)));
    return RBF_OK;
}

rbf_status rbf_count_neighbors(rbf_ctx* ctx, int64_t* total, rbf_stream stream)
{
    if (!ctx || !total) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_count_neighbors: call rbf_bin first");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    return neighbor_lists(ctx, nullptr, nullptr, 0, total, S(stream));
}

rbf_status rbf_count_candidates(rbf_ctx* ctx, int grid, int64_t* total, rbf_stream stream)
{
    if (!ctx || !total || (grid != 0 && grid != 1)) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_count_candidates: call rbf_bin first");
    if (grid == 1 && !ctx->in.ready)
        return fail(ctx, RBF_ERR_STATE, "rbf_count_candidates: no inner grid (run a mixed solve with inner_cutoff > 0)");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    return count_candidates(ctx, grid, total, S(stream));
}

rbf_status rbf_debug_inner_matvec(rbf_ctx* ctx, double inner_cutoff, const double* w_dev, double* y_dev, int variant,
                                  rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_debug_inner_matvec: call rbf_bin first");
    if (!w_dev || !y_dev || !(inner_cutoff > 0.0) || (variant != 0 && variant != 1))
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_debug_inner_matvec: bad argument");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_CHECK(ensure(ctx, ctx->vec_a, ctx->n));
    RBF_CHECK(ensure(ctx, ctx->vec_b, ctx->n));
    RBF_CHECK(permute_to_sorted(ctx, w_dev, ctx->vec_a.p, S(stream)));
    RBF_CHECK(inner_matvec_debug(ctx, inner_cutoff, ctx->vec_a.p, ctx->vec_b.p, variant, S(stream)));
    return permute_to_user(ctx, ctx->vec_b.p, y_dev, S(stream));
}

rbf_status rbf_count_pairs(rbf_ctx* ctx, int grid, int64_t* total, rbf_stream stream)
{
    if (!ctx || !total || (grid != 0 && grid != 1)) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_count_pairs: call rbf_bin first");
    if (grid == 1 && !ctx->in.ready)
        return fail(ctx, RBF_ERR_STATE, "rbf_count_pairs: no inner grid (run a mixed solve with inner_cutoff > 0)");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    return count_pairs(ctx, grid, total, S(stream));
}

rbf_status rbf_profile_enable(rbf_ctx* ctx, int enable)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    ctx->prof = enable != 0;
    return RBF_OK;
}

rbf_status rbf_profile_classes(rbf_ctx* ctx, unsigned mask)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    ctx->prof_mask = mask;
    return RBF_OK;
}

rbf_status rbf_profile_read(rbf_ctx* ctx, int kernel, int64_t* launches, double* total_ms)
{
    if (!ctx || kernel < 0 || kernel >= RBF_PROF_COUNT) return RBF_ERR_INVALID_ARG;
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    rbf_prof_slot& s = ctx->prof_slots[kernel];
    double tot = 0.0;
    for (int64_t i = 0; i < s.used; ++i) {
        RBF_CUDA(ctx, cudaEventSynchronize(s.ev[2 * i + 1]));
        float ms = 0.f;
        RBF_CUDA(ctx, cudaEventElapsedTime(&ms, s.ev[2 * i], s.ev[2 * i + 1]));
        tot += ms;
    }
    if (launches) *launches = s.used + s.graph_launches;
    if (total_ms) *total_ms = tot + s.graph_ms;
    s.used = 0;
    s.graph_ms = 0.0;
    s.graph_launches = 0;
    return RBF_OK;
}

rbf_status rbf_eval(rbf_ctx* ctx, const double* xe_dev, int64_t m, const double* w_dev, double* s_dev,
                    rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_eval: call rbf_bin first");
    if (ctx->nprob != 1) return fail(ctx, RBF_ERR_STATE, "rbf_eval: the context holds a batch of problems");
    if (m < 0 || m > (int64_t)0x7fffffff - 1)
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_eval: need 0 <= m < 2^31 (m = %lld)", (long long)m);
    if (m == 0) return RBF_OK;
    if (!xe_dev || !w_dev || !s_dev) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_eval: null buffer");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t st = S(stream);
    RBF_CHECK(bin_targets(ctx, xe_dev, m, st));
    EvalBins& E = ctx->ev;
    RBF_CHECK(ensure(ctx, E.w_s, ctx->n));
    RBF_CHECK(ensure(ctx, E.s_s, m));
    RBF_CHECK(permute_to_sorted(ctx, w_dev, E.w_s.p, st));
    RBF_CHECK(eval_sorted_f64(ctx, E.xy_s.p, E.loc.p, E.cell_start.p, E.work.p, E.nwork, E.w_s.p, E.s_s.p, st));
    return targets_to_user(ctx, E.s_s.p, s_dev, st);
}

rbf_status rbf_debug_kernel_pairs(rbf_ctx* ctx, const double* pairs_dev, double* out_dev, int64_t n,
                                  rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_debug_kernel_pairs: call rbf_bin first");
    if (n < 0 || (n > 0 && (!pairs_dev || !out_dev)))
        return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_debug_kernel_pairs: bad buffers");
    if (n == 0) return RBF_OK;
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_LAUNCH(ctx, k_debug_kernel_pairs, blocks_for(n, 256), 256, 0, S(stream), pairs_dev, out_dev, n,
               ctx->prob.p, ctx->fxtab.p);
    return RBF_OK;
}

rbf_status rbf_debug_exp(rbf_ctx* ctx, const double* t_dev, double* out_dev, int64_t n, int variant,
                         rbf_stream stream)
{
    if (!ctx || !t_dev || !out_dev || n < 0 || variant < 0 || variant > 2) return RBF_ERR_INVALID_ARG;
    if (n == 0) return RBF_OK;
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    RBF_LAUNCH(ctx, k_debug_exp, blocks_for(n, 256), 256, 0, S(stream), t_dev, out_dev, n, variant, ctx->expc,
               ctx->exp2048.p, ctx->exp2048_c[0], ctx->exp2048_c[1], ctx->exp2048_c[2]);
    return RBF_OK;
}

rbf_status rbf_get_neighbors(rbf_ctx* ctx, int64_t* ptr_dev, int32_t* idx_dev, int64_t capacity, rbf_stream stream)
{
    if (!ctx) return RBF_ERR_INVALID_ARG;
    if (!ctx->binned) return fail(ctx, RBF_ERR_STATE, "rbf_get_neighbors: call rbf_bin first");
    if (!ptr_dev || !idx_dev || capacity < 0) return fail(ctx, RBF_ERR_INVALID_ARG, "rbf_get_neighbors: bad output");
    RBF_CUDA(ctx, cudaSetDevice(ctx->device));
    int64_t total = 0;
    return neighbor_lists(ctx, ptr_dev, idx_dev, capacity, &total, S(stream));
}

}  // extern "C"
