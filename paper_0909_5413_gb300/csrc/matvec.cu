// matvec.cu -- the truncated Gaussian matvec y = A~ w of Sec. 2.3, matrix-free:
// for each target i (cell order), the sum over the sources j of the
// (2k+1) x (2k+1) neighbour cells with r2_ij <= r_c^2 of
// exp(-r2_ij / (2 sigma^2)) w_j. Each stencil row is one contiguous range of
// cell-ordered sources, read straight from HBM/L2 (no ghost exchange on one GPU).
//
// FP64 kernel. GB300 issues FP64 at 1/73 of the FP32 rate, so the pair's
// kernel value is computed on the integer pipes (fixexp.cuh: exact
// fixed-point offsets, table-driven exp in 64-bit fixed point, FP64 bits
// assembled at the end) and the FP64 pipe only does the accumulate FMA. One
// block per (cell, T targets), T = 32, 64 or 128 (the tile; autotuned with the
// cell size by rbf_tune), with four threads per target (its quarters) mapped
// densely onto the block's 4T threads, so that a cell with fewer than T
// targets leaves whole warps idle rather than lanes of every warp. The
// stencil's sources are staged in shared memory; each target tests its
// candidates in FP32 on scaled cell-local offsets, word w of 32 sources by
// quarter w mod 4 (a thin band around the cutoff is re-tested exactly in FP64
// with the same IEEE operations as the index-list definition), keeping a
// bitmask of accepted sources; each quarter then walks one of four near-equal
// contiguous parts of its target's accepted sources, two per step. The four
// partial sums of a target are added in quarter order (deterministic).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "matvec_sym.cuh"

namespace rbf {
namespace {

constexpr int kMvQ = 4;                        // source quarters of the FP64 kernel
constexpr int kMvStage = 1152;                 // FP64: sources staged per pass at most (3 x 3 cells of ~115 points)
constexpr int kMv32StageMax = 1536;            // FP32: the same
constexpr int kMvMaxRows = 129;                // 2k + 1 with k <= 64

// Stage size for the largest stencil of a binning: rounded up to 32, capped.
inline int round_stage(int stage_max, int cap)
{
    const int s = ((std::max(stage_max, 1) + 31) / 32) * 32;
    return std::min(s, cap);
}

inline int stage_for(const rbf_ctx* ctx, int cap) { return round_stage(ctx->stage_max, cap); }

// Dynamic shared memory of the FP64 kernel for tile T and stage S: tables, staged
// FP64 and fixed-point coordinates, weights, partial sums, FP32 offsets, masks.
__host__ __device__ constexpr size_t mv64_smem(int T, int S)
{
    return 2 * kFxTab * sizeof(unsigned long long) + (size_t)S * (2 * sizeof(double) + 2 * sizeof(long long) +
                                                                   sizeof(double) + 2 * sizeof(float)) +
           (size_t)kMvQ * T * sizeof(double) + (size_t)(S / 32) * T * 4;
}

// The FP64 matvec's pair values kept in device memory: MODE 1 counts, per work
// item of the full list, its value slots and its 32-source words; MODE 2
// stores the accept masks and the kernel values (MODE 4 also forms the product
// with them, as MODE 0 would); MODE 3 replays the matvec from them: the same
// values, the same sums, bit for bit, without the filter or the kernel
// evaluations. The values are laid out for the lockstep walk
// below: per pass, per warp, per step of the walk, 64 doubles, lane l's one or
// two values of that step at 2l and 2l + 1 (a slot of a lane with nothing at
// that step is written as zeros and never read), so that a step loads 512
// contiguous bytes per warp. A warp takes, per pass, as many steps as its
// busiest lane: ceil(share / 2), its share being a quarter of its target's
// accepted sources in the pass.
constexpr int kReplayAhead = 3;   // replay: walk steps whose values are in flight

struct F64Store {
    int64_t* cnt;               // MODE 1: value slots of each item (doubles, a multiple of 64)
    int64_t* nwords;            // MODE 1: 32-source words of each item (all passes)
    const int64_t* val_off;     // MODE 2, 3: first value of each item
    const int64_t* mask_off;    // MODE 2, 3: first word of each item (T masks per word)
    double* val;
    uint32_t* mask;
};

// Exclusive prefix of v over the block's threads in thread order, and the
// block's total. sh: one V per warp.
template <class V>
__device__ __forceinline__ V block_excl_scan(V v, V* sh, V& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwp = blockDim.x >> 5;
    V x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const V u = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += u;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        V z = lane < nwp ? sh[lane] : V(0);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const V u = __shfl_up_sync(0xffffffffu, z, d);
            if (lane >= d) z += u;
        }
        if (lane < nwp) sh[lane] = z;
    }
    __syncthreads();
    const V pre = (wid ? sh[wid - 1] : V(0)) + x - v;
    total = sh[nwp - 1];
    __syncthreads();
    return pre;
}

template <int T, int MODE>
__global__ void __launch_bounds__(T * kMvQ, 256 / T) k_matvec_f64(MvParams P, const double* __restrict__ w,
                                                                 double* __restrict__ y, F64Store FS)
{
    constexpr int kThreads = T * kMvQ;
    constexpr bool kEval = MODE == 0 || MODE == 2 || MODE == 4;   // kernel values computed here
    constexpr bool kFilter = MODE != 3;                            // accept masks computed here
    constexpr bool kStore = MODE == 2 || MODE == 4;                // masks and values written
    constexpr bool kSum = MODE == 0 || MODE == 3 || MODE == 4;     // the product formed
    const int kStage = P.stage;
    extern __shared__ unsigned long long smem_u64[];
    unsigned long long* T1 = smem_u64;
    unsigned long long* T2 = T1 + kFxTab;
    double* SX = (double*)(T2 + kFxTab);
    long long* SXF = (long long*)(SX + 2 * kStage);
    double* SW = (double*)(SXF + 2 * kStage);
    double* PART = SW + kStage;
    float* SF = (float*)(PART + kMvQ * T);
    uint32_t* MASK = (uint32_t*)(SF + 2 * kStage);
    __shared__ int row_beg[kMvMaxRows], row_pre[kMvMaxRows + 1];
    __shared__ long long scan_sh[kThreads / 32];
    __shared__ int CNT[kThreads];   // accepted sources per (quarter, target) in this pass

    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t item = blockIdx.x;
    const int cell = P.work[2 * item], first = P.work[2 * item + 1];
    const int pcell = P.pid_cell[cell];
    if (P.active && !P.active[pcell]) return;   // masked problem (the whole block belongs to it)
    if (kEval)
        for (int i = tid; i < 2 * kFxTab; i += kThreads) T1[i] = P.fxtab[i];
    const Prob& pr = P.prob[pcell];
    const int ncx = (int)pr.ncx, ncy = (int)pr.ncy, kst = pr.k, cbase = (int)pr.cellbase;
    const double rc2 = pr.rc2, knorm = pr.knorm, fxs = pr.fx_scale;
    const int sh = pr.fx_sh, F = pr.fx_F;
    const unsigned long long M = pr.fx_M;
    const float ca = pr.ca, rc2f_lo = pr.rc2f_lo, rc2f_hi = pr.rc2f_hi;
    const int cb = P.tcell_start[cell], ce = P.tcell_start[cell + 1];
    // the item's targets (at most T) and their quarters, densely over the
    // block's threads: thread k < kMvQ * nt takes target k % nt and quarter
    // k / nt; the threads past them (whole warps but one) stay idle
    const int nt = min(T, ce - cb - first);
    const bool active = tid < kMvQ * nt;
    const int t = active ? tid % nt : 0, qtr = active ? tid / nt : 0;
    const int p = cb + first + t;
    const int cx = (cell - cbase) % ncx, cy = (cell - cbase) / ncx;
    const int y0 = max(cy - kst, 0), y1 = min(cy + kst, ncy - 1);
    const int x0 = max(cx - kst, 0), x1 = min(cx + kst, ncx - 1);
    const int nrow = y1 - y0 + 1;
    if (tid == 0) {
        int s = 0;
        for (int r = 0; r < nrow; ++r) {
            int yy = y0 + r;
            int b = P.cell_start[cbase + yy * ncx + x0], e = P.cell_start[cbase + yy * ncx + x1 + 1];
            row_beg[r] = b;
            row_pre[r] = s;
            s += e - b;
        }
        row_pre[nrow] = s;
    }
    double xi = 0.0, yi = 0.0;
    long long xf = 0, yf = 0;
    float fx = 0.f, fy = 0.f;
    if (active && kFilter) {
        xi = P.txy[2 * p];
        yi = P.txy[2 * p + 1];
        xf = fx_coord(xi, fxs, sh);
        yf = fx_coord(yi, fxs, sh);
        fx = P.tloc[2 * p];
        fy = P.tloc[2 * p + 1];
    }
    __syncthreads();
    const int S = row_pre[nrow];
    if (MODE == 1 && tid == 0) FS.nwords[item] = (S + 31) / 32;
    int64_t vbase = (MODE >= 2) ? FS.val_off[item] : 0;   // this pass's first slot (block-uniform)
    long long slots = 0;                                  // MODE 1: this warp's slots so far
    double acc = 0.0;
    for (int base = 0; base < S; base += kStage) {
        const int ns = min(kStage, S - base);
        if (base > 0) __syncthreads();   // the previous pass is done with the staged data
        for (int idx = tid; idx < ns; idx += kThreads) {
            int g = base + idx;
            int r = 0;
            while (r + 1 < nrow && g >= row_pre[r + 1]) ++r;
            int q = row_beg[r] + (g - row_pre[r]);
            if (kFilter) {
                const double qx = P.xy[2 * q], qy = P.xy[2 * q + 1];
                SX[2 * idx] = qx;
                SX[2 * idx + 1] = qy;
                if (kEval) {
                    SXF[2 * idx] = fx_coord(qx, fxs, sh);
                    SXF[2 * idx + 1] = fx_coord(qy, fxs, sh);
                }
                int cq = P.cell_s[q] - cbase;
                // FP32 offsets, two sources per float4: (x_a, x_b, y_a, y_b)
                SF[4 * (idx >> 1) + (idx & 1)] = P.loc[2 * q] + (float)(cq % ncx - cx) * ca;
                SF[4 * (idx >> 1) + 2 + (idx & 1)] = P.loc[2 * q + 1] + (float)(cq / ncx - cy) * ca;
            }
            if (kSum) SW[idx] = w[q];
        }
        __syncthreads();
        const int nw = (ns + 31) >> 5;
        const int64_t mbase = (MODE >= 2) ? (FS.mask_off[item] + (base >> 5)) * T : 0;
        int c = 0;   // accepted sources of this thread's target in its words (q, q + 4, ...)
        if (kFilter && active) {
            // FP32 filter: one accept bit per staged source. Sources in the thin
            // band around the cutoff get a second bit and are settled afterwards
            // by the exact FP64 test, in a loop of its own so that no FP64
            // instruction is issued (predicated or not) for the ordinary
            // candidates. Two candidates per packed f32x2 step; a partial last
            // word is masked.
            const float2 fx2 = make_float2(fx, fx), fy2 = make_float2(fy, fy);
            for (int wi = qtr; wi < nw; wi += kMvQ) {
                uint32_t m = 0, mh = 0;
                const float4* S4 = reinterpret_cast<const float4*>(SF) + wi * 16;
#pragma unroll
                for (int b = 0; b < 32; b += 2) {
                    const float4 v = S4[b >> 1];
                    const float2 dx = f2_sub(fx2, make_float2(v.x, v.y));
                    const float2 dy = f2_sub(fy2, make_float2(v.z, v.w));
                    const float2 r2 = f2_fma(dy, dy, f2_mul(dx, dx));
                    m |= (r2.x < rc2f_lo ? 1u << b : 0u) | (r2.y < rc2f_lo ? 2u << b : 0u);
                    mh |= (r2.x <= rc2f_hi ? 1u << b : 0u) | (r2.y <= rc2f_hi ? 2u << b : 0u);
                }
                const int lim = ns - wi * 32;
                if (lim < 32) {
                    const uint32_t keep = (1u << lim) - 1u;
                    m &= keep;
                    mh &= keep;
                }
                uint32_t band = mh & ~m;
                while (band != 0u) {
                    const int b = __ffs(band) - 1;
                    band &= band - 1u;
                    const int idx = wi * 32 + b;
                    double ex = __dsub_rn(xi, SX[2 * idx]), ey = __dsub_rn(yi, SX[2 * idx + 1]);
                    if (__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) <= rc2) m |= 1u << b;
                }
                MASK[wi * T + t] = m;
                c += __popc(m);
                if (kStore) FS.mask[mbase + (int64_t)wi * T + t] = m;
            }
        } else if (!kFilter && active) {   // MODE 3: the stored masks
            for (int wi = qtr; wi < nw; wi += kMvQ) {
                const uint32_t m = __ldg(FS.mask + mbase + (int64_t)wi * T + t);
                MASK[wi * T + t] = m;
                c += __popc(m);
            }
        }
        if (active) CNT[qtr * T + t] = c;
        __syncthreads();
        // this thread's share of its target's accepted sources in this pass:
        // ranks [lo, hi) in source order, quarter q taking the q-th of four
        // near-equal contiguous parts (word boundaries do not matter)
        int lo = 0, cntq = 0;
        if (active) {
            int n = 0;
#pragma unroll
            for (int q = 0; q < kMvQ; ++q) n += CNT[q * T + t];
            lo = (qtr * n) / kMvQ;
            cntq = ((qtr + 1) * n) / kMvQ - lo;
        }
        const int steps = (cntq + 1) >> 1;   // walk steps: two sources per step
        if (MODE == 1) {
            slots += 64 * (long long)__reduce_max_sync(0xffffffffu, steps);
            continue;
        }
        // the lo-th accepted source: its word wi and the word's bits from it on
        int wi = 0;
        uint32_t cur = 0u;
        if (cntq > 0) {
            int r = lo;
            for (;;) {
                cur = MASK[wi * T + t];
                const int pc = __popc(cur);
                if (r < pc) break;
                r -= pc;
                ++wi;
            }
            for (; r > 0; --r) cur &= cur - 1u;
        }
        // the next accepted source in order (called exactly cntq times)
        auto next_src = [&]() -> int {
            while (cur == 0u) cur = MASK[++wi * T + t];
            const int i = wi * 32 + (__ffs(cur) - 1);
            cur &= cur - 1u;
            return i;
        };
        // this warp's value slots in this pass: after the earlier warps' (warp
        // order), after the block's earlier passes
        int64_t wbase = 0;
        int wsteps = 0;   // MODE 2, 3, 4: the warp's steps (its busiest lane's)
        if (MODE >= 2) {
            wsteps = __reduce_max_sync(0xffffffffu, steps);
            const long long ws = lane == 0 ? 64 * (long long)wsteps : 0LL;
            long long total = 0;
            const long long pre = block_excl_scan(ws, scan_sh, total);
            wbase = vbase + __shfl_sync(0xffffffffu, pre, 0);
            vbase += total;
        }
        // pairs: step s takes the share's sources 2s and 2s + 1 (two
        // independent evaluation chains), accumulated in source order
        auto walk = [&](auto k52) {
            auto kval = [&](int idx) {
                const long long du = (long long)((unsigned long long)xf - (unsigned long long)SXF[2 * idx]);
                const long long dv = (long long)((unsigned long long)yf - (unsigned long long)SXF[2 * idx + 1]);
                if constexpr (decltype(k52)::value) return kernel_fx52(du, dv, M, T1, T2);
                else return kernel_fx(du, dv, F, M, T1, T2);
            };
            if constexpr (kStore) {
                // every lane writes its slot of each of the warp's steps (zeros
                // past its own), 512 contiguous bytes per step
                for (int st = 0; st < wsteps; ++st) {
                    double2 v = make_double2(0.0, 0.0);
                    if (st < steps) {
                        const int i0 = next_src();
                        const bool two = 2 * st + 1 < cntq;
                        const int i1 = two ? next_src() : i0;
                        v.x = kval(i0);
                        if (two) v.y = kval(i1);
                        if constexpr (MODE == 4) {   // the sums of MODE 0
                            acc = fma(v.x, SW[i0], acc);
                            if (two) acc = fma(v.y, SW[i1], acc);
                        }
                    }
                    *reinterpret_cast<double2*>(FS.val + wbase + (int64_t)st * 64 + 2 * lane) = v;
                }
            } else {
                for (int st = 0; st < steps; ++st) {
                    const int i0 = next_src();
                    const bool two = 2 * st + 1 < cntq;
                    const int i1 = two ? next_src() : i0;
                    const double k0 = kval(i0), k1 = kval(i1);
                    acc = fma(k0, SW[i0], acc);
                    if (two) acc = fma(k1, SW[i1], acc);
                }
            }
        };
        if constexpr (MODE == 3) {
            // the same shares over the stored masks, the warp's step count
            // known: a ring of kReplayAhead loads stays in flight, the load of
            // step s + kReplayAhead issued as step s's value is taken (lane
            // l's slot of step s at 64 s + 2 l, as they were stored)
            const double2* vp = reinterpret_cast<const double2*>(FS.val + wbase) + lane;
            double2 kv[kReplayAhead];
#pragma unroll
            for (int k = 0; k < kReplayAhead; ++k)
                kv[k] = k < wsteps ? __ldg(vp + (int64_t)k * 32) : make_double2(0.0, 0.0);
            for (int j0 = 0; j0 < wsteps; j0 += kReplayAhead) {
#pragma unroll
                for (int k = 0; k < kReplayAhead; ++k) {
                    const int st = j0 + k;
                    const double2 v = kv[k];
                    const int nx = st + kReplayAhead;
                    kv[k] = nx < wsteps ? __ldg(vp + (int64_t)nx * 32) : make_double2(0.0, 0.0);
                    if (st < steps) {
                        const int i0 = next_src();
                        acc = fma(v.x, SW[i0], acc);
                        if (2 * st + 1 < cntq) {
                            const int i1 = next_src();
                            acc = fma(v.y, SW[i1], acc);
                        }
                    }
                }
            }
        } else {
            if (F == 52) walk(std::true_type{});   // block-uniform
            else walk(std::false_type{});
        }
    }
    if constexpr (MODE == 1) {
        long long total = 0;
        block_excl_scan(lane == 0 ? slots : 0LL, scan_sh, total);
        if (tid == 0) FS.cnt[item] = total;
    } else if constexpr (kSum) {
        if (active) PART[qtr * T + t] = acc;
        __syncthreads();
        if (active && qtr == 0) y[p] = (((PART[t] + PART[T + t]) + PART[2 * T + t]) + PART[3 * T + t]) * knorm;
    }
}


// FP32 matvec for the inner solves of the mixed form: block per (cell, T
// targets), sources staged in shared memory as FP32 offsets from the target
// cell's corner (scaled so the kernel is exp2(-|dX|^2)), four sources per
// step as two packed f32x2 pairs (three 128-bit shared loads). No cutoff
// mask: every source of the 3 x 3 stencil counts. On cells of side r_c the
// entries this adds beyond r_c are below 2^-53 relative to the diagonal, far
// under FP32 rounding; on the inner grid (cells of side r_i < r_c) every pair
// within r_i counts and the pairs beyond r_i that are dropped are below
// exp(-r_i^2 / (2 sigma^2)) each. The outer FP64 residual uses the exact
// truncated matrix either way.
template <int T>
__global__ void __launch_bounds__(T) k_matvec_f32v2(MvParams P, const float* __restrict__ w, float* __restrict__ y)
{
    const int kStage = P.stage;
    extern __shared__ __align__(16) float smem_f32[];
    float* SXs = smem_f32;                 // kStage + 4 each (16-byte aligned)
    float* SYs = SXs + kStage + 4;
    float* SWs = SYs + kStage + 4;
    __shared__ int row_beg[kMvMaxRows], row_pre[kMvMaxRows + 1];
    const int tid = threadIdx.x;
    const int cell = P.work[2 * blockIdx.x], first = P.work[2 * blockIdx.x + 1];
    const int pcell = P.pid_cell[cell];
    if (P.active && !P.active[pcell]) return;   // masked problem (the whole block belongs to it)
    const Prob& pr = P.prob[pcell];
    const int ncx = (int)pr.ncx, ncy = (int)pr.ncy, kst = pr.k, cbase = (int)pr.cellbase;
    const float ca = pr.ca, knorm = (float)pr.knorm;
    const int cb = P.cell_start[cell], ce = P.cell_start[cell + 1];
    const int p = cb + first + tid;
    const bool active = p < ce;
    const int cx = (cell - cbase) % ncx, cy = (cell - cbase) / ncx;
    const int y0 = max(cy - kst, 0), y1 = min(cy + kst, ncy - 1);
    const int x0 = max(cx - kst, 0), x1 = min(cx + kst, ncx - 1);
    const int nrow = y1 - y0 + 1;
    if (tid == 0) {
        int s = 0;
        for (int r = 0; r < nrow; ++r) {
            int yy = y0 + r;
            int b = P.cell_start[cbase + yy * ncx + x0], e = P.cell_start[cbase + yy * ncx + x1 + 1];
            row_beg[r] = b;
            row_pre[r] = s;
            s += e - b;
        }
        row_pre[nrow] = s;
    }
    float2 t2 = make_float2(0.f, 0.f), u2 = make_float2(0.f, 0.f);
    if (active) {
        float fx = P.loc[2 * p], fy = P.loc[2 * p + 1];
        t2 = make_float2(fx, fx);
        u2 = make_float2(fy, fy);
    }
    __syncthreads();
    const int S = row_pre[nrow];
    float2 acc2 = make_float2(0.f, 0.f), acc2b = make_float2(0.f, 0.f);
    for (int base = 0; base < S; base += kStage) {
        const int ns = min(kStage, S - base);
        if (base > 0) __syncthreads();
        for (int idx = tid; idx < ns; idx += T) {
            const int g = base + idx;
            int r = 0;
            while (r + 1 < nrow && g >= row_pre[r + 1]) ++r;
            const int q = row_beg[r] + (g - row_pre[r]);
            const int yy = y0 + r;                           // the stencil row gives the cell's y
            const int xq = P.cell_s[q] - cbase - yy * ncx;   // and its x
            const float2 l = reinterpret_cast<const float2*>(P.loc)[q];
            SXs[idx] = l.x + (float)(xq - cx) * ca;
            SYs[idx] = l.y + (float)(yy - cy) * ca;
            SWs[idx] = w[q];
        }
        if (tid < ((4 - (ns & 3)) & 3)) {   // pad to a multiple of 4 with far, zero-weight sources
            SXs[ns + tid] = 1.0e4f;
            SYs[ns + tid] = 1.0e4f;
            SWs[ns + tid] = 0.0f;
        }
        __syncthreads();
        const int ns4 = (ns + 3) >> 2;
#pragma unroll 8
        for (int s = 0; s < ns4; ++s) {
            const float4 sx = reinterpret_cast<const float4*>(SXs)[s];
            const float4 sy = reinterpret_cast<const float4*>(SYs)[s];
            const float4 sw = reinterpret_cast<const float4*>(SWs)[s];
            const float2 dx0 = f2_sub(t2, make_float2(sx.x, sx.y)), dy0 = f2_sub(u2, make_float2(sy.x, sy.y));
            const float2 dx1 = f2_sub(t2, make_float2(sx.z, sx.w)), dy1 = f2_sub(u2, make_float2(sy.z, sy.w));
            const float2 r0 = f2_fma(dy0, dy0, f2_mul(dx0, dx0));
            const float2 r1 = f2_fma(dy1, dy1, f2_mul(dx1, dx1));
            const float2 e0 = make_float2(ex2_approx(-r0.x), ex2_approx(-r0.y));
            const float2 e1 = make_float2(ex2_approx(-r1.x), ex2_approx(-r1.y));
            acc2 = f2_fma(e0, make_float2(sw.x, sw.y), acc2);
            acc2b = f2_fma(e1, make_float2(sw.z, sw.w), acc2b);
        }
    }
    if (active) y[p] = ((acc2.x + acc2.y) + (acc2b.x + acc2b.y)) * knorm;
}

// One warp per cell of one size class (TPL targets per lane, 32 (TPL - 1) <
// points <= 32 TPL): the list holds (cell, 0) items of that class, and each
// class has a kernel of its own register budget.
template <int TPL>
__global__ void __launch_bounds__(kSymWarps * 32, TPL == 1 ? 8 : (TPL == 2 ? 8 : 4))
    k_matvec_f32_sym(MvParams P, const int32_t* __restrict__ cells, int64_t ncells, const float* __restrict__ w,
                     float* __restrict__ rowslot, float* __restrict__ colslot, int64_t n)
{
    __shared__ __align__(16) SymWarp sm_all[kSymWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kSymWarps + warp;
    if (item >= ncells) return;
    const int cell = cells[2 * item];
    const int pcell = P.pid_cell[cell];
    if (P.active && !P.active[pcell]) return;
    const Prob& pr = P.prob[pcell];
    const int cb = P.cell_start[cell], cnt = P.cell_start[cell + 1] - cb;
    sym_cell<TPL>(P, sm_all[warp], lane, cell, cb, cnt, pr, w, rowslot, colslot, n);
}

// y_p = row slot + the four column slots in the order of d (a missing
// backward neighbour's slot holds zero); the slots already carry the
// normalisation. Points of masked problems, and of problems the symmetric
// kernel does not serve (served[b] == 0), are left alone.
__global__ void k_sym_gather(const float* __restrict__ rowslot, const float* __restrict__ colslot, int64_t n,
                             const int32_t* __restrict__ pid, const int32_t* __restrict__ active,
                             const int32_t* __restrict__ served, float* __restrict__ y)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int pb = pid[p];
    if ((active && !active[pb]) || !served[pb]) return;
    y[p] = (((rowslot[p] + colslot[p]) + colslot[n + p]) + colslot[2 * n + p]) + colslot[3 * n + p];
}

// Symmetric FP64 matvec (the exact truncated operator): one warp per cell C of
// at most 160 points (TPL = ceil(points / 32) targets per lane), with the 3 x
// 3 stencil of cells as wide as r_c. As in the FP32 kernel, C takes itself (row
// sums only) and its four forward neighbours D; each accepted pair (i, j) --
// the packed FP32 filter, the exact FP64 pair test in the thin band around
// r_c -- gets its kernel value once, by the fixed-point evaluation, which
// feeds i's row sum (registers) and, through the lane's row of a shared FP64
// tile (lane i adds k_ij w_i at column j), j's column sum: lane j adds the
// warp's 32 rows in order. A missing backward neighbour's slot gets zero.
// FP64 work stays one FMA per directed pair (row or column), the integer
// work of the kernel values is halved.
constexpr int kSym64Warps = 4;
constexpr int kSym64Stage = 160 + 32;
constexpr int kSym64Tld = 33;

struct Sym64Warp {
    double sx[2 * kSym64Stage];          // staged FP64 coordinates (x, y) for the exact band test
    long long sxf[2 * kSym64Stage];      // pre-shifted fixed-point coordinates
    double sw[kSym64Stage];
    float sf[2 * kSym64Stage];           // FP32 offsets from C's corner, (x_a, x_b, y_a, y_b) per source pair
    double T[32 * kSym64Tld];            // column tile: lane r's contributions at columns 0..31
};

template <int TPL, bool COL, bool F52>
__device__ __forceinline__ void sym64_pass(Sym64Warp& S, int lane, const Prob& pr, const unsigned long long* T1,
                                           const unsigned long long* T2, const double (&xi)[TPL],
                                           const double (&yi)[TPL], const long long (&xf)[TPL],
                                           const long long (&yf)[TPL], const float (&fx)[TPL], const float (&fy)[TPL],
                                           const double (&wt)[TPL], double (&acc)[TPL], int dn,
                                           double* __restrict__ colout, double knorm)
{
    const double rc2 = pr.rc2;
    const float rc2f_lo = pr.rc2f_lo, rc2f_hi = pr.rc2f_hi;
    const int F = pr.fx_F;
    const unsigned long long M = pr.fx_M;
    const int nw = (dn + 31) >> 5;
    for (int wi = 0; wi < nw; ++wi) {
        if (COL) {
#pragma unroll 8
            for (int b = 0; b < 32; ++b) S.T[lane * kSym64Tld + b] = 0.0;
        }
        const int lim = dn - wi * 32;
        const float4* S4 = reinterpret_cast<const float4*>(S.sf) + wi * 16;
#pragma unroll
        for (int t = 0; t < TPL; ++t) {
            // FP32 filter of the word's 32 sources against target t, the band settled in FP64
            uint32_t m = 0, mh = 0;
            const float2 fx2 = make_float2(fx[t], fx[t]), fy2 = make_float2(fy[t], fy[t]);
#pragma unroll
            for (int b = 0; b < 32; b += 2) {
                const float4 v = S4[b >> 1];
                const float2 dx = f2_sub(fx2, make_float2(v.x, v.y));
                const float2 dy = f2_sub(fy2, make_float2(v.z, v.w));
                const float2 r2 = f2_fma(dy, dy, f2_mul(dx, dx));
                m |= (r2.x < rc2f_lo ? 1u << b : 0u) | (r2.y < rc2f_lo ? 2u << b : 0u);
                mh |= (r2.x <= rc2f_hi ? 1u << b : 0u) | (r2.y <= rc2f_hi ? 2u << b : 0u);
            }
            if (lim < 32) {
                const uint32_t keep = (1u << lim) - 1u;
                m &= keep;
                mh &= keep;
            }
            uint32_t band = mh & ~m;
            while (band != 0u) {
                const int b = __ffs(band) - 1;
                band &= band - 1u;
                const int idx = wi * 32 + b;
                const double ex = __dsub_rn(xi[t], S.sx[2 * idx]), ey = __dsub_rn(yi[t], S.sx[2 * idx + 1]);
                if (__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) <= rc2) m |= 1u << b;
            }
            // the accepted sources, two per step, the warp in lockstep
            uint32_t cur = m;
            for (;;) {
                const bool has = cur != 0u;
                if (!__any_sync(0xffffffffu, has)) break;
                if (has) {
                    const int b0 = __ffs(cur) - 1;
                    cur &= cur - 1u;
                    const bool two = cur != 0u;
                    const int b1 = two ? __ffs(cur) - 1 : b0;
                    cur &= cur - (two ? 1u : 0u);
                    const int i0 = wi * 32 + b0, i1 = wi * 32 + b1;
                    const long long du0 = (long long)((unsigned long long)xf[t] - (unsigned long long)S.sxf[2 * i0]);
                    const long long dv0 = (long long)((unsigned long long)yf[t] - (unsigned long long)S.sxf[2 * i0 + 1]);
                    const long long du1 = (long long)((unsigned long long)xf[t] - (unsigned long long)S.sxf[2 * i1]);
                    const long long dv1 = (long long)((unsigned long long)yf[t] - (unsigned long long)S.sxf[2 * i1 + 1]);
                    double k0, k1;
                    if (F52) {
                        k0 = kernel_fx52(du0, dv0, M, T1, T2);
                        k1 = kernel_fx52(du1, dv1, M, T1, T2);
                    } else {
                        k0 = kernel_fx(du0, dv0, F, M, T1, T2);
                        k1 = kernel_fx(du1, dv1, F, M, T1, T2);
                    }
                    acc[t] = fma(k0, S.sw[i0], acc[t]);
                    if (two) acc[t] = fma(k1, S.sw[i1], acc[t]);
                    if (COL) {
                        double* row = S.T + lane * kSym64Tld;
                        row[b0] = fma(k0, wt[t], row[b0]);
                        if (two) row[b1] = fma(k1, wt[t], row[b1]);
                    }
                }
            }
        }
        if (COL) {
            __syncwarp();
            double sum = 0.0;
#pragma unroll 8
            for (int r = 0; r < 32; ++r) sum += S.T[r * kSym64Tld + lane];
            __syncwarp();
            if (lane < lim) colout[wi * 32 + lane] = sum * knorm;
        }
    }
}

template <int TPL, bool F52>
__device__ __forceinline__ void sym64_cell(const MvParams& P, Sym64Warp& S, int lane, int cell, int cb, int cnt,
                                           const Prob& pr, const double* __restrict__ w, double* __restrict__ rowslot,
                                           double* __restrict__ colslot, int64_t n)
{
    const int ncx = (int)pr.ncx, ncy = (int)pr.ncy, cbase = (int)pr.cellbase;
    const float ca = pr.ca;
    const double knorm = pr.knorm, fxs = pr.fx_scale;
    const int sh = pr.fx_sh;
    const int cx = (cell - cbase) % ncx, cy = (cell - cbase) / ncx;
    double xi[TPL], yi[TPL], wt[TPL], acc[TPL];
    long long xf[TPL], yf[TPL];
    float fx[TPL], fy[TPL];
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int q = lane + 32 * t;
        const bool ok = q < cnt;
        const int p = cb + (ok ? q : 0);
        xi[t] = P.xy[2 * (int64_t)p];
        yi[t] = P.xy[2 * (int64_t)p + 1];
        xf[t] = fx_coord(xi[t], fxs, sh);
        yf[t] = fx_coord(yi[t], fxs, sh);
        fx[t] = ok ? P.loc[2 * (int64_t)p] : -1.0e4f;   // a missing target accepts no source
        fy[t] = ok ? P.loc[2 * (int64_t)p + 1] : -1.0e4f;
        wt[t] = ok ? w[p] : 0.0;
        acc[t] = 0.0;
    }
    {   // zero slots of the backward directions whose source cell is missing
        const int bx[4] = {cx - 1, cx + 1, cx, cx - 1}, by[4] = {cy, cy - 1, cy - 1, cy - 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bool missing = bx[q] < 0 || bx[q] >= ncx || by[q] < 0;
            if (!missing) {
                const int c = cbase + by[q] * ncx + bx[q];
                missing = P.cell_start[c + 1] == P.cell_start[c];
            }
            if (missing)
                for (int t = lane; t < cnt; t += 32) colslot[(int64_t)q * n + cb + t] = 0.0;
        }
    }
    const unsigned long long* T1 = P.fxtab;
    const unsigned long long* T2 = P.fxtab + kFxTab;
#pragma unroll 1
    for (int pass = 0; pass < 5; ++pass) {
        const int dx = (pass == 1 || pass == 4) ? 1 : (pass == 2 ? -1 : 0);
        const int dy = pass >= 2 ? 1 : 0;
        const int nx = cx + dx, ny = cy + dy;
        if (nx < 0 || nx >= ncx || ny >= ncy) continue;
        const int dcell = cbase + ny * ncx + nx;
        const int db = P.cell_start[dcell], dn = P.cell_start[dcell + 1] - db;
        if (dn == 0) continue;
        const int dnp = (dn + 31) & ~31;
        for (int s = lane; s < dnp; s += 32) {
            float lx = 1.0e4f, ly = 1.0e4f;
            if (s < dn) {
                const int64_t q = db + s;
                const double x = P.xy[2 * q], y = P.xy[2 * q + 1];
                S.sx[2 * s] = x;
                S.sx[2 * s + 1] = y;
                S.sxf[2 * s] = fx_coord(x, fxs, sh);
                S.sxf[2 * s + 1] = fx_coord(y, fxs, sh);
                S.sw[s] = w[q];
                lx = P.loc[2 * q] + (float)dx * ca;
                ly = P.loc[2 * q + 1] + (float)dy * ca;
            } else {
                S.sw[s] = 0.0;
            }
            S.sf[4 * (s >> 1) + (s & 1)] = lx;
            S.sf[4 * (s >> 1) + 2 + (s & 1)] = ly;
        }
        __syncwarp();
        if (pass == 0)
            sym64_pass<TPL, false, F52>(S, lane, pr, T1, T2, xi, yi, xf, yf, fx, fy, wt, acc, dn, nullptr, knorm);
        else
            sym64_pass<TPL, true, F52>(S, lane, pr, T1, T2, xi, yi, xf, yf, fx, fy, wt, acc, dn,
                                       colslot + (int64_t)(pass - 1) * n + db, knorm);
        __syncwarp();
    }
#pragma unroll
    for (int t = 0; t < TPL; ++t) {
        const int q = lane + 32 * t;
        if (q < cnt) rowslot[cb + q] = acc[t] * knorm;
    }
}

template <int TPL>
__global__ void __launch_bounds__(kSym64Warps * 32)
    k_matvec_f64_sym(MvParams P, const int32_t* __restrict__ cells, int64_t ncells, const double* __restrict__ w,
                     double* __restrict__ rowslot, double* __restrict__ colslot, int64_t n)
{
    extern __shared__ __align__(16) unsigned char sym64_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * kSym64Warps + warp;
    if (item >= ncells) return;
    const int cell = cells[2 * item];
    const int pcell = P.pid_cell[cell];
    if (P.active && !P.active[pcell]) return;
    const Prob& pr = P.prob[pcell];
    const int cb = P.cell_start[cell], cnt = P.cell_start[cell + 1] - cb;
    Sym64Warp& S = reinterpret_cast<Sym64Warp*>(sym64_raw)[warp];
    if (pr.fx_F == 52) sym64_cell<TPL, true>(P, S, lane, cell, cb, cnt, pr, w, rowslot, colslot, n);
    else sym64_cell<TPL, false>(P, S, lane, cell, cb, cnt, pr, w, rowslot, colslot, n);
}

// y_p = row slot + the four column slots in the order of d (each already
// carrying the normalisation), for the points of the problems the symmetric
// kernel serves; points of masked problems are left alone.
__global__ void k_sym64_gather(const double* __restrict__ rowslot, const double* __restrict__ colslot, int64_t n,
                               const int32_t* __restrict__ pid, const int32_t* __restrict__ active,
                               const int32_t* __restrict__ served, double* __restrict__ y)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int pb = pid[p];
    if ((active && !active[pb]) || !served[pb]) return;   // served: the problems of the symmetric kernel
    y[p] = (((rowslot[p] + colslot[p]) + colslot[n + p]) + colslot[2 * n + p]) + colslot[3 * n + p];
}

__global__ void k_to_f32(const double* __restrict__ in, int64_t n, float* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)in[i];
}

__global__ void k_to_f64(const float* __restrict__ in, int64_t n, double* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

MvParams mv_params(const rbf_ctx* ctx)
{
    MvParams P;
    P.xy = ctx->xy_s.p;
    P.loc = ctx->loc32.p;
    P.cell_s = ctx->cell_s.p;
    P.cell_start = ctx->cell_start.p;
    P.work = ctx->mv_work.p;
    P.txy = ctx->xy_s.p;
    P.tloc = ctx->loc32.p;
    P.tcell_start = ctx->cell_start.p;
    P.fxtab = ctx->fxtab.p;
    P.prob = ctx->prob.p;
    P.pid_cell = ctx->pid_cell.p;
    P.active = ctx->active_mask;
    P.stage = 0;
    return P;
}

template <int T, int MODE>
rbf_status prepare_f64_mode(rbf_ctx* ctx)
{
    RBF_CUDA(ctx, cudaFuncSetAttribute(k_matvec_f64<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)mv64_smem(T, kMvStage)));
    RBF_CUDA(ctx, cudaFuncSetAttribute(k_matvec_f64<T, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       cudaSharedmemCarveoutMaxShared));
    return RBF_OK;
}

template <int T>
rbf_status prepare_f64(rbf_ctx* ctx)
{
    RBF_CHECK((prepare_f64_mode<T, 0>(ctx)));
    RBF_CHECK((prepare_f64_mode<T, 1>(ctx)));
    RBF_CHECK((prepare_f64_mode<T, 2>(ctx)));
    RBF_CHECK((prepare_f64_mode<T, 3>(ctx)));
    return prepare_f64_mode<T, 4>(ctx);
}

template <int T, int MODE>
rbf_status launch_f64(rbf_ctx* ctx, const MvParams& P, int64_t nwork, const double* w, double* y,
                      const F64Store& FS, cudaStream_t st)
{
    RBF_LAUNCH(ctx, (k_matvec_f64<T, MODE>), (unsigned)nwork, T * kMvQ, mv64_smem(T, P.stage), st, P, w, y, FS);
    return RBF_OK;
}

template <int MODE>
rbf_status dispatch_f64_mode(rbf_ctx* ctx, MvParams P, int64_t nwork, const double* w, double* y, const F64Store& FS,
                             cudaStream_t st)
{
    if (nwork == 0) return RBF_OK;
    P.stage = stage_for(ctx, kMvStage);
    switch (ctx->tile64) {
    case 32: return launch_f64<32, MODE>(ctx, P, nwork, w, y, FS, st);
    case 64: return launch_f64<64, MODE>(ctx, P, nwork, w, y, FS, st);
    default: return launch_f64<128, MODE>(ctx, P, nwork, w, y, FS, st);
    }
}

rbf_status dispatch_f64(rbf_ctx* ctx, MvParams P, int64_t nwork, const double* w, double* y, cudaStream_t st)
{
    return dispatch_f64_mode<0>(ctx, P, nwork, w, y, F64Store{}, st);
}

template <int T>
rbf_status launch_f32(rbf_ctx* ctx, MvParams P, int64_t nwork, const float* w, float* y, cudaStream_t st)
{
    const size_t smem = 3 * (size_t)(P.stage + 4) * sizeof(float);
    RBF_LAUNCH(ctx, k_matvec_f32v2<T>, (unsigned)nwork, T, smem, st, P, w, y);
    return RBF_OK;
}

}  // namespace

bool inner_sym_params(rbf_ctx* ctx, MvParams* P, const int32_t** cells, int64_t* ncells)
{
    if (!ctx->inner_on || !ctx->in.sym_all || ctx->sym_mode == 1) return false;
    const InnerGrid& G = ctx->in;
    *P = mv_params(ctx);
    P->loc = G.loc.p;
    P->cell_s = G.cell_s.p;
    P->cell_start = G.cell_start.p;
    P->prob = G.prob.p;
    P->pid_cell = G.pid_cell.p;
    *cells = ctx->al.on ? ctx->al.symw.p : G.symw.p;
    *ncells = ctx->al.on ? ctx->al.symoff[4] : G.symoff[4];
    return true;
}

template <int TPL>
static rbf_status prepare_sym64(rbf_ctx* ctx)
{
    RBF_CUDA(ctx, cudaFuncSetAttribute(k_matvec_f64_sym<TPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(sizeof(Sym64Warp) * kSym64Warps)));
    return RBF_OK;
}

rbf_status matvec_prepare(rbf_ctx* ctx)
{
    RBF_CHECK(prepare_f64<32>(ctx));
    RBF_CHECK(prepare_f64<64>(ctx));
    RBF_CHECK(prepare_f64<128>(ctx));
    RBF_CHECK(prepare_sym64<1>(ctx));
    RBF_CHECK(prepare_sym64<2>(ctx));
    RBF_CHECK(prepare_sym64<3>(ctx));
    RBF_CHECK(prepare_sym64<4>(ctx));
    return prepare_sym64<5>(ctx);
}

rbf_status matvec_sorted_f64_plain(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st)
{
    if (ctx->sym64 && ctx->sym64_mode == 0) {
        // each neighbouring pair of cells once, then the fixed-order gather, for
        // the problems the symmetric kernel serves; the stencil kernel for the others
        const int64_t n = ctx->n;
        if (ctx->sym64_slots.count < (size_t)(5 * n))
            return fail(ctx, RBF_ERR_STATE, "symmetric FP64 matvec: slots not allocated");
        MvParams P = mv_params(ctx);
        double* rowslot = ctx->sym64_slots.p;
        double* colslot = rowslot + n;
        const size_t smem = sizeof(Sym64Warp) * kSym64Warps;
        const int32_t* lists = ctx->al.on ? ctx->al.sym64w.p : ctx->sym64w.p;
        const int64_t* off = ctx->al.on ? ctx->al.sym64off : ctx->sym64off;
        for (int t = 1; t <= 5; ++t) {
            const int64_t cnt = off[t] - off[t - 1];
            if (cnt == 0) continue;
            const int32_t* cl = lists + 2 * off[t - 1];
            const unsigned nb = blocks_for(cnt, kSym64Warps);
            switch (t) {
            case 1: RBF_LAUNCH(ctx, k_matvec_f64_sym<1>, nb, kSym64Warps * 32, smem, st, P, cl, cnt, w, rowslot, colslot, n); break;
            case 2: RBF_LAUNCH(ctx, k_matvec_f64_sym<2>, nb, kSym64Warps * 32, smem, st, P, cl, cnt, w, rowslot, colslot, n); break;
            case 3: RBF_LAUNCH(ctx, k_matvec_f64_sym<3>, nb, kSym64Warps * 32, smem, st, P, cl, cnt, w, rowslot, colslot, n); break;
            case 4: RBF_LAUNCH(ctx, k_matvec_f64_sym<4>, nb, kSym64Warps * 32, smem, st, P, cl, cnt, w, rowslot, colslot, n); break;
            default: RBF_LAUNCH(ctx, k_matvec_f64_sym<5>, nb, kSym64Warps * 32, smem, st, P, cl, cnt, w, rowslot, colslot, n);
            }
        }
        RBF_LAUNCH(ctx, k_sym64_gather, blocks_for(n, 256), 256, 0, st, rowslot, colslot, n, ctx->pid.p, P.active,
                   ctx->sym64_prob.p, y);
        if (ctx->sym64_all) return RBF_OK;
        MvParams Q = mv_params(ctx);
        Q.work = ctx->al.on ? ctx->al.w64ns.p : ctx->mv_work_ns.p;
        return dispatch_f64(ctx, Q, ctx->al.on ? ctx->al.n64ns : ctx->n_work_ns, w, y, st);
    }
    if (ctx->al.on) {   // batched solve: only the work items of active problems
        MvParams P = mv_params(ctx);
        P.work = ctx->al.w64.p;
        return dispatch_f64(ctx, P, ctx->al.n64, w, y, st);
    }
    if (ctx->f64s.valid && ctx->f64s.tile == ctx->tile64) {   // the kept pair values, the same sums
        F64Store FS{};
        FS.val_off = ctx->f64s.val_off.p;
        FS.mask_off = ctx->f64s.mask_off.p;
        FS.val = ctx->f64s.val.p;
        FS.mask = ctx->f64s.mask.p;
        return dispatch_f64_mode<3>(ctx, mv_params(ctx), ctx->n_work, w, y, FS, st);
    }
    return dispatch_f64(ctx, mv_params(ctx), ctx->n_work, w, y, st);
}

void f64_store_release(rbf_ctx* ctx)
{
    F64Keep& K = ctx->f64s;
    K.valid = false;
    release(ctx, K.val.p);
    K.val = {};
    release(ctx, K.mask.p);
    K.mask = {};
}

namespace {

// Counts and keeps the pair values of the current binning when they fit; with
// w, forms y = A~ w from them in the same pass (*formed). Nothing is kept, and
// *formed stays false, when the option is off, the values are kept already,
// the symmetric FP64 kernel serves the products, a cycle is being captured, or
// (with w) a batched solve runs on the lists of its active problems.
rbf_status f64_store_build(rbf_ctx* ctx, const double* w, double* y, bool* formed, cudaStream_t st)
{
    *formed = false;
    F64Keep& K = ctx->f64s;
    if (ctx->store_mode == 0 || (K.valid && K.tile == ctx->tile64) || K.tried || ctx->n_work == 0) return RBF_OK;
    if (ctx->sym64 && ctx->sym64_mode == 0) return RBF_OK;   // the symmetric kernel serves those problems
    if (ctx->capturing || (w && ctx->al.on)) return RBF_OK;
    K.valid = false;
    const int64_t nwork = ctx->n_work;
    MvParams P = mv_params(ctx);
    P.active = nullptr;   // every problem's pairs
    RBF_CHECK(ensure(ctx, K.cnt, (size_t)nwork + 1));
    RBF_CHECK(ensure(ctx, K.nwords, (size_t)nwork + 1));
    RBF_CHECK(ensure(ctx, K.val_off, (size_t)nwork + 1));
    RBF_CHECK(ensure(ctx, K.mask_off, (size_t)nwork + 1));
    F64Store FS{};
    FS.cnt = K.cnt.p;
    FS.nwords = K.nwords.p;
    RBF_CHECK(dispatch_f64_mode<1>(ctx, P, nwork, nullptr, nullptr, FS, st));
    RBF_CHECK(exclusive_scan_i64(ctx, K.cnt.p, K.val_off.p, nwork, st));
    RBF_CHECK(exclusive_scan_i64(ctx, K.nwords.p, K.mask_off.p, nwork, st));
    int64_t tot[2] = {0, 0};
    RBF_CUDA(ctx, cudaMemcpyAsync(&tot[0], K.val_off.p + nwork, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaMemcpyAsync(&tot[1], K.mask_off.p + nwork, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RBF_CUDA(ctx, cudaStreamSynchronize(st));
    const int64_t nmask = tot[1] * ctx->tile64;
    const size_t need = (size_t)tot[0] * sizeof(double) + (size_t)nmask * sizeof(uint32_t);
    // only when it fits beside everything else: the device's free memory less
    // a margin (and the context's own limit); otherwise the matvec stays
    // matrix-free
    size_t free_b = 0, total_b = 0;
    RBF_CUDA(ctx, cudaMemGetInfo(&free_b, &total_b));
    const size_t have = (K.val.count * sizeof(double) + K.mask.count * sizeof(uint32_t));
    const size_t margin = (size_t)8 << 30;
    const bool fits = !(need > have && need - have + margin > free_b) &&
                      !(ctx->mem_limit > 0 && ctx->dev_bytes + (int64_t)(need > have ? need - have : 0) > ctx->mem_limit);
    if (!fits) {
        K.tried = true;   // the later products of this binning stay matrix-free without counting again
        return RBF_OK;
    }
    // an allocation that fails all the same (the device shared with another
    // process) leaves the matvec matrix-free rather than failing the solve
    if (ensure(ctx, K.val, (size_t)tot[0]) != RBF_OK || ensure(ctx, K.mask, (size_t)nmask) != RBF_OK) {
        f64_store_release(ctx);
        K.tried = true;
        return RBF_OK;
    }
    FS = F64Store{};
    FS.val_off = K.val_off.p;
    FS.mask_off = K.mask_off.p;
    FS.val = K.val.p;
    FS.mask = K.mask.p;
    if (w) {
        RBF_CHECK(dispatch_f64_mode<4>(ctx, P, nwork, w, y, FS, st));
        *formed = true;
    } else {
        RBF_CHECK(dispatch_f64_mode<2>(ctx, P, nwork, nullptr, nullptr, FS, st));
    }
    K.valid = true;
    K.tile = ctx->tile64;
    K.bytes = (int64_t)need;
    return RBF_OK;
}

rbf_status f64_store_build_timed(rbf_ctx* ctx, const double* w, double* y, bool* formed, cudaStream_t st)
{
    *formed = false;
    const F64Keep& K = ctx->f64s;
    if (ctx->store_mode == 0 || (K.valid && K.tile == ctx->tile64) || K.tried) return RBF_OK;   // nothing to time
    RBF_CHECK(prof_begin(ctx, RBF_PROF_STORE_F64, st));
    RBF_CHECK(f64_store_build(ctx, w, y, formed, st));
    return prof_end(ctx, RBF_PROF_STORE_F64, st);
}

}  // namespace

rbf_status f64_store_prepare(rbf_ctx* ctx, cudaStream_t st)
{
    bool formed = false;
    return f64_store_build_timed(ctx, nullptr, nullptr, &formed, st);
}

rbf_status matvec_sorted_f64_keep(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st)
{
    bool formed = false;
    RBF_CHECK(f64_store_build_timed(ctx, w, y, &formed, st));
    return formed ? RBF_OK : matvec_sorted_f64(ctx, w, y, st);
}

// s = sum_j k(|t - x_j|) w_j for the cell-sorted targets of another point
// set binned into the same grid (txy, tloc, tcell_start, twork, nwork).
rbf_status eval_sorted_f64(rbf_ctx* ctx, const double* txy, const float* tloc, const int32_t* tcell_start,
                           const int32_t* twork, int64_t nwork, const double* w, double* s, cudaStream_t st)
{
    MvParams P = mv_params(ctx);
    P.work = twork;
    P.txy = txy;
    P.tloc = tloc;
    P.tcell_start = tcell_start;
    return dispatch_f64(ctx, P, nwork, w, s, st);
}

rbf_status matvec_sorted_f64(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st)
{
    RBF_CHECK(prof_begin(ctx, RBF_PROF_MATVEC_F64, st));
    RBF_CHECK(matvec_sorted_f64_plain(ctx, w, y, st));
    return prof_end(ctx, RBF_PROF_MATVEC_F64, st);
}

rbf_status ensure_local_coords(rbf_ctx* ctx, float2** loc, cudaStream_t)
{
    *loc = (float2*)ctx->loc32.p;
    return RBF_OK;
}

rbf_status matvec_f32_raw(rbf_ctx* ctx, const float2*, const float* w, float* y, cudaStream_t st)
{
    RBF_CHECK(prof_begin(ctx, RBF_PROF_MATVEC_F32, st));
    MvParams P = mv_params(ctx);
    int tile = ctx->tile32;
    int64_t nwork = ctx->n_work32;
    P.work = ctx->mv_work32.p;
    P.stage = stage_for(ctx, kMv32StageMax);
    if (ctx->inner_on) {   // the mixed form's inner grid (shorter cutoff, its own order)
        const InnerGrid& G = ctx->in;
        P.loc = G.loc.p;
        P.cell_s = G.cell_s.p;
        P.cell_start = G.cell_start.p;
        P.work = G.work.p;
        P.prob = G.prob.p;
        P.pid_cell = G.pid_cell.p;
        P.stage = round_stage(G.stage_max, kMv32StageMax);
        tile = G.tile;
        nwork = G.n_work;
    }
    if (ctx->al.on) {   // batched solve: only the work items of active problems
        P.work = ctx->al.w32.p;
        nwork = ctx->al.n32;
    }
    if (nwork > 0 && ctx->inner_on && ctx->in.sym && ctx->sym_mode != 1) {
        // each neighbouring pair of inner cells once, then the fixed-order gather
        const int64_t n = ctx->n;
        if (ctx->sym_slots.count < (size_t)(5 * n))   // allocated with the inner grid (never inside a capture)
            return fail(ctx, RBF_ERR_STATE, "symmetric FP32 matvec: slots not allocated");
        float* rowslot = ctx->sym_slots.p;
        float* colslot = rowslot + n;
        const InnerGrid& G = ctx->in;
        const int32_t* lists = ctx->al.on ? ctx->al.symw.p : G.symw.p;
        const int64_t* off = ctx->al.on ? ctx->al.symoff : G.symoff;
        for (int t = 1; t <= 4; ++t) {
            const int64_t cnt = off[t] - off[t - 1];
            if (cnt == 0) continue;
            const int32_t* cl = lists + 2 * off[t - 1];
            const unsigned nb = blocks_for(cnt, kSymWarps);
            switch (t) {
            case 1: RBF_LAUNCH(ctx, k_matvec_f32_sym<1>, nb, kSymWarps * 32, 0, st, P, cl, cnt, w, rowslot, colslot, n); break;
            case 2: RBF_LAUNCH(ctx, k_matvec_f32_sym<2>, nb, kSymWarps * 32, 0, st, P, cl, cnt, w, rowslot, colslot, n); break;
            case 3: RBF_LAUNCH(ctx, k_matvec_f32_sym<3>, nb, kSymWarps * 32, 0, st, P, cl, cnt, w, rowslot, colslot, n); break;
            default: RBF_LAUNCH(ctx, k_matvec_f32_sym<4>, nb, kSymWarps * 32, 0, st, P, cl, cnt, w, rowslot, colslot, n);
            }
        }
        RBF_LAUNCH(ctx, k_sym_gather, blocks_for(n, 256), 256, 0, st, rowslot, colslot, n, ctx->pid.p, P.active,
                   G.sym_prob.p, y);
        if (!G.sym_all) {   // the stencil kernel for the problems the symmetric one does not serve
            P.work = ctx->al.on ? ctx->al.w32ns.p : G.work_ns.p;
            const int64_t nns = ctx->al.on ? ctx->al.n32ns : G.n_work_ns;
            if (nns > 0) {
                switch (tile) {
                case 32: RBF_CHECK(launch_f32<32>(ctx, P, nns, w, y, st)); break;
                case 64: RBF_CHECK(launch_f32<64>(ctx, P, nns, w, y, st)); break;
                default: RBF_CHECK(launch_f32<128>(ctx, P, nns, w, y, st)); break;
                }
            }
        }
    } else if (nwork > 0) {
        switch (tile) {
        case 32: RBF_CHECK(launch_f32<32>(ctx, P, nwork, w, y, st)); break;
        case 64: RBF_CHECK(launch_f32<64>(ctx, P, nwork, w, y, st)); break;
        default: RBF_CHECK(launch_f32<128>(ctx, P, nwork, w, y, st)); break;
        }
    }
    return prof_end(ctx, RBF_PROF_MATVEC_F32, st);
}

rbf_status matvec_sorted_f32(rbf_ctx* ctx, const double* w, double* y, cudaStream_t st)
{
    float2* loc = nullptr;
    RBF_CHECK(ensure_local_coords(ctx, &loc, st));
    RBF_CHECK(ensure(ctx, ctx->vec_c, (size_t)ctx->n));   // two FP32 vectors
    float* wf = (float*)ctx->vec_c.p;
    float* yf = wf + ctx->n;
    RBF_LAUNCH(ctx, k_to_f32, blocks_for(ctx->n, 256), 256, 0, st, w, ctx->n, wf);
    RBF_CHECK(matvec_f32_raw(ctx, loc, wf, yf, st));
    RBF_LAUNCH(ctx, k_to_f64, blocks_for(ctx->n, 256), 256, 0, st, yf, ctx->n, y);
    return RBF_OK;
}

}  // namespace rbf
