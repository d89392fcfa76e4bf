// server.cu -- serving loop: independent interpolation requests admitted while
// others run. Host code only; every request runs through the library's own
// calls (rbf_bin, rbf_rasm_setup, rbf_solve) on a context of its slot.
//
// Each slot is a worker thread with a context, a non-blocking stream and a
// staging buffer for the request's points, values and weights; all of them
// stay allocated from request to request (the "resident" state a request
// reuses). Admission: FIFO, a request is taken by an idle slot when its
// estimated footprint fits in the budget next to what the other slots hold or
// have reserved; a smaller request behind a head that does not fit may go
// first, at most `slots` times in a row. An idle slot whose resident buffers
// keep the head from fitting releases them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rbf.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Ticket {
    rbf_request req;
    rbf_request_result res;
    int64_t est = 0;
    int bypassed = 0;
    bool done = false;
};

struct Slot {
    rbf_ctx* ctx = nullptr;
    cudaStream_t st = nullptr;
    double* buf = nullptr;   // staging: xy (2 cap), f (cap), w (cap)
    int64_t cap = 0;
    int64_t held = 0;        // device bytes held while idle (context + staging)
    int64_t reserved = 0;    // bytes charged while a request runs
    bool busy = false;
    std::thread th;
};

constexpr int64_t kFixedBytes = 16ll << 20;   // per-request tables, scan scratch, exp table

}  // namespace

struct rbf_server {
    int device = 0;
    int nslots = 0;
    int64_t budget = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Ticket> tickets;
    std::vector<Slot> slots;
    bool stop = false;
    int64_t next = 1, submitted = 0, completed = 0, trims = 0, peak = 0, launches = 0;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }

    int64_t charge(const Slot& s) const { return s.busy ? std::max(s.held, s.reserved) : s.held; }

    int64_t total_charge() const
    {
        int64_t t = 0;
        for (const Slot& s : slots) t += charge(s);
        return t;
    }

    void worker(int i);
    rbf_status run(Slot& s, Ticket& t);
    void release_slot(Slot& s);
};

void rbf_server::release_slot(Slot& s)
{
    if (s.ctx) rbf_destroy(s.ctx);
    s.ctx = nullptr;
    if (s.buf) cudaFree(s.buf);
    s.buf = nullptr;
    s.cap = 0;
}

rbf_status rbf_server::run(Slot& s, Ticket& t)
{
    const rbf_request& r = t.req;
    if (cudaSetDevice(device) != cudaSuccess) return RBF_ERR_CUDA;
    if (!s.st && cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess) return RBF_ERR_CUDA;
    if (!s.ctx) {
        rbf_status c = rbf_create(&s.ctx, device);
        if (c != RBF_OK) return c;
        // the slots run at once on their own streams: no cooperative (fused)
        // Arnoldi steps, whose grid would have to share the SMs with the
        // other slots' kernels
        c = rbf_set_option(s.ctx, RBF_OPT_FUSED_STEP, 0);
        // nor kept FP64 pair values: admission counts each request's own footprint
        if (c == RBF_OK) c = rbf_set_option(s.ctx, RBF_OPT_STORE_F64, 0);
        if (c != RBF_OK) return c;
    }
    const int64_t n = r.n;
    if (s.cap < n) {
        if (s.buf) cudaFree(s.buf);
        s.buf = nullptr;
        s.cap = 0;
        if (cudaMalloc(&s.buf, sizeof(double) * 4 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return RBF_ERR_OOM;
        }
        s.cap = n;
    }
    double* xy = s.buf;
    double* f = xy + 2 * s.cap;
    double* w = f + s.cap;
    rbf_stream st = (rbf_stream)s.st;
    if (cudaMemcpyAsync(xy, r.xy, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
        cudaMemcpyAsync(f, r.f, sizeof(double) * n, cudaMemcpyHostToDevice, s.st) != cudaSuccess ||
        cudaMemsetAsync(w, 0, sizeof(double) * n, s.st) != cudaSuccess)
        return RBF_ERR_CUDA;
    rbf_status rs = rbf_bin(s.ctx, xy, n, &r.kernel, st);
    if (rs == RBF_OK) rs = rbf_rasm_setup(s.ctx, &r.rasm, st);
    if (rs != RBF_OK) return rs;
    rs = rbf_solve(s.ctx, f, w, &r.solve, &t.res.info, st);
    if (rs == RBF_OK || rs == RBF_ERR_NOT_CONVERGED) {
        if (cudaMemcpyAsync(r.w, w, sizeof(double) * n, cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
            cudaStreamSynchronize(s.st) != cudaSuccess)
            return RBF_ERR_CUDA;
    }
    return rs;
}

void rbf_server::worker(int i)
{
    Slot& me = slots[i];
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        if (stop) return;
        // the first queued request that fits next to the other slots' charges
        int64_t others = total_charge() - charge(me);
        int64_t pick = -1;
        bool head_blocked = false;
        for (size_t q = 0; q < queue.size(); ++q) {
            Ticket& t = tickets[queue[q]];
            if (others + std::max(me.held, t.est) <= budget) {
                pick = (int64_t)q;
                break;
            }
            if (q == 0) {
                head_blocked = true;
                if (t.bypassed >= nslots) break;   // no more overtaking of this head
            }
        }
        if (pick < 0) {
            if (!queue.empty() && me.held > 0) {
                // idle buffers keep the head out: give them back and look again
                lk.unlock();
                release_slot(me);
                lk.lock();
                me.held = 0;
                ++trims;
                continue;
            }
            cv_work.wait(lk);
            continue;
        }
        if (pick > 0 && head_blocked) tickets[queue[0]].bypassed++;
        const int64_t id = queue[(size_t)pick];
        queue.erase(queue.begin() + pick);
        Ticket& t = tickets[id];
        me.busy = true;
        me.reserved = t.est;
        peak = std::max(peak, total_charge());
        t.res.t_admit = now();
        t.res.slot = i;
        lk.unlock();

        const uint64_t l0 = me.ctx ? rbf_launch_count(me.ctx) : 0;
        rbf_status st = run(me, t);
        const uint64_t l1 = me.ctx ? rbf_launch_count(me.ctx) : 0;
        if (st == RBF_ERR_CUDA || st == RBF_ERR_OOM) {
            cudaGetLastError();
            release_slot(me);   // start the next request from a fresh context
        }
        int64_t held = (me.ctx ? rbf_device_bytes(me.ctx) : 0) + (int64_t)sizeof(double) * 4 * me.cap;

        lk.lock();
        t.res.status = st;
        t.res.t_done = now();
        t.done = true;
        me.busy = false;
        me.reserved = 0;
        me.held = held;
        peak = std::max(peak, total_charge());
        launches += (int64_t)(l1 >= l0 ? l1 - l0 : l1);
        ++completed;
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

extern "C" {

int64_t rbf_request_footprint(const rbf_request* r)
{
    if (!r || r->n < 1) return 0;
    const double n = (double)r->n;
    double area = 0.0;
    if (r->xy) {
        double x0 = r->xy[0], x1 = x0, y0 = r->xy[1], y1 = y0;
        for (int64_t i = 1; i < r->n; ++i) {
            const double x = r->xy[2 * i], y = r->xy[2 * i + 1];
            x0 = std::min(x0, x);
            x1 = std::max(x1, x);
            y0 = std::min(y0, y);
            y1 = std::max(y1, y);
        }
        area = (x1 - x0) * (y1 - y0);
    }
    const int cap = (r->rasm.max_sub_points > 0 && r->rasm.max_sub_points <= 192) ? r->rasm.max_sub_points : 192;
    double n_ov = cap, n_core = 1.0;
    if (area > 0.0 && r->rasm.core_size > 0.0) {
        const double rho = n / area, B = r->rasm.core_size, D = B + 2.0 * std::max(r->rasm.overlap, 0.0);
        n_ov = std::min((double)cap, std::max(1.0, rho * D * D));
        n_core = std::min(n_ov, std::max(1.0, rho * B * B));
    }
    const int m = (r->solve.restart > 0 && r->solve.restart <= 32) ? r->solve.restart : 30;
    const bool mixed = r->solve.mixed != 0;
    const bool f32 = r->rasm.precision != RBF_FP64;
    double per = 32.0;                                 // staging xy, f, w
    per += 60.0;                                       // sorted points, permutations, cell ids, FP32 offsets
    per += 8.0 + 4.0 * n_ov / n_core;                  // core and overlap lists
    per += 40.0;                                       // solver vectors
    per += mixed ? 4.0 * (m + 3) : 8.0 * (m + 1);      // Krylov basis
    per += (f32 ? 4.0 : 8.0) * n_ov;                   // subdomain inverses W_i (n_ov per core point)
    if (mixed && !f32) per += 4.0 * n_ov;              // FP32 copy made for the inner solve
    if (mixed && r->solve.inner_cutoff > 0.0)          // inner grid: order, coordinates, re-indexed lists
        per += 52.0 + 4.0 * n_ov / n_core;
    return (int64_t)(n * per * 1.05) + kFixedBytes;
}

rbf_status rbf_server_create(rbf_server** out, const rbf_server_params* p)
{
    if (!out || !p) return RBF_ERR_INVALID_ARG;
    *out = nullptr;
    if (p->slots < 1 || p->slots > 64 || p->mem_budget < 0) return RBF_ERR_INVALID_ARG;
    int64_t budget = p->mem_budget;
    if (budget == 0) {
        if (cudaSetDevice(p->device) != cudaSuccess) return RBF_ERR_CUDA;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return RBF_ERR_CUDA;
        budget = (int64_t)(0.9 * (double)fr);
    }
    rbf_server* s = new rbf_server();
    s->device = p->device;
    s->nslots = p->slots;
    s->budget = budget;
    s->t0 = Clock::now();
    s->slots.resize((size_t)p->slots);
    for (int i = 0; i < p->slots; ++i) s->slots[(size_t)i].th = std::thread([s, i] { s->worker(i); });
    *out = s;
    return RBF_OK;
}

void rbf_server_destroy(rbf_server* s)
{
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // admitted requests finish; queued ones fail
        for (int64_t id : s->queue) {
            Ticket& t = s->tickets[id];
            t.res.status = RBF_ERR_STATE;
            t.res.t_done = s->now();
            t.done = true;
        }
        s->queue.clear();
        s->stop = true;
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    for (Slot& sl : s->slots)
        if (sl.th.joinable()) sl.th.join();
    cudaSetDevice(s->device);
    for (Slot& sl : s->slots) {
        s->release_slot(sl);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    delete s;
}

rbf_status rbf_server_submit(rbf_server* s, const rbf_request* req, int64_t* ticket)
{
    if (!s || !req || !ticket) return RBF_ERR_INVALID_ARG;
    if (!req->xy || !req->f || !req->w || req->n < 1 || req->n > (int64_t)0x7fffffff - 1) return RBF_ERR_INVALID_ARG;
    const int64_t est = rbf_request_footprint(req);
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) return RBF_ERR_STATE;
    if (est > s->budget) return RBF_ERR_OOM;
    const int64_t id = s->next++;
    Ticket& t = s->tickets[id];
    t.req = *req;
    std::memset(&t.res, 0, sizeof(t.res));
    t.res.t_submit = s->now();
    t.res.footprint = est;
    t.res.slot = -1;
    t.est = est;
    s->queue.push_back(id);
    ++s->submitted;
    *ticket = id;
    s->cv_work.notify_all();
    return RBF_OK;
}

rbf_status rbf_server_wait(rbf_server* s, int64_t ticket, double timeout_s, rbf_request_result* result)
{
    if (!s) return RBF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return RBF_ERR_INVALID_ARG;
    auto ready = [&] { return s->tickets[ticket].done; };
    if (timeout_s < 0.0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return RBF_ERR_TIMEOUT;
    }
    Ticket& t = s->tickets[ticket];
    if (result) *result = t.res;
    s->tickets.erase(ticket);
    return RBF_OK;
}

rbf_status rbf_server_get_stats(rbf_server* s, rbf_server_stats* out)
{
    if (!s || !out) return RBF_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->queued = (int64_t)s->queue.size();
    for (const Slot& sl : s->slots) out->running += sl.busy ? 1 : 0;
    out->resident_bytes = s->total_charge();
    out->mem_budget = s->budget;
    out->peak_resident_bytes = s->peak;
    out->trims = s->trims;
    out->launches = s->launches;
    return RBF_OK;
}

double rbf_server_clock(rbf_server* s)
{
    return s ? s->now() : 0.0;
}

}  // extern "C"
