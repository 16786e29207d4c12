// server.cu -- continuous batching of sFFT requests on one GPU (sfft_server_*).
//
// A host scheduler thread admits queued requests, grouped by plan, onto free worker
// workspaces while fewer than max_slots groups are in flight, and launches each admitted
// group with the batched path on the worker's own stream, so groups that arrive while
// others run overlap on the device.  A group's completion is reported by a host function
// enqueued on its stream after its kernels (cudaLaunchHostFunc): it records the requests'
// status and latency, frees the worker and wakes the scheduler, which otherwise sleeps on a
// condition variable until a request arrives or a group finishes.
//
// Worker workspaces are clones of the caller's plan (same tables and options, their own
// bins and decode state, kGroupMax signals each) with a stream.  They
// are created only by sfft_server_reserve, or by the first sfft_submit of a plan that has
// none -- in the caller's thread, before the request is queued -- and they are freed only
// there too (an idle workspace of another plan makes room when the memory budget is
// full) or by sfft_server_destroy.  So in the steady state the scheduler allocates,
// frees and synchronises nothing.  A plan's workspaces are not freed while one of its
// requests is queued.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sfft.h"
#include "sfft_plan.h"

namespace sfft {
int execute_group(sfft_plan_s* p, int n, const void* const* xs, int64_t* const* idx,
                  void* const* val, int32_t* const* rows, cudaStream_t st, bool host);
}

namespace {

constexpr int kGroupMax = 32;  // signals per launch group

double now_us()
{
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket;
    sfft_plan_t plan;
    const void* x;
    int64_t* idx;
    void* val;
    int32_t* info;
    double t_submit;
};

struct Done {
    int status;
    double latency_us;
};

}  // namespace

struct sfft_server_s;

namespace {

struct Worker {
    sfft_server_s* srv = nullptr;
    sfft_plan_t src = nullptr;   // caller plan it clones
    sfft_plan_t plan = nullptr;  // clone with max_batch = kGroupMax
    cudaStream_t stream = nullptr;
    size_t bytes = 0;
    bool busy = false;
    std::vector<Request> reqs;   // the group in flight
};

}  // namespace

struct sfft_server_s {
    size_t budget = 0;
    int max_slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;       // scheduler: work queued or a group finished
    std::condition_variable done_cv;  // drain: a group finished
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Done> done;
    std::vector<std::unique_ptr<Worker>> workers;
    int running = 0;
    size_t used = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    int in_flight = 0;  // queued + running requests
    int error = 0;
    std::thread th;
};

namespace {

size_t worker_need(const sfft_plan_s* p)
{
    return p->footprint / (size_t)p->max_batch * kGroupMax + 4096;
}

sfft_plan_t clone_plan(sfft_plan_t p, int batch)
{
    sfft_opts o = p->opts;
    o.max_batch = batch;
    std::vector<int64_t> f(p->pd.D), dl((size_t)p->pd.D * p->pd.R);
    for (int d = 0; d < p->pd.D; ++d) {
        f[d] = p->pd.st[d].L;
        for (int r = 0; r < p->pd.R; ++r) dl[(size_t)d * p->pd.R + r] = p->pd.st[d].tau[r];
    }
    sfft_plan_t c = nullptr;
    if (sfft_plan_create(&c, p->pd.N, p->pd.K, p->pd.D, f.data(), p->pd.R, dl.data(), &o) != SFFT_OK)
        return nullptr;
    return c;
}

void free_worker(Worker* w)
{
    if (w->plan) sfft_plan_destroy(w->plan);
    if (w->stream) cudaStreamDestroy(w->stream);
}

// Host function at the end of a group's stream work: the group is complete.  Makes no CUDA
// call (host functions may not).
void CUDART_CB group_done(void* arg)
{
    Worker* w = static_cast<Worker*>(arg);
    sfft_server_s* s = w->srv;
    const double t = now_us();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& r : w->reqs) s->done[r.ticket] = Done{SFFT_OK, t - r.t_submit};
        s->in_flight -= (int)w->reqs.size();
        w->reqs.clear();
        w->busy = false;
        --s->running;
    }
    s->cv.notify_one();
    s->done_cv.notify_all();
}

// whether a queued request waits for plan p (its workspaces must stay); mutex held
bool queued_for(const sfft_server_s* s, sfft_plan_t p)
{
    for (const auto& q : s->queue)
        if (q.plan == p) return true;
    return false;
}

// Create up to n workspaces of plan p within the budget (caller's thread, server mutex
// not held while allocating).  Idle workspaces of other plans are freed to make room.
// Returns the number of p's workspaces afterwards, or a negative error.
int reserve_workers(sfft_server_s* s, sfft_plan_t p, int n)
{
    const size_t need = worker_need(p);
    if (need > s->budget) return SFFT_EADMIT;
    int have = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& w : s->workers) have += w->src == p;
    }
    while (have < n) {
        std::unique_ptr<Worker> victim;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->used + need > s->budget) {
                for (size_t i = 0; i < s->workers.size(); ++i)
                    if (!s->workers[i]->busy && s->workers[i]->src != p &&
                        !queued_for(s, s->workers[i]->src)) {
                        victim = std::move(s->workers[i]);
                        s->workers.erase(s->workers.begin() + i);
                        s->used -= victim->bytes;
                        break;
                    }
                if (!victim) break;  // the budget is full of busy or own workspaces
            } else {
                s->used += need;  // claimed before allocating
            }
        }
        if (victim) {
            free_worker(victim.get());
            continue;
        }
        auto w = std::make_unique<Worker>();
        w->srv = s;
        w->src = p;
        w->bytes = need;
        w->plan = clone_plan(p, kGroupMax);
        cudaError_t e = cudaSuccess;
        if (w->plan) e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
        if (!w->plan || e != cudaSuccess) {
            free_worker(w.get());
            std::lock_guard<std::mutex> lk(s->mu);
            s->used -= need;
            return SFFT_ENOMEM;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->workers.push_back(std::move(w));
        ++have;
    }
    s->cv.notify_one();
    return have;
}

void scheduler_loop(sfft_server_s* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // admit: the oldest queued request whose plan has an idle workspace, with up to
        // kGroupMax queued requests of the same plan, in arrival order
        Worker* w = nullptr;
        if (s->running < s->max_slots) {
            for (auto& q : s->queue) {
                for (auto& wk : s->workers)
                    if (!wk->busy && wk->src == q.plan) {
                        w = wk.get();
                        break;
                    }
                if (w) break;
            }
        }
        if (!w) {
            if (s->stop && s->queue.empty() && s->running == 0) break;
            s->cv.wait(lk);
            continue;
        }
        std::vector<Request> grp;
        for (auto it = s->queue.begin(); it != s->queue.end() && (int)grp.size() < kGroupMax;) {
            if (it->plan == w->src) {
                grp.push_back(*it);
                it = s->queue.erase(it);
            } else {
                ++it;
            }
        }
        w->busy = true;
        ++s->running;
        lk.unlock();
        std::vector<const void*> xs;
        std::vector<int64_t*> ix;
        std::vector<void*> vs;
        std::vector<int32_t*> rows;
        for (auto& r : grp) {
            xs.push_back(r.x);
            ix.push_back(r.idx);
            vs.push_back(r.val);
            rows.push_back(r.info);
        }
        int rc = sfft::execute_group(w->plan, (int)grp.size(), xs.data(), ix.data(), vs.data(),
                                     rows.data(), w->stream, false);
        if (rc == SFFT_OK) {
            lk.lock();
            w->reqs = std::move(grp);
            lk.unlock();
            if (cudaLaunchHostFunc(w->stream, group_done, w) != cudaSuccess) rc = SFFT_ECUDA;
            lk.lock();
            if (rc != SFFT_OK) grp = std::move(w->reqs);
        } else {
            lk.lock();
        }
        if (rc != SFFT_OK) {
            // the launch failed: report it on every request of the group
            const double t = now_us();
            for (auto& r : grp) s->done[r.ticket] = Done{rc, t - r.t_submit};
            s->in_flight -= (int)grp.size();
            w->reqs.clear();
            w->busy = false;
            --s->running;
            s->error = rc;
            s->done_cv.notify_all();
        }
    }
}

}  // namespace

extern "C" int sfft_server_create(sfft_server_t* out, size_t hbm_budget, int32_t max_slots)
{
    if (!out || max_slots < 1 || hbm_budget == 0) return SFFT_EINVAL;
    sfft_server_s* s = new (std::nothrow) sfft_server_s();
    if (!s) return SFFT_ENOMEM;
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    cudaGetDevice(&s->device);
    s->th = std::thread(scheduler_loop, s);
    *out = s;
    return SFFT_OK;
}

extern "C" int sfft_server_reserve(sfft_server_t s, sfft_plan_t plan, int32_t n_workspaces)
{
    if (!s || !plan || n_workspaces < 1) return SFFT_EINVAL;
    if (!plan->layers.empty()) return SFFT_EINVAL;
    const int rc = reserve_workers(s, plan, std::min(n_workspaces, s->max_slots));
    if (rc < 0) return rc;
    return rc > 0 ? SFFT_OK : SFFT_EADMIT;
}

extern "C" int sfft_submit(sfft_server_t s, sfft_plan_t plan, const void* x, int64_t* out_idx,
                           void* out_val, int32_t* out_info, uint64_t* ticket)
{
    if (!s || !plan || !x || !out_idx || !out_val || !out_info || !ticket) return SFFT_EINVAL;
    if (!plan->layers.empty()) return SFFT_EINVAL;  // DSFFT plans are host-driven, not served
    if (worker_need(plan) > s->budget) return SFFT_EADMIT;
    bool has = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error) return s->error;
        for (auto& w : s->workers) has |= w->src == plan;
    }
    if (!has) {
        // first request of this plan: its workspaces, before the request is queued
        const int rc = reserve_workers(s, plan, s->max_slots);
        if (rc < 0) return rc;
        if (rc == 0) return SFFT_EADMIT;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Request r{s->next_ticket++, plan, x, out_idx, out_val, out_info, now_us()};
    s->queue.push_back(r);
    s->in_flight++;
    *ticket = r.ticket;
    s->cv.notify_one();
    return SFFT_OK;
}

extern "C" int sfft_poll(sfft_server_t s, uint64_t ticket, int32_t* status, double* latency_us)
{
    if (!s || !status) return SFFT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (ticket == 0 || ticket >= s->next_ticket) return SFFT_ENOTFOUND;
        *status = SFFT_PENDING;
        if (latency_us) *latency_us = 0;
        return SFFT_OK;
    }
    *status = it->second.status;
    if (latency_us) *latency_us = it->second.latency_us;
    return SFFT_OK;
}

extern "C" int sfft_server_drain(sfft_server_t s)
{
    if (!s) return SFFT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->done_cv.wait(lk, [&] { return s->in_flight == 0 || s->error != 0; });
    return s->error;
}

extern "C" void sfft_server_destroy(sfft_server_t s)
{
    if (!s) return;
    sfft_server_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto& w : s->workers) {
        if (w->stream) cudaStreamSynchronize(w->stream);
        free_worker(w.get());
    }
    delete s;
}
