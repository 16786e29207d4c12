// server.cu -- continuous batching of sFFT requests on one GPU (sfft_server_*).
//
// A host scheduler thread runs iteration-level batching: every pass it (1) retires the
// groups whose completion event has fired, (2) admits queued requests, grouped by plan,
// onto free worker workspaces while their device footprint fits the memory budget and
// fewer than max_slots groups are in flight, and (3) launches each admitted group with the
// batched path on the group's own stream, so groups that arrive while others run overlap
// on the device.  Worker workspaces are clones of the caller's plan (same tables and
// options, their own bins and decode state) created on demand and kept for reuse.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sfft.h"
#include "sfft_plan.h"

namespace sfft {
int execute_group(sfft_plan_s* p, int n, const void* const* xs, int64_t* const* idx,
                  void* const* val, int32_t* infos, cudaStream_t st, bool host);
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

struct Worker {
    sfft_plan_t src = nullptr;   // caller plan it clones
    sfft_plan_t plan = nullptr;  // clone with max_batch = kGroupMax
    size_t bytes = 0;
    bool busy = false;
    int32_t* d_infos = nullptr;  // group info rows, copied to each request's info
};

struct Group {
    Worker* w;
    cudaStream_t stream;
    cudaEvent_t done;
    std::vector<Request> reqs;
};

struct Done {
    int status;
    double latency_us;
};

}  // namespace

struct sfft_server_s {
    size_t budget = 0;
    int max_slots = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, Done> done;
    std::vector<std::unique_ptr<Worker>> workers;
    std::vector<cudaStream_t> free_streams;
    std::vector<Group> running;
    size_t used = 0;
    uint64_t next_ticket = 1;
    std::atomic<bool> stop{false};
    std::atomic<int> in_flight{0};
    int error = 0;
    std::thread th;
};

namespace {

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

// One scheduler pass; called with the server mutex released.
void scheduler_loop(sfft_server_s* s)
{
    cudaSetDevice(s->device);
    while (true) {
        std::vector<Request> admitted;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->running.empty() && s->queue.empty()) {
                if (s->stop) break;
                s->cv.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
        }
        // (1) retire finished groups
        {
            std::lock_guard<std::mutex> lk(s->mu);
            for (size_t i = 0; i < s->running.size();) {
                Group& g = s->running[i];
                if (cudaEventQuery(g.done) == cudaSuccess) {
                    const double t = now_us();
                    for (auto& r : g.reqs) s->done[r.ticket] = Done{SFFT_OK, t - r.t_submit};
                    g.w->busy = false;
                    s->free_streams.push_back(g.stream);
                    cudaEventDestroy(g.done);
                    s->in_flight -= (int)g.reqs.size();
                    s->running.erase(s->running.begin() + i);
                } else {
                    ++i;
                }
            }
        }
        // (2) admit and (3) launch
        while (true) {
            std::vector<Request> grp;
            Worker* w = nullptr;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (s->queue.empty() || (int)s->running.size() >= s->max_slots) break;
                sfft_plan_t p = s->queue.front().plan;
                for (auto& wk : s->workers)
                    if (!wk->busy && wk->src == p) {
                        w = wk.get();
                        break;
                    }
                if (!w) {
                    // a new workspace if the budget allows (plans are sized from the source)
                    const size_t need = p->footprint / (size_t)p->max_batch * kGroupMax + 4096;
                    if (s->used + need > s->budget) {
                        // evict an idle workspace of another plan, else wait
                        bool freed = false;
                        for (size_t i = 0; i < s->workers.size(); ++i)
                            if (!s->workers[i]->busy) {
                                sfft_plan_destroy(s->workers[i]->plan);
                                cudaFree(s->workers[i]->d_infos);
                                s->used -= s->workers[i]->bytes;
                                s->workers.erase(s->workers.begin() + i);
                                freed = true;
                                break;
                            }
                        if (!freed || s->used + need > s->budget) break;
                    }
                    auto wk = std::make_unique<Worker>();
                    wk->src = p;
                    wk->plan = clone_plan(p, kGroupMax);
                    if (!wk->plan || cudaMalloc(&wk->d_infos, 16 * kGroupMax) != cudaSuccess) {
                        if (wk->plan) sfft_plan_destroy(wk->plan);
                        s->error = SFFT_ENOMEM;
                        break;
                    }
                    wk->bytes = wk->plan->footprint + 16 * kGroupMax;
                    s->used += wk->bytes;
                    w = wk.get();
                    s->workers.push_back(std::move(wk));
                }
                // take up to kGroupMax queued requests of this plan, in arrival order
                for (auto it = s->queue.begin(); it != s->queue.end() && (int)grp.size() < kGroupMax;) {
                    if (it->plan == p) {
                        grp.push_back(*it);
                        it = s->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                w->busy = true;
            }
            cudaStream_t st;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                if (!s->free_streams.empty()) {
                    st = s->free_streams.back();
                    s->free_streams.pop_back();
                } else {
                    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
                }
            }
            std::vector<const void*> xs;
            std::vector<int64_t*> ix;
            std::vector<void*> vs;
            for (auto& r : grp) {
                xs.push_back(r.x);
                ix.push_back(r.idx);
                vs.push_back(r.val);
            }
            int rc = sfft::execute_group(w->plan, (int)grp.size(), xs.data(), ix.data(), vs.data(),
                                         w->d_infos, st, false);
            for (size_t i = 0; i < grp.size() && rc == SFFT_OK; ++i)
                if (cudaMemcpyAsync(grp[i].info, w->d_infos + 4 * i, 16, cudaMemcpyDeviceToDevice,
                                    st) != cudaSuccess)
                    rc = SFFT_ECUDA;
            std::lock_guard<std::mutex> lk(s->mu);
            if (rc != SFFT_OK) {
                // the launch failed: report it on every request of the group
                const double t = now_us();
                for (auto& r : grp) s->done[r.ticket] = Done{rc, t - r.t_submit};
                s->in_flight -= (int)grp.size();
                w->busy = false;
                s->free_streams.push_back(st);
                s->error = rc;
                continue;
            }
            Group g;
            g.w = w;
            g.stream = st;
            g.reqs = std::move(grp);
            cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
            cudaEventRecord(g.done, st);
            s->running.push_back(std::move(g));
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" int sfft_server_create(sfft_server_t* out, size_t hbm_budget, int32_t max_slots)
{
    if (!out || max_slots < 1 || hbm_budget == 0) return SFFT_EINVAL;
    sfft_server_s* s = new sfft_server_s();
    s->budget = hbm_budget;
    s->max_slots = max_slots;
    cudaGetDevice(&s->device);
    s->th = std::thread(scheduler_loop, s);
    *out = s;
    return SFFT_OK;
}

extern "C" int sfft_submit(sfft_server_t s, sfft_plan_t plan, const void* x, int64_t* out_idx,
                           void* out_val, int32_t* out_info, uint64_t* ticket)
{
    if (!s || !plan || !x || !out_idx || !out_val || !out_info || !ticket) return SFFT_EINVAL;
    if (!plan->layers.empty()) return SFFT_EINVAL;  // DSFFT plans are host-driven, not served
    const size_t need = plan->footprint / (size_t)plan->max_batch * kGroupMax + 4096;
    if (need > s->budget) return SFFT_EADMIT;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return s->error;
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
    while (s->in_flight.load() > 0) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->error) return s->error;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    return SFFT_OK;
}

extern "C" void sfft_server_destroy(sfft_server_t s)
{
    if (!s) return;
    sfft_server_drain(s);
    s->stop = true;
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto& w : s->workers) {
        sfft_plan_destroy(w->plan);
        cudaFree(w->d_infos);
    }
    for (auto st : s->free_streams) cudaStreamDestroy(st);
    delete s;
}
