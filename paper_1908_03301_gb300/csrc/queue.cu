// queue.cu -- continuous-batching request queue (netq_* of the C ABI).
//
// A worker thread owns the device work.  Between batch steps (every K
// sweeps) it admits queued requests while their estimated device footprint
// fits in the memory budget and a slot is free, creates their networks and
// adds them to the running batch; requests whose refinement loop finished
// leave at once, returning their memory and slot.  Requests therefore overlap
// on the device with whatever is already running, and every running network
// keeps its CG state resident between steps.  Latency is measured from
// netq_submit to the end of the request's solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/netsolve.h"
#include "batch.h"
#include "runtime_internal.h"

using namespace netsolve;

namespace {

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2 };

struct Req {
    uint64_t ticket = 0;
    net_desc desc{};
    std::vector<unsigned char> bonds[3];
    size_t foot = 0;
    int state = Q_QUEUED;
    net_result res{};
    std::string err;  // error message of a request that ended non-OK
    BatchItem item;
    net_t *net = nullptr;
    std::chrono::steady_clock::time_point t_submit, t_admit;
    long long co_running = 0;  // requests on the device when this one was admitted
};

}  // namespace

struct netq_s {
    int device = 0;
    cudaStream_t st = nullptr;
    size_t budget = 0, used = 0;
    int max_slots = 1;
    int running = 0;
    net_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::unordered_map<uint64_t, Req *> all;
    std::vector<double> lat_ms;
    uint64_t next = 1;
    bool stopping = false;
    std::thread worker;
};

namespace {

void finalize_locked(netq_t *q, Req *r, net_status st) {
    r->res.status = st;
    if (r->state == Q_RUNNING) {
        r->res.queue_ms = std::chrono::duration<double, std::milli>(r->t_admit - r->t_submit).count();
        r->res.co_running = r->co_running;
    }
    if (st != NET_OK && r->err.empty()) r->err = last_error();
    r->state = Q_DONE;
    q->lat_ms.push_back(
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - r->t_submit).count());
}

void worker_main(netq_t *q) {
    cudaSetDevice(q->device);
    BatchEngine eng(q->device, q->st);
    std::vector<Req *> active;
    const int K = q->opts.check_every > 0 ? q->opts.check_every : 16;
    while (true) {
        std::vector<Req *> admit;
        {
            std::unique_lock<std::mutex> lk(q->mu);
            if (q->stopping) break;
            while (!q->pending.empty() && q->running < q->max_slots &&
                   q->used + q->pending.front()->foot <= q->budget) {
                Req *r = q->pending.front();
                q->pending.pop_front();
                r->state = Q_RUNNING;
                r->t_admit = std::chrono::steady_clock::now();
                r->co_running = (long long)eng.running();
                q->used += r->foot;
                q->running++;
                admit.push_back(r);
            }
            if (admit.empty() && eng.running() == 0) {
                q->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
        }
        // set up the admitted networks (outside the lock)
        std::vector<BatchItem *> items;
        for (Req *r : admit) {
            const void *ptr[3] = {nullptr, nullptr, nullptr};
            for (int d = 0; d < r->desc.ndim; d++) ptr[d] = r->bonds[d].empty() ? nullptr : r->bonds[d].data();
            net_desc dd = r->desc;
            dd.on_device = 0;
            dd.stream = nullptr;
            net_status s = net_create(&dd, ptr, &r->net);
            for (int d = 0; d < 3; d++) std::vector<unsigned char>().swap(r->bonds[d]);
            if (s != NET_OK) {
                std::lock_guard<std::mutex> lk(q->mu);
                r->res = net_result{};
                finalize_locked(q, r, s);
                q->used -= r->foot;
                q->running--;
                q->cv_done.notify_all();
                continue;
            }
            r->item = BatchItem{};
            r->item.net = r->net;
            r->item.opts = q->opts;
            r->item.user = r->ticket;
            items.push_back(&r->item);
            active.push_back(r);
        }
        net_status es = NET_OK;
        if (!items.empty()) es = eng.add(items);
        if (es == NET_OK && eng.running() > 0) es = eng.step(K);
        std::vector<BatchItem *> done = eng.take_done();
        if (es != NET_OK) {
            // the device failed: every running request ends with that status
            for (Req *r : active)
                if (!r->item.done) {
                    r->item.res.status = es;
                    r->item.err = last_error();
                    r->item.done = true;
                    done.push_back(&r->item);
                }
        }
        if (done.empty()) continue;
        std::lock_guard<std::mutex> lk(q->mu);
        for (BatchItem *it : done) {
            auto f = q->all.find(it->user);
            if (f == q->all.end()) continue;
            Req *r = f->second;
            r->res = it->res;
            r->err = it->err;
            net_destroy(r->net);
            r->net = nullptr;
            finalize_locked(q, r, it->res.status);
            q->used -= r->foot;
            q->running--;
            active.erase(std::remove(active.begin(), active.end(), r), active.end());
        }
        q->cv_done.notify_all();
        if (es != NET_OK) break;
    }
    // shutting down: running requests end as cancelled
    std::lock_guard<std::mutex> lk(q->mu);
    for (Req *r : active) {
        if (r->state == Q_DONE) continue;
        if (r->net) net_destroy(r->net);
        r->net = nullptr;
        r->res = net_result{};
        r->err = "queue destroyed while the request was running";
        finalize_locked(q, r, NET_ECANCELLED);
    }
    q->cv_done.notify_all();
}

}  // namespace

#define NET_API extern "C" __attribute__((visibility("default")))

NET_API net_status netq_create(size_t mem_budget_bytes, int max_slots, const net_opts *opts,
                               netq_t **out) {
    if (!out || max_slots < 1 || mem_budget_bytes == 0) {
        set_error("netq_create: bad arguments");
        return NET_EINVAL;
    }
    *out = nullptr;
    netq_t *q = new netq_t();
    cudaGetDevice(&q->device);
    q->budget = mem_budget_bytes;
    q->max_slots = max_slots;
    net_opts_default(&q->opts);
    if (opts) q->opts = *opts;
    q->opts.x0 = nullptr;
    q->opts.stream = nullptr;
    if (!opts_valid(q->opts)) {
        delete q;
        set_error("netq_create: %s", std::string(last_error()).c_str());
        return NET_EINVAL;
    }
    if (cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete q;
        set_error("netq_create: stream");
        return NET_ECUDA;
    }
    q->worker = std::thread(worker_main, q);
    *out = q;
    return NET_OK;
}

NET_API net_status netq_submit(netq_t *q, const net_desc *desc, const void *const g[3],
                               uint64_t *ticket) {
    if (!q || !desc || !ticket) {
        set_error("netq_submit: NULL argument");
        return NET_EINVAL;
    }
    Geom G;
    net_status s = make_geom(desc, &G);
    if (s != NET_OK) return s;
    if (desc->on_device) {
        set_error("netq_submit: bond planes must be host pointers");
        return NET_EINVAL;
    }
    const int f32 = desc->bond_dtype == NET_F32;
    const size_t foot = net_footprint_bytes(G, f32);
    if (foot > q->budget) {
        set_error("netq_submit: request needs %zu bytes, budget is %zu", foot, q->budget);
        return NET_EBUDGET;
    }
    Req *r = new Req();
    r->desc = *desc;
    r->foot = foot;
    const size_t es = f32 ? 4 : 8;
    for (int d = 0; d < G.ndim; d++) {
        const size_t m = (size_t)plane_elems(G, d);
        if (m == 0) continue;
        if (!g || !g[d]) {
            delete r;
            set_error("netq_submit: bond plane %d is NULL", d);
            return NET_EINVAL;
        }
        r->bonds[d].resize(m * es);
        memcpy(r->bonds[d].data(), g[d], m * es);
    }
    r->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> lk(q->mu);
    if (q->stopping) {
        delete r;
        set_error("netq_submit: queue is shutting down");
        return NET_ECANCELLED;
    }
    r->ticket = q->next++;
    q->all[r->ticket] = r;
    q->pending.push_back(r);
    *ticket = r->ticket;
    q->cv_work.notify_one();
    return NET_OK;
}

NET_API net_status netq_poll(netq_t *q, uint64_t ticket, net_result *out) {
    if (!q) {
        set_error("netq_poll: NULL queue");
        return NET_EINVAL;
    }
    std::lock_guard<std::mutex> lk(q->mu);
    auto f = q->all.find(ticket);
    if (f == q->all.end()) {
        set_error("netq_poll: unknown or already read ticket");
        return NET_EINVAL;
    }
    Req *r = f->second;
    if (r->state != Q_DONE) return NET_EBUSY;
    if (out) *out = r->res;
    const net_status st = r->res.status;
    if (st != NET_OK) set_error("request %llu: %s", (unsigned long long)ticket, r->err.c_str());
    q->all.erase(f);
    delete r;
    return st;
}

NET_API net_status netq_wait(netq_t *q, uint64_t ticket, int timeout_ms, net_result *out) {
    if (!q) {
        set_error("netq_wait: NULL queue");
        return NET_EINVAL;
    }
    std::unique_lock<std::mutex> lk(q->mu);
    auto ready = [&] {
        auto f = q->all.find(ticket);
        return f == q->all.end() || f->second->state == Q_DONE;
    };
    if (timeout_ms < 0) q->cv_done.wait(lk, ready);
    else if (!q->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return NET_ETIMEOUT;
    auto f = q->all.find(ticket);
    if (f == q->all.end()) {
        set_error("netq_wait: unknown or already read ticket");
        return NET_EINVAL;
    }
    Req *r = f->second;
    if (out) *out = r->res;
    const net_status st = r->res.status;
    if (st != NET_OK) set_error("request %llu: %s", (unsigned long long)ticket, r->err.c_str());
    q->all.erase(f);
    delete r;
    return st;
}

NET_API net_status netq_cancel(netq_t *q, uint64_t ticket) {
    if (!q) {
        set_error("netq_cancel: NULL queue");
        return NET_EINVAL;
    }
    std::lock_guard<std::mutex> lk(q->mu);
    auto f = q->all.find(ticket);
    if (f == q->all.end()) {
        set_error("netq_cancel: unknown ticket");
        return NET_EINVAL;
    }
    Req *r = f->second;
    if (r->state == Q_RUNNING) return NET_EBUSY;
    if (r->state == Q_DONE) return NET_OK;
    q->pending.erase(std::remove(q->pending.begin(), q->pending.end(), r), q->pending.end());
    r->res = net_result{};
    r->res.status = NET_ECANCELLED;
    r->err = "cancelled before it started";
    r->state = Q_DONE;
    q->cv_done.notify_all();
    return NET_OK;
}

NET_API net_status netq_stats(netq_t *q, double *p50_ms, double *p99_ms, uint64_t *completed) {
    if (!q) {
        set_error("netq_stats: NULL queue");
        return NET_EINVAL;
    }
    std::vector<double> v;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        v = q->lat_ms;
    }
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
        return v[i];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (completed) *completed = v.size();
    return NET_OK;
}

NET_API net_status netq_destroy(netq_t *q) {
    if (!q) return NET_OK;
    {
        std::lock_guard<std::mutex> lk(q->mu);
        q->stopping = true;
        for (Req *r : q->pending) {
            r->res = net_result{};
            r->res.status = NET_ECANCELLED;
            r->err = "queue destroyed before the request started";
            r->state = Q_DONE;
        }
        q->pending.clear();
    }
    q->cv_work.notify_all();
    if (q->worker.joinable()) q->worker.join();
    for (auto &kv : q->all) delete kv.second;
    q->all.clear();
    if (q->st) cudaStreamDestroy(q->st);
    delete q;
    return NET_OK;
}
