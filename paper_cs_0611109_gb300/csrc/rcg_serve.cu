// rcg_serve.cu -- the serving engine: a request loop with continuous batching
// on top of the batched tile engine.
//
// Requests (an rcg_job on caller-owned device stripes, an arrival time and an
// HBM footprint) are queued with rcg_serve_submit.  A scheduler thread owns
// the context while the server runs and repeats:
//   1. retire: launches whose completion event has fired complete their
//      requests (completion time = when the host sees the event), freeing
//      their HBM footprint and in-flight slots;
//   2. admit: requests whose arrival time has passed are admitted in arrival
//      order while the in-flight slot count and the HBM budget allow -- a
//      request on a stripe that an earlier admitted request still uses waits
//      (two jobs on one stripe must not share a batch);
//   3. launch: while fewer than two launches are in flight, everything
//      admitted and not yet launched (up to max_batch_jobs) goes out as ONE
//      persistent-kernel batch -- so requests that arrived while the previous
//      batch ran join the next one (continuous batching), and the next batch
//      is prepared on the host while the GPU runs the current one.
// In per-job mode (the comparison) each admitted request is launched on its
// own with the single-operation call.  Latency = completion - arrival.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rcg.h"
#include "rcg_internal.h"

namespace {

uint64_t mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return static_cast<uint64_t>(ts.tv_sec) * 1000000000ull + ts.tv_nsec;
}

struct Request {
    rcg_serve_request req;
    uint64_t id;
    uint64_t footprint;
    uint64_t admit_ns = 0, launch_ns = 0, complete_ns = 0;
    uint32_t status = RCG_OK;
    uint32_t batch = 0;
};

struct Launch {
    std::vector<uint64_t> ids;   // requests in this launch
    cudaEvent_t done = nullptr;
    uint64_t ticket = 0;         // batch mode
};

uint64_t job_footprint(const rcg_job &j) {
    const rcg_layout &L = j.layout;
    const uint64_t rs = L.row_stride ? L.row_stride : L.row_bytes;
    const uint64_t ss = L.strip_stride ? L.strip_stride : (L.p - 1ull) * rs;
    uint64_t fp = (L.n_data + 2ull) * ss * j.n_stripes;
    if (j.op == RCG_OP_DEGRADED_READ || j.op == RCG_OP_UPDATE) fp += (L.p - 1ull) * L.row_bytes * j.n_stripes;
    return fp;
}

}  // namespace

struct rcg_server {
    rcg_ctx *ctx = nullptr;
    rcg_serve_config cfg;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<Request> reqs;          // by id
    std::deque<uint64_t> pending;       // submitted, not admitted (arrival order of submission)
    std::deque<uint64_t> admitted;      // admitted, not launched
    std::deque<Launch> inflight;        // launched, not retired
    std::unordered_map<uintptr_t, uint32_t> busy;  // stripe base -> requests admitted on it
    std::vector<cudaEvent_t> free_events;
    uint64_t budget_used = 0;
    uint32_t inflight_jobs = 0;
    uint64_t start_ns = 0;
    uint64_t completed = 0;
    uint32_t batches = 0;
    std::atomic<bool> stop{false};
    std::atomic<bool> running{false};
    rcg_status error = RCG_OK;
};

namespace {

cudaEvent_t get_event(rcg_server *s) {
    if (!s->free_events.empty()) {
        cudaEvent_t e = s->free_events.back();
        s->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
}

uintptr_t stripe_key(const rcg_job &j) {
    const rcg_layout &L = j.layout;
    const uint64_t rs = L.row_stride ? L.row_stride : L.row_bytes;
    const uint64_t ss = L.strip_stride ? L.strip_stride : (L.p - 1ull) * rs;
    const uint64_t st = L.stripe_stride ? L.stripe_stride : (L.n_data + 2ull) * ss;
    return reinterpret_cast<uintptr_t>(L.base) + j.first_stripe * st;
}

rcg_status launch_single_job(rcg_ctx *ctx, const rcg_job &j, cudaStream_t s) {
    switch (j.op) {
        case RCG_OP_ENCODE:
            return rcg_encode(ctx, &j.layout, j.first_stripe, j.n_stripes, s);
        case RCG_OP_RECOVER:
            if (j.n_stripes != 1) return RCG_EINVAL;
            return rcg_recover(ctx, &j.layout, j.first_stripe, j.i, j.j, s);
        case RCG_OP_DEGRADED_READ:
            if (j.n_stripes != 1) return RCG_EINVAL;
            return rcg_degraded_read(ctx, &j.layout, j.first_stripe, j.j, const_cast<void *>(j.aux),
                                     j.aux_row_stride, s);
        case RCG_OP_UPDATE:
            if (j.n_stripes != 1) return RCG_EINVAL;
            return rcg_update(ctx, &j.layout, j.first_stripe, j.i, j.aux, j.aux_row_stride, s);
    }
    return RCG_EINVAL;
}

// One pass of the scheduler; returns true when it did something.
bool tick(rcg_server *s) {
    bool did = false;
    const uint64_t now = mono_ns() - s->start_ns;
    std::unique_lock<std::mutex> lock(s->mu);
    // 1. retire, in launch order
    while (!s->inflight.empty()) {
        Launch &L = s->inflight.front();
        const cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) break;
        for (uint64_t id : L.ids) {
            Request &r = s->reqs[id];
            r.complete_ns = now;  // the tick's clock: frees precede this tick's admissions
            if (q != cudaSuccess) r.status = RCG_ECUDA;
            s->budget_used -= r.footprint;
            --s->inflight_jobs;
            auto it = s->busy.find(stripe_key(r.req.job));
            if (it != s->busy.end() && --it->second == 0) s->busy.erase(it);
        }
        s->completed += L.ids.size();
        s->free_events.push_back(L.done);
        s->inflight.pop_front();
        did = true;
        s->cv.notify_all();
    }
    // 2. admit arrived requests in order while slots and HBM allow; a request
    //    on a stripe still in use waits (without blocking the ones behind it)
    for (auto it = s->pending.begin(); it != s->pending.end();) {
        Request &r = s->reqs[*it];
        if (r.req.arrival_ns > now) break;
        if (s->inflight_jobs >= s->cfg.max_inflight_jobs) break;
        if (s->budget_used + r.footprint > s->cfg.hbm_budget_bytes) break;
        const uintptr_t key = stripe_key(r.req.job);
        if (s->busy.count(key)) {
            ++it;
            continue;
        }
        s->busy[key] = 1;
        s->budget_used += r.footprint;
        ++s->inflight_jobs;
        r.admit_ns = now;
        s->admitted.push_back(*it);
        it = s->pending.erase(it);
        did = true;
    }
    // 3. launch what is admitted, keeping at most two launches in flight
    if (!s->admitted.empty() && s->inflight.size() < 2) {
        const uint32_t n = static_cast<uint32_t>(std::min<size_t>(s->admitted.size(), s->cfg.max_batch_jobs));
        std::vector<uint64_t> ids(s->admitted.begin(), s->admitted.begin() + n);
        s->admitted.erase(s->admitted.begin(), s->admitted.begin() + n);
        std::vector<rcg_job> jobs(n);
        for (uint32_t k = 0; k < n; ++k) jobs[k] = s->reqs[ids[k]].req.job;
        const uint32_t batch_no = ++s->batches;
        lock.unlock();  // host preparation runs without the lock
        const uint64_t t_launch = mono_ns() - s->start_ns;
        rcg_status st = RCG_OK;
        Launch L;
        if (s->cfg.per_job_launches) {
            for (uint32_t k = 0; k < n && st == RCG_OK; ++k) {
                st = launch_single_job(s->ctx, jobs[k], s->stream);
                if (st == RCG_OK && k + 1 < n) {  // one completion event per job
                    Launch one;
                    one.ids.push_back(ids[k]);
                    one.done = get_event(s);
                    cudaEventRecord(one.done, s->stream);
                    lock.lock();
                    s->reqs[ids[k]].launch_ns = t_launch;
                    s->reqs[ids[k]].batch = batch_no;
                    s->inflight.push_back(std::move(one));
                    lock.unlock();
                    ids[k] = ~0ull;
                }
            }
        } else {
            st = rcg_batch_submit(s->ctx, jobs.data(), n, s->stream, &L.ticket);
        }
        lock.lock();
        for (uint64_t id : ids)
            if (id != ~0ull) {
                L.ids.push_back(id);
                s->reqs[id].launch_ns = t_launch;
                s->reqs[id].batch = batch_no;
                if (st != RCG_OK) s->reqs[id].status = st;
            }
        if (!L.ids.empty()) {
            L.done = get_event(s);
            cudaEventRecord(L.done, s->stream);
            s->inflight.push_back(std::move(L));
        }
        if (st != RCG_OK && s->error == RCG_OK) s->error = st;
        did = true;
    }
    return did;
}

void worker_main(rcg_server *s) {
    cudaSetDevice(rcg::ctx_device(s->ctx));
    while (!s->stop.load()) {
        if (tick(s)) continue;
        // idle: nothing retired, admitted or launched; poll again shortly
        timespec ts = {0, 2000};
        nanosleep(&ts, nullptr);
    }
}

}  // namespace

extern "C" {

rcg_status rcg_serve_create(rcg_ctx *ctx, const rcg_serve_config *cfg, rcg_server **out) {
    if (!ctx || !out) return RCG_EINVAL;
    *out = nullptr;
    rcg_server *s = new (std::nothrow) rcg_server();
    if (!s) return RCG_ENOMEM;
    s->ctx = ctx;
    memset(&s->cfg, 0, sizeof(s->cfg));
    if (cfg) s->cfg = *cfg;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(rcg::ctx_device(ctx));
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if (s->cfg.hbm_budget_bytes == 0) s->cfg.hbm_budget_bytes = std::min<uint64_t>(120000000000ull, free_b);
    if (s->cfg.max_batch_jobs == 0) s->cfg.max_batch_jobs = 2048;
    // room for two full batches in flight, so the next one is prepared while one runs
    if (s->cfg.max_inflight_jobs == 0) s->cfg.max_inflight_jobs = 4 * s->cfg.max_batch_jobs;
    const cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        delete s;
        return RCG_ECUDA;
    }
    *out = s;
    return RCG_OK;
}

rcg_status rcg_serve_submit(rcg_server *s, const rcg_serve_request *reqs, uint32_t n, uint64_t *first_id) {
    if (!s || (n && !reqs)) return RCG_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    const uint64_t first = s->reqs.size();
    for (uint32_t k = 0; k < n; ++k) {
        const rcg_job &j = reqs[k].job;
        if (j.n_stripes != 1 && j.op != RCG_OP_ENCODE) return RCG_EINVAL;
        Request r;
        r.req = reqs[k];
        r.id = first + k;
        r.footprint = reqs[k].footprint_bytes ? reqs[k].footprint_bytes : job_footprint(j);
        if (r.footprint > s->cfg.hbm_budget_bytes) return RCG_EINVAL;  // could never be admitted
        s->reqs.push_back(r);
        s->pending.push_back(r.id);
    }
    if (first_id) *first_id = first;
    return RCG_OK;
}

rcg_status rcg_serve_start(rcg_server *s) {
    if (!s || s->running.load()) return RCG_EINVAL;
    s->stop = false;
    s->start_ns = mono_ns();
    s->running = true;
    s->worker = std::thread(worker_main, s);
    return RCG_OK;
}

rcg_status rcg_serve_drain(rcg_server *s, uint64_t timeout_ns) {
    if (!s) return RCG_EINVAL;
    const uint64_t t0 = mono_ns();
    std::unique_lock<std::mutex> lock(s->mu);
    while (s->completed < s->reqs.size()) {
        if (mono_ns() - t0 > timeout_ns) return RCG_ETIMEOUT;
        s->cv.wait_for(lock, std::chrono::milliseconds(1));
    }
    return s->error;
}

rcg_status rcg_serve_results(rcg_server *s, rcg_serve_result *out, uint64_t max, uint64_t *n) {
    if (!s || !n || (max && !out)) return RCG_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    const uint64_t m = std::min<uint64_t>(max, s->reqs.size());
    for (uint64_t k = 0; k < m; ++k) {
        const Request &r = s->reqs[k];
        out[k].id = r.id;
        out[k].arrival_ns = r.req.arrival_ns;
        out[k].admit_ns = r.admit_ns;
        out[k].launch_ns = r.launch_ns;
        out[k].complete_ns = r.complete_ns;
        out[k].status = r.complete_ns ? r.status : RCG_EBUSY;
        out[k].batch = r.batch;
    }
    *n = m;
    return RCG_OK;
}

rcg_status rcg_serve_destroy(rcg_server *s) {
    if (!s) return RCG_EINVAL;
    s->stop = true;
    if (s->worker.joinable()) s->worker.join();
    s->running = false;
    cudaStreamSynchronize(s->stream);
    for (auto &L : s->inflight)
        if (L.done) cudaEventDestroy(L.done);
    for (auto e : s->free_events) cudaEventDestroy(e);
    cudaStreamDestroy(s->stream);
    delete s;
    return RCG_OK;
}

}  // extern "C"
