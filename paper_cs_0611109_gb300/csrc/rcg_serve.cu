// rcg_serve.cu -- the serving engine: a request loop with continuous batching
// on top of the batched tile engine.
//
// Requests (an rcg_job on caller-owned device stripes, an arrival time and an
// HBM footprint) are queued with rcg_serve_submit.  A scheduler thread owns
// the context while the server runs and repeats:
//   1. retire: launches whose completion event has fired complete their
//      requests (completion time = when the host sees the event), freeing
//      their HBM footprint, in-flight slots and device byte ranges;
//   2. admit: requests whose arrival time has passed are admitted in arrival
//      order while the in-flight count and the HBM budget allow.  A request
//      whose device bytes (its stripes' extent, and its aux buffer's) overlap
//      those of an admitted request -- or of an earlier request that is still
//      waiting -- waits, so requests on the same bytes run in arrival order
//      and never share a launch;
//   3. launch: batched mode -- while fewer than max_inflight_batches launches
//      are in flight, everything admitted and not yet launched (up to
//      max_batch_jobs) goes out as ONE persistent-kernel batch, so requests
//      that arrived while the previous batch ran join the next one (continuous
//      batching) and the next batch is prepared on the host while the GPU runs
//      the current one; per-job mode (the comparison) -- every admitted
//      request is launched at once with its own single-operation call and
//      completion event.  Launches go round-robin over the server's streams.
// Latency = completion - arrival.
#include <cuda_runtime.h>
#if defined(__linux__)
#include <sys/prctl.h>
#endif
#include <stdint.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/rcg.h"
#include "rcg_admission.h"
#include "rcg_internal.h"

namespace {

uint64_t mono_ns() {
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return static_cast<uint64_t>(ts.tv_sec) * 1000000000ull + ts.tv_nsec;
}

using rcg::Extent;

struct Request {
    rcg_serve_request req;
    uint64_t id;
    uint64_t footprint;
    Extent ext[2];
    uint32_t n_ext = 0;
    uint64_t admit_ns = 0, launch_ns = 0, complete_ns = 0;
    uint32_t status = RCG_OK;
    uint32_t batch = 0;
};

struct Launch {
    std::vector<uint64_t> ids;   // requests in this launch
    cudaEvent_t done = nullptr;
    uint64_t ticket = 0;         // batch mode
};

// The server's streams.  Launches go round-robin over them -- per-job
// launches (a request's single-stripe kernel fills a fraction of the GPU, so
// several run at once) and batches alike (a small batch at low load starts
// at once, and one batch's tail overlaps the next one's start).  Admission
// keeps requests on the same bytes from being in flight together, so
// launches on different streams never touch the same bytes.
constexpr int kServeStreams = 8;

struct Strides {
    uint64_t rs, ss, st, ars, ass;
};

Strides strides_of(const rcg_job &j) {
    const rcg_layout &L = j.layout;
    Strides s;
    s.rs = L.row_stride ? L.row_stride : L.row_bytes;
    s.ss = L.strip_stride ? L.strip_stride : (L.p - 1ull) * s.rs;
    s.st = L.stripe_stride ? L.stripe_stride : (L.n_data + 2ull) * s.ss;
    s.ars = j.aux_row_stride ? j.aux_row_stride : L.row_bytes;
    s.ass = j.aux_stripe_stride ? j.aux_stripe_stride : (L.p - 1ull) * s.ars;
    return s;
}

bool uses_aux(const rcg_job &j) { return j.op == RCG_OP_DEGRADED_READ || j.op == RCG_OP_UPDATE; }

uint64_t job_footprint(const rcg_job &j) {
    const rcg_layout &L = j.layout;
    const Strides s = strides_of(j);
    uint64_t fp = (L.n_data + 2ull) * s.ss * j.n_stripes;
    if (uses_aux(j)) fp += (L.p - 1ull) * L.row_bytes * j.n_stripes;
    return fp;
}

// The device bytes a job touches: from its first stripe's first byte to one
// past the last byte of row p-2 of strip N+1 of its last stripe, and the same
// for the aux buffer of a degraded read or small write.  Overlapping extents
// are merged.
uint32_t job_extents(const rcg_job &j, Extent *out) {
    const rcg_layout &L = j.layout;
    const Strides s = strides_of(j);
    const uint64_t n = j.n_stripes ? j.n_stripes : 1;
    uint32_t k = 0;
    out[k].lo = reinterpret_cast<uintptr_t>(L.base) + j.first_stripe * s.st;
    out[k].hi = out[k].lo + (n - 1) * s.st + (L.n_data + 1ull) * s.ss + (L.p - 2ull) * s.rs + L.row_bytes;
    ++k;
    if (uses_aux(j) && j.aux) {
        // an aux extent overlapping the stripes is merged by Admission::add
        out[k].lo = reinterpret_cast<uintptr_t>(j.aux);
        out[k].hi = out[k].lo + (n - 1) * s.ass + (L.p - 2ull) * s.ars + L.row_bytes;
        ++k;
    }
    return k;
}

}  // namespace

struct rcg_server {
    rcg_ctx *ctx = nullptr;
    rcg_serve_config cfg;
    cudaStream_t streams[kServeStreams] = {};
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    std::vector<Request> reqs;          // by id
    std::unique_ptr<rcg::Admission> adm;  // which requests may start (rcg_admission.h)
    std::deque<uint64_t> admitted;      // admitted, not launched
    std::deque<Launch> inflight[kServeStreams];  // launched, not retired, per stream (in launch order)
    uint32_t n_inflight = 0;
    std::vector<cudaEvent_t> free_events;
    uint64_t start_ns = 0;
    uint64_t completed = 0;
    uint32_t launches = 0;              // launch numbers handed out (batches, or single jobs)
    uint64_t kernel_launches = 0;
    uint32_t max_inflight_launches = 0;
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

void note_launch(rcg_server *s) {
    s->max_inflight_launches = std::max<uint32_t>(s->max_inflight_launches, s->n_inflight);
}

// One pass of the scheduler; returns true when it did something.
bool tick(rcg_server *s) {
    bool did = false;
    const uint64_t now = mono_ns() - s->start_ns;
    std::unique_lock<std::mutex> lock(s->mu);
    // 1. retire: each stream's launches finish in their launch order
    for (auto &queue : s->inflight) {
        while (!queue.empty()) {
            Launch &L = queue.front();
            const cudaError_t q = cudaEventQuery(L.done);
            if (q == cudaErrorNotReady) break;
            for (uint64_t id : L.ids) {
                Request &r = s->reqs[id];
                r.complete_ns = now;  // the tick's clock: frees precede this tick's admissions
                if (q != cudaSuccess) r.status = RCG_ECUDA;
                s->adm->retire(id);
            }
            s->completed += L.ids.size();
            s->free_events.push_back(L.done);
            queue.pop_front();
            --s->n_inflight;
            did = true;
            s->cv.notify_all();
        }
    }
    // 2. admit arrived requests in order while slots and HBM allow; a request
    //    whose bytes overlap an admitted one's, or an earlier waiting one's,
    //    waits (the ones behind it that do not overlap go ahead)
    if (s->adm->admit(now, [&](uint64_t id) {
            s->reqs[id].admit_ns = now;
            s->admitted.push_back(id);
        }))
        did = true;
    // 3a. per-job mode: every admitted request goes out at once, on its own
    if (s->cfg.per_job_launches) {
        while (!s->admitted.empty()) {
            const uint64_t id = s->admitted.front();
            s->admitted.pop_front();
            const rcg_job job = s->reqs[id].req.job;
            const uint32_t launch_no = ++s->launches;
            const int q = static_cast<int>(launch_no % kServeStreams);
            lock.unlock();
            const uint64_t t_launch = mono_ns() - s->start_ns;
            const rcg_status st = launch_single_job(s->ctx, job, s->streams[q]);
            Launch one;
            one.ids.push_back(id);
            one.done = get_event(s);
            cudaEventRecord(one.done, s->streams[q]);
            lock.lock();
            Request &r = s->reqs[id];
            r.launch_ns = t_launch;
            r.batch = launch_no;
            if (st != RCG_OK) {
                r.status = st;
                if (s->error == RCG_OK) s->error = st;
            } else {
                ++s->kernel_launches;
            }
            s->inflight[q].push_back(std::move(one));
            ++s->n_inflight;
            note_launch(s);
            did = true;
        }
        return did;
    }
    // 3b. batched mode: what is admitted goes out as one batch while fewer
    //     than max_inflight_batches are in flight
    if (!s->admitted.empty() && s->n_inflight < s->cfg.max_inflight_batches) {
        const uint32_t n = static_cast<uint32_t>(std::min<size_t>(s->admitted.size(), s->cfg.max_batch_jobs));
        std::vector<uint64_t> ids(s->admitted.begin(), s->admitted.begin() + n);
        s->admitted.erase(s->admitted.begin(), s->admitted.begin() + n);
        std::vector<rcg_job> jobs(n);
        for (uint32_t k = 0; k < n; ++k) jobs[k] = s->reqs[ids[k]].req.job;
        const uint32_t launch_no = ++s->launches;
        const int q = static_cast<int>(launch_no % kServeStreams);
        lock.unlock();  // host preparation runs without the lock
        const uint64_t t_launch = mono_ns() - s->start_ns;
        Launch L;
        // a batch of one request gains nothing from the batch tables: it goes
        // out as that request's single-operation call
        const rcg_status st = n == 1 ? launch_single_job(s->ctx, jobs[0], s->streams[q])
                                     : rcg_batch_submit(s->ctx, jobs.data(), n, s->streams[q], &L.ticket);
        L.done = get_event(s);
        cudaEventRecord(L.done, s->streams[q]);
        lock.lock();
        L.ids = ids;
        for (uint64_t id : ids) {
            s->reqs[id].launch_ns = t_launch;
            s->reqs[id].batch = launch_no;
            if (st != RCG_OK) s->reqs[id].status = st;
        }
        if (st == RCG_OK) ++s->kernel_launches;
        s->inflight[q].push_back(std::move(L));
        ++s->n_inflight;
        note_launch(s);
        if (st != RCG_OK && s->error == RCG_OK) s->error = st;
        did = true;
    }
    return did;
}

void worker_main(rcg_server *s) {
    cudaSetDevice(rcg::ctx_device(s->ctx));
#if defined(__linux__)
    // The idle poll below sleeps 2 us; with the default timer slack (50 us)
    // the kernel may stretch each sleep to about 50 us, which then delays
    // every admission and completion.  The slack is this thread's own.
    prctl(PR_SET_TIMERSLACK, 1000UL, 0UL, 0UL, 0UL);
#endif
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
    if (s->cfg.max_inflight_batches == 0) s->cfg.max_inflight_batches = kServeStreams;
    if (s->cfg.max_inflight_batches > static_cast<uint32_t>(kServeStreams)) {
        if (prev >= 0) cudaSetDevice(prev);
        delete s;
        return RCG_EINVAL;
    }
    // room for four full batches admitted at once, so the next ones are prepared while one runs
    if (s->cfg.max_inflight_jobs == 0) s->cfg.max_inflight_jobs = 4 * s->cfg.max_batch_jobs;
    s->adm.reset(new (std::nothrow) rcg::Admission(s->cfg.hbm_budget_bytes, s->cfg.max_inflight_jobs));
    if (!s->adm) {
        if (prev >= 0) cudaSetDevice(prev);
        delete s;
        return RCG_ENOMEM;
    }
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < kServeStreams && e == cudaSuccess; ++q)
        e = cudaStreamCreateWithFlags(&s->streams[q], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        for (auto st : s->streams)
            if (st) cudaStreamDestroy(st);
    }
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
    // validate every request before queueing any (all or nothing)
    std::vector<Request> batch(n);
    for (uint32_t k = 0; k < n; ++k) {
        const rcg_job &j = reqs[k].job;
        if (j.n_stripes == 0 || (j.n_stripes != 1 && j.op != RCG_OP_ENCODE)) return RCG_EINVAL;
        if (!j.layout.base || j.layout.p < 3 || j.layout.n_data < 1 || j.layout.row_bytes == 0) return RCG_EINVAL;
        Request &r = batch[k];
        r.req = reqs[k];
        r.footprint = reqs[k].footprint_bytes ? reqs[k].footprint_bytes : job_footprint(j);
        if (r.footprint > s->cfg.hbm_budget_bytes) return RCG_EINVAL;  // could never be admitted
        r.n_ext = job_extents(j, r.ext);
    }
    std::lock_guard<std::mutex> lock(s->mu);
    const uint64_t first = s->reqs.size();
    for (uint32_t k = 0; k < n; ++k) {
        batch[k].id = first + k;
        s->reqs.push_back(batch[k]);
        rcg::Admission::Item it;
        it.arrival_ns = batch[k].req.arrival_ns;
        it.footprint = batch[k].footprint;
        it.n_ext = batch[k].n_ext;
        for (uint32_t e = 0; e < batch[k].n_ext; ++e) it.ext[e] = batch[k].ext[e];
        s->adm->add(it);  // the same id
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

rcg_status rcg_serve_get_stats(rcg_server *s, rcg_serve_stats *out) {
    if (!s || !out) return RCG_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    out->kernel_launches = s->kernel_launches;
    out->completed = s->completed;
    out->conflict_waits = s->adm->conflict_waits();
    out->max_inflight_launches = s->max_inflight_launches;
    out->max_inflight_jobs = s->adm->max_inflight_seen();
    return RCG_OK;
}

rcg_status rcg_serve_destroy(rcg_server *s) {
    if (!s) return RCG_EINVAL;
    s->stop = true;
    if (s->worker.joinable()) s->worker.join();
    s->running = false;
    for (auto st : s->streams) cudaStreamSynchronize(st);
    for (auto &queue : s->inflight)
        for (auto &L : queue)
            if (L.done) cudaEventDestroy(L.done);
    for (auto e : s->free_events) cudaEventDestroy(e);
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
    return RCG_OK;
}

}  // extern "C"
