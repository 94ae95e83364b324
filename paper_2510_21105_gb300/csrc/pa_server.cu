// pa_server.cu -- continuous-batching request loop over the library's anneals.
//
// Two background host threads make every CUDA call of the server:
//   admission   (admission thread) requests wait in FIFO order until their estimated device
//               memory fits under the HBM budget (the oldest request is
//               always admitted when nothing else runs), then get a context
//               (graph upload) and an initialised population;
//   ticks       (tick thread) each active request (at most n_streams at once, each on its
//               own stream) gets its next steps_per_tick temperature steps
//               enqueued; a request keeps at most two ticks in flight, so
//               arrivals join within one tick;
//   completion  a request whose last tick has finished on the device records
//               its best cut and configuration and releases its memory and
//               its copies of the caller's inputs;
//   timeout     a request with timeout_ms > 0 that has not completed that
//               long after its admission is cancelled: its enqueued ticks
//               drain (every kernel is bounded), its memory is released and
//               it reports PA_ETIMEOUT; the other requests carry on.
// Populations stay resident between ticks. Results are bit-identical to a
// lone pa_anneal of the same request: all randomness is keyed by seed, slot,
// step, sweep and vertex, never by scheduling.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/pa.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    // copies of the caller's inputs
    int32_t n = 0;
    std::vector<uint32_t> rp;
    std::vector<uint16_t> col;
    std::vector<int8_t> w;
    bool has_w = false;
    std::vector<double> betas;
    int32_t K = 0, R = 0, S = 0;
    uint64_t seed = 0;
    pa_anneal_opts opts{};
    double timeout_ms = 0.0;
    size_t bytes = 0;
    // state
    bool held = false;               // testing hook: no further ticks are enqueued
    pa_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;   // one stream per admitted request
    int32_t k_enq = 0;
    std::deque<cudaEvent_t> inflight;
    int status = 0;   // 0 queued, 1 running, 2 done, <0 error
    pa_response resp{};
    std::vector<int8_t> config;
};

}  // namespace

struct pa_server {
    int device = 0;
    size_t budget = 0, used = 0;
    int32_t steps_per_tick = 8;
    int32_t slots = 16;               // maximum concurrently running requests
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> active;
    std::map<uint64_t, std::shared_ptr<Request>> all;
    uint64_t next_id = 1;
    bool stopping = false;
    int preparing = 0;                // requests being admitted by the admission thread
    std::thread worker, admitter;
    Clock::time_point t0;
    pa_server_stats_t stats{};
};

namespace {

double ms_since(const pa_server *s) {
    return std::chrono::duration<double, std::milli>(Clock::now() - s->t0).count();
}

// Device bytes a request will hold: two population buffers (int8 spins +
// int16 fields), energies, parents, resampling scratch, tables and records.
size_t estimate_bytes(const Request &q) {
    const size_t np = (size_t)((q.n + 15) & ~15);
    const size_t rpad = (size_t)((q.R + 31) & ~31);
    const size_t m2 = q.rp.empty() ? 0 : q.rp.back();
    int32_t maxdeg = 0;
    for (int32_t i = 0; i < q.n; ++i) maxdeg = std::max<int32_t>(maxdeg, (int32_t)(q.rp[i + 1] - q.rp[i]));
    const size_t K = (size_t)std::max(q.K, 1);
    size_t b = 2 * np * rpad * 3 + 4 * 4 * rpad + 16 * 2 * rpad;
    b += (rpad / 4) * (np + 16);                    // best records and configurations
    b += K * (size_t)(maxdeg + 1) * 4 + K * 32 * 8 + K * (64 + 4 * (size_t)std::max(q.S, 1));
    b += m2 * 6 + np * 24;                          // graph copies
    if (q.opts.nlm_period > 0) b += (size_t)q.R * 12 + 16384;
    return b + (1u << 20);
}

void finish(pa_server *s, Request &q, int status) {
    if (q.ctx) {
        if (status == 2) {
            int64_t cut = 0;
            int32_t E = 0, step = -1, sweep = -1, slot = -1;
            q.config.assign(q.n, 0);
            if (pa_best_record(q.ctx, &E, &step, &sweep, &slot) == PA_OK &&
                pa_best(q.ctx, &cut, q.config.data(), nullptr, nullptr) == PA_OK) {
                q.resp.cut = cut;
                q.resp.energy = E;
                q.resp.step = step;
                q.resp.sweep = sweep;
                q.resp.slot = slot;
            } else {
                status = PA_ESTATE;
            }
            pa_stats_t st;
            if (pa_stats(q.ctx, &st) == PA_OK) q.resp.attempts = st.attempts;
        }
        pa_destroy(q.ctx);
        q.ctx = nullptr;
    }
    for (cudaEvent_t e : q.inflight) cudaEventDestroy(e);
    q.inflight.clear();
    if (q.stream) {
        cudaStreamDestroy(q.stream);
        q.stream = nullptr;
    }
    // The inputs are not needed any more; only the response and configuration stay.
    std::vector<uint32_t>().swap(q.rp);
    std::vector<uint16_t>().swap(q.col);
    std::vector<int8_t>().swap(q.w);
    std::vector<double>().swap(q.betas);
    q.resp.finish_ms = ms_since(s);
    q.resp.status = status == 2 ? PA_OK : status;
    std::lock_guard<std::mutex> lock(s->mu);
    q.status = status;
    s->used -= q.bytes;
    s->stats.completed += 1;
    s->stats.attempts += q.resp.attempts;
}

bool admit_one(pa_server *s, const std::shared_ptr<Request> &q) {
    q->resp.start_ms = ms_since(s);
    int rc = pa_create(&q->ctx, q->n, q->rp.data(), q->col.data(), q->has_w ? q->w.data() : nullptr);
    if (rc == PA_OK && cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking) != cudaSuccess) rc = PA_ECUDA;
    if (rc == PA_OK) {
        pa_anneal_opts o = q->opts;
        o.stream = q->stream;
        o.time_kernels = 0;
        // Layout by load: an automatic-layout request admitted while others run
        // shares the device, so it takes the cheapest attempt (multi-spin coded,
        // every word in one-CTA blocks); admitted alone it keeps the automatic
        // single-instance choice. Results do not depend on the layout.
        bool shared;
        {
            std::lock_guard<std::mutex> lock(s->mu);
            shared = !s->active.empty() || s->preparing > 1;
        }
        int32_t maxdeg = 0;
        for (int32_t i = 0; i < q->n; ++i) maxdeg = std::max<int32_t>(maxdeg, (int32_t)(q->rp[i + 1] - q->rp[i]));
        if (o.variant == PA_VARIANT_AUTO && shared && maxdeg <= 127) {
            o.variant = PA_VARIANT_MSC;
            o.msc_no_split = 1;
        }
        rc = pa_anneal_begin(q->ctx, q->betas.empty() ? nullptr : q->betas.data(), q->K, q->R, q->S, q->seed, &o);
    }
    if (rc != PA_OK) {
        finish(s, *q, rc);
        return false;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    q->status = 1;
    s->active.push_back(q);
    s->stats.admitted += 1;
    return true;
}

// Admission thread: moves queued requests to the active set (graph upload,
// tables, population initialisation) while the tick thread keeps the device
// busy with the requests already running.
void admission_loop(pa_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::shared_ptr<Request> q;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            for (;;) {
                if (!s->queue.empty()) {
                    auto &f = s->queue.front();
                    const bool idle = s->active.empty() && s->preparing == 0;
                    if (idle || (s->used + f->bytes <= s->budget &&
                                 (int32_t)s->active.size() + s->preparing < s->slots))
                        break;
                } else if (s->stopping) {
                    return;
                }
                s->cv.wait_for(lock, std::chrono::milliseconds(2));
            }
            q = s->queue.front();
            s->queue.pop_front();
            s->used += q->bytes;
            s->preparing += 1;
        }
        admit_one(s, q);
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->preparing -= 1;
        }
        s->cv.notify_all();
    }
}

// Tick thread: retires finished ticks and requests, enqueues new ticks.
void worker_loop(pa_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<std::shared_ptr<Request>> act;
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->active.empty()) {
                if (s->stopping && s->queue.empty() && s->preparing == 0) return;
                s->cv.wait_for(lock, std::chrono::milliseconds(2));
                continue;
            }
            act = s->active;
        }
        bool progressed = false;
        for (auto &q : act) {
            while (!q->inflight.empty() && cudaEventQuery(q->inflight.front()) == cudaSuccess) {
                cudaEventDestroy(q->inflight.front());
                q->inflight.pop_front();
                progressed = true;
            }
            if (q->k_enq >= q->K && q->inflight.empty()) {
                finish(s, *q, 2);
                progressed = true;
            } else if (q->timeout_ms > 0.0 && ms_since(s) - q->resp.start_ms > q->timeout_ms) {
                finish(s, *q, PA_ETIMEOUT);   // pa_destroy waits for the enqueued ticks
                progressed = true;
            }
        }
        {
            std::lock_guard<std::mutex> lock(s->mu);
            s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                           [](const std::shared_ptr<Request> &q) { return q->status != 1; }),
                            s->active.end());
            act = s->active;
        }
        if (progressed) s->cv.notify_all();
        for (auto &q : act) {
            bool held;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                held = q->held;
            }
            if (held || q->k_enq >= q->K || q->inflight.size() >= 2) continue;
            const int32_t k_end = std::min(q->K, q->k_enq + s->steps_per_tick);
            if (pa_anneal_run(q->ctx, k_end) != PA_OK) {
                finish(s, *q, PA_ECUDA);
                continue;
            }
            q->k_enq = k_end;
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
                cudaEventRecord(e, q->stream);
                q->inflight.push_back(e);
            }
            progressed = true;
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(100));
    }
}

}  // namespace

extern "C" {

int pa_server_start(pa_server **out, size_t hbm_budget_bytes, int32_t n_streams, int32_t steps_per_tick) {
    if (!out || hbm_budget_bytes == 0 || n_streams < 0 || n_streams > 64 || steps_per_tick < 0) return PA_EINVAL;
    pa_server *s = new (std::nothrow) pa_server();
    if (!s) return PA_ENOMEM;
    cudaGetDevice(&s->device);
    s->budget = hbm_budget_bytes;
    s->steps_per_tick = steps_per_tick ? steps_per_tick : 8;
    s->slots = n_streams ? n_streams : 16;
    s->t0 = Clock::now();
    s->worker = std::thread(worker_loop, s);
    s->admitter = std::thread(admission_loop, s);
    *out = s;
    return PA_OK;
}

int pa_server_submit(pa_server *s, const pa_request *req, uint64_t *id) {
    if (!s || !req || !req->row_ptr || req->n < 1 || req->n > 65536 || req->R < 1 || req->K < 0 ||
        req->sweeps < 0 || (!req->opts.adaptive && req->K > 0 && !req->betas) || !(req->timeout_ms >= 0.0))
        return PA_EINVAL;
    auto q = std::make_shared<Request>();
    q->n = req->n;
    q->rp.assign(req->row_ptr, req->row_ptr + req->n + 1);
    const uint32_t m2 = q->rp.back();
    if (m2 && !req->col) return PA_EINVAL;
    q->col.assign(req->col, req->col + m2);
    if (req->w) {
        q->has_w = true;
        q->w.assign(req->w, req->w + m2);
    }
    if (!req->opts.adaptive) q->betas.assign(req->betas, req->betas + req->K);
    q->K = req->K;
    q->R = req->R;
    q->S = req->sweeps;
    q->seed = req->seed;
    q->opts = req->opts;
    q->timeout_ms = req->timeout_ms;
    q->bytes = estimate_bytes(*q);
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->stopping) return PA_ESTATE;
        q->id = s->next_id++;
        q->resp.submit_ms = ms_since(s);
        s->queue.push_back(q);
        s->all[q->id] = q;
        s->stats.submitted += 1;
    }
    s->cv.notify_one();
    if (id) *id = q->id;
    return PA_OK;
}

int pa_server_poll(pa_server *s, uint64_t id, int32_t *state) {
    if (!s || !state) return PA_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return PA_EINVAL;
    const int st = it->second->status;
    *state = st == 2 ? 2 : (st < 0 ? st : st);
    return PA_OK;
}

int pa_server_result(pa_server *s, uint64_t id, pa_response *out, int8_t *config) {
    if (!s || !out) return PA_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return PA_EINVAL;
    const Request &q = *it->second;
    if (q.status == 0 || q.status == 1) return PA_EBUSY;
    *out = q.resp;
    if (config && !q.config.empty()) std::memcpy(config, q.config.data(), q.config.size());
    return q.status == 2 ? PA_OK : q.status;
}

int pa_server_release(pa_server *s, uint64_t id) {
    if (!s) return PA_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return PA_EINVAL;
    if (it->second->status == 0 || it->second->status == 1) return PA_EBUSY;
    s->all.erase(it);
    return PA_OK;
}

int pa_server_hold(pa_server *s, uint64_t id, int32_t hold) {
    if (!s) return PA_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return PA_EINVAL;
    it->second->held = hold != 0;
    return PA_OK;
}

int pa_server_stats(pa_server *s, pa_server_stats_t *out) {
    if (!s || !out) return PA_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->stats;
    out->queued = (int64_t)s->queue.size();
    out->running = (int64_t)s->active.size();
    out->bytes_in_use = (int64_t)s->used;
    out->elapsed_ms = ms_since(s);
    return PA_OK;
}

int pa_server_stop(pa_server *s) {
    if (!s) return PA_EINVAL;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    if (s->admitter.joinable()) s->admitter.join();
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return PA_OK;
}

}  // extern "C"
