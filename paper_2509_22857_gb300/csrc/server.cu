// Continuous-batching inference server.
//
// One server per context (one parameter set and key set).  Every registered
// model gets a pipeline (see model.cu) and a worker thread.  Requests queue
// per model; at each tick the worker admits up to `group` queued requests into
// the pipeline while earlier requests are still inside it, so their work
// overlaps on the device, and the workers of different models tick
// concurrently on their own streams.  A model is admitted only if free device
// memory covers its pipeline's estimate.  Results are bit-identical to
// one-image fhe_infer (the arithmetic of an image does not depend on what it
// is batched with).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "host.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    std::vector<fhe_ct *> in;   // owned by the server until admitted
    clk::time_point t_submit;
};

struct Result {
    bool done = false;
    int error = FHE_OK;
    std::vector<fhe_ct *> out;
    double latency_ms = 0;
};

struct ModelSlot {
    const fhe_model *model = nullptr;
    fhe_pipeline *pipe = nullptr;
    int group = 1, n_in = 1, n_out = 1, segments = 1;
    std::deque<Request> queue;
    std::unordered_map<long long, std::vector<Request>> in_flight;   // entry tick -> requests
    long long tick = 0;
    std::thread worker;
};

}  // namespace

struct fhe_server {
    fhe_ctx *ctx = nullptr;
    const fhe_evk *evk = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    bool paused = false;      // workers run no tick while set (a stalled host worker)
    uint64_t next_ticket = 1;
    std::vector<std::unique_ptr<ModelSlot>> models;
    std::unordered_map<uint64_t, Result> results;
    std::vector<double> latencies;
    int error = FHE_OK;
    std::string error_msg;
};

static void worker_loop(fhe_server *sv, ModelSlot *ms) {
    cudaSetDevice(sv->ctx->dev);
    std::vector<fhe_ct *> out((size_t)ms->group * ms->n_out);
    for (;;) {
        std::vector<Request> admit;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait(lk, [&] {
                return sv->stop || (!sv->paused && (!ms->queue.empty() || !ms->in_flight.empty()));
            });
            if (sv->stop) return;
            while (!ms->queue.empty() && (int)admit.size() < ms->group) {
                admit.push_back(std::move(ms->queue.front()));
                ms->queue.pop_front();
            }
        }
        std::vector<const fhe_ct *> in;
        for (auto &r : admit)
            for (auto *c : r.in) in.push_back(c);
        size_t n_done = 0;
        int64_t tag = -1, before = 0, after = 0;
        fhe_pipeline_ticks(ms->pipe, &before);
        const int rc = fhe_pipeline_tick(ms->pipe, in.data(), admit.size(), out.data(), &n_done, &tag);
        fhe_pipeline_ticks(ms->pipe, &after);
        for (auto &r : admit)
            for (auto *c : r.in) fhe_ct_free(c);
        std::lock_guard<std::mutex> lk(sv->mu);
        // the pipeline's tick counter is the entry tick of each admitted group
        const long long entry = before;
        ms->tick = after;
        if (rc != FHE_OK) {
            sv->error = rc;
            sv->error_msg = fhe_last_error();
            auto fail = [&](const Request &r) {
                Result &res = sv->results[r.ticket];
                res.done = true;
                res.error = rc;
            };
            // this tick's admissions failed with it (refused before launch:
            // they never entered; failed after: their state is unknown)
            for (auto &r : admit) fail(r);
            // the group that was due to leave lost its outputs
            if (tag >= 0) {
                auto it = ms->in_flight.find(tag);
                if (it != ms->in_flight.end()) {
                    for (auto &r : it->second) fail(r);
                    ms->in_flight.erase(it);
                }
            }
            sv->cv.notify_all();
            continue;
        }
        if (!admit.empty()) {
            for (auto &r : admit) r.in.clear();
            ms->in_flight[entry] = std::move(admit);
        }
        if (n_done) {
            auto it = ms->in_flight.find(tag);
            if (it != ms->in_flight.end()) {
                const auto now = clk::now();
                for (size_t j = 0; j < it->second.size(); j++) {
                    Result &res = sv->results[it->second[j].ticket];
                    res.out.assign(out.begin() + j * ms->n_out, out.begin() + (j + 1) * ms->n_out);
                    res.latency_ms = std::chrono::duration<double, std::milli>(now - it->second[j].t_submit).count();
                    res.done = true;
                    sv->latencies.push_back(res.latency_ms);
                }
                ms->in_flight.erase(it);
            }
        }
        // groups still inside keep the pipeline ticking (empty admissions drain it)
        sv->cv.notify_all();
    }
}

extern "C" int fhe_server_create(fhe_ctx *c, const fhe_evk *evk, fhe_server **out) {
    if (!c || !evk || !out) return fhe_fail(FHE_E_INVAL, "null argument");
    fhe_server *sv = new fhe_server();
    sv->ctx = c;
    sv->evk = evk;
    *out = sv;
    return FHE_OK;
}

extern "C" int fhe_server_add_model(fhe_server *sv, const fhe_model *model, int group, size_t reserve_bytes,
                                    int *model_id) {
    if (!sv || !model || !model_id || group < 1) return fhe_fail(FHE_E_INVAL, "bad argument");
    FHE_CU(cudaSetDevice(sv->ctx->dev));
    size_t free_b = 0, total_b = 0;
    FHE_CU(pool_trim());   // freed temporaries held by the pool count as free
    FHE_CU(cudaMemGetInfo(&free_b, &total_b));
    if (reserve_bytes && free_b < reserve_bytes)
        return fhe_fail(FHE_E_OOM, "not enough free device memory to admit this model (" + std::to_string(free_b) +
                                       " < " + std::to_string(reserve_bytes) + " bytes)");
    std::unique_ptr<ModelSlot> ms(new ModelSlot());
    ms->model = model;
    ms->group = group;
    FHE_TRY(fhe_pipeline_create(sv->ctx, model, sv->evk, group, 1, &ms->pipe));
    fhe_pipeline_info(ms->pipe, &ms->segments, nullptr, &ms->n_in, &ms->n_out);
    std::lock_guard<std::mutex> lk(sv->mu);
    *model_id = (int)sv->models.size();
    ModelSlot *raw = ms.get();
    sv->models.push_back(std::move(ms));
    raw->worker = std::thread(worker_loop, sv, raw);
    return FHE_OK;
}

extern "C" int fhe_server_submit(fhe_server *sv, int model_id, fhe_ct *const *in, uint64_t *ticket) {
    if (!sv || !in || !ticket) return fhe_fail(FHE_E_INVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (model_id < 0 || model_id >= (int)sv->models.size()) return fhe_fail(FHE_E_INVAL, "no such model");
    ModelSlot *ms = sv->models[model_id].get();
    Request r;
    r.ticket = sv->next_ticket++;
    r.in.assign(in, in + ms->n_in);
    r.t_submit = clk::now();
    *ticket = r.ticket;
    sv->results[r.ticket] = Result();
    ms->queue.push_back(std::move(r));
    sv->cv.notify_all();
    return FHE_OK;
}

extern "C" int fhe_server_pause(fhe_server *sv, int paused) {
    if (!sv) return fhe_fail(FHE_E_INVAL, "null argument");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->paused = paused != 0;
    }
    sv->cv.notify_all();
    return FHE_OK;
}

extern "C" int fhe_server_poll(fhe_server *sv, uint64_t ticket, int timeout_ms, fhe_ct **out, size_t cap,
                               size_t *n_out, double *latency_ms) {
    if (!sv || !n_out) return fhe_fail(FHE_E_INVAL, "null argument");
    *n_out = 0;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return fhe_fail(FHE_E_INVAL, "unknown ticket");
    // the entry stays in the map until it is returned, so the reference is stable under the lock
    const auto done = [&] { return sv->results[ticket].done; };
    if (timeout_ms < 0) {
        sv->cv.wait(lk, done);
    } else if (timeout_ms > 0 && !sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), done)) {
        return fhe_fail(FHE_E_TIMEOUT, "request " + std::to_string(ticket) + " not done within " +
                                           std::to_string(timeout_ms) + " ms");
    }
    Result &r = sv->results[ticket];
    if (!r.done) return FHE_OK;
    if (r.error != FHE_OK) {
        const int e = r.error;
        sv->results.erase(ticket);
        return fhe_fail(e, "request failed: " + sv->error_msg);
    }
    if (cap < r.out.size()) return fhe_fail(FHE_E_INVAL, "output capacity too small");
    for (size_t k = 0; k < r.out.size(); k++) out[k] = r.out[k];
    *n_out = r.out.size();
    if (latency_ms) *latency_ms = r.latency_ms;
    sv->results.erase(ticket);
    return FHE_OK;
}

extern "C" int fhe_server_stats(fhe_server *sv, uint64_t *completed, double *p50_ms, double *p99_ms) {
    if (!sv) return fhe_fail(FHE_E_INVAL, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> l = sv->latencies;
    std::sort(l.begin(), l.end());
    if (completed) *completed = l.size();
    auto q = [&](double f) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
    if (p50_ms) *p50_ms = q(0.50);
    if (p99_ms) *p99_ms = q(0.99);
    return FHE_OK;
}

extern "C" int fhe_server_destroy(fhe_server *sv) {
    if (!sv) return FHE_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    for (auto &ms : sv->models)
        if (ms->worker.joinable()) ms->worker.join();
    for (auto &ms : sv->models) {
        for (auto &r : ms->queue)
            for (auto *c : r.in) fhe_ct_free(c);
        fhe_pipeline_free(ms->pipe);
    }
    for (auto &kv : sv->results)
        for (auto *c : kv.second.out) fhe_ct_free(c);
    delete sv;
    return FHE_OK;
}
