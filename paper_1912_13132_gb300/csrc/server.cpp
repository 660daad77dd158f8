// server.cpp -- continuous-batching request loop over several device-resident datasets.
//
// The paper's Algorithm 1 evaluates one parameter configuration after another for
// an outer optimiser (Sec. 4.4: a grid of configurations evaluated sequentially).
// Here many clients submit CV-loss evaluations and prediction requests at any time:
//   * every dataset has `lanes` lanes (default two): its own context and a clone over
//     the same device-resident data (ctx_clone), each with a worker thread and a
//     stream.  An idle lane takes the CV requests queued for its dataset (up to
//     max_batch) as one batch, or every queued prediction with the same parameters as
//     one call; so a request that arrives while a batch runs starts on the other lane
//     at once, and its persistent launch takes over the SMs that the running launch
//     frees as its last tasks finish (or the SMs it never used) -- admission as slots
//     free up, with the two launches overlapping on the device;
//   * lanes of different datasets run concurrently as well;
//   * predictions use the kriging weights that CV evaluations of the same
//     configuration kept (the lanes of a dataset share that cache), so a prediction at
//     a recently evaluated configuration factors nothing;
//   * every lane's work memory is reserved when the server is created, budget
//     permitting (a device allocation waits for the kernels already running, so a
//     lane allocating at its first batch would wait for the other lanes' launches);
//   * a batch is admitted only when its lane's work memory fits the server's HBM
//     budget; idle lanes' work memory is released, least recently used first, to make
//     room, otherwise the worker waits for running batches to finish;
//   * results do not depend on the batching or the lane: every (subset,
//     configuration) task is computed on its own, lanes are identical clones, and the
//     per-configuration sum has a fixed order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pcv_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum class Kind { Cv, Predict };

struct Request {
    int64_t id;
    Kind kind;
    int32_t dataset;
    double params[3];
    std::vector<double> xy;        // prediction locations (m x 2)
    Clock::time_point t_submit, t_done;
    bool done = false;
    int32_t status = PCV_OK;
    double sspe = 0.0;
    std::vector<double> yhat;
};

struct Lane {
    pcv_ctx* ctx = nullptr;
    bool owned = false;             // a clone the server made (freed with the server)
    bool busy = false;
    bool evicting = false;
    int64_t resident = 0;           // work-memory bytes accounted to this lane
    Clock::time_point last_used;
    std::thread worker;
    cudaStream_t stream = nullptr;
};

struct Dataset {
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::unique_ptr<Lane>> lanes;
};

}  // namespace

struct pcv_server {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::unique_ptr<Dataset>> ds;
    std::unordered_map<int64_t, std::shared_ptr<Request>> reqs;
    int64_t next_id = 1;
    int32_t max_batch = 16;
    int32_t lanes = 2;
    bool by_work = true;            // stream priorities by work per configuration (else all equal)
    int32_t precision = PCV_PREC_MIXED;
    double budget = 0.0;            // 0: unlimited
    int64_t used = 0;
    bool stop = false;
    // statistics
    std::vector<double> lat_ms;
    int64_t cv_done = 0, pred_done = 0, batches = 0, evictions = 0, pred_calls = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
};

namespace {

// Admission: make room for lane L's work memory (called with the lock held).
bool admit(pcv_server* s, Lane& L, std::unique_lock<std::mutex>& lk) {
    for (;;) {
        if (s->stop) return false;
        const int64_t need = pcv::ctx_workspace_estimate(L.ctx, s->precision);
        if (s->budget <= 0.0 || (double)(s->used + need) <= s->budget) {
            s->used += need;
            L.resident += need;
            return true;
        }
        // evict the least recently used idle lane that holds memory
        Lane* victim = nullptr;
        for (auto& d : s->ds)
            for (auto& lp : d->lanes) {
                Lane& V = *lp;
                if (&V == &L || V.busy || V.evicting || V.resident == 0) continue;
                if (!victim || V.last_used < victim->last_used) victim = &V;
            }
        if (victim) {
            Lane& V = *victim;
            V.evicting = true;
            lk.unlock();
            pcv::ctx_release_workspace(V.ctx);
            lk.lock();
            s->used -= V.resident;
            V.resident = 0;
            V.evicting = false;
            ++s->evictions;
            s->cv.notify_all();
            continue;
        }
        if (s->used == 0) return true;   // alone and still too big: run anyway, it cannot fit otherwise
        s->cv.wait(lk);                  // wait for running batches to finish
    }
}

// The next batch of dataset D for an idle lane (lock held): every queued prediction with
// the front prediction's parameters (one call), or up to max_batch CV requests.
void take_batch(pcv_server* s, Dataset& D, std::vector<std::shared_ptr<Request>>& batch) {
    batch.clear();
    const Kind kind = D.queue.front()->kind;
    const double* p = D.queue.front()->params;
    for (auto it = D.queue.begin(); it != D.queue.end();) {
        const Request& r = **it;
        const bool take = r.kind == kind &&
                          (kind == Kind::Cv ? (int)batch.size() < s->max_batch
                                            : std::memcmp(r.params, p, sizeof r.params) == 0);
        if (take) {
            batch.push_back(*it);
            it = D.queue.erase(it);
        } else {
            ++it;
        }
    }
}

void worker(pcv_server* s, size_t d, size_t l) {
    Dataset& D = *s->ds[d];
    Lane& L = *D.lanes[l];
    cudaSetDevice(pcv::ctx_device(L.ctx));
    std::vector<std::shared_ptr<Request>> batch;
    std::vector<double> params, sspe, xy, yhat;
    std::vector<int32_t> status;
    for (;;) {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [&] { return s->stop || (!D.queue.empty() && !L.evicting); });
        if (s->stop) return;
        take_batch(s, D, batch);
        L.busy = true;
        if (!admit(s, L, lk)) {
            L.busy = false;
            return;
        }
        ++s->batches;
        lk.unlock();
        s->cv.notify_all();   // the other lane may take what is still queued

        // run the batch (synchronous on this lane's stream; other lanes proceed)
        if (batch[0]->kind == Kind::Cv) {
            const int32_t B = (int32_t)batch.size();
            params.resize(3 * B);
            sspe.assign(B, 0.0);
            status.assign(B, 0);
            for (int32_t b = 0; b < B; ++b) std::memcpy(&params[3 * b], batch[b]->params, sizeof(double) * 3);
            pcv_status st = pcv_cv_loss(L.ctx, params.data(), B, s->precision, sspe.data(), nullptr, nullptr, nullptr,
                                        status.data(), L.stream);
            for (int32_t b = 0; b < B; ++b) {
                batch[b]->sspe = st == PCV_OK ? sspe[b] : NAN;
                batch[b]->status = st == PCV_OK ? status[b] : (int32_t)st;
            }
        } else {
            // predictions with one configuration: one call over all their locations
            xy.clear();
            for (auto& r : batch) xy.insert(xy.end(), r->xy.begin(), r->xy.end());
            const int64_t m = (int64_t)xy.size() / 2;
            yhat.assign(m, 0.0);
            const pcv_status st = pcv_predict(L.ctx, batch[0]->params, xy.data(), m, s->precision, yhat.data(),
                                              L.stream);
            int64_t off = 0;
            for (auto& r : batch) {
                const int64_t mr = (int64_t)r->xy.size() / 2;
                r->yhat.assign(yhat.begin() + off, yhat.begin() + off + mr);
                r->status = st;
                off += mr;
            }
        }

        lk.lock();
        const auto now = Clock::now();
        s->t_last = now;
        if (batch[0]->kind == Kind::Predict) ++s->pred_calls;
        for (auto& r : batch) {
            r->t_done = now;
            r->done = true;
            s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
            if (r->kind == Kind::Cv) ++s->cv_done; else ++s->pred_done;
        }
        L.busy = false;
        L.last_used = now;
        // the workspace estimate is now zero; keep the accounted bytes as resident
        lk.unlock();
        s->cv.notify_all();
    }
}

pcv_status submit(pcv_server* s, std::shared_ptr<Request> r, int64_t* id) {
    if (r->dataset < 0 || r->dataset >= (int32_t)s->ds.size()) return PCV_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return PCV_ERR_BUSY;
        r->id = s->next_id++;
        r->t_submit = Clock::now();
        if (!s->any) {
            s->any = true;
            s->t_first = r->t_submit;
        }
        s->reqs[r->id] = r;
        s->ds[r->dataset]->queue.push_back(r);
        if (id) *id = r->id;
    }
    s->cv.notify_all();
    return PCV_OK;
}

}  // namespace

PCV_API pcv_status pcv_server_create(pcv_ctx* const* ctxs, int32_t n_ctx, const pcv_server_options* opts,
                                     pcv_server** out) {
    if (!out || !ctxs || n_ctx < 1) return PCV_ERR_ARG;
    *out = nullptr;
    for (int32_t i = 0; i < n_ctx; ++i)
        if (!ctxs[i]) return PCV_ERR_ARG;
    std::unique_ptr<pcv_server> s(new (std::nothrow) pcv_server);
    if (!s) return PCV_ERR_OOM;
    if (opts) {
        if (opts->struct_size != 0 && opts->struct_size != (int32_t)sizeof(pcv_server_options)) return PCV_ERR_ARG;
        if (opts->max_batch > 0) s->max_batch = opts->max_batch;
        if (opts->lanes > 0) s->lanes = std::min(opts->lanes, 4);
        if (opts->priorities == 1) s->by_work = false;
        if (opts->precision == PCV_PREC_FP64 || opts->precision == PCV_PREC_MIXED) s->precision = opts->precision;
        if (opts->hbm_budget_bytes > 0) s->budget = opts->hbm_budget_bytes;
    }
    // Stream priorities: the dataset with the least work per configuration gets the
    // highest priority, so that when launches of several datasets wait for SMs the
    // short ones are scheduled first (shortest job first lowers the mean latency;
    // a running launch is never pre-empted, so long jobs are delayed, not starved).
    std::vector<double> work(n_ctx);
    for (int32_t i = 0; i < n_ctx; ++i) work[i] = pcv::ctx_work_estimate(ctxs[i]);
    auto cleanup = [&]() {
        for (auto& e : s->ds)
            for (auto& l : e->lanes) {
                if (l->stream) cudaStreamDestroy(l->stream);
                if (l->owned) pcv::ctx_free(l->ctx);
            }
    };
    for (int32_t i = 0; i < n_ctx; ++i) {
        auto d = std::make_unique<Dataset>();
        cudaSetDevice(pcv::ctx_device(ctxs[i]));
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
        int rank = 0;   // datasets with strictly less work
        for (int32_t j = 0; j < n_ctx; ++j) rank += work[j] < work[i];
        const int levels = least - greatest + 1;   // greatest is numerically smallest
        const int prio = !s->by_work ? least
                         : n_ctx > 1 ? greatest + (int)((int64_t)rank * (levels - 1) / (n_ctx - 1)) : least;
        for (int32_t l = 0; l < s->lanes; ++l) {
            auto L = std::make_unique<Lane>();
            L->ctx = l == 0 ? ctxs[i] : pcv::ctx_clone(ctxs[i]);
            L->owned = l > 0;
            L->last_used = Clock::now();
            const bool ok = L->ctx && cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking, prio) == cudaSuccess;
            if (ok) {
                // the lane's work memory now, budget permitting: a lane whose first batch
                // allocated it would wait for the launches already running on the device
                const int64_t need = pcv::ctx_workspace_estimate(L->ctx, s->precision);
                if (s->budget <= 0.0 ||
                    (double)(s->used + pcv::ctx_workspace_resident(L->ctx) + need) <= s->budget)
                    if (pcv::ctx_reserve(L->ctx, s->precision, s->max_batch) != PCV_OK)
                        cudaGetLastError();   // the lane allocates at its first batch instead
            }
            if (L->ctx) {
                L->resident = pcv::ctx_workspace_resident(L->ctx);
                s->used += L->resident;
            }
            d->lanes.push_back(std::move(L));
            if (!ok) {
                s->ds.push_back(std::move(d));
                cleanup();
                return PCV_ERR_CUDA;
            }
        }
        s->ds.push_back(std::move(d));
    }
    pcv_server* raw = s.get();
    for (size_t i = 0; i < raw->ds.size(); ++i)
        for (size_t l = 0; l < raw->ds[i]->lanes.size(); ++l)
            raw->ds[i]->lanes[l]->worker = std::thread(worker, raw, i, l);
    *out = s.release();
    return PCV_OK;
}

PCV_API pcv_status pcv_server_submit_cv(pcv_server* s, int32_t dataset, const double* params3, int64_t* request_id) {
    if (!s || !params3) return PCV_ERR_ARG;
    auto r = std::make_shared<Request>();
    r->kind = Kind::Cv;
    r->dataset = dataset;
    std::memcpy(r->params, params3, sizeof(double) * 3);
    return submit(s, r, request_id);
}

PCV_API pcv_status pcv_server_submit_predict(pcv_server* s, int32_t dataset, const double* params3,
                                             const double* xy_new, int64_t m, int64_t* request_id) {
    if (!s || !params3 || m < 0 || (m > 0 && !xy_new)) return PCV_ERR_ARG;
    auto r = std::make_shared<Request>();
    r->kind = Kind::Predict;
    r->dataset = dataset;
    std::memcpy(r->params, params3, sizeof(double) * 3);
    r->xy.assign(xy_new, xy_new + 2 * m);
    return submit(s, r, request_id);
}

PCV_API pcv_status pcv_server_wait(pcv_server* s, int64_t request_id, double timeout_s, double* sspe,
                                   int32_t* status, double* yhat, double* latency_ms) {
    if (!s) return PCV_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return PCV_ERR_ARG;
    std::shared_ptr<Request> r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    if (!s->cv.wait_until(lk, deadline, [&] { return r->done || s->stop; })) return PCV_ERR_TIMEOUT;
    if (!r->done) return PCV_ERR_BUSY;
    if (sspe) *sspe = r->sspe;
    if (status) *status = r->status;
    if (yhat && !r->yhat.empty()) std::memcpy(yhat, r->yhat.data(), r->yhat.size() * sizeof(double));
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
    s->reqs.erase(it);
    return PCV_OK;
}

PCV_API pcv_status pcv_server_stats(pcv_server* s, double* p50_ms, double* p99_ms, double* cv_evals_per_s,
                                    int64_t* completed, int64_t* batches, int64_t* evictions) {
    if (!s) return PCV_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
        if (v.empty()) return 0.0;
        const size_t i = std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5));
        return v[i];
    };
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (cv_evals_per_s) {
        const double dt = s->any ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
        *cv_evals_per_s = dt > 0 ? (double)s->cv_done / dt : 0.0;
    }
    if (completed) *completed = s->cv_done + s->pred_done;
    if (batches) *batches = s->batches;
    if (evictions) *evictions = s->evictions;
    return PCV_OK;
}

PCV_API void pcv_server_destroy(pcv_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto& d : s->ds)
        for (auto& l : d->lanes) {
            if (l->worker.joinable()) l->worker.join();
            if (l->stream) cudaStreamDestroy(l->stream);
            if (l->owned) pcv::ctx_free(l->ctx);
        }
    delete s;
}
