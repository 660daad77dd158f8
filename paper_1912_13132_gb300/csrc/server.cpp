// server.cpp -- continuous-batching request loop over several device-resident datasets.
//
// The paper's Algorithm 1 evaluates one parameter configuration after another for
// an outer optimiser (Sec. 4.4: a grid of configurations evaluated sequentially).
// Here many clients submit CV-loss evaluations and prediction requests at any time:
//   * every dataset (a pcv_ctx) has a worker thread with its own stream; a worker
//     takes *all* CV requests queued for its dataset (up to max_batch) as one batch,
//     so requests that arrive while a batch runs join the next one;
//   * workers of different datasets run concurrently, so their kernels overlap on
//     the device;
//   * a batch is admitted only when its dataset's work memory fits the server's HBM
//     budget; idle datasets' work memory is released, least recently used first, to
//     make room, otherwise the worker waits for running batches to finish;
//   * results do not depend on the batching: every (subset, configuration) task is
//     computed on its own and the per-configuration sum has a fixed order.
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

struct Dataset {
    pcv_ctx* ctx;
    std::deque<std::shared_ptr<Request>> queue;
    bool busy = false;
    bool evicting = false;
    int64_t resident = 0;           // work-memory bytes accounted to this dataset
    Clock::time_point last_used;
    std::thread worker;
    cudaStream_t stream = nullptr;
};

}  // namespace

struct pcv_server {
    std::mutex mu;
    std::condition_variable cv;
    std::vector<std::unique_ptr<Dataset>> ds;
    std::unordered_map<int64_t, std::shared_ptr<Request>> reqs;
    int64_t next_id = 1;
    int32_t max_batch = 16;
    int32_t precision = PCV_PREC_MIXED;
    double budget = 0.0;            // 0: unlimited
    int64_t used = 0;
    bool stop = false;
    // statistics
    std::vector<double> lat_ms;
    int64_t cv_done = 0, pred_done = 0, batches = 0, evictions = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
};

namespace {

// Admission: make room for dataset d's work memory (called with the lock held).
bool admit(pcv_server* s, size_t d, std::unique_lock<std::mutex>& lk) {
    Dataset& D = *s->ds[d];
    for (;;) {
        if (s->stop) return false;
        const int64_t need = pcv::ctx_workspace_estimate(D.ctx, s->precision);
        if (s->budget <= 0.0 || (double)(s->used + need) <= s->budget) {
            s->used += need;
            D.resident += need;
            return true;
        }
        // evict the least recently used idle dataset that holds memory
        int victim = -1;
        for (size_t j = 0; j < s->ds.size(); ++j) {
            Dataset& V = *s->ds[j];
            if (j == d || V.busy || V.evicting || V.resident == 0) continue;
            if (victim < 0 || V.last_used < s->ds[victim]->last_used) victim = (int)j;
        }
        if (victim >= 0) {
            Dataset& V = *s->ds[victim];
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

void worker(pcv_server* s, size_t d) {
    Dataset& D = *s->ds[d];
    cudaSetDevice(pcv::ctx_device(D.ctx));
    std::vector<std::shared_ptr<Request>> batch;
    std::vector<double> params, sspe;
    std::vector<int32_t> status;
    for (;;) {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.wait(lk, [&] { return s->stop || (!D.queue.empty() && !D.evicting); });
        if (s->stop) return;
        batch.clear();
        if (D.queue.front()->kind == Kind::Predict) {
            batch.push_back(D.queue.front());
            D.queue.pop_front();
        } else {
            while (!D.queue.empty() && D.queue.front()->kind == Kind::Cv && (int)batch.size() < s->max_batch) {
                batch.push_back(D.queue.front());
                D.queue.pop_front();
            }
        }
        D.busy = true;
        if (!admit(s, d, lk)) {
            D.busy = false;
            return;
        }
        ++s->batches;
        lk.unlock();

        // run the batch (synchronous on this dataset's stream; other datasets proceed)
        if (batch[0]->kind == Kind::Cv) {
            const int32_t B = (int32_t)batch.size();
            params.resize(3 * B);
            sspe.assign(B, 0.0);
            status.assign(B, 0);
            for (int32_t b = 0; b < B; ++b) std::memcpy(&params[3 * b], batch[b]->params, sizeof(double) * 3);
            pcv_status st = pcv_cv_loss(D.ctx, params.data(), B, s->precision, sspe.data(), nullptr, nullptr, nullptr,
                                        status.data(), D.stream);
            for (int32_t b = 0; b < B; ++b) {
                batch[b]->sspe = st == PCV_OK ? sspe[b] : NAN;
                batch[b]->status = st == PCV_OK ? status[b] : (int32_t)st;
            }
        } else {
            Request& R = *batch[0];
            const int64_t m = (int64_t)R.xy.size() / 2;
            R.yhat.assign(m, 0.0);
            R.status = pcv_predict(D.ctx, R.params, R.xy.data(), m, s->precision, R.yhat.data(), D.stream);
        }

        lk.lock();
        const auto now = Clock::now();
        s->t_last = now;
        for (auto& r : batch) {
            r->t_done = now;
            r->done = true;
            s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
            if (r->kind == Kind::Cv) ++s->cv_done; else ++s->pred_done;
        }
        D.busy = false;
        D.last_used = now;
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
        if (opts->precision == PCV_PREC_FP64 || opts->precision == PCV_PREC_MIXED) s->precision = opts->precision;
        if (opts->hbm_budget_bytes > 0) s->budget = opts->hbm_budget_bytes;
    }
    // Stream priorities: the dataset with the least work per configuration gets the
    // highest priority, so that when launches of several datasets wait for SMs the
    // short ones are scheduled first (shortest job first lowers the mean latency;
    // a running launch is never pre-empted, so long jobs are delayed, not starved).
    std::vector<double> work(n_ctx);
    for (int32_t i = 0; i < n_ctx; ++i) work[i] = pcv::ctx_work_estimate(ctxs[i]);
    for (int32_t i = 0; i < n_ctx; ++i) {
        auto d = std::make_unique<Dataset>();
        d->ctx = ctxs[i];
        d->last_used = Clock::now();
        d->resident = pcv::ctx_workspace_resident(ctxs[i]);
        s->used += d->resident;
        cudaSetDevice(pcv::ctx_device(ctxs[i]));
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
        int rank = 0;   // datasets with strictly less work
        for (int32_t j = 0; j < n_ctx; ++j) rank += work[j] < work[i];
        const int levels = least - greatest + 1;   // greatest is numerically smallest
        const int prio = n_ctx > 1 ? greatest + (int)((int64_t)rank * (levels - 1) / (n_ctx - 1)) : least;
        if (cudaStreamCreateWithPriority(&d->stream, cudaStreamNonBlocking, prio) != cudaSuccess) {
            for (auto& e : s->ds) cudaStreamDestroy(e->stream);
            return PCV_ERR_CUDA;
        }
        s->ds.push_back(std::move(d));
    }
    pcv_server* raw = s.get();
    for (size_t i = 0; i < raw->ds.size(); ++i) raw->ds[i]->worker = std::thread(worker, raw, i);
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
    for (auto& d : s->ds) {
        if (d->worker.joinable()) d->worker.join();
        if (d->stream) cudaStreamDestroy(d->stream);
    }
    delete s;
}
