// api.cu -- the C ABI of include/pcv.h: plans, device contexts and dispatch.
//
// pcv_create builds the subset membership (Sec. 2.3) once on the host and keeps
// the data and the membership resident in device memory (Algorithm 1: "dividing
// and reading the data have to be done once" for many parameter configurations).
// pcv_cv_loss then runs one persistent launch over all (subset, configuration)
// tasks and the fixed-order combine (Eq. 6).
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "pcv_internal.h"

namespace {

thread_local std::string g_err;

pcv_status fail(pcv_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

pcv_status cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PCV_ERR_OOM : PCV_ERR_CUDA;
}

#define CUDA_TRY(expr)                                              \
    do {                                                            \
        cudaError_t e_ = (expr);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr);         \
    } while (0)

// Device buffer that grows on demand.  Growing never frees the old allocation at once:
// cudaFree waits for the whole device, which would stall a call behind kernels other
// streams (other serving lanes) are running; the old block is kept until release() (the
// context idle or destroyed), and growth is geometric so that few such blocks pile up.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    std::vector<T*> retired;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        for (T* q : retired) cudaFree(q);
        retired.clear();
        p = nullptr;
        n = 0;
    }
    cudaError_t reserve(size_t want) {
        want = std::max<size_t>(want, 1);
        if (want <= n && p) return cudaSuccess;
        size_t cnt = std::max(want, n + n / 2);
        T* q = nullptr;
        cudaError_t e = cudaMalloc(&q, cnt * sizeof(T));
        if (e != cudaSuccess && cnt > want) {   // the geometric size did not fit: the exact one may
            cudaGetLastError();
            cnt = want;
            e = cudaMalloc(&q, cnt * sizeof(T));
        }
        if (e != cudaSuccess) return e;
        if (p) retired.push_back(p);
        p = q;
        n = cnt;
        return cudaSuccess;
    }
};

struct Workspace {
    DevBuf<unsigned char> mem;
    DevBuf<unsigned char> planes;          // mixed path, tensor engines: 16-bit planes of the factors
    int64_t plane_elems = 0;
    alignas(64) unsigned char maps[3 * 128];   // CUtensorMap x 3 over the planes
    int grid = 0;
    int32_t ld = 0;
    int64_t slot_bytes = 0;
};

// One size bucket of the mixed CV launch: the active subsets whose training sizes fall
// in [klo, khi], their own slot size (ld), factorisation engine, workspace, task counter
// and stream (buckets run side by side, forked from and joined to the caller's stream).
struct Bucket {
    int32_t klo = 0, khi = 0;
    int engine = 0;
    double work = 0.0;                    // sum of k^3 over the bucket's subsets
    std::vector<int32_t> subsets;         // longest first
    DevBuf<int32_t> order;
    Workspace ws;
    DevBuf<unsigned int> counter;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    ~Bucket() {
        if (done) cudaEventDestroy(done);
        if (stream) cudaStreamDestroy(stream);
    }
};

// Kriging weights of recent configurations: a pool of `cap` rows of T_off[N] doubles,
// one row per (rho, lambda, precision), least recently used replaced first; a row in
// use by a running call is pinned and never replaced.  Guarded by mu (serving lanes of
// one dataset share it from their worker threads).
struct AlphaEntry {
    double rho = 0.0, lam = 0.0;
    int32_t prec = -1;
    std::vector<uint8_t> have;   // subsets whose weights the row holds
    uint64_t used = 0;
    int pins = 0;
};
struct AlphaCache {
    std::mutex mu;
    int cap = 0;
    DevBuf<double> pool;
    std::vector<AlphaEntry> rows;
    uint64_t clock = 0;
    int64_t hits = 0, misses = 0;
};

}  // namespace

struct pcv_plan {
    pcv::Plan p;
};

struct pcv_ctx {
    int device = 0;
    int sms = 0;
    pcv::Plan plan;
    pcv_options opts{};
    DevBuf<double> X, Y, V;                 // all points
    DevBuf<int64_t> Toff, Voff;
    DevBuf<int32_t> Tidx;
    DevBuf<double> Vx, Vy, Vv;              // validation points in membership order
    // lattice data: all points at integer multiples of (lat_hx, lat_hy) from one origin
    bool lattice = false;
    double lat_hx = 0.0, lat_hy = 0.0;
    int64_t lat_cap = 0;                    // largest covariance table of a subset (entries)
    DevBuf<int32_t> LX, LY, VLX, VLY;       // lattice indices of all points and of the validation points
    DevBuf<int32_t> order;                  // subsets with validation data, longest first
    int32_t n_active = 0;
    int32_t kmax = 0;
    int64_t mmax = 0;
    int64_t nV = 0;
    double coord_scale = 1.0;               // power of two, window offsets scaled below 1
    DevBuf<int32_t> fb_list;                // mixed path: tasks handed to the FP64 kernel
    DevBuf<unsigned int> fb_count;
    // per-call buffers
    DevBuf<double> z, params, sspe;
    DevBuf<double> lik, lik_total;          // local -2 log-likelihoods and their sums
    DevBuf<int32_t> tst, status;
    DevBuf<unsigned int> counter;
    // work memory: [0] FP64, [2] FP64 fallback of the mixed path, [3 + e] mixed engine e
    Workspace ws[3 + pcv::kMixedEngines];
    int32_t tc_stages_set = 0;              // ring depth the caller asked for (0: each engine's default)
    // prediction buffers
    DevBuf<double> Px, Py, Pyhat;
    DevBuf<double> yv;                      // validation predictions of the host-buffer CV call
    DevBuf<int64_t> Poff;
    DevBuf<int32_t> Porder;
    DevBuf<int32_t> prow;                   // parameter row of each subset (local predictions)
    DevBuf<double> rhs;                     // several right-hand sides (GLS), column-major n x r
    std::vector<double> hxy;                // host copy of the coordinates (GLS)
    std::vector<double> hv;                 // host copy of the values (GLS)
    // optional kernel timing (events on the launching stream)
    bool timing = false;
    bool timed_task = false, timed_combine = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    DevBuf<unsigned long long> phase;       // per-phase cycle counters of the mixed kernel
    // size buckets of the mixed CV launch (built at the first mixed CV call)
    std::vector<std::unique_ptr<Bucket>> buckets;
    bool buckets_tuned = false;             // the engines were chosen by timing, not by rule
    cudaEvent_t fork = nullptr;
    std::string bucket_desc;
    // CUDA graph of the mixed CV call (the buckets' launches, the FP64 fallback and the
    // combine), captured at the second call of a shape and replayed while the buffers it
    // names stay in place; parameters and results pass through the context's buffers
    // kriging weights of recent configurations (pcv_cv_loss and pcv_predict keep them),
    // so that predictions at new locations need no factorisation; shared with the
    // context's serving lanes (ctx_clone)
    std::shared_ptr<AlphaCache> alpha;
    DevBuf<int32_t> alpha_slot;             // the current call's row per configuration
    bool alpha_call = false;                // this call stores weights (alpha_slot is set)
    bool alpha_in_call = false;             // this call predicts from stored weights
    cudaGraphExec_t gexec = nullptr;
    int64_t gkey = -1, gseen = -1;
    std::vector<const void*> gprint;
    cudaStream_t gcap = nullptr;
    bool capturing = false;
    int64_t graph_launches = 0;             // replays so far
    uint64_t mem_gen = 0;                   // bumped whenever work memory is released or buckets rebuilt
    int64_t graph_kernels = 0;              // kernel launches inside the captured graph
    DevBuf<double> gparams, gsspe, gyhat;
    DevBuf<int32_t> gstatus;
    ~pcv_ctx() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gcap) cudaStreamDestroy(gcap);
        buckets.clear();
        if (fork) cudaEventDestroy(fork);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace {

pcv_options default_options(const pcv_options* o) {
    pcv_options d{};
    d.struct_size = sizeof(pcv_options);
    d.max_slots = 0;
    d.workspace_fraction = 0.5;
    d.refine_max_iter = 6;
    d.refine_tol = 2e-8;
    d.factor_engine = pcv::kMixedEngineTensor;
    d.tc_stages = 0;
    d.refine_loss_tol = 2e-8;
    d.bucketing = 0;
    d.graph = 0;
    d.alpha_cache = 32;
    d.test_wait_us = 0;
    d.refine_loss_guard = 1000.0;
    d.test_withhold_task = 0;
    if (o) {
        if (o->struct_size != 0 && o->struct_size != (int32_t)sizeof(pcv_options)) return d;
        if (o->max_slots > 0) d.max_slots = o->max_slots;
        if (o->workspace_fraction > 0 && o->workspace_fraction <= 0.95) d.workspace_fraction = o->workspace_fraction;
        if (o->refine_max_iter > 0) d.refine_max_iter = o->refine_max_iter;
        if (o->refine_tol > 0) d.refine_tol = o->refine_tol;
        if (o->factor_engine > 0 && o->factor_engine < pcv::kMixedEngines) d.factor_engine = o->factor_engine;
        if (o->tc_stages >= 2 && o->tc_stages <= 4) d.tc_stages = o->tc_stages;
        if (o->bucketing == 1) d.bucketing = 1;
        if (o->graph == 1) d.graph = 1;
        if (o->alpha_cache > 0) d.alpha_cache = std::min(o->alpha_cache, 4096);
        else if (o->alpha_cache < 0) d.alpha_cache = 0;
        if (o->test_wait_us > 0) d.test_wait_us = o->test_wait_us;
        if (o->refine_loss_guard > 0) d.refine_loss_guard = o->refine_loss_guard;
        else if (o->refine_loss_guard < 0) d.refine_loss_guard = 0.0;   // no guard
        if (o->test_withhold_task > 0) d.test_withhold_task = o->test_withhold_task;
        if (o->refine_loss_tol > 0) d.refine_loss_tol = o->refine_loss_tol;
        else if (o->refine_loss_tol < 0) d.refine_loss_tol = 0.0;   // solution rule only
    }
    if (d.tc_stages == 0) d.tc_stages = pcv::mixed_default_stages(d.factor_engine);
    // (the explicit engine modes take their own default depth unless the caller set one)
    return d;
}

int32_t round_up(int64_t v, int64_t m) { return (int32_t)(((std::max<int64_t>(v, 1) + m - 1) / m) * m); }

// Allocate the per-CTA workspace slots of one precision (once per context).
constexpr int kFallbackWs = 2;          // index of the fallback workspace
constexpr int kMixedWs0 = 3;            // workspace of mixed engine e: kMixedWs0 + e

bool is_mixed(int32_t prec) { return prec != PCV_PREC_FP64; }

// The factorisation engine of a mixed precision mode (-1 for FP64).
int engine_of(const pcv_ctx* c, int32_t prec) {
    switch (prec) {
        case PCV_PREC_MIXED: return c->opts.factor_engine;
        case PCV_PREC_MIXED_TF32: return pcv::kMixedEngineTensorTF32;
        case PCV_PREC_MIXED_TF32X3: return pcv::kMixedEngineTensorTF32x3;
        case PCV_PREC_MIXED_BF16X3: return pcv::kMixedEngineTensorBF16;
        case PCV_PREC_MIXED_F16X2: return pcv::kMixedEngineTensor;
        default: return -1;
    }
}

// Workspace index of a precision mode.
int ws_of(const pcv_ctx* c, int32_t prec) { return is_mixed(prec) ? kMixedWs0 + engine_of(c, prec) : 0; }

// TMA ring depth of an engine: the caller's choice, else the engine's default.
int32_t stages_for(const pcv_ctx* c, int engine) {
    return c->tc_stages_set ? c->tc_stages_set : pcv::mixed_default_stages(engine);
}
constexpr int kFallbackSlots = 32;      // tasks needing the FP64 fallback are rare

// Slot count (before the free-memory clamp) and bytes per slot of workspace `wi`
// (0 FP64, kFallbackWs, or kMixedWs0 + engine).
void workspace_shape(const pcv_ctx* c, int wi, int64_t& g, int64_t& sb, int64_t& pb, int32_t& ld) {
    const bool fallback = wi == kFallbackWs;
    const bool mixed = wi >= kMixedWs0;
    const int prec = mixed ? PCV_PREC_MIXED : PCV_PREC_FP64;
    const int engine = mixed ? wi - kMixedWs0 : -1;
    ld = round_up(c->kmax, 128);
    const int planes = mixed ? pcv::mixed_planes(engine) : 0;
    const bool tensor = planes > 0;
    sb = prec == PCV_PREC_FP64 ? pcv::slot_bytes_fp64(ld, c->mmax)
                               : pcv::slot_bytes_mixed(ld, c->mmax, c->lattice ? c->lat_cap : 0);
    pb = (int64_t)planes * ld * ld * (tensor ? pcv::mixed_term_bytes(engine) : 0);   // planes per slot
    // CTAs per SM: two for both mixed engines (the tensor engine holds half of an
    // SM's tensor memory per CTA), one for the FP64 kernel
    const int per_sm = prec == PCV_PREC_MIXED ? 2 : 1;
    g = c->opts.max_slots > 0 ? c->opts.max_slots : (int64_t)c->sms * per_sm;
    if (tensor) g = std::min<int64_t>(g, 2 * (int64_t)c->sms);
    if (fallback) g = std::min<int64_t>(g, kFallbackSlots);
}

// Allocate `g` slots of sb bytes plus pb bytes of planes each (at most the context's
// share of free device memory) for slots of leading dimension ld, with the tensor maps
// of a tensor engine's `np` planes.
pcv_status alloc_workspace(pcv_ctx* c, Workspace& w, int64_t g, int64_t sb, int64_t pb, int32_t ld, int np,
                           int term_bytes = 2) {
    size_t free_b = 0, total_b = 0;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    const double budget = c->opts.workspace_fraction * (double)free_b;
    g = std::min<int64_t>(g, (int64_t)(budget / (double)(sb + pb)));
    if (g < 1) return fail(PCV_ERR_OOM, "workspace for one task does not fit in device memory");
    cudaError_t e = w.mem.reserve((size_t)(g * sb));
    if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    if (pb > 0) {
        w.plane_elems = g * (int64_t)ld * ld * (term_bytes / 2);   // 16-bit units per plane
        e = w.planes.reserve((size_t)(np * w.plane_elems * 2));
        if (e != cudaSuccess) return cuda_fail(e, "plane allocation");
        if (!pcv::mixed_make_maps(w.planes.p, w.plane_elems, ld, (int)g, np, term_bytes, w.maps))
            return fail(PCV_ERR_CUDA, "tensor map encoding failed");
    }
    w.grid = (int)g;
    w.ld = ld;
    w.slot_bytes = sb;
    return PCV_OK;
}

pcv_status ensure_workspace(pcv_ctx* c, int wi) {
    Workspace& w = c->ws[wi];
    if (w.grid > 0) return PCV_OK;
    int64_t g, sb, pb;
    int32_t ld;
    workspace_shape(c, wi, g, sb, pb, ld);
    const int engine = wi >= kMixedWs0 ? wi - kMixedWs0 : -1;
    return alloc_workspace(c, w, g, sb, pb, ld, pb > 0 ? pcv::mixed_planes(engine) : 0,
                           pb > 0 ? pcv::mixed_term_bytes(engine) : 2);
}

// Mixed-path slot shape of a given slot size and engine (two CTAs per SM).
void mixed_shape(const pcv_ctx* c, int32_t ld, int engine, int64_t& g, int64_t& sb, int64_t& pb) {
    const int planes = pcv::mixed_planes(engine);
    sb = pcv::slot_bytes_mixed(ld, c->mmax, c->lattice ? c->lat_cap : 0);
    pb = (int64_t)planes * ld * ld * pcv::mixed_term_bytes(engine);
    g = c->opts.max_slots > 0 ? c->opts.max_slots : 2 * (int64_t)c->sms;
    if (planes > 0) g = std::min<int64_t>(g, 2 * (int64_t)c->sms);
}

bool bad_precision(int32_t p) { return p < PCV_PREC_FP64 || p > PCV_PREC_MIXED_F16X2; }

// Whether the values v all lie on v0 + i h for integers 0 <= i < 2^31, h the smallest
// gap between distinct values refined over the whole range.  The slack is a few FP64
// ulps of the largest coordinate (16 eps (max|v| / h + steps) in units of h): snapping a
// point to its lattice node then moves it no more than the rounding of its coordinate
// already did, so the tabulated covariances equal the exact ones to FP64 input accuracy.
bool lattice_axis(const std::vector<double>& v, double& v0, double& h, std::vector<int32_t>& idx) {
    std::vector<double> u(v);
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
    idx.assign(v.size(), 0);
    if (u.empty()) return false;
    v0 = u[0];
    if (u.size() == 1) {
        h = 1.0;
        return true;
    }
    double g = INFINITY;
    for (size_t q = 1; q < u.size(); ++q) g = std::min(g, u[q] - u[q - 1]);
    if (!(g > 0.0)) return false;
    const double span = u.back() - u[0];
    const double steps = std::nearbyint(span / g);
    if (!(steps >= 1.0) || steps > 2147483647.0) return false;
    h = span / steps;
    const double tol = 16.0 * DBL_EPSILON * (std::max(std::fabs(u.front()), std::fabs(u.back())) / h + steps);
    for (size_t q = 0; q < v.size(); ++q) {
        const double t = (v[q] - v0) / h;
        const double r = std::nearbyint(t);
        if (!(std::fabs(t - r) <= tol) || r < 0.0 || r > 2147483647.0) return false;
        idx[q] = (int32_t)r;
    }
    return true;
}

}  // namespace

// ----------------------------------------------------------------- helpers for the server

static pcv_status ensure_buckets(pcv_ctx* c, const double* d_params, int32_t B, cudaStream_t s);

namespace pcv {

int64_t ctx_workspace_estimate(pcv_ctx* c, int32_t prec) {
    int64_t total = 0;
    const int list[2] = {ws_of(c, prec), is_mixed(prec) ? kFallbackWs : -1};
    for (int wi : list) {
        if (wi < 0 || c->ws[wi].grid > 0) continue;
        if (prec == PCV_PREC_MIXED && wi == ws_of(c, prec) && !c->buckets.empty()) continue;   // buckets are held
        int64_t g, sb, pb;
        int32_t ld;
        workspace_shape(c, wi, g, sb, pb, ld);
        total += g * (sb + pb);
    }
    return total;
}

// Everything a CV call of up to Bmax configurations in precision prec allocates (work
// memory, per-call buffers and, for PCV_PREC_MIXED, the size buckets with theirs),
// allocated now, so that such a call allocates nothing: a device allocation is ordered
// after the kernels already running in other streams, and a serving lane whose first
// call allocated would wait for the other lanes' launches.  The buckets are built here
// when the process holds the autotuner's choice for this context's subset sizes;
// otherwise the first call builds them (tuning needs its parameters).
pcv_status ctx_reserve(pcv_ctx* c, int32_t prec, int32_t Bmax) {
    if (!c || bad_precision(prec) || Bmax < 1) return PCV_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    const int32_t N = c->plan.N;
    CUDA_TRY(c->params.reserve((size_t)3 * Bmax));
    CUDA_TRY(c->sspe.reserve(Bmax));
    CUDA_TRY(c->status.reserve(Bmax));
    CUDA_TRY(c->alpha_slot.reserve(Bmax));
    CUDA_TRY(c->z.reserve((size_t)Bmax * N));
    CUDA_TRY(c->tst.reserve((size_t)Bmax * N));
    if (c->n_active == 0) return PCV_OK;
    if (is_mixed(prec)) {
        const int e = pcv::mixed_prepare(c->device);
        if (e) return cuda_fail((cudaError_t)e, "mixed-path set-up");
    }
    if (prec == PCV_PREC_MIXED) {
        if (ensure_buckets(c, nullptr, Bmax, nullptr) != PCV_OK) cudaGetLastError();   // the first call builds them
    } else {
        const pcv_status st = ensure_workspace(c, ws_of(c, prec));
        if (st != PCV_OK) return st;
    }
    if (is_mixed(prec)) {
        const pcv_status st = ensure_workspace(c, kFallbackWs);
        if (st != PCV_OK) return st;
        CUDA_TRY(c->fb_list.reserve((size_t)c->n_active * Bmax));
        CUDA_TRY(c->fb_count.reserve(2));
    }
    return PCV_OK;
}

int64_t ctx_workspace_resident(pcv_ctx* c) {
    int64_t t = 0;
    for (const auto& w : c->ws) t += (int64_t)(w.mem.n * sizeof(unsigned char) + w.planes.n);
    for (const auto& b : c->buckets) t += (int64_t)(b->ws.mem.n + b->ws.planes.n);
    return t;
}

void ctx_release_workspace(pcv_ctx* c) {
    cudaSetDevice(c->device);
    for (auto& w : c->ws) {
        w.mem.release();
        w.planes.release();
        w.grid = 0;
        w.plane_elems = 0;
    }
    c->buckets.clear();   // rebuilt at the next mixed CV call (the tuner's choice is cached)
    ++c->mem_gen;         // a captured graph of the CV call names freed memory now
}

int ctx_device(const pcv_ctx* c) { return c->device; }

// A second context over the same data on the same device (a serving lane): the plan,
// options and device arrays are copied, the kriging-weight cache is shared, work memory
// and per-call buffers are its own.  nullptr on failure.
template <class T>
static bool copy_buf(DevBuf<T>& dst, const DevBuf<T>& src) {
    if (!src.p) return true;
    if (dst.reserve(src.n) != cudaSuccess) return false;
    return cudaMemcpy(dst.p, src.p, src.n * sizeof(T), cudaMemcpyDeviceToDevice) == cudaSuccess;
}

pcv_ctx* ctx_clone(const pcv_ctx* c) {
    if (cudaSetDevice(c->device) != cudaSuccess) return nullptr;
    std::unique_ptr<pcv_ctx> d(new (std::nothrow) pcv_ctx);
    if (!d) return nullptr;
    try {
        d->device = c->device;
        d->sms = c->sms;
        d->plan = c->plan;
        d->opts = c->opts;
        d->hxy = c->hxy;
        d->hv = c->hv;
    } catch (const std::bad_alloc&) {
        return nullptr;
    }
    d->lattice = c->lattice;
    d->lat_hx = c->lat_hx;
    d->lat_hy = c->lat_hy;
    d->lat_cap = c->lat_cap;
    d->n_active = c->n_active;
    d->kmax = c->kmax;
    d->mmax = c->mmax;
    d->nV = c->nV;
    d->coord_scale = c->coord_scale;
    d->alpha = c->alpha;
    const bool ok = copy_buf(d->X, c->X) && copy_buf(d->Y, c->Y) && copy_buf(d->V, c->V) &&
                    copy_buf(d->Toff, c->Toff) && copy_buf(d->Voff, c->Voff) && copy_buf(d->Tidx, c->Tidx) &&
                    copy_buf(d->Vx, c->Vx) && copy_buf(d->Vy, c->Vy) && copy_buf(d->Vv, c->Vv) &&
                    copy_buf(d->LX, c->LX) && copy_buf(d->LY, c->LY) && copy_buf(d->VLX, c->VLX) &&
                    copy_buf(d->VLY, c->VLY) && copy_buf(d->order, c->order) &&
                    d->counter.reserve(1) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return nullptr;
    }
    return d.release();
}

void ctx_free(pcv_ctx* c) { pcv_destroy(c); }

double ctx_work_estimate(const pcv_ctx* c) {
    const Plan& P = c->plan;
    double w = 0.0;
    for (int32_t i = 0; i < P.N; ++i) {
        if (P.V_off[i + 1] == P.V_off[i]) continue;
        const double k = (double)(P.T_off[i + 1] - P.T_off[i]);
        w += k * k * k;
    }
    return w;
}

}  // namespace pcv

// ----------------------------------------------------------------- plans

PCV_API pcv_status pcv_plan_create(const double* xy, const uint8_t* role, int64_t n, const pcv_layout* layout,
                                   pcv_plan** out) {
    if (!out) return fail(PCV_ERR_ARG, "NULL out");
    *out = nullptr;
    std::unique_ptr<pcv_plan> p(new (std::nothrow) pcv_plan);
    if (!p) return fail(PCV_ERR_OOM, "host allocation");
    std::string err;
    try {
        pcv_status s = pcv::build_plan(xy, role, n, layout, p->p, err);
        if (s != PCV_OK) return fail(s, err);
    } catch (const std::bad_alloc&) {
        return fail(PCV_ERR_OOM, "host allocation");
    }
    *out = p.release();
    return PCV_OK;
}

static pcv_status plan_views(const pcv::Plan& P, int32_t* N, const int64_t** To, const int64_t** Ti,
                             const int64_t** Vo, const int64_t** Vi) {
    if (N) *N = P.N;
    if (To) *To = P.T_off.data();
    if (Ti) *Ti = P.T_idx.data();
    if (Vo) *Vo = P.V_off.data();
    if (Vi) *Vi = P.V_idx.data();
    return PCV_OK;
}

PCV_API pcv_status pcv_plan_info(const pcv_plan* plan, int32_t* N, const int64_t** T_off, const int64_t** T_idx,
                                 const int64_t** V_off, const int64_t** V_idx) {
    if (!plan) return fail(PCV_ERR_ARG, "NULL plan");
    return plan_views(plan->p, N, T_off, T_idx, V_off, V_idx);
}

PCV_API pcv_status pcv_plan_cores(const pcv_plan* plan, pcv_rect* cores) {
    if (!plan || !cores) return fail(PCV_ERR_ARG, "NULL argument");
    std::copy(plan->p.cores.begin(), plan->p.cores.end(), cores);
    return PCV_OK;
}

PCV_API void pcv_plan_destroy(pcv_plan* plan) { delete plan; }

// ----------------------------------------------------------------- contexts

PCV_API pcv_status pcv_create(const double* xy, const double* v, const uint8_t* role, int64_t n,
                              const pcv_layout* layout, int32_t device, const pcv_options* opts, pcv_ctx** out) {
    if (!out) return fail(PCV_ERR_ARG, "NULL out");
    *out = nullptr;
    if (n > 0 && !v) return fail(PCV_ERR_ARG, "NULL values");
    for (int64_t j = 0; j < n; ++j)
        if (!std::isfinite(v[j])) return fail(PCV_ERR_ARG, "non-finite value");
    std::unique_ptr<pcv_ctx> c(new (std::nothrow) pcv_ctx);
    if (!c) return fail(PCV_ERR_OOM, "host allocation");
    std::string err;
    try {
        pcv_status s = pcv::build_plan(xy, role, n, layout, c->plan, err);
        if (s != PCV_OK) return fail(s, err);
    } catch (const std::bad_alloc&) {
        return fail(PCV_ERR_OOM, "host allocation");
    }
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(PCV_ERR_ARG, "bad device index");
    CUDA_TRY(cudaSetDevice(device));
    c->device = device;
    CUDA_TRY(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device));
    c->opts = default_options(opts);
    c->tc_stages_set = opts && (opts->struct_size == 0 || opts->struct_size == (int32_t)sizeof(pcv_options)) &&
                               opts->tc_stages >= 2 && opts->tc_stages <= 4 ? opts->tc_stages : 0;
    c->alpha = std::make_shared<AlphaCache>();
    c->alpha->cap = c->opts.alpha_cache;
    const pcv::Plan& P = c->plan;
    const int32_t N = P.N;

    c->hxy.assign(xy, xy + 2 * n);
    c->hv.assign(v, v + n);
    // points as SoA
    std::vector<double> hx(n), hy(n);
    for (int64_t j = 0; j < n; ++j) { hx[j] = xy[2 * j]; hy[j] = xy[2 * j + 1]; }
    CUDA_TRY(c->X.reserve(n));
    CUDA_TRY(c->Y.reserve(n));
    CUDA_TRY(c->V.reserve(n));
    if (n) {
        CUDA_TRY(cudaMemcpy(c->X.p, hx.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->Y.p, hy.data(), n * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->V.p, v, n * sizeof(double), cudaMemcpyHostToDevice));
    }
    // membership
    std::vector<int32_t> tidx(P.T_idx.begin(), P.T_idx.end());
    CUDA_TRY(c->Toff.reserve(N + 1));
    CUDA_TRY(c->Voff.reserve(N + 1));
    CUDA_TRY(c->Tidx.reserve(tidx.size()));
    CUDA_TRY(cudaMemcpy(c->Toff.p, P.T_off.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c->Voff.p, P.V_off.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    if (!tidx.empty()) CUDA_TRY(cudaMemcpy(c->Tidx.p, tidx.data(), tidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    // validation points in membership order
    const int64_t nV = P.V_off[N];
    c->nV = nV;
    std::vector<double> vx(nV), vy(nV), vv(nV);
    for (int64_t q = 0; q < nV; ++q) {
        const int64_t j = P.V_idx[q];
        vx[q] = xy[2 * j];
        vy[q] = xy[2 * j + 1];
        vv[q] = v[j];
    }
    CUDA_TRY(c->Vx.reserve(nV));
    CUDA_TRY(c->Vy.reserve(nV));
    CUDA_TRY(c->Vv.reserve(nV));
    if (nV) {
        CUDA_TRY(cudaMemcpy(c->Vx.p, vx.data(), nV * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->Vy.p, vy.data(), nV * sizeof(double), cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(c->Vv.p, vv.data(), nV * sizeof(double), cudaMemcpyHostToDevice));
    }
    // active subsets (with validation data, Sec. 4.3.1), longest first
    std::vector<int32_t> ord;
    for (int32_t i = 0; i < N; ++i)
        if (P.V_off[i + 1] > P.V_off[i]) ord.push_back(i);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
        return (P.T_off[a + 1] - P.T_off[a]) > (P.T_off[b + 1] - P.T_off[b]);
    });
    c->n_active = (int32_t)ord.size();
    c->kmax = 0;
    c->mmax = 0;
    for (int32_t i : ord) {
        c->kmax = std::max<int32_t>(c->kmax, (int32_t)(P.T_off[i + 1] - P.T_off[i]));
        c->mmax = std::max<int64_t>(c->mmax, P.V_off[i + 1] - P.V_off[i]);
    }
    // power-of-two scale so that offsets between training points of one window are below 1
    double wmax = 0.0;
    for (const pcv_rect& r : P.cores) wmax = std::max({wmax, r.x1 - r.x0, r.y1 - r.y0});
    wmax += 2.0 * P.delta;
    c->coord_scale = wmax > 0.0 ? std::ldexp(1.0, -std::ilogb(wmax) - 1) : 1.0;
    CUDA_TRY(c->order.reserve(ord.size()));
    if (!ord.empty()) CUDA_TRY(cudaMemcpy(c->order.p, ord.data(), ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    // lattice data: covariances then depend on the index offsets only, and the mixed
    // path tabulates them per task (the largest table over the subsets sizes the slots)
    {
        double x0 = 0.0, y0 = 0.0;
        std::vector<int32_t> ix, iy;
        if (n > 0 && lattice_axis(hx, x0, c->lat_hx, ix) && lattice_axis(hy, y0, c->lat_hy, iy)) {
            int64_t cap = 0;
            for (int32_t i : ord) {
                int32_t a0 = INT32_MAX, a1 = INT32_MIN, b0 = INT32_MAX, b1 = INT32_MIN;
                auto take = [&](int64_t j) {
                    a0 = std::min(a0, ix[j]); a1 = std::max(a1, ix[j]);
                    b0 = std::min(b0, iy[j]); b1 = std::max(b1, iy[j]);
                };
                for (int64_t q = P.T_off[i]; q < P.T_off[i + 1]; ++q) take(P.T_idx[q]);
                for (int64_t q = P.V_off[i]; q < P.V_off[i + 1]; ++q) take(P.V_idx[q]);
                if (a1 >= a0) cap = std::max<int64_t>(cap, (int64_t)(a1 - a0 + 1) * (b1 - b0 + 1));
            }
            // tables up to 2^21 entries (16 MB per slot); beyond that the general path
            if (cap > 0 && cap <= (1 << 21)) {
                c->lattice = true;
                c->lat_cap = cap;
                std::vector<int32_t> vix(nV), viy(nV);
                for (int64_t q = 0; q < nV; ++q) { vix[q] = ix[P.V_idx[q]]; viy[q] = iy[P.V_idx[q]]; }
                CUDA_TRY(c->LX.reserve(n));
                CUDA_TRY(c->LY.reserve(n));
                CUDA_TRY(c->VLX.reserve(nV));
                CUDA_TRY(c->VLY.reserve(nV));
                CUDA_TRY(cudaMemcpy(c->LX.p, ix.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
                CUDA_TRY(cudaMemcpy(c->LY.p, iy.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
                if (nV) {
                    CUDA_TRY(cudaMemcpy(c->VLX.p, vix.data(), nV * sizeof(int32_t), cudaMemcpyHostToDevice));
                    CUDA_TRY(cudaMemcpy(c->VLY.p, viy.data(), nV * sizeof(int32_t), cudaMemcpyHostToDevice));
                }
            }
        }
    }
    CUDA_TRY(c->counter.reserve(1));
    *out = c.release();
    return PCV_OK;
}

PCV_API pcv_status pcv_subset_info(const pcv_ctx* c, int32_t* N, const int64_t** T_off, const int64_t** T_idx,
                                   const int64_t** V_off, const int64_t** V_idx) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    return plan_views(c->plan, N, T_off, T_idx, V_off, V_idx);
}

// The fields of a task-kernel launch that do not depend on the workspace.
static pcv::TaskArgs base_args(pcv_ctx* c, const double* d_params, int32_t B, const int64_t* P_off, const double* Px,
                               const double* Py, const double* Pv, const int32_t* order, int32_t n_order,
                               double* d_yhat, int64_t yhat_stride, bool want_lik, const int32_t* d_param_row,
                               const double* d_rhs, int32_t nrhs, bool lattice) {
    pcv::TaskArgs a{};
    a.X = c->X.p;
    a.Y = c->Y.p;
    a.Vals = c->V.p;
    a.T_off = c->Toff.p;
    a.T_idx = c->Tidx.p;
    a.P_off = P_off;
    a.Px = Px;
    a.Py = Py;
    a.Pv = Pv;
    a.order = order;
    a.n_order = n_order;
    a.params = d_params;
    a.B = B;
    a.N = c->plan.N;
    a.z = c->z.p;
    a.lik = want_lik ? c->lik.p : nullptr;
    a.param_row = d_param_row;
    a.rhs = d_rhs;
    a.nrhs = nrhs;
    a.rhs_stride = (int64_t)c->plan.n;
    // the slots hold the lattice table whenever the data are a lattice; the lattice
    // variant runs where the prediction points are lattice points too (the CV loss)
    a.lat_cap = c->lattice ? c->lat_cap : 0;
    if (lattice && c->lattice) {
        a.LX = c->LX.p;
        a.LY = c->LY.p;
        a.PLX = c->VLX.p;
        a.PLY = c->VLY.p;
        a.lat_hx = c->lat_hx;
        a.lat_hy = c->lat_hy;
    }
    a.tstatus = c->tst.p;
    a.yhat = d_yhat;
    a.yhat_stride = yhat_stride;
    a.counter = c->counter.p;
    a.refine_max_iter = c->opts.refine_max_iter;
    a.refine_tol = c->opts.refine_tol;
    a.refine_loss_tol = c->opts.refine_loss_tol;
    a.refine_loss_guard = c->opts.refine_loss_guard;
    a.coord_scale = c->coord_scale;
    a.fb_list = c->fb_list.p;
    a.fb_count = c->fb_count.p;
    a.phase_cycles = c->timing ? c->phase.p : nullptr;
    a.tc_stages = c->opts.tc_stages;
    a.test_wait_ns = c->opts.test_wait_us > 0 ? (uint64_t)c->opts.test_wait_us * 1000ull : 0;
    a.test_withhold_task = c->opts.test_withhold_task > 0 ? c->opts.test_withhold_task : 0;
    if (c->alpha_call || c->alpha_in_call) {
        if (c->alpha_in_call) a.alpha_in = c->alpha->pool.p;
        else a.alpha_out = c->alpha->pool.p;
        a.alpha_slot = c->alpha_slot.p;
        a.alpha_stride = c->plan.T_off[c->plan.N];
    }
    return a;
}

// ---------------------------------------------------------------- kriging-weight cache

// The row of (rho, lambda, precision), or -1 (cache lock held).
static int alpha_find(const AlphaCache& A, double rho, double lam, int32_t prec) {
    for (size_t q = 0; q < A.rows.size(); ++q) {
        const auto& e = A.rows[q];
        if (e.prec == prec && e.rho == rho && e.lam == lam) return (int)q;
    }
    return -1;
}

// A pinned row for (rho, lambda, precision): its own if cached, else a free or the
// least recently used unpinned one (its weights forgotten); -1 when the cache is off or
// every row is pinned (cache lock held).
static int alpha_take(pcv_ctx* c, AlphaCache& A, double rho, double lam, int32_t prec) {
    if (A.cap <= 0) return -1;
    const int64_t T = c->plan.T_off[c->plan.N];
    if (T <= 0) return -1;
    if (!A.pool.p) {
        if (A.pool.reserve((size_t)A.cap * T) != cudaSuccess) {
            cudaGetLastError();
            A.cap = 0;   // no room: run without the cache
            return -1;
        }
        A.rows.assign(A.cap, {});
    }
    int q = alpha_find(A, rho, lam, prec);
    if (q < 0) {
        uint64_t oldest = UINT64_MAX;
        for (int r = 0; r < A.cap; ++r)
            if (A.rows[r].pins == 0 && A.rows[r].used < oldest) {
                oldest = A.rows[r].used;
                q = r;
            }
        if (q < 0) return -1;
        auto& e = A.rows[q];
        e.rho = rho;
        e.lam = lam;
        e.prec = prec;
        e.have.assign(c->plan.N, 0);
    }
    A.rows[q].used = ++A.clock;
    ++A.rows[q].pins;
    return q;
}

static void with_workspace(pcv::TaskArgs& a, const Workspace& w) {
    a.work = reinterpret_cast<double*>(w.mem.p);
    a.slot_bytes = w.slot_bytes;
    a.ld = w.ld;
    a.planes = w.planes.p;
    a.plane_elems = w.plane_elems;
}

// ---------------------------------------------------------------- size buckets

// Training-size classes of the autotuner: class c holds sizes below kClassEdge[c] (and at
// least the previous edge).  Adjacent classes that take the same engine form one bucket.
static const int32_t kClassEdge[] = {128, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 6144, 8192,
                                     12288, 16384, INT32_MAX};
constexpr int kClasses = (int)(sizeof(kClassEdge) / sizeof(kClassEdge[0]));
constexpr int32_t kSimtMaxK = 2048;   // the FP32 SIMT engine is a candidate below this size

static int size_class(int32_t k) {
    int c = 0;
    while (k >= kClassEdge[c]) ++c;
    return c;
}

static std::mutex g_tune_mu;       // guards the cache below
static std::mutex g_tune_run_mu;   // held from the cache lookup through tuning: contexts with one key tune once
static std::map<std::string, std::vector<int>> g_tune_cache;   // key -> engine per class

// Time the mixed task kernel with `engine` on a sample of subsets (each evaluated with
// Bt copies of one parameter row, enough tasks to fill the device); ms per task.
static pcv_status time_engine(pcv_ctx* c, const std::vector<int32_t>& sample, int engine, int32_t ld,
                              const double* d_prow, int32_t Bt, cudaStream_t s, double& ms_per_task) {
    Workspace w;
    int64_t g, sb, pb;
    mixed_shape(c, ld, engine, g, sb, pb);
    g = std::min<int64_t>(g, (int64_t)sample.size() * Bt);
    pcv_status st = alloc_workspace(c, w, g, sb, pb, ld, pcv::mixed_planes(engine), pcv::mixed_term_bytes(engine));
    if (st != PCV_OK) return st;
    DevBuf<int32_t> ord;
    DevBuf<unsigned int> cnt;
    CUDA_TRY(ord.reserve(sample.size()));
    CUDA_TRY(cnt.reserve(1));
    CUDA_TRY(cudaMemcpyAsync(ord.p, sample.data(), sample.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const int32_t N = c->plan.N;
    CUDA_TRY(c->z.reserve((size_t)Bt * N));
    CUDA_TRY(c->tst.reserve((size_t)Bt * N));
    CUDA_TRY(c->fb_list.reserve((size_t)sample.size() * Bt));
    CUDA_TRY(c->fb_count.reserve(2));
    pcv::TaskArgs a = base_args(c, d_prow, Bt, c->Voff.p, c->Vx.p, c->Vy.p, c->Vv.p, ord.p, (int32_t)sample.size(),
                                nullptr, 0, false, nullptr, nullptr, 0, true);
    a.phase_cycles = nullptr;
    a.counter = cnt.p;
    with_workspace(a, w);
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float ms = 0.f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 2 && err == cudaSuccess; ++rep) {   // the first launch warms up
        cudaMemsetAsync(cnt.p, 0, sizeof(unsigned int), s);
        cudaMemsetAsync(c->fb_count.p, 0, 2 * sizeof(unsigned int), s);
        cudaEventRecord(e0, s);
        err = (cudaError_t)pcv::launch_task_mixed(a, w.maps, engine, (int)w.grid, s);
        cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "autotuner launch");
    ms_per_task = (double)ms / (double)(sample.size() * Bt);
    return PCV_OK;
}

// Build the size buckets of the mixed CV launch (once per context).  With bucketing on
// and the default engine, every training-size class present gets the engine that ran
// its sample fastest (cached per process by the class histogram); adjacent classes with
// the same engine merge.  Otherwise one bucket takes every subset with factor_engine.
static pcv_status build_buckets(pcv_ctx* c, const double* d_params, int32_t B, cudaStream_t s);

static pcv_status ensure_buckets(pcv_ctx* c, const double* d_params, int32_t B, cudaStream_t s) {
    if (!c->buckets.empty()) return PCV_OK;
    ++c->mem_gen;
    const pcv_status st = build_buckets(c, d_params, B, s);
    if (st != PCV_OK) {
        c->buckets.clear();   // no half-built list: the next call starts over
        c->bucket_desc.clear();
    }
    return st;
}

static pcv_status build_buckets(pcv_ctx* c, const double* d_params, int32_t B, cudaStream_t s) {
    const pcv::Plan& P = c->plan;
    std::vector<int32_t> act;
    for (int32_t i = 0; i < P.N; ++i)
        if (P.V_off[i + 1] > P.V_off[i]) act.push_back(i);
    std::stable_sort(act.begin(), act.end(), [&](int32_t a2, int32_t b2) {
        return (P.T_off[a2 + 1] - P.T_off[a2]) > (P.T_off[b2 + 1] - P.T_off[b2]);
    });
    auto ksz = [&](int32_t i) { return (int32_t)(P.T_off[i + 1] - P.T_off[i]); };
    std::vector<int> eng(kClasses, c->opts.factor_engine);
    std::string tune_notes;
    std::vector<std::vector<int32_t>> cls(kClasses);
    for (int32_t i : act) cls[size_class(ksz(i))].push_back(i);
    const bool tune = c->opts.bucketing == 0 && c->opts.factor_engine == pcv::kMixedEngineTensor;
    c->buckets_tuned = false;
    if (tune) {
        std::string key = "sms=" + std::to_string(c->sms) + ";lat=" + std::to_string((int)c->lattice) +
                          ";tc=" + std::to_string(c->opts.tc_stages) + ";hist=";
        for (int q = 0; q < kClasses; ++q)
            if (!cls[q].empty()) key += std::to_string(q) + ":" + std::to_string(cls[q].size()) + ",";
        bool cached = false;
        std::lock_guard<std::mutex> run_lk(g_tune_run_mu);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                eng = it->second;
                cached = true;
            }
        }
        if (!cached && !d_params) return PCV_ERR_ARG;   // tuning needs the call's parameters
        if (!cached) {
            // the first valid parameter row of the call, repeated to fill the device
            std::vector<double> hp((size_t)3 * B);
            CUDA_TRY(cudaMemcpyAsync(hp.data(), d_params, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            int32_t row = -1;
            for (int32_t b = 0; b < B && row < 0; ++b) {
                const double s2 = hp[3 * b], rho = hp[3 * b + 1], t2 = hp[3 * b + 2];
                if (s2 > 0 && rho > 0 && t2 >= 0 && std::isfinite(s2) && std::isfinite(rho) && std::isfinite(t2))
                    row = b;
            }
            bool timed = false;
            if (row >= 0) {
                const int64_t fill = 2 * (int64_t)c->sms;
                for (int q = 0; q < kClasses; ++q) {
                    const auto& L = cls[q];
                    if (L.empty() || ksz(L.front()) >= kSimtMaxK) continue;   // one candidate: no timing
                    const int64_t ns = std::min<int64_t>((int64_t)L.size(), fill);
                    std::vector<int32_t> sample;
                    for (int64_t j = 0; j < ns; ++j) sample.push_back(L[(size_t)(j * (int64_t)L.size() / ns)]);
                    const int32_t Bt = (int32_t)std::min<int64_t>(8, (fill + ns - 1) / ns);
                    DevBuf<double> prow;
                    CUDA_TRY(prow.reserve((size_t)3 * Bt));
                    for (int32_t b = 0; b < Bt; ++b)
                        CUDA_TRY(cudaMemcpyAsync(prow.p + 3 * b, hp.data() + 3 * row, 3 * sizeof(double),
                                                 cudaMemcpyHostToDevice, s));
                    const int32_t ld = round_up(ksz(L.front()), 128);
                    double t_tc = 0.0, t_simt = 0.0;
                    pcv_status st = time_engine(c, sample, pcv::kMixedEngineTensor, ld, prow.p, Bt, s, t_tc);
                    if (st == PCV_OK) st = time_engine(c, sample, pcv::kMixedEngineSimt, ld, prow.p, Bt, s, t_simt);
                    if (st != PCV_OK) return st;
                    // the SIMT engine must win clearly (timing noise must not flip the choice)
                    eng[q] = t_simt < 0.9 * t_tc ? pcv::kMixedEngineSimt : pcv::kMixedEngineTensor;
                    timed = true;
                    char line[200];
                    std::snprintf(line, sizeof line, "tuned k %d-%d (%lld sampled x %d): tensor %.4f ms/task, simt %.4f ms/task\n",
                                  ksz(L.back()), ksz(L.front()), (long long)ns, Bt, t_tc, t_simt);
                    tune_notes += line;
                }
            }
            c->buckets_tuned = timed;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_cache[key] = eng;
        } else {
            c->buckets_tuned = true;
        }
    }
    // merge classes into buckets (largest sizes first), one bucket when not tuning
    c->bucket_desc.clear();
    for (int q = kClasses - 1; q >= 0; --q) {
        if (cls[q].empty()) continue;
        const int e = tune ? eng[q] : c->opts.factor_engine;
        if (c->buckets.empty() || (tune && c->buckets.back()->engine != e)) {
            c->buckets.emplace_back(new Bucket);
            c->buckets.back()->engine = e;
        }
        Bucket& bk = *c->buckets.back();
        bk.subsets.insert(bk.subsets.end(), cls[q].begin(), cls[q].end());
    }
    for (auto& bp : c->buckets) {
        Bucket& bk = *bp;
        bk.khi = ksz(bk.subsets.front());
        bk.klo = ksz(bk.subsets.back());
        for (int32_t i : bk.subsets) bk.work += std::pow((double)ksz(i), 3.0);
        const int32_t ld = round_up(bk.khi, 128);
        int64_t g, sb, pb;
        mixed_shape(c, ld, bk.engine, g, sb, pb);
        g = std::min<int64_t>(g, (int64_t)bk.subsets.size() * std::max(B, 1));
        pcv_status st = alloc_workspace(c, bk.ws, g, sb, pb, ld, pcv::mixed_planes(bk.engine),
                                        pcv::mixed_term_bytes(bk.engine));
        if (st != PCV_OK) return st;
        CUDA_TRY(bk.order.reserve(bk.subsets.size()));
        CUDA_TRY(cudaMemcpy(bk.order.p, bk.subsets.data(), bk.subsets.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice));
        CUDA_TRY(bk.counter.reserve(1));
        CUDA_TRY(cudaStreamCreateWithFlags(&bk.stream, cudaStreamNonBlocking));
        CUDA_TRY(cudaEventCreateWithFlags(&bk.done, cudaEventDisableTiming));
        static const char* names[] = {"tensor-f16x2", "simt-f32", "tensor-bf16x3", "tensor-tf32", "tensor-tf32x3"};
        char line[256];
        std::snprintf(line, sizeof line, "k %d-%d: %zu subsets, engine %s, ld %d, %d slots%s\n", bk.klo, bk.khi,
                      bk.subsets.size(), names[bk.engine], ld, bk.ws.grid, c->buckets_tuned ? " (tuned)" : "");
        c->bucket_desc += line;
    }
    c->bucket_desc += tune_notes;
    std::stable_sort(c->buckets.begin(), c->buckets.end(),
                     [](const std::unique_ptr<Bucket>& x, const std::unique_ptr<Bucket>& y) { return x->work > y->work; });
    if (!c->fork) CUDA_TRY(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
    return PCV_OK;
}

static pcv_status run_tasks(pcv_ctx* c, const double* d_params, int32_t B, int32_t prec, const int64_t* P_off,
                            const double* Px, const double* Py, const double* Pv, const int32_t* order,
                            int32_t n_order, double* d_yhat, int64_t yhat_stride, void* stream,
                            bool want_lik = false, const int32_t* d_param_row = nullptr,
                            const double* d_rhs = nullptr, int32_t nrhs = 0, bool lattice = false,
                            bool bucketed = false) {
    const int32_t N = c->plan.N;
    CUDA_TRY(c->z.reserve((size_t)B * N));
    CUDA_TRY(c->tst.reserve((size_t)B * N));
    cudaStream_t s = (cudaStream_t)stream;
    // the size buckets serve the context's own mixed mode (PCV_PREC_MIXED); the explicit
    // engine modes run one launch with their engine
    bucketed = bucketed && prec == PCV_PREC_MIXED;
    if ((int64_t)n_order * B > 0 && is_mixed(prec)) {
        int e = pcv::mixed_prepare(c->device);
        if (e) return cuda_fail((cudaError_t)e, "mixed-path set-up");
        if (bucketed) {
            pcv_status st = ensure_buckets(c, d_params, B, s);
            if (st != PCV_OK) return st;
            CUDA_TRY(c->z.reserve((size_t)B * N));
            CUDA_TRY(c->tst.reserve((size_t)B * N));
        }
    }
    CUDA_TRY(cudaMemsetAsync(c->z.p, 0, (size_t)B * N * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(c->tst.p, 0, (size_t)B * N * sizeof(int32_t), s));
    if (want_lik) {
        CUDA_TRY(c->lik.reserve((size_t)B * N));
        CUDA_TRY(cudaMemsetAsync(c->lik.p, 0, (size_t)B * N * sizeof(double), s));
    }
    if ((int64_t)n_order * B == 0) return PCV_OK;
    pcv_status st = PCV_OK;
    if (!bucketed) {
        st = ensure_workspace(c, ws_of(c, prec));
        if (st != PCV_OK) return st;
    }
    if (is_mixed(prec)) {
        st = ensure_workspace(c, kFallbackWs);   // fallback tasks run in FP64
        if (st != PCV_OK) return st;
        CUDA_TRY(c->fb_list.reserve((size_t)n_order * B));
        CUDA_TRY(c->fb_count.reserve(2));
        CUDA_TRY(cudaMemsetAsync(c->fb_count.p, 0, 2 * sizeof(unsigned int), s));
    }
    pcv::TaskArgs a = base_args(c, d_params, B, P_off, Px, Py, Pv, order, n_order, d_yhat, yhat_stride, want_lik,
                                d_param_row, d_rhs, nrhs, lattice);
    const bool timing = c->timing && !c->capturing;   // a captured record would not time the replay
    if (timing) CUDA_TRY(cudaEventRecord(c->ev[0], s));
    if (bucketed) {
        // the buckets' persistent launches side by side, forked from and joined to `s`
        CUDA_TRY(cudaEventRecord(c->fork, s));
        for (auto& bp : c->buckets) {
            Bucket& bk = *bp;
            CUDA_TRY(cudaStreamWaitEvent(bk.stream, c->fork, 0));
            CUDA_TRY(cudaMemsetAsync(bk.counter.p, 0, sizeof(unsigned int), bk.stream));
            pcv::TaskArgs ab = a;
            ab.order = bk.order.p;
            ab.n_order = (int32_t)bk.subsets.size();
            ab.counter = bk.counter.p;
            with_workspace(ab, bk.ws);
            const int grid = (int)std::min<int64_t>(bk.ws.grid, (int64_t)ab.n_order * B);
            int e = pcv::launch_task_mixed(ab, bk.ws.maps, bk.engine, grid, bk.stream);
            if (e) return cuda_fail((cudaError_t)e, "task kernel launch");
            CUDA_TRY(cudaEventRecord(bk.done, bk.stream));
            CUDA_TRY(cudaStreamWaitEvent(s, bk.done, 0));
        }
    } else {
        Workspace& w = c->ws[ws_of(c, prec)];
        a.tc_stages = is_mixed(prec) ? stages_for(c, engine_of(c, prec)) : a.tc_stages;
        CUDA_TRY(cudaMemsetAsync(c->counter.p, 0, sizeof(unsigned int), s));
        with_workspace(a, w);
        const int grid = (int)std::min<int64_t>(w.grid, (int64_t)n_order * B);
        int e = prec == PCV_PREC_FP64 ? pcv::launch_task_fp64(a, grid, stream)
                                      : pcv::launch_task_mixed(a, w.maps, engine_of(c, prec), grid, stream);
        if (e) return cuda_fail((cudaError_t)e, "task kernel launch");
    }
    if (timing) {
        CUDA_TRY(cudaEventRecord(c->ev[1], s));
        c->timed_task = true;
    }
    if (is_mixed(prec)) {
        // tasks the mixed kernel could not finish run again in FP64 (the list and
        // its length stay on the device; CTAs beyond the list exit at once)
        Workspace& w64 = c->ws[kFallbackWs];
        pcv::TaskArgs f = a;
        with_workspace(f, w64);
        f.planes = nullptr;
        f.counter = c->fb_count.p + 1;
        f.order = nullptr;                 // list entries are subset * B + configuration
        f.task_list = c->fb_list.p;
        f.task_count = c->fb_count.p;
        f.list_status = PCV_REFINE_FALLBACK;
        int e = pcv::launch_task_fp64(f, (int)std::min<int64_t>(w64.grid, (int64_t)n_order * B), stream);
        if (e) return cuda_fail((cudaError_t)e, "fallback kernel launch");
    }
    return PCV_OK;
}

// Device buffers a captured graph of the CV call names; a graph is replayed only while
// they are all where they were at capture time.
static std::vector<const void*> graph_fingerprint(const pcv_ctx* c) {
    std::vector<const void*> f = {c->z.p, c->tst.p, c->fb_list.p, c->fb_count.p, c->ws[kFallbackWs].mem.p,
                                  c->phase.p, c->gparams.p, c->gsspe.p, c->gstatus.p, c->gyhat.p,
                                  c->alpha->pool.p, c->alpha_slot.p, (const void*)(uintptr_t)c->mem_gen};
    for (const auto& b : c->buckets) {
        f.push_back(b->ws.mem.p);
        f.push_back(b->ws.planes.p);
        f.push_back(b->order.p);
        f.push_back(b->counter.p);
    }
    return f;
}

// The CV call's device work: the task launches (bucketed for the mixed path), the FP64
// fallback and the fixed-order combine.
static pcv_status cv_work(pcv_ctx* c, const double* d_params, int32_t B, int32_t prec, double* d_sspe,
                          double* d_yhat_valid, int32_t* d_status, cudaStream_t s) {
    pcv_status st = run_tasks(c, d_params, B, prec, c->Voff.p, c->Vx.p, c->Vy.p, c->Vv.p, c->order.p, c->n_active,
                              d_yhat_valid, c->nV, s, false, nullptr, nullptr, 0, true, true);
    if (st != PCV_OK) return st;
    const bool timing = c->timing && !c->capturing;
    if (timing) CUDA_TRY(cudaEventRecord(c->ev[2], s));
    int e = pcv::launch_combine(c->z.p, c->tst.p, d_params, B, c->plan.N, d_sspe, d_status, s);
    if (e) return cuda_fail((cudaError_t)e, "combine launch");
    if (timing) {
        CUDA_TRY(cudaEventRecord(c->ev[3], s));
        c->timed_combine = true;
    }
    return PCV_OK;
}

// Capture cv_work for B configurations into c->gexec (on the context's own capture
// stream, so that any caller stream can replay it).  False if the capture did not work
// out (the call then runs eagerly and this shape is not captured again).
static bool capture_cv_graph(pcv_ctx* c, const double* d_params, int32_t B, bool want_yhat, cudaStream_t s) {
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->gparams.reserve((size_t)3 * B) != cudaSuccess || c->gsspe.reserve(B) != cudaSuccess ||
        c->gstatus.reserve(B) != cudaSuccess || (want_yhat && c->gyhat.reserve((size_t)B * c->nV) != cudaSuccess))
        return false;
    // everything the call allocates is allocated before the capture (a released work
    // memory, say, is rebuilt here): nothing inside may allocate or synchronise
    if (pcv::mixed_prepare(c->device) != 0 || ensure_buckets(c, d_params, B, s) != PCV_OK ||
        ensure_workspace(c, kFallbackWs) != PCV_OK)
        return false;
    const int32_t N = c->plan.N;
    if (c->z.reserve((size_t)B * N) != cudaSuccess || c->tst.reserve((size_t)B * N) != cudaSuccess ||
        c->fb_list.reserve((size_t)c->n_active * B) != cudaSuccess || c->fb_count.reserve(2) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return false;
    if (!c->gcap && cudaStreamCreateWithFlags(&c->gcap, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaStreamBeginCapture(c->gcap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
    c->capturing = true;
    const int64_t launches0 = pcv_launch_count(0);
    const pcv_status st = cv_work(c, c->gparams.p, B, PCV_PREC_MIXED, c->gsspe.p, want_yhat ? c->gyhat.p : nullptr,
                                  c->gstatus.p, c->gcap);
    c->capturing = false;
    // the captured kernels run at each replay, not now
    c->graph_kernels = pcv_launch_count(0) - launches0;
    pcv::count_launch((int)-c->graph_kernels);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->gcap, &g);
    bool ok = st == PCV_OK && e == cudaSuccess && g;
    if (ok) ok = cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();   // a failed capture leaves no sticky error
    if (!ok) {
        c->gexec = nullptr;
        return false;
    }
    c->gprint = graph_fingerprint(c);
    return true;
}

PCV_API pcv_status pcv_cv_loss_device(pcv_ctx* c, const double* d_params, int32_t B, int32_t prec, double* d_sspe,
                                      double* d_sspe_per_subset, double* d_yhat_valid, int32_t* d_status,
                                      void* stream) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    if (B < 0) return fail(PCV_ERR_ARG, "B < 0");
    if (B == 0) return PCV_OK;
    if (!d_params || !d_sspe) return fail(PCV_ERR_ARG, "NULL params or sspe");
    if (bad_precision(prec)) return fail(PCV_ERR_ARG, "unknown precision");
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t N = c->plan.N;
    // repeated mixed calls of one shape replay a captured graph of the whole call
    const bool graphable = prec == PCV_PREC_MIXED && c->opts.graph == 0 && c->n_active > 0;
    const int64_t key = (int64_t)B * 8 + (c->alpha_call ? 4 : 0) + (d_yhat_valid ? 2 : 0) + (c->timing ? 1 : 0);
    bool replay = false;
    if (graphable) {
        if (c->gexec && c->gkey == key && graph_fingerprint(c) == c->gprint) {
            replay = true;
        } else if (c->gseen == key) {
            replay = capture_cv_graph(c, d_params, B, d_yhat_valid != nullptr, s);
            c->gkey = replay ? key : -1;
            if (!replay) c->gseen = -2;
        } else if (c->gseen != -2) {
            c->gseen = key;
        }
    }
    if (replay) {
        CUDA_TRY(cudaMemcpyAsync(c->gparams.p, d_params, (size_t)3 * B * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (c->timing) CUDA_TRY(cudaEventRecord(c->ev[0], s));
        CUDA_TRY(cudaGraphLaunch(c->gexec, s));
        pcv::count_launch((int)c->graph_kernels);
        ++c->graph_launches;
        if (c->timing) {
            CUDA_TRY(cudaEventRecord(c->ev[1], s));
            c->timed_task = true;
            c->timed_combine = false;   // the combine is inside the timed graph
        }
        CUDA_TRY(cudaMemcpyAsync(d_sspe, c->gsspe.p, B * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (d_status) CUDA_TRY(cudaMemcpyAsync(d_status, c->gstatus.p, B * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        if (d_yhat_valid && c->nV)
            CUDA_TRY(cudaMemcpyAsync(d_yhat_valid, c->gyhat.p, (size_t)B * c->nV * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
    } else {
        pcv_status st = cv_work(c, d_params, B, prec, d_sspe, d_yhat_valid, d_status, s);
        if (st != PCV_OK) return st;
    }
    if (d_sspe_per_subset)
        CUDA_TRY(cudaMemcpyAsync(d_sspe_per_subset, c->z.p, (size_t)B * N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    return PCV_OK;
}

PCV_API pcv_status pcv_cv_loss(pcv_ctx* c, const double* params, int32_t B, int32_t prec, double* sspe,
                               double* sspe_per_subset, double* yhat_valid, int64_t* n_valid, int32_t* status,
                               void* stream) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    if (B < 0) return fail(PCV_ERR_ARG, "B < 0");
    if (n_valid) *n_valid = c->nV;
    if (B == 0) return PCV_OK;
    if (!params || !sspe) return fail(PCV_ERR_ARG, "NULL params or sspe");
    if (bad_precision(prec)) return fail(PCV_ERR_ARG, "unknown precision");
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t N = c->plan.N;
    CUDA_TRY(c->params.reserve((size_t)3 * B));
    CUDA_TRY(c->sspe.reserve(B));
    CUDA_TRY(c->status.reserve(B));
    DevBuf<double>& yv = c->yv;   // (a context buffer: no allocation and free per call)
    if (yhat_valid) CUDA_TRY(yv.reserve((size_t)B * c->nV));
    CUDA_TRY(cudaMemcpyAsync(c->params.p, params, (size_t)3 * B * sizeof(double), cudaMemcpyHostToDevice, s));
    // rows of the kriging-weight cache for the valid configurations of the batch
    std::vector<int32_t> rows(B, -1);
    AlphaCache& A = *c->alpha;
    bool store = false;
    if (c->n_active > 0) {
        std::lock_guard<std::mutex> lk(A.mu);
        for (int32_t b = 0; b < B; ++b) {
            const double s2 = params[3 * b], rho = params[3 * b + 1], t2 = params[3 * b + 2];
            if (!(s2 > 0 && rho > 0 && t2 >= 0 && std::isfinite(s2) && std::isfinite(rho) && std::isfinite(t2)))
                continue;
            rows[b] = alpha_take(c, A, rho, t2 / s2, prec);
            store = store || rows[b] >= 0;
        }
    }
    bool unpinned = false;
    auto unpin = [&](bool good_call, const int32_t* st) {
        if (unpinned) return;
        unpinned = true;
        std::lock_guard<std::mutex> lk(A.mu);
        for (int32_t b = 0; b < B; ++b) {
            if (rows[b] < 0) continue;
            auto& e = A.rows[rows[b]];
            // the row now holds the weights of every subset with validation data, unless
            // a task of this configuration failed
            const bool good = good_call && (st[b] == PCV_OK || st[b] == PCV_REFINE_FALLBACK);
            for (int32_t i = 0; i < N; ++i)
                if (c->plan.V_off[i + 1] > c->plan.V_off[i]) e.have[i] = good ? 1 : 0;
            --e.pins;
        }
    };
    std::vector<int32_t> hst(B, PCV_ERR_CUDA);
    struct Guard {   // an early return leaves no row pinned (after the stream's work ends)
        std::function<void()> f;
        ~Guard() { if (f) f(); }
    } guard{[&] {
        if (!unpinned) {
            cudaStreamSynchronize(s);
            unpin(false, hst.data());
        }
    }};
    if (store) {
        CUDA_TRY(c->alpha_slot.reserve(B));
        CUDA_TRY(cudaMemcpyAsync(c->alpha_slot.p, rows.data(), B * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    c->alpha_call = store;
    pcv_status st = pcv_cv_loss_device(c, c->params.p, B, prec, c->sspe.p, nullptr, yhat_valid ? yv.p : nullptr,
                                       c->status.p, stream);
    c->alpha_call = false;
    if (st != PCV_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(sspe, c->sspe.p, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(hst.data(), c->status.p, B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (sspe_per_subset)
        CUDA_TRY(cudaMemcpyAsync(sspe_per_subset, c->z.p, (size_t)B * N * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (yhat_valid && c->nV)
        CUDA_TRY(cudaMemcpyAsync(yhat_valid, yv.p, (size_t)B * c->nV * sizeof(double), cudaMemcpyDeviceToHost, s));
    const cudaError_t se = cudaStreamSynchronize(s);
    unpin(se == cudaSuccess, hst.data());
    if (se != cudaSuccess) return cuda_fail(se, "cudaStreamSynchronize");
    if (status) std::copy(hst.begin(), hst.end(), status);
    return PCV_OK;
}

PCV_API pcv_status pcv_neg2loglik(pcv_ctx* c, const double* params, int32_t B, int32_t prec, double* total,
                                  double* per_subset, int32_t* status, void* stream) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    if (B < 0) return fail(PCV_ERR_ARG, "B < 0");
    if (B == 0) return PCV_OK;
    if (!params || !total) return fail(PCV_ERR_ARG, "NULL params or total");
    if (bad_precision(prec)) return fail(PCV_ERR_ARG, "unknown precision");
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t N = c->plan.N;
    if (is_mixed(prec) && engine_of(c, prec) != pcv::kMixedEngineTensor && engine_of(c, prec) != pcv::kMixedEngineSimt)
        return fail(PCV_ERR_ARG, "the local log-likelihood in mixed precision needs the FP16 tensor or the SIMT engine");
    CUDA_TRY(c->params.reserve((size_t)3 * B));
    CUDA_TRY(c->lik_total.reserve(B));
    CUDA_TRY(c->status.reserve(B));
    CUDA_TRY(c->sspe.reserve(B));
    CUDA_TRY(cudaMemcpyAsync(c->params.p, params, (size_t)3 * B * sizeof(double), cudaMemcpyHostToDevice, s));
    pcv_status st = run_tasks(c, c->params.p, B, prec, c->Voff.p, c->Vx.p, c->Vy.p, c->Vv.p, c->order.p,
                              c->n_active, nullptr, c->nV, stream, true);
    if (st != PCV_OK) return st;
    // fixed-order sums: the likelihood's, and the SSPE's for the per-configuration status
    int e = pcv::launch_combine(c->lik.p, c->tst.p, c->params.p, B, N, c->lik_total.p, nullptr, stream);
    if (!e) e = pcv::launch_combine(c->z.p, c->tst.p, c->params.p, B, N, c->sspe.p, c->status.p, stream);
    if (e) return cuda_fail((cudaError_t)e, "combine launch");
    CUDA_TRY(cudaMemcpyAsync(total, c->lik_total.p, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (status) CUDA_TRY(cudaMemcpyAsync(status, c->status.p, B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if (per_subset)
        CUDA_TRY(cudaMemcpyAsync(per_subset, c->lik.p, (size_t)B * N * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return PCV_OK;
}

// Core containing each location after clamping onto D: regular layouts search their cut
// points; other layouts take the first core containing the point, else the nearest.
static int32_t core_of_point(const pcv::Plan& P, double x, double y) {
    x = std::min(std::max(x, P.domain.x0), P.domain.x1);
    y = std::min(std::max(y, P.domain.y0), P.domain.y1);
    if (P.nx > 0) {
        auto cell = [](const std::vector<double>& b, double v) {
            const int n = (int)b.size() - 1;
            int c = (int)(std::upper_bound(b.begin(), b.end(), v) - b.begin()) - 1;
            return std::min(std::max(c, 0), n - 1);
        };
        return cell(P.by, y) * P.nx + cell(P.bx, x);
    }
    int32_t best = -1;
    double bestd = INFINITY;
    for (int32_t i = 0; i < P.N; ++i) {
        const pcv_rect& r = P.cores[i];
        const bool xc = (r.x1 == P.domain.x1), yc = (r.y1 == P.domain.y1);
        const bool in = x >= r.x0 && (xc ? x <= r.x1 : x < r.x1) && y >= r.y0 && (yc ? y <= r.y1 : y < r.y1);
        if (in) return i;
        const double dx = std::max(std::max(r.x0 - x, 0.0), x - r.x1);
        const double dy = std::max(std::max(r.y0 - y, 0.0), y - r.y1);
        const double dd = dx * dx + dy * dy;
        if (dd < bestd) { bestd = dd; best = i; }
    }
    return best;
}

// Predictions at m locations; params: nrows x 3 host rows, row_of_subset: the row each
// subset uses (empty: row 0 for all).
static pcv_status predict_impl(pcv_ctx* c, const double* params, int32_t nrows,
                               const std::vector<int32_t>& row_of_subset, const double* xy_new, int64_t m,
                               int32_t prec, double* yhat, void* stream) {
    const pcv::Plan& P = c->plan;
    const int32_t N = P.N;
    std::vector<int32_t> core(m);
    for (int64_t j = 0; j < m; ++j) {
        const double x = xy_new[2 * j], y = xy_new[2 * j + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) return fail(PCV_ERR_ARG, "non-finite location");
        core[j] = core_of_point(P, x, y);
    }
    std::vector<int64_t> off(N + 1, 0);
    for (int64_t j = 0; j < m; ++j) off[core[j] + 1]++;
    for (int32_t i = 0; i < N; ++i) off[i + 1] += off[i];
    std::vector<int64_t> pos(off.begin(), off.end() - 1), perm(m);
    std::vector<double> px(m), py(m);
    for (int64_t j = 0; j < m; ++j) {
        const int64_t q = pos[core[j]]++;
        perm[q] = j;
        px[q] = xy_new[2 * j];
        py[q] = xy_new[2 * j + 1];
    }
    std::vector<int32_t> ord;
    for (int32_t i = 0; i < N; ++i)
        if (off[i + 1] > off[i]) ord.push_back(i);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
        return (P.T_off[a + 1] - P.T_off[a]) > (P.T_off[b + 1] - P.T_off[b]);
    });
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c->Px.reserve(m));
    CUDA_TRY(c->Py.reserve(m));
    CUDA_TRY(c->Pyhat.reserve(m));
    CUDA_TRY(c->Poff.reserve(N + 1));
    CUDA_TRY(c->Porder.reserve(ord.size()));
    CUDA_TRY(c->params.reserve((size_t)3 * nrows));
    CUDA_TRY(cudaMemcpyAsync(c->Px.p, px.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Py.p, py.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Poff.p, off.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Porder.p, ord.data(), ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->params.p, params, (size_t)3 * nrows * sizeof(double), cudaMemcpyHostToDevice, s));
    const int32_t* d_rows = nullptr;
    if (!row_of_subset.empty()) {
        CUDA_TRY(c->prow.reserve(N));
        CUDA_TRY(cudaMemcpyAsync(c->prow.p, row_of_subset.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        d_rows = c->prow.p;
    }
    // one configuration for every subset: its kriging weights may be kept (alpha_cache);
    // when they are, for every subset the locations need, no matrix is factored
    int row = -1;
    bool from_cache = false;
    AlphaCache& A = *c->alpha;
    if (row_of_subset.empty()) {
        const double rho = params[1], lam = params[2] / params[0];
        if (params[0] > 0 && rho > 0 && params[2] >= 0 && std::isfinite(rho) && std::isfinite(lam)) {
            std::lock_guard<std::mutex> lk(A.mu);
            const int q = alpha_find(A, rho, lam, prec);
            if (q >= 0) {
                from_cache = true;
                for (int32_t i : ord) from_cache = from_cache && A.rows[q].have[i];
            }
            row = alpha_take(c, A, rho, lam, prec);
            if (row < 0) from_cache = false;
            if (row >= 0) ++(from_cache ? A.hits : A.misses);
        }
    }
    struct Guard {   // the row is released (after the stream's work ends) on every return
        std::function<void()> f;
        ~Guard() { if (f) f(); }
    } guard{[&] {
        if (row < 0) return;
        cudaStreamSynchronize(s);
        std::lock_guard<std::mutex> lk(A.mu);
        --A.rows[row].pins;
    }};
    if (row >= 0) {
        CUDA_TRY(c->alpha_slot.reserve(1));
        CUDA_TRY(cudaMemcpyAsync(c->alpha_slot.p, &row, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        (from_cache ? c->alpha_in_call : c->alpha_call) = true;
    }
    // predictions need the slot for matrices as large as the largest training set
    pcv_status st = run_tasks(c, c->params.p, 1, prec, c->Poff.p, c->Px.p, c->Py.p, nullptr, c->Porder.p,
                              (int32_t)ord.size(), c->Pyhat.p, 0, stream, false, d_rows);
    c->alpha_call = c->alpha_in_call = false;
    if (st != PCV_OK) return st;
    std::vector<double> out(m);
    std::vector<int32_t> tst(N);
    CUDA_TRY(cudaMemcpyAsync(out.data(), c->Pyhat.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(tst.data(), c->tst.p, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int64_t q = 0; q < m; ++q) yhat[perm[q]] = out[q];
    pcv_status worst = PCV_OK;
    for (int32_t i : ord)
        if (tst[i] != PCV_OK && tst[i] != PCV_REFINE_FALLBACK) worst = (pcv_status)tst[i];
    if (row >= 0 && !from_cache) {   // the weights just computed for these subsets are kept
        std::lock_guard<std::mutex> lk(A.mu);
        for (int32_t i : ord) A.rows[row].have[i] = (tst[i] == PCV_OK || tst[i] == PCV_REFINE_FALLBACK);
    }
    if (worst != PCV_OK) return fail(worst, "prediction failed for at least one subset");
    return PCV_OK;
}

PCV_API pcv_status pcv_predict(pcv_ctx* c, const double* params3, const double* xy_new, int64_t m, int32_t prec,
                               double* yhat, void* stream) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    if (m < 0) return fail(PCV_ERR_ARG, "m < 0");
    if (m == 0) return PCV_OK;
    if (!params3 || !xy_new || !yhat) return fail(PCV_ERR_ARG, "NULL argument");
    if (bad_precision(prec)) return fail(PCV_ERR_ARG, "unknown precision");
    return predict_impl(c, params3, 1, {}, xy_new, m, prec, yhat, stream);
}

PCV_API pcv_status pcv_predict_local(pcv_ctx* c, const double* params, int32_t B, const double* sspe_per_subset,
                                     const double* xy_new, int64_t m, int32_t prec, double* yhat, int32_t* best,
                                     void* stream) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    if (B < 1 || m < 0) return fail(PCV_ERR_ARG, "B < 1 or m < 0");
    if (!params || !sspe_per_subset || (m > 0 && (!xy_new || !yhat))) return fail(PCV_ERR_ARG, "NULL argument");
    if (bad_precision(prec)) return fail(PCV_ERR_ARG, "unknown precision");
    const pcv::Plan& P = c->plan;
    const int32_t N = P.N;
    // the globally best row: smallest sum of the local losses, rows with a non-finite one excluded
    int32_t gbest = -1;
    double gmin = INFINITY;
    for (int32_t b = 0; b < B; ++b) {
        double t = 0.0;
        for (int32_t i = 0; i < N; ++i) t += sspe_per_subset[(int64_t)b * N + i];
        if (std::isfinite(t) && t < gmin) { gmin = t; gbest = b; }
    }
    if (gbest < 0) return fail(PCV_ERR_ARG, "no configuration has finite local losses");
    std::vector<int32_t> row(N, gbest);
    for (int32_t i = 0; i < N; ++i) {
        if (P.V_off[i + 1] == P.V_off[i]) continue;   // no validation data: the global choice
        double zmin = INFINITY;
        for (int32_t b = 0; b < B; ++b) {
            const double z = sspe_per_subset[(int64_t)b * N + i];
            if (std::isfinite(z) && z < zmin) { zmin = z; row[i] = b; }
        }
    }
    if (best) std::copy(row.begin(), row.end(), best);
    if (m == 0) return PCV_OK;
    return predict_impl(c, params, B, row, xy_new, m, prec, yhat, stream);
}

PCV_API pcv_status pcv_gls(pcv_ctx* c, const double* X, int32_t p, const double* params3, int32_t prec,
                           double* beta, void* stream) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    if (p < 1 || p > 64) return fail(PCV_ERR_ARG, "need 1 <= p <= 64 covariates");
    if (!X || !params3 || !beta) return fail(PCV_ERR_ARG, "NULL argument");
    if (bad_precision(prec)) return fail(PCV_ERR_ARG, "unknown precision");
    const double s2 = params3[0], rho = params3[1], tau2 = params3[2];
    if (!(s2 > 0.0) || !(rho > 0.0) || !(tau2 > 0.0) || !std::isfinite(s2) || !std::isfinite(rho) ||
        !std::isfinite(tau2))
        return fail(PCV_ERR_ARG, "GLS needs sigma2 > 0, rho > 0 and a nugget tau2 > 0");
    if (is_mixed(prec) && engine_of(c, prec) != pcv::kMixedEngineTensor)
        return fail(PCV_ERR_ARG, "GLS in mixed precision needs the default tensor engine");
    const pcv::Plan& P = c->plan;
    const int32_t N = P.N;
    const int64_t n = P.n;
    // every TRAIN point of D once, from the subset whose core holds it: the prediction
    // locations of H (core training points of each subset, in subset order)
    std::vector<int64_t> off(N + 1, 0), who;
    std::vector<double> px, py;
    for (int32_t i = 0; i < N; ++i) {
        const pcv_rect& r = P.cores[i];
        const bool xc = r.x1 == P.domain.x1, yc = r.y1 == P.domain.y1;
        for (int64_t q = P.T_off[i]; q < P.T_off[i + 1]; ++q) {
            const int64_t j = P.T_idx[q];
            const double x = c->hxy[2 * j], y = c->hxy[2 * j + 1];
            if (x >= r.x0 && (xc ? x <= r.x1 : x < r.x1) && y >= r.y0 && (yc ? y <= r.y1 : y < r.y1)) {
                who.push_back(j);
                px.push_back(x);
                py.push_back(y);
            }
        }
        off[i + 1] = (int64_t)who.size();
    }
    const int64_t m = (int64_t)who.size();
    if (m == 0) return fail(PCV_ERR_ARG, "no training points inside the cores");
    std::vector<int32_t> ord;
    for (int32_t i = 0; i < N; ++i)
        if (off[i + 1] > off[i]) ord.push_back(i);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a2, int32_t b2) {
        return (P.T_off[a2 + 1] - P.T_off[a2]) > (P.T_off[b2 + 1] - P.T_off[b2]);
    });
    // right-hand sides: the p covariate columns, then y
    const int32_t nr = p + 1;
    std::vector<double> R((size_t)nr * n);
    for (int32_t col = 0; col < p; ++col)
        for (int64_t j = 0; j < n; ++j) R[(size_t)col * n + j] = X[(size_t)j * p + col];
    std::copy(c->hv.begin(), c->hv.end(), R.begin() + (size_t)p * n);
    CUDA_TRY(cudaSetDevice(c->device));
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(c->rhs.reserve((size_t)nr * n));
    CUDA_TRY(c->Px.reserve(m));
    CUDA_TRY(c->Py.reserve(m));
    CUDA_TRY(c->Pyhat.reserve((size_t)nr * m));
    CUDA_TRY(c->Poff.reserve(N + 1));
    CUDA_TRY(c->Porder.reserve(ord.size()));
    CUDA_TRY(c->params.reserve(3));
    CUDA_TRY(cudaMemcpyAsync(c->rhs.p, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Px.p, px.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Py.p, py.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Poff.p, off.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Porder.p, ord.data(), ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->params.p, params3, 3 * sizeof(double), cudaMemcpyHostToDevice, s));
    // H applied to every column at the core training points: one factorisation per subset
    pcv_status st = run_tasks(c, c->params.p, 1, prec, c->Poff.p, c->Px.p, c->Py.p, nullptr, c->Porder.p,
                              (int32_t)ord.size(), c->Pyhat.p, m, stream, false, nullptr, c->rhs.p, nr);
    if (st != PCV_OK) return st;
    std::vector<double> H((size_t)nr * m);
    std::vector<int32_t> tst(N);
    CUDA_TRY(cudaMemcpyAsync(H.data(), c->Pyhat.p, H.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(tst.data(), c->tst.p, N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    for (int32_t i : ord)
        if (tst[i] != PCV_OK && tst[i] != PCV_REFINE_FALLBACK) return fail((pcv_status)tst[i], "GLS solve failed");
    // M^-1 v = (v - H v) / lambda; the 1 / lambda cancels in beta:
    // (X^T (X - H X)) beta = X^T (y - H y), summed over the points in subset order
    std::vector<double> A((size_t)p * p, 0.0), rhsb(p, 0.0);
    for (int64_t q = 0; q < m; ++q) {
        const int64_t j = who[q];
        const double* xj = X + (size_t)j * p;
        for (int32_t u = 0; u < p; ++u) {
            for (int32_t w = 0; w < p; ++w) A[(size_t)u * p + w] += xj[u] * (xj[w] - H[(size_t)w * m + q]);
            rhsb[u] += xj[u] * (c->hv[j] - H[(size_t)p * m + q]);
        }
    }
    // p x p solve: Gaussian elimination with partial pivoting
    for (int32_t col = 0; col < p; ++col) {
        int32_t piv = col;
        for (int32_t r2 = col + 1; r2 < p; ++r2)
            if (std::fabs(A[(size_t)r2 * p + col]) > std::fabs(A[(size_t)piv * p + col])) piv = r2;
        if (!(std::fabs(A[(size_t)piv * p + col]) > 0.0)) return fail(PCV_NOT_SPD, "singular GLS system");
        if (piv != col) {
            for (int32_t w = 0; w < p; ++w) std::swap(A[(size_t)piv * p + w], A[(size_t)col * p + w]);
            std::swap(rhsb[piv], rhsb[col]);
        }
        for (int32_t r2 = col + 1; r2 < p; ++r2) {
            const double f = A[(size_t)r2 * p + col] / A[(size_t)col * p + col];
            for (int32_t w = col; w < p; ++w) A[(size_t)r2 * p + w] -= f * A[(size_t)col * p + w];
            rhsb[r2] -= f * rhsb[col];
        }
    }
    for (int32_t col = p - 1; col >= 0; --col) {
        double t = rhsb[col];
        for (int32_t w = col + 1; w < p; ++w) t -= A[(size_t)col * p + w] * beta[w];
        beta[col] = t / A[(size_t)col * p + col];
    }
    return PCV_OK;
}

PCV_API pcv_status pcv_set_timing(pcv_ctx* c, int32_t enable) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    CUDA_TRY(cudaSetDevice(c->device));
    for (auto& e : c->ev)
        if (!e) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(c->phase.reserve(pcv::kPhaseCount));
    CUDA_TRY(cudaMemset(c->phase.p, 0, pcv::kPhaseCount * sizeof(unsigned long long)));
    c->timing = enable != 0;
    c->timed_task = c->timed_combine = false;
    return PCV_OK;
}

PCV_API pcv_status pcv_kernel_time(pcv_ctx* c, double* task_ms, double* combine_ms) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    if (!c->timing || !c->timed_task) return fail(PCV_ERR_ARG, "no timed launch");
    float t = 0.f;
    CUDA_TRY(cudaEventSynchronize(c->ev[1]));
    CUDA_TRY(cudaEventElapsedTime(&t, c->ev[0], c->ev[1]));
    if (task_ms) *task_ms = t;
    if (combine_ms) {
        *combine_ms = 0.0;
        if (c->timed_combine) {
            CUDA_TRY(cudaEventSynchronize(c->ev[3]));
            CUDA_TRY(cudaEventElapsedTime(&t, c->ev[2], c->ev[3]));
            *combine_ms = t;
        }
    }
    return PCV_OK;
}

PCV_API pcv_status pcv_phase_cycles(pcv_ctx* c, uint64_t* out, int32_t reset) {
    if (!c || !out) return fail(PCV_ERR_ARG, "NULL argument");
    if (!c->phase.p) return fail(PCV_ERR_ARG, "timing was never enabled");
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemcpy(out, c->phase.p, pcv::kPhaseCount * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (reset) CUDA_TRY(cudaMemset(c->phase.p, 0, pcv::kPhaseCount * sizeof(unsigned long long)));
    return PCV_OK;
}

PCV_API void pcv_destroy(pcv_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    delete c;
}

PCV_API const char* pcv_status_str(int32_t s) {
    switch (s) {
        case PCV_OK: return "ok";
        case PCV_ERR_ARG: return "invalid argument";
        case PCV_ERR_OOM: return "out of memory";
        case PCV_ERR_CUDA: return "CUDA error";
        case PCV_ERR_TIMEOUT: return "device wait timed out";
        case PCV_ERR_BUSY: return "context busy";
        case PCV_NOT_SPD: return "matrix not positive definite";
        case PCV_REFINE_FALLBACK: return "refinement fell back to FP64";
        case PCV_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

PCV_API const char* pcv_last_error(void) { return g_err.c_str(); }

PCV_API int32_t pcv_version(void) { return 1; }

PCV_API pcv_status pcv_alpha_cache_stats(const pcv_ctx* c, int64_t* hits, int64_t* misses, int32_t* rows_held) {
    if (!c) return fail(PCV_ERR_ARG, "NULL ctx");
    AlphaCache& A = *c->alpha;
    std::lock_guard<std::mutex> lk(A.mu);
    if (hits) *hits = A.hits;
    if (misses) *misses = A.misses;
    if (rows_held) {
        int32_t n = 0;
        for (const auto& e : A.rows) n += e.prec >= 0;
        *rows_held = n;
    }
    return PCV_OK;
}

PCV_API int32_t pcv_buckets(const pcv_ctx* c, char* buf, int32_t cap) {
    if (!c) return 0;
    const std::string& d = c->bucket_desc;
    if (buf && cap > 0) {
        const size_t n = std::min<size_t>(d.size(), (size_t)cap - 1);
        std::memcpy(buf, d.data(), n);
        buf[n] = 0;
    }
    return (int32_t)d.size();
}

PCV_API int32_t pcv_lattice(const pcv_ctx* c, double* hx, double* hy) {
    if (!c || !c->lattice) return 0;
    if (hx) *hx = c->lat_hx;
    if (hy) *hy = c->lat_hy;
    return 1;
}

PCV_API int32_t pcv_lattice_detect(const double* xy, int64_t n, double* x0, double* hx, double* y0, double* hy) {
    if (!xy || n <= 0) return 0;
    std::vector<double> vx((size_t)n), vy((size_t)n);
    for (int64_t q = 0; q < n; ++q) {
        vx[q] = xy[2 * q];
        vy[q] = xy[2 * q + 1];
        if (!std::isfinite(vx[q]) || !std::isfinite(vy[q])) return 0;
    }
    double ox = 0.0, oy = 0.0, sx = 0.0, sy = 0.0;
    std::vector<int32_t> ix, iy;
    if (!lattice_axis(vx, ox, sx, ix) || !lattice_axis(vy, oy, sy, iy)) return 0;
    if (x0) *x0 = ox;
    if (hx) *hx = sx;
    if (y0) *y0 = oy;
    if (hy) *hy = sy;
    return 1;
}
