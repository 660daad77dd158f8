// no_alloc.cu -- an allocation-free variant of the FP64 cross-validation launch.
//
// Some callers cannot call cudaMalloc: a host application that hands out all
// device memory from its own pool and forbids allocations behind its back, or a
// latency-critical loop in which cudaMalloc/cudaFree, which may synchronise the
// whole device, are not acceptable.  pcv_cv_loss_fp64_static serves them: it runs
// the same FP64 task kernel and combine kernel as pcv_cv_loss_device, but every
// work buffer (task counter, subset order, per-task losses and statuses, and the
// per-CTA matrix slots) lives in one file-scope device array of fixed size,
// PCV_STATIC_SCRATCH_BYTES, which every GPU that loads this library holds until
// the process exits.  It allocates nothing, on the device or through any library.
//
// The paper has no counterpart to this entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "pcv_internal.h"

namespace pcv {
namespace {

constexpr size_t kScratchBytes = PCV_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kOrderThreads = 1024;

// The scratch array.  In host code `g_scratch` is only a host-side stand-in: its
// device address comes from cudaGetSymbolAddress, once per device.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Region layout inside the scratch array (byte offsets, 256-aligned).
struct Layout {
    size_t counter, toff, voff, order, z, tst, slots, slot_bytes;
    int grid;
    int32_t ld;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Subsets with validation data, longest training set first, so that the persistent
// CTAs finish together (the order pcv_cv_loss_device uses): one CTA, a counting sort by
// training size in shared memory (sizes 0 .. kmax, kmax <= kMaxOrderK; ties in any
// order, which changes no result: every task is computed on its own and the losses
// are summed in subset order).
constexpr int kMaxOrderK = 4096;
__global__ void __launch_bounds__(kOrderThreads) k_active_order(const int64_t* T_off, const int64_t* V_off, int32_t N,
                                                              int32_t kmax, int32_t* order) {
    __shared__ int32_t cnt[kMaxOrderK + 1];
    __shared__ int32_t part[kOrderThreads];
    const int t = threadIdx.x;
    for (int q = t; q <= kmax; q += kOrderThreads) cnt[q] = 0;
    __syncthreads();
    for (int32_t i = t; i < N; i += kOrderThreads)
        if (V_off[i + 1] > V_off[i]) atomicAdd(&cnt[(int)(T_off[i + 1] - T_off[i])], 1);
    __syncthreads();
    // exclusive scan from the largest size down: start[q] = active subsets larger than q.
    // Thread t owns sizes kmax - t*per .. (descending), a chunk of per values.
    const int per = (kmax + 1 + kOrderThreads - 1) / kOrderThreads;
    const int hi = kmax - t * per, lo = max(-1, hi - per);   // sizes hi down to lo + 1
    int32_t c = 0;
    for (int q = hi; q > lo; --q) c += cnt[q];
    part[t] = c;
    __syncthreads();
    for (int off = 1; off < kOrderThreads; off <<= 1) {   // inclusive Hillis-Steele scan
        const int32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = part[t] - c;
    for (int q = hi; q > lo; --q) {
        const int32_t n = cnt[q];
        cnt[q] = run;
        run += n;
    }
    __syncthreads();
    for (int32_t i = t; i < N; i += kOrderThreads)
        if (V_off[i + 1] > V_off[i]) order[atomicAdd(&cnt[(int)(T_off[i + 1] - T_off[i])], 1)] = i;
}

cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace pcv

using namespace pcv;

PCV_API pcv_status pcv_cv_loss_fp64_static(const double* d_x, const double* d_y, const double* d_v, int32_t N,
                                           const int64_t* h_T_off, const int32_t* d_T_idx, const int64_t* h_V_off,
                                           const double* d_Vx, const double* d_Vy, const double* d_Vv,
                                           const double* d_params, int32_t B, double* d_sspe,
                                           double* d_sspe_per_subset, int32_t* d_status, void* stream) {
    if (N < 1 || B < 0 || !h_T_off || !h_V_off) return PCV_ERR_ARG;
    if (B == 0) return PCV_OK;
    if (!d_x || !d_y || !d_v || !d_T_idx || !d_Vx || !d_Vy || !d_Vv || !d_params || !d_sspe) return PCV_ERR_ARG;
    // offsets index the caller's arrays from their first entry on
    if (h_T_off[0] < 0 || h_V_off[0] < 0) return PCV_ERR_ARG;
    // the per-task results (12 bytes each) alone must fit, checked before any size
    // arithmetic that could wrap
    if ((uint64_t)B * (uint64_t)N > (uint64_t)(kScratchBytes / 12)) return PCV_ERR_ARG;
    int32_t kmax = 0, n_active = 0;
    int64_t mmax = 0;
    for (int32_t i = 0; i < N; ++i) {
        const int64_t k = h_T_off[i + 1] - h_T_off[i], m = h_V_off[i + 1] - h_V_off[i];
        if (k < 0 || m < 0) return PCV_ERR_ARG;
        if (m > 0) {
            ++n_active;
            kmax = (int32_t)std::max<int64_t>(kmax, k);
            mmax = std::max(mmax, m);
        }
    }
    // fixed layout of the scratch array for this call
    Layout L{};
    L.ld = (int32_t)((std::max(kmax, 1) + 127) / 128 * 128);
    L.counter = 0;
    L.toff = 256;
    L.voff = align256(L.toff + (size_t)(N + 1) * sizeof(int64_t));
    L.order = align256(L.voff + (size_t)(N + 1) * sizeof(int64_t));
    L.z = align256(L.order + (size_t)N * sizeof(int32_t));
    L.tst = align256(L.z + (size_t)B * N * sizeof(double));
    L.slots = align256(L.tst + (size_t)B * N * sizeof(int32_t));
    L.slot_bytes = (size_t)slot_bytes_fp64(L.ld, mmax);
    if (L.slots + L.slot_bytes > kScratchBytes) return PCV_ERR_ARG;   // problem exceeds the static scratch
    static_assert((size_t)8 * kMaxOrderK * kMaxOrderK > kScratchBytes, "a slot bounds the training size");
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PCV_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PCV_ERR_CUDA;
    L.grid = (int)std::min<size_t>({(size_t)sms, (kScratchBytes - L.slots) / L.slot_bytes,
                                    (size_t)n_active * (size_t)B});
    unsigned char* base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) return PCV_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t* Toff = reinterpret_cast<int64_t*>(base + L.toff);
    int64_t* Voff = reinterpret_cast<int64_t*>(base + L.voff);
    int32_t* order = reinterpret_cast<int32_t*>(base + L.order);
    double* z = reinterpret_cast<double*>(base + L.z);
    int32_t* tst = reinterpret_cast<int32_t*>(base + L.tst);
    unsigned int* counter = reinterpret_cast<unsigned int*>(base + L.counter);
    // every call shares the array and finds the previous call's contents: reset
    // what must start at zero
    if (cudaMemcpyAsync(Toff, h_T_off, (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(Voff, h_V_off, (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(counter, 0, 256, s) != cudaSuccess ||
        cudaMemsetAsync(z, 0, (size_t)B * N * sizeof(double), s) != cudaSuccess ||
        cudaMemsetAsync(tst, 0, (size_t)B * N * sizeof(int32_t), s) != cudaSuccess)
        return PCV_ERR_CUDA;
    k_active_order<<<1, kOrderThreads, 0, s>>>(Toff, Voff, N, kmax, order);
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return PCV_ERR_CUDA;
    if (n_active > 0) {
        TaskArgs a{};
        a.X = d_x;
        a.Y = d_y;
        a.Vals = d_v;
        a.T_off = Toff;
        a.T_idx = d_T_idx;
        a.P_off = Voff;
        a.Px = d_Vx;
        a.Py = d_Vy;
        a.Pv = d_Vv;
        a.order = order;
        a.n_order = n_active;
        a.params = d_params;
        a.B = B;
        a.N = N;
        a.z = z;
        a.tstatus = tst;
        a.yhat = nullptr;
        a.yhat_stride = 0;
        a.counter = counter;
        a.work = reinterpret_cast<double*>(base + L.slots);
        a.slot_bytes = (int64_t)L.slot_bytes;
        a.ld = L.ld;
        if (launch_task_fp64(a, L.grid, stream) != 0) return PCV_ERR_CUDA;
    }
    if (launch_combine(z, tst, d_params, B, N, d_sspe, d_status, stream) != 0) return PCV_ERR_CUDA;
    if (d_sspe_per_subset &&
        cudaMemcpyAsync(d_sspe_per_subset, z, (size_t)B * N * sizeof(double), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        return PCV_ERR_CUDA;
    return PCV_OK;
}
