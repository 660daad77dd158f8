// peaks.cu -- throughput probes for the roofline denominators of the task kernels:
// FP64 and FP32 fused multiply-add on the SIMT pipes, and the tcgen05 tensor pipe at
// kind::tf32, kind::f16 with BF16 and with FP16 operands (dense, FP32 accumulators in
// TMEM).  Each probe keeps its pipe busy for a requested wall time and reports the
// achieved rate; nothing here belongs to the cross-validation path itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "pcv_internal.h"
#include "umma.cuh"

namespace {

constexpr int kFmaChains = 8;   // independent accumulator chains per thread

// Every thread runs kFmaChains independent FMA chains for `iters` rounds; the result
// is written (conditionally, never in practice) so the compiler keeps the work.
template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(int64_t iters, T a, T b, T* sink) {
    T x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
#pragma unroll
            for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    if (s == (T)-12345.678) *sink = s;
}

// Tensor-pipe probe: one CTA per SM, one thread issues M = 128, N = 256 MMAs from two
// fixed shared-memory tiles (A 128 x 32 bytes of K, B 256 x 32 bytes, 64-byte swizzle
// layout) into alternating halves of the CTA's 512 TMEM columns.  Every kBatch MMAs are
// committed to an mbarrier and the issuer waits (bounded) for the batch before the
// previous one, so at most two batches are in flight.  FMT: 2 = kind::tf32, otherwise
// the kind::f16 format code (0 FP16, 1 BF16).
constexpr int kBatch = 64;
constexpr int kPeakN = 256;
constexpr int kATileBytes = 128 * 64;
constexpr int kBTileBytes = kPeakN * 64;

struct PeakSmem {
    uint64_t bar[2];
    uint32_t tmem;
};

template <int FMT>
__global__ void __launch_bounds__(128, 1) k_tensor_peak(int64_t batches, int* err) {
    using namespace pcv::umma;
    extern __shared__ __align__(1024) unsigned char raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    uint8_t* A = base;
    uint8_t* B = base + kATileBytes;
    PeakSmem& sm = *reinterpret_cast<PeakSmem*>(base + kATileBytes + kBTileBytes);
    // operands: small values of either sign (the same bit patterns whatever the format)
    for (int e = threadIdx.x; e < (kATileBytes + kBTileBytes) / 4; e += blockDim.x) {
        const uint32_t h = (uint32_t)e * 2654435761u;
        uint32_t w;
        if (FMT == kFmtTF32) {
            const float f = ((float)(h >> 8) * (1.0f / 16777216.0f) - 0.5f) * 0.25f;
            w = __float_as_uint(f);
        } else {
            const float f0 = ((float)((h >> 8) & 0xFFF) / 4096.0f - 0.5f) * 0.25f;
            const float f1 = ((float)((h >> 20) & 0xFFF) / 4096.0f - 0.5f) * 0.25f;
            uint16_t u0, u1;
            if (FMT == 1) {
                u0 = __bfloat16_as_ushort(__float2bfloat16_rn(f0));
                u1 = __bfloat16_as_ushort(__float2bfloat16_rn(f1));
            } else {
                u0 = __half_as_ushort(__float2half_rn(f0));
                u1 = __half_as_ushort(__float2half_rn(f1));
            }
            w = (uint32_t)u0 | ((uint32_t)u1 << 16);
        }
        reinterpret_cast<uint32_t*>(base)[e] = w;
    }
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    fence_proxy_async();   // generic-proxy writes of the tiles, read by the tensor pipe
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tmem_alloc(&sm.tmem, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_f16kind(128, kPeakN, FMT);
        const uint64_t ad = smem_desc_sw64(smem_u32(A)), bd = smem_desc_sw64(smem_u32(B));
        bool ok = true;
        uint32_t issued = 0;
        for (int64_t bt = 0; bt < batches && ok; ++bt) {
            const int slot = (int)(bt & 1);
            // before reusing this batch barrier, the batch committed to it two rounds ago
            // must have completed (phase parity of that round)
            if (bt >= 2 && !mbar_wait(&sm.bar[slot], (uint32_t)(((bt - 2) >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t d = sm.tmem + (uint32_t)(slot * kPeakN);
            for (int q = 0; q < kBatch; ++q) {
                const uint32_t kb = (uint32_t)(q & 1) * 2;   // second K-step: +32 bytes (>> 4)
                if (FMT == kFmtTF32) mma_tf32kind(d, ad + kb, bd + kb, idesc, q > 0 ? 1u : 0u);
                else mma_f16kind(d, ad + kb, bd + kb, idesc, q > 0 ? 1u : 0u);
            }
            mma_commit(&sm.bar[slot]);
            ++issued;
        }
        // drain: the last one or two commits
        for (int64_t bt = std::max<int64_t>(0, (int64_t)issued - 2); bt < (int64_t)issued; ++bt)
            if (!mbar_wait(&sm.bar[bt & 1], (uint32_t)((bt >> 1) & 1))) ok = false;
        if (!ok) atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(sm.tmem, kTmemCols);
}

// more shared memory than two CTAs can hold, so that each SM runs exactly one probe CTA
// (and its 512 TMEM columns)
template <int FMT>
constexpr int tensor_peak_smem() { return 120 * 1024; }
static_assert(1024 + kATileBytes + kBTileBytes + (int)sizeof(PeakSmem) <= 120 * 1024, "probe tiles");

}  // namespace

// kind: 0 FP64 FMA, 1 FP32 FMA, 2 tcgen05 kind::tf32, 3 kind::f16 BF16, 4 kind::f16 FP16.
PCV_API pcv_status pcv_measure_peak(int32_t kind, double seconds, double* tflops, double* elapsed_s) {
    if (kind < 0 || kind > 4 || !tflops || !(seconds > 0.0) || seconds > 60.0) return PCV_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PCV_ERR_CUDA;
    double* sink = nullptr;
    int* err = nullptr;
    if (cudaMalloc(&sink, 8) != cudaSuccess) return PCV_ERR_OOM;
    if (cudaMalloc(&err, 4) != cudaSuccess) {
        cudaFree(sink);
        return PCV_ERR_OOM;
    }
    cudaMemset(err, 0, 4);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    pcv_status st = PCV_OK;
    // grid shapes: SIMT probes 8 CTAs of 256 threads per SM; tensor probes one CTA per SM
    const int grid_simt = 8 * sms;
    auto run = [&](int64_t n) -> double {
        cudaEventRecord(e0);
        switch (kind) {
            case 0: k_fma_peak<double><<<grid_simt, 256>>>(n, 0.999999, 1e-7, sink); break;
            case 1: k_fma_peak<float><<<grid_simt, 256>>>(n, 0.999999f, 1e-7f, reinterpret_cast<float*>(sink)); break;
            case 2: k_tensor_peak<2><<<sms, 128, tensor_peak_smem<2>()>>>(n, err); break;
            case 3: k_tensor_peak<1><<<sms, 128, tensor_peak_smem<1>()>>>(n, err); break;
            default: k_tensor_peak<0><<<sms, 128, tensor_peak_smem<0>()>>>(n, err); break;
        }
        pcv::count_launch();
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms * 1e-3;
    };
    // flops per unit of n: SIMT 2 flops x 16 x chains per thread; tensor 2 M N K per MMA
    // x kBatch (K = 16 for kind::f16, 8 for kind::tf32)
    const double per = kind < 2 ? 2.0 * 16 * kFmaChains * 256.0 * grid_simt
                                : 2.0 * 128 * kPeakN * (kind == 2 ? 8 : 16) * kBatch * (double)sms;
    if (kind >= 2) {
        cudaFuncSetAttribute(k_tensor_peak<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, tensor_peak_smem<2>());
        cudaFuncSetAttribute(k_tensor_peak<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, tensor_peak_smem<1>());
        cudaFuncSetAttribute(k_tensor_peak<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, tensor_peak_smem<0>());
    }
    // calibrate on a short run, then one run of about `seconds`
    int64_t n = 64;
    double t = run(n);
    while (t >= 0.0 && t < 0.05 && n < ((int64_t)1 << 40)) {
        n *= 4;
        t = run(n);
    }
    if (t > 0.0) {
        n = std::max<int64_t>(1, (int64_t)((double)n * seconds / t));
        t = run(n);
    }
    int herr = 0;
    if (t <= 0.0 || cudaGetLastError() != cudaSuccess) st = PCV_ERR_CUDA;
    else if (cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = PCV_ERR_CUDA;
    else if (herr) st = PCV_ERR_TIMEOUT;
    if (st == PCV_OK) {
        *tflops = per * (double)n / t / 1e12;
        if (elapsed_s) *elapsed_s = t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(err);
    return st;
}
