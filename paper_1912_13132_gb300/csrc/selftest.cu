// selftest.cu -- checks of the double-float arithmetic (df.cuh) used by the
// mixed-precision refinement: the same routines evaluated on the host and on the
// device, so tests can compare them with libm / CUDA's FP64 functions.
#include <cuda_runtime.h>

#include "df.cuh"
#include "pcv_internal.h"

namespace {

using pcv::dfm::df;

PCV_HD double eval(int op, double a, double b, const pcv::dfm::ExpConsts& k) {
    using namespace pcv::dfm;
    const df x = from_double(a), y = from_double(b);
    switch (op) {
        case 0: return to_double(exp_neg(x, k));
        case 1: return to_double(sqrt_df(x));
        case 2: return to_double(mul(x, y));
        case 3: return to_double(add(x, y));
        default: return 0.0;
    }
}

__global__ void k_selftest(int op, const double* a, const double* b, int64_t n, double* out,
                           pcv::dfm::ExpConsts k) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = eval(op, a[i], b ? b[i] : 0.0, k);
}

}  // namespace

PCV_API pcv_status pcv_selftest_df(int32_t op, const double* a, const double* b, int64_t n, double* out) {
    if (op < 0 || op > 3 || n < 0 || (n > 0 && (!a || !out))) return PCV_ERR_ARG;
    pcv::dfm::ExpConsts k;
    pcv::dfm::exp_constants(k);
    for (int64_t i = 0; i < n; ++i) out[i] = eval(op, a[i], b ? b[i] : 0.0, k);
    return PCV_OK;
}

PCV_API pcv_status pcv_selftest_df_device(int32_t op, const double* d_a, const double* d_b, int64_t n,
                                          double* d_out, void* stream) {
    if (op < 0 || op > 3 || n < 0 || (n > 0 && (!d_a || !d_out))) return PCV_ERR_ARG;
    if (n == 0) return PCV_OK;
    pcv::dfm::ExpConsts k;
    pcv::dfm::exp_constants(k);
    const int T = 256;
    k_selftest<<<(unsigned)((n + T - 1) / T), T, 0, (cudaStream_t)stream>>>(op, d_a, d_b, n, d_out, k);
    pcv::count_launch();
    return cudaGetLastError() == cudaSuccess ? PCV_OK : PCV_ERR_CUDA;
}

// ---------------------------------------------------------------- tensor-core pipeline self-test
#include <vector>

#include "umma.cuh"

namespace {

__global__ void k_split(const float* x, int64_t n, __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) pcv::umma::split3(x[i], p0[i], p1[i], p2[i]);
}

struct UmmaTestSmem {
    pcv::umma::Pipe pipe;
    int err;
};

constexpr int kTestStages = 3;
constexpr int kTestStageBytes = pcv::umma::stage_bytes<pcv::umma::SplitBF16x3>(pcv::umma::kTilesPerPass);

__global__ void __launch_bounds__(256, 1) k_umma_test(const __grid_constant__ CUtensorMap m0,
                                                      const __grid_constant__ CUtensorMap m1,
                                                      const __grid_constant__ CUtensorMap m2, int M, int K, float* C,
                                                      int* err) {
    using namespace pcv::umma;
    extern __shared__ __align__(1024) unsigned char raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stages = base;
    UmmaTestSmem& sm = *reinterpret_cast<UmmaTestSmem*>(base + kTestStages * kTestStageBytes);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        pipe_init(sm.pipe, kTestStages);
        sm.err = 0;
        prefetch_map(&m0);
        prefetch_map(&m1);
        prefetch_map(&m2);
    }
    if (warp == 1) tmem_alloc(&sm.pipe.tmem_base, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    Phases ph;
    auto epi = [&](int row0, int quad, uint32_t taddr) {
        const int r = row0 - kTileM + quad * 32 + (threadIdx.x & 31);   // A rows start at plane row 128
        for (int c0 = 0; c0 < kTileN; c0 += 32) {
            float v[32];
            tmem_ld32(taddr + c0, v);
            if (r < M)
                for (int j = 0; j < 32; ++j) C[(int64_t)r * kTileN + c0 + j] = v[j];
        }
    };
    // two calls in a row to exercise the phase bookkeeping across block columns
    for (int rep = 0; rep < 2; ++rep) {
        const bool ok = block_column(sm.pipe, ph, stages, &m0, &m1, &m2, 0, kTileM, M, 0, K, epi);
        if (!ok) atomicExch(&sm.err, 1);
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(sm.pipe.tmem_base, kTmemCols);
    if (threadIdx.x == 0) *err = sm.err;
}

// ---- the same product with any operand scheme (16-bit or TF32 terms)

template <class Sch>
__global__ void k_split_scheme(const float* x, int64_t n, uint16_t* planes, int64_t plane_units) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (Sch::kElem == 2) {
        uint16_t t[Sch::kPlanes];
        pcv::umma::split_terms(Sch{}, x[i], t);
        for (int p = 0; p < Sch::kPlanes; ++p) planes[p * plane_units + i] = t[p];
    } else {
        uint32_t t[Sch::kPlanes];
        pcv::umma::split_terms(Sch{}, x[i], t);
        for (int p = 0; p < Sch::kPlanes; ++p) reinterpret_cast<uint32_t*>(planes + p * plane_units)[i] = t[p];
    }
}

template <class Sch>
__global__ void __launch_bounds__(256, 1) k_umma_test_scheme(const __grid_constant__ CUtensorMap m0,
                                                             const __grid_constant__ CUtensorMap m1,
                                                             const __grid_constant__ CUtensorMap m2, int M, int K,
                                                             float* C, int* err) {
    using namespace pcv::umma;
    extern __shared__ __align__(1024) unsigned char raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stages = base;
    UmmaTestSmem& sm = *reinterpret_cast<UmmaTestSmem*>(base + kTestStages * stage_bytes<Sch>(kTilesPerPass));
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        pipe_init(sm.pipe, kTestStages);
        sm.err = 0;
    }
    if (warp == 1) tmem_alloc(&sm.pipe.tmem_base, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    Phases ph;
    auto epi = [&](int row0, int quad, uint32_t taddr) {
        const int r = row0 - kTileM + quad * 32 + (threadIdx.x & 31);
        for (int c0 = 0; c0 < kTileN; c0 += 32) {
            float v[32];
            tmem_ld32(taddr + c0, v);
            if (r < M)
                for (int j = 0; j < 32; ++j) C[(int64_t)r * kTileN + c0 + j] = v[j];
        }
    };
    const bool ok = block_column<false, kTilesPerPass, Sch>(sm.pipe, ph, stages, &m0, &m1, &m2, 0, kTileM, M, 0,
                                                            K * (Sch::kElem / 2), epi);
    if (!ok) atomicExch(&sm.err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(sm.pipe.tmem_base, kTmemCols);
    if (threadIdx.x == 0) *err = sm.err;
}

template <class Sch>
pcv_status umma_scheme_test(const float* A, int32_t M, const float* B, int32_t K, float* C) {
    using namespace pcv::umma;
    const int Mp = (M + kTileM - 1) / kTileM * kTileM;
    const int64_t rows = kTileM + Mp;
    std::vector<float> X((size_t)rows * K, 0.0f);
    for (int r = 0; r < kTileM; ++r)
        for (int k = 0; k < K; ++k) X[(size_t)r * K + k] = B[(size_t)r * K + k];
    for (int r = 0; r < M; ++r)
        for (int k = 0; k < K; ++k) X[(size_t)(kTileM + r) * K + k] = A[(size_t)r * K + k];
    const int64_t n = rows * K;
    const int64_t units = n * (Sch::kElem / 2);   // 16-bit units per plane
    float *dX = nullptr, *dC = nullptr;
    uint16_t* dP = nullptr;
    int* dErr = nullptr;
    pcv_status st = PCV_OK;
    if (cudaMalloc(&dX, n * 4) || cudaMalloc(&dP, Sch::kPlanes * units * 2) ||
        cudaMalloc(&dC, (size_t)M * kTileN * 4) || cudaMalloc(&dErr, 4)) {
        st = PCV_ERR_OOM;
    } else {
        cudaMemcpy(dX, X.data(), n * 4, cudaMemcpyHostToDevice);
        k_split_scheme<Sch><<<(unsigned)((n + 255) / 256), 256>>>(dX, n, dP, units);
        CUtensorMap m[3];
        bool ok = true;
        for (int p = 0; p < 3; ++p)
            ok = ok && make_plane_map(&m[p], dP + std::min(p, Sch::kPlanes - 1) * units,
                                      (uint64_t)K * (Sch::kElem / 2), (uint64_t)rows);
        if (!ok) {
            st = PCV_ERR_CUDA;
        } else {
            const int smem = kTestStages * stage_bytes<Sch>(kTilesPerPass) + (int)sizeof(UmmaTestSmem) + 1024;
            cudaFuncSetAttribute(k_umma_test_scheme<Sch>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_umma_test_scheme<Sch><<<1, 256, smem>>>(m[0], m[1], m[2], M, K, dC, dErr);
            pcv::count_launch(2);
            int herr = 0;
            if (cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = PCV_ERR_CUDA;
            else if (herr) st = PCV_ERR_TIMEOUT;
            else if (cudaMemcpy(C, dC, (size_t)M * kTileN * 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = PCV_ERR_CUDA;
        }
    }
    cudaFree(dX);
    cudaFree(dP);
    cudaFree(dC);
    cudaFree(dErr);
    return st;
}

}  // namespace

// The block-column product of the mixed path's factorisation with one operand scheme:
// scheme 0 = three BF16 terms, 1 = two FP16 terms, 2 = TF32, 3 = two TF32 terms.
PCV_API pcv_status pcv_selftest_umma_scheme(int32_t scheme, const float* A, int32_t M, const float* B, int32_t K,
                                            float* C) {
    using namespace pcv::umma;
    if (!A || !B || !C || M < 1 || K < kChunkK || K % kChunkK) return PCV_ERR_ARG;
    switch (scheme) {
        case 0: return umma_scheme_test<SplitBF16x3>(A, M, B, K, C);
        case 1: return umma_scheme_test<SplitF16x2>(A, M, B, K, C);
        case 2: return umma_scheme_test<SplitTF32x1>(A, M, B, K, C);
        case 3: return umma_scheme_test<SplitTF32x3>(A, M, B, K, C);
        default: return PCV_ERR_ARG;
    }
}

// C (M x 128, row-major) = A (M x K) * B (128 x K)^T through the split-BF16 tensor-core
// pipeline; K a positive multiple of 32.  Host arrays.  Returns PCV_ERR_TIMEOUT if a
// bounded wait ran out inside the kernel.
PCV_API pcv_status pcv_selftest_umma(const float* A, int32_t M, const float* B, int32_t K, float* C) {
    using namespace pcv::umma;
    if (!A || !B || !C || M < 1 || K < kChunkK || K % kChunkK) return PCV_ERR_ARG;
    const int Mp = (M + kTileM - 1) / kTileM * kTileM;
    const int64_t rows = kTileM + Mp;
    std::vector<float> X((size_t)rows * K, 0.0f);
    for (int r = 0; r < kTileM; ++r)
        for (int k = 0; k < K; ++k) X[(size_t)r * K + k] = B[(size_t)r * K + k];
    for (int r = 0; r < M; ++r)
        for (int k = 0; k < K; ++k) X[(size_t)(kTileM + r) * K + k] = A[(size_t)r * K + k];
    float *dX = nullptr, *dC = nullptr;
    __nv_bfloat16* dP = nullptr;
    int* dErr = nullptr;
    const int64_t n = rows * K;
    pcv_status st = PCV_OK;
    if (cudaMalloc(&dX, n * 4) || cudaMalloc(&dP, 3 * n * 2) || cudaMalloc(&dC, (size_t)M * kTileN * 4) ||
        cudaMalloc(&dErr, 4)) {
        st = PCV_ERR_OOM;
    } else {
        cudaMemcpy(dX, X.data(), n * 4, cudaMemcpyHostToDevice);
        k_split<<<(unsigned)((n + 255) / 256), 256>>>(dX, n, dP, dP + n, dP + 2 * n);
        CUtensorMap m[3];
        bool ok = true;
        for (int p = 0; p < 3; ++p) ok = ok && make_plane_map(&m[p], dP + p * n, (uint64_t)K, (uint64_t)rows);
        if (!ok) {
            st = PCV_ERR_CUDA;
        } else {
            const int smem = kTestStages * kTestStageBytes + (int)sizeof(UmmaTestSmem) + 1024;
            cudaFuncSetAttribute(k_umma_test, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            k_umma_test<<<1, 256, smem>>>(m[0], m[1], m[2], M, K, dC, dErr);
            pcv::count_launch(2);
            int herr = 0;
            if (cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = PCV_ERR_CUDA;
            else if (herr) st = PCV_ERR_TIMEOUT;
            else if (cudaMemcpy(C, dC, (size_t)M * kTileN * 4, cudaMemcpyDeviceToHost) != cudaSuccess) st = PCV_ERR_CUDA;
        }
    }
    cudaFree(dX);
    cudaFree(dP);
    cudaFree(dC);
    cudaFree(dErr);
    return st;
}
