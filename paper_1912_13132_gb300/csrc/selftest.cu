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
