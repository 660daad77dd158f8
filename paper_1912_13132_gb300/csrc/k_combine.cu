// k_combine.cu -- Algorithm 1's combine step (z = sum_i z_i, Eq. 6) on the device.
//
// One CTA per configuration sums the N local SSPEs in a fixed order (thread-strided
// partial sums, then a fixed tree), so the result does not depend on how the tasks
// were scheduled.  The configuration's status is the most severe task status, or
// PCV_ERR_ARG when its parameters are invalid.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>

#include "pcv_internal.h"

namespace pcv {
namespace {

constexpr int CT = 256;

__device__ __forceinline__ int severity(int st) {
    switch (st) {
        case PCV_OK: return 0;
        case PCV_REFINE_FALLBACK: return 1;
        case PCV_NOT_SPD: return 2;
        default: return 3;
    }
}

__global__ void __launch_bounds__(CT) k_combine(const double* z, const int32_t* tst, const double* params,
                                                int N, double* sspe, int32_t* status) {
    __shared__ double part[CT];
    __shared__ int sev;
    const int b = blockIdx.x, tid = threadIdx.x;
    if (tid == 0) sev = 0;
    __syncthreads();
    double s = 0.0;
    int mysev = 0;
    for (int i = tid; i < N; i += CT) {
        s += z[(int64_t)b * N + i];
        mysev = max(mysev, severity(tst[(int64_t)b * N + i]));
    }
    part[tid] = s;
    if (mysev) atomicMax(&sev, mysev);
    __syncthreads();
    for (int w = CT / 2; w > 0; w >>= 1) {
        if (tid < w) part[tid] += part[tid + w];
        __syncthreads();
    }
    if (tid == 0) {
        const double s2 = params[3 * b], rho = params[3 * b + 1], tau2 = params[3 * b + 2];
        const bool bad = !(s2 > 0.0) || !(rho > 0.0) || !(tau2 >= 0.0) || !isfinite(s2) || !isfinite(rho) || !isfinite(tau2);
        int st = PCV_OK;
        if (bad) st = PCV_ERR_ARG;
        else if (sev == 2) st = PCV_NOT_SPD;
        else if (sev == 3) st = PCV_ERR_ARG;
        else if (sev == 1) st = PCV_REFINE_FALLBACK;
        sspe[b] = (st == PCV_ERR_ARG || st == PCV_NOT_SPD) ? NAN : part[0];
        if (status) status[b] = st;
    }
}

thread_local int64_t g_launches = 0;

}  // namespace

void count_launch(int n) { g_launches += n; }

int launch_combine(const double* z, const int32_t* tstatus, const double* params, int32_t B, int32_t N,
                   double* sspe, int32_t* status, void* stream) {
    if (B <= 0) return 0;
    k_combine<<<B, CT, 0, (cudaStream_t)stream>>>(z, tstatus, params, N, sspe, status);
    count_launch();
    return (int)cudaGetLastError();
}

}  // namespace pcv

PCV_API int64_t pcv_launch_count(int32_t reset) {
    int64_t v = pcv::g_launches;
    if (reset) pcv::g_launches = 0;
    return v;
}
