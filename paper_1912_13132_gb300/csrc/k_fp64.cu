// k_fp64.cu -- the all-FP64 GPU path of parallel cross-validation (arXiv 1912.13132).
//
// One persistent launch evaluates every (subset, configuration) task: Algorithm 1's
// "parallel for" over subsets, extended over the batch of configurations.  A CTA
// takes tasks from a global counter (longest subset first) and runs one task at a
// time in its own workspace slot:
//   gather    training coordinates/values of subset i             (Algorithm 1, read step)
//   assemble  A = Sigma(rho) + lambda I, lambda = tau2 / sigma2  (Eq. 3, second line; Sec. 3)
//   factor    A = L L^T, left-looking, 64-wide block columns
//   solve     alpha = L^-T L^-1 y_T
//   predict   yhat_j = sum_a exp(-||p_j - s_a|| / rho) alpha_a   (Eq. 3)
//   loss      z = sum_j (yhat_j - y_V,j)^2                        (Eq. 4)
// GB300's FP64 rate is a small fraction of its FP32 rate, so this path is the
// correctness reference on the device; the mixed path is the fast one.
#include <cuda_runtime.h>

#include <cmath>

#include <mutex>

#include "pcv_internal.h"

namespace pcv {
namespace {

constexpr int NB = 64;    // block-column width
constexpr int NT = 256;   // threads per CTA
constexpr int KC = 16;    // K chunk of the trailing update

struct Slot64 {
    double* A;    // ld x ld, column-major, lower triangle used
    double* sx;   // ld
    double* sy;   // ld
    double* yt;   // ld: training values
    double* al;   // ld: right-hand side -> w -> alpha
    double* ep;   // mmax: squared errors
};

__device__ __forceinline__ Slot64 slot_of(const TaskArgs& a) {
    char* base = reinterpret_cast<char*>(a.work) + (int64_t)blockIdx.x * a.slot_bytes;
    Slot64 s;
    const int64_t ld = a.ld;
    s.A = reinterpret_cast<double*>(base);
    s.sx = s.A + ld * ld;
    s.sy = s.sx + ld;
    s.yt = s.sy + ld;
    s.al = s.yt + ld;
    s.ep = s.al + ld;
    return s;
}

__device__ __forceinline__ double cov64(double ax, double ay, double bx, double by, double rho) {
    const double dx = ax - bx, dy = ay - by;
    return exp(-sqrt(dx * dx + dy * dy) / rho);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Smem64 {
    double L[NB][NB + 1];     // diagonal block
    double Ta[KC][NB + 1];    // trailing-update staging: rows of the updated tile
    double Tb[KC][NB + 1];    // trailing-update staging: rows of the block column's top
    double red[NT / 32];
    double red2[NT / 32];
    int flag;
    int task;
};

// C[r0:r0+rb, j0:j0+jb] -= L[r0:r0+rb, 0:j0] * L[j0:j0+jb, 0:j0]^T (j0 is a multiple of NB)
__device__ void update_tile(Smem64& sm, double* A, int64_t ld, int r0, int rb, int j0, int jb) {
    const int tid = threadIdx.x;
    const int ty = tid / 16, tx = tid % 16;
    double acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
    for (int p0 = 0; p0 < j0; p0 += KC) {
        for (int e = tid; e < KC * NB; e += NT) {
            const int r = e % NB, q = e / NB;
            sm.Ta[q][r] = (r < rb) ? A[(int64_t)(r0 + r) + (int64_t)(p0 + q) * ld] : 0.0;
            sm.Tb[q][r] = (r < jb) ? A[(int64_t)(j0 + r) + (int64_t)(p0 + q) * ld] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < KC; ++q) {
            double ar[4], bc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) ar[u] = sm.Ta[q][ty * 4 + u];
#pragma unroll
            for (int v = 0; v < 4; ++v) bc[v] = sm.Tb[q][tx * 4 + v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(ar[u], bc[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = ty * 4 + u, c = tx * 4 + v;
            if (r < rb && c < jb) A[(int64_t)(r0 + r) + (int64_t)(j0 + c) * ld] -= acc[u][v];
        }
}

// Factor task (subset i, configuration b); returns the task status.
__device__ int run_task(Smem64& sm, const TaskArgs& a, int i, int b) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int pr = a.param_row ? a.param_row[i] : b;   // the subset's own row, or the task's
    const double s2 = a.params[3 * pr], rho = a.params[3 * pr + 1], tau2 = a.params[3 * pr + 2];
    const int64_t zoff = (int64_t)b * a.N + i;
    const int64_t p0 = a.P_off[i];
    const int m = (int)(a.P_off[i + 1] - p0);
    const bool bad = !(s2 > 0.0) || !(rho > 0.0) || !(tau2 >= 0.0) || !isfinite(s2) || !isfinite(rho) || !isfinite(tau2);
    if (bad) {
        if (a.yhat)
            for (int j = tid; j < m; j += NT) a.yhat[(int64_t)b * a.yhat_stride + p0 + j] = NAN;
        if (tid == 0) {
            a.z[zoff] = NAN;
            if (a.lik) a.lik[zoff] = NAN;
            a.tstatus[zoff] = PCV_ERR_ARG;
        }
        return PCV_ERR_ARG;
    }
    const double lam = tau2 / s2;
    const int64_t t0 = a.T_off[i];
    const int k = (int)(a.T_off[i + 1] - t0);
    const int64_t ld = a.ld;
    Slot64 S = slot_of(a);

    // gather (Algorithm 1: read the subset's data)
    for (int t = tid; t < k; t += NT) {
        const int g = a.T_idx[t0 + t];
        S.sx[t] = a.X[g];
        S.sy[t] = a.Y[g];
        S.yt[t] = a.Vals[g];
        S.al[t] = a.Vals[g];
    }
    __syncthreads();

    // predictions from kriging weights computed earlier (alpha_in): no matrix, no solve
    const bool pred_only = a.alpha_in != nullptr;
    // assemble the lower triangle of Sigma + lambda I (column-major)
    const int nb = pred_only ? 0 : (k + NB - 1) / NB;
    for (int bj = 0; bj < nb; ++bj)
        for (int bi = bj; bi < nb; ++bi)
            for (int e = tid; e < NB * NB; e += NT) {
                const int r = bi * NB + (e % NB), c = bj * NB + (e / NB);
                if (r < k && c <= r)
                    S.A[r + (int64_t)c * ld] = (r == c) ? 1.0 + lam : cov64(S.sx[r], S.sy[r], S.sx[c], S.sy[c], rho);
            }
    __syncthreads();

    // left-looking blocked Cholesky
    for (int J = 0; J < nb; ++J) {
        const int j0 = J * NB, jb = min(NB, k - j0);
        if (j0 > 0) {
            for (int R = J; R < nb; ++R) update_tile(sm, S.A, ld, R * NB, min(NB, k - R * NB), j0, jb);
            __syncthreads();   // the updated block column is read by other threads below
        }
        // diagonal block: Cholesky-Crout in shared memory
        for (int e = tid; e < NB * NB; e += NT) {
            const int r = e % NB, c = e / NB;
            if (r < jb && c <= r) sm.L[r][c] = S.A[(j0 + r) + (int64_t)(j0 + c) * ld];
        }
        if (tid == 0) sm.flag = 0;
        __syncthreads();
        for (int c = 0; c < jb; ++c) {
            if (tid == 0) {
                double s = sm.L[c][c];
                for (int p = 0; p < c; ++p) s -= sm.L[c][p] * sm.L[c][p];
                if (!(s > 0.0)) { sm.flag = 1; s = 1.0; }
                sm.L[c][c] = sqrt(s);
            }
            __syncthreads();
            const double d = sm.L[c][c];
            for (int r = c + 1 + tid; r < jb; r += NT) {
                double s = sm.L[r][c];
                for (int p = 0; p < c; ++p) s -= sm.L[r][p] * sm.L[c][p];
                sm.L[r][c] = s / d;
            }
            __syncthreads();
        }
        if (sm.flag) {
            if (a.yhat)
                for (int j = tid; j < m; j += NT) a.yhat[(int64_t)b * a.yhat_stride + p0 + j] = NAN;
            if (tid == 0) {
                a.z[zoff] = NAN;
                if (a.lik) a.lik[zoff] = NAN;
                a.tstatus[zoff] = PCV_NOT_SPD;
            }
            __syncthreads();
            return PCV_NOT_SPD;
        }
        for (int e = tid; e < NB * NB; e += NT) {
            const int r = e % NB, c = e / NB;
            if (r < jb && c <= r) S.A[(j0 + r) + (int64_t)(j0 + c) * ld] = sm.L[r][c];
        }
        // rows below: x L_JJ^T = c  (triangular solve per row)
        for (int r = j0 + jb + tid; r < k; r += NT) {
            for (int c = 0; c < jb; ++c) {
                double s = S.A[r + (int64_t)(j0 + c) * ld];
                for (int p = 0; p < c; ++p) s -= S.A[r + (int64_t)(j0 + p) * ld] * sm.L[c][p];
                S.A[r + (int64_t)(j0 + c) * ld] = s / sm.L[c][c];
            }
        }
        __syncthreads();
    }

    // several right-hand sides (a.rhs): one factorisation, each column solved and predicted
    const int nrhs = a.rhs ? a.nrhs : 1;
    for (int rh = 0; rh < nrhs; ++rh) {
        if (a.rhs) {   // this column's values (the factor stays)
            for (int t = tid; t < k; t += NT) S.al[t] = a.rhs[rh * a.rhs_stride + a.T_idx[t0 + t]];
            __syncthreads();
        }
        // forward substitution L w = y
        for (int J = 0; J < nb; ++J) {
            const int j0 = J * NB, jb = min(NB, k - j0);
            for (int r = warp; r < jb; r += NT / 32) {
                double s = 0.0;
                for (int p = lane; p < j0; p += 32) s += S.A[(j0 + r) + (int64_t)p * ld] * S.al[p];
                s = warp_sum(s);
                if (lane == 0) S.al[j0 + r] -= s;
            }
            __syncthreads();
            if (tid == 0)
                for (int c = 0; c < jb; ++c) {
                    double s = S.al[j0 + c];
                    for (int p = 0; p < c; ++p) s -= S.A[(j0 + c) + (int64_t)(j0 + p) * ld] * S.al[j0 + p];
                    S.al[j0 + c] = s / S.A[(j0 + c) + (int64_t)(j0 + c) * ld];
                }
            __syncthreads();
        }
        // back substitution L^T alpha = w
        for (int J = nb - 1; J >= 0; --J) {
            const int j0 = J * NB, jb = min(NB, k - j0);
            for (int c = warp; c < jb; c += NT / 32) {
                double s = 0.0;
                for (int p = j0 + jb + lane; p < k; p += 32) s += S.A[p + (int64_t)(j0 + c) * ld] * S.al[p];
                s = warp_sum(s);
                if (lane == 0) S.al[j0 + c] -= s;
            }
            __syncthreads();
            if (tid == 0)
                for (int c = jb - 1; c >= 0; --c) {
                    double s = S.al[j0 + c];
                    for (int p = c + 1; p < jb; ++p) s -= S.A[(j0 + p) + (int64_t)(j0 + c) * ld] * S.al[j0 + p];
                    S.al[j0 + c] = s / S.A[(j0 + c) + (int64_t)(j0 + c) * ld];
                }
            __syncthreads();
        }

        if (pred_only) {
            const double* al = a.alpha_in + (int64_t)(a.alpha_slot ? a.alpha_slot[b] : 0) * a.alpha_stride + t0;
            for (int t = tid; t < k; t += NT) S.al[t] = al[t];
            __syncthreads();
        } else if (a.alpha_out && a.alpha_slot && a.alpha_slot[b] >= 0 && !a.rhs) {
            // keep the kriging weights for later predictions at new locations
            double* al = a.alpha_out + (int64_t)a.alpha_slot[b] * a.alpha_stride + t0;
            for (int t = tid; t < k; t += NT) al[t] = S.al[t];
        }
        // local -2 log-likelihood (Eq. 2) of the training data from the same factor:
        // log det(sigma2 A) = k log sigma2 + 2 sum log L_jj, y^T (sigma2 A)^-1 y = y^T alpha / sigma2
        if (a.lik && rh == 0) {
            double ldet = 0.0, quad = 0.0;
            for (int q = tid; q < k; q += NT) {
                ldet += log(S.A[q + (int64_t)q * ld]);
                quad += a.Vals[a.T_idx[t0 + q]] * S.al[q];
            }
            ldet = warp_sum(ldet);
            quad = warp_sum(quad);
            if (lane == 0) { sm.red[warp] = ldet; sm.red2[warp] = quad; }
            __syncthreads();
            if (tid == 0) {
                double l = 0.0, qf = 0.0;
                for (int w = 0; w < NT / 32; ++w) { l += sm.red[w]; qf += sm.red2[w]; }
                a.lik[zoff] = k * log(2.0 * M_PI) + k * log(s2) + 2.0 * l + qf / s2;
            }
            __syncthreads();
        }

        // predict (Eq. 3) and squared errors (Eq. 4)
        for (int j = warp; j < m; j += NT / 32) {
            const double px = a.Px[p0 + j], py = a.Py[p0 + j];
            double s = 0.0;
            for (int t = lane; t < k; t += 32) s += cov64(px, py, S.sx[t], S.sy[t], rho) * S.al[t];
            s = warp_sum(s);
            if (lane == 0) {
                if (a.yhat) a.yhat[(int64_t)(a.rhs ? rh : b) * a.yhat_stride + p0 + j] = s;
                if (a.Pv) {
                    const double e = s - a.Pv[p0 + j];
                    S.ep[j] = e * e;
                }
            }
        }
        __syncthreads();
        if (a.Pv) {
            double s = 0.0;
            for (int j = tid; j < m; j += NT) s += S.ep[j];
            s = warp_sum(s);
            if (lane == 0) sm.red[warp] = s;
            __syncthreads();
            if (tid == 0) {
                double zz = 0.0;
                for (int w = 0; w < NT / 32; ++w) zz += sm.red[w];
                a.z[zoff] = zz;
            }
        }
    }
    if (tid == 0) a.tstatus[zoff] = a.task_list ? a.list_status : PCV_OK;
    __syncthreads();
    return PCV_OK;
}

__global__ void __launch_bounds__(NT, 1) k_cv_fp64(TaskArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem64& sm = *reinterpret_cast<Smem64*>(smem_raw);
    const int ntask = a.task_list ? (int)*a.task_count : a.n_order * a.B;
    for (;;) {
        if (threadIdx.x == 0) sm.task = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        int t = sm.task;
        __syncthreads();
        if (t >= ntask) break;
        if (a.task_list) t = a.task_list[t];
        run_task(sm, a, a.order ? a.order[t / a.B] : t / a.B, t % a.B);
    }
}

}  // namespace

int64_t slot_bytes_fp64(int32_t ld, int64_t mmax) {
    int64_t e = (int64_t)ld * ld + 4 * (int64_t)ld + mmax + 32;
    return ((e * 8 + 255) / 256) * 256;
}

int launch_task_fp64(const TaskArgs& a, int grid, void* stream) {
    // the shared-memory opt-in is a per-device function attribute; contexts on
    // several devices and the serving workers may get here concurrently
    static std::mutex mu;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!attr_set[dev]) {
            e = cudaFuncSetAttribute(k_cv_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem64));
            if (e != cudaSuccess) return (int)e;
            attr_set[dev] = true;
        }
    }
    k_cv_fp64<<<grid, NT, sizeof(Smem64), (cudaStream_t)stream>>>(a);
    count_launch();
    return (int)cudaGetLastError();
}

}  // namespace pcv
