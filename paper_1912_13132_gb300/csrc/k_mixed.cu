// k_mixed.cu -- mixed-precision path of parallel cross-validation (arXiv 1912.13132).
//
// Same task decomposition as the FP64 path (Algorithm 1's parallel loop over
// subsets, extended over the batch of configurations), different arithmetic:
//   gather     training coordinates as offsets from the subset's first training
//              point in units of rho, split in double-float (high parts on a
//              power-of-two grid so that differences of high parts are exact)
//   assemble   A32 = Sigma(rho) + lambda I in FP32                  (Eq. 3, Sec. 3);
//              on lattice data (the LAT variant) every entry comes from a per-task
//              FP64 table of covariances by index offset, and only the 128 x 128
//              diagonal blocks are stored (the factorisation reads the rest from it)
//   factor     A32 ~ L L^T, left-looking: tensor engine (k_cv_mixed_tc) with
//              128-wide block columns whose trailing updates and panels run on
//              tcgen05 from 16-bit planes (two FP16 terms per value by default,
//              three BF16 terms as an option); FP32 engine (k_cv_mixed) with
//              64-wide blocks.  The first forward solve rides on the panels.
//   refine     x <- x + L^-T L^-1 r,  r = y - A x with A's entries and the sums
//              in double-float (exp by Tang's method, see df.cuh), until the error
//              left, estimated as |d_i|^2 / |d_i-1|, is below refine_tol |x|
//   predict    yhat_j = sum_a exp(-||p_j - s_a|| / rho) x_a in double-float (Eq. 3)
//   loss       z = sum_j (yhat_j - y_V,j)^2 in FP64                  (Eq. 4)
// A task whose FP32 factorisation breaks down or whose refinement does not
// converge is appended to a fallback list that the FP64 kernel then runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstddef>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "df.cuh"
#include "pcv_internal.h"
#include "umma.cuh"

namespace pcv {
namespace {

using dfm::df;

constexpr int NB = 64;   // block-column width of the factorisation and of the residual tiles
constexpr int NT = 256;  // threads per CTA
constexpr int KC = 16;   // K chunk of the trailing update

__constant__ dfm::ExpConsts c_exp;

// Per-phase cycle counters (thread 0 of each CTA adds its elapsed clock64 cycles).
__device__ __forceinline__ long long now_cycles() {
    long long t;
    asm volatile("mov.u64 %0, %%clock64;" : "=l"(t));
    return t;
}

struct PhaseTimer {
    unsigned long long* out;
    long long t;
    __device__ explicit PhaseTimer(unsigned long long* o) : out(o), t(0) {
        if (o) t = now_cycles();
    }
    __device__ void lap(int ph) {
        if (!out) return;
        const long long n = now_cycles();
        if (threadIdx.x == 0) atomicAdd(out + ph, (unsigned long long)(n - t));
        t = n;
    }
};

struct SlotM {
    float* L;      // ld x ld, column-major, lower triangle
    double* yv;    // training values
    double* xs;    // solution
    double* rr;    // residual
    double* ep;    // squared errors (mmax)
    float *xh, *xl, *yh, *yl;   // double-float scaled offsets of the training points
    float* w;      // solve vector
    float *qh, *ql;             // solution in double-float
    float *ah, *al;             // residual accumulators
    float2* tab;                // lattice data: covariance table (hi, lo) by index offset
};

__device__ __forceinline__ SlotM slot_of(const TaskArgs& a) {
    char* base = reinterpret_cast<char*>(a.work) + (int64_t)blockIdx.x * a.slot_bytes;
    const int64_t ld = a.ld;
    SlotM s;
    s.L = reinterpret_cast<float*>(base);
    double* d = reinterpret_cast<double*>(base + ld * ld * 4);
    s.yv = d;
    s.xs = d + ld;
    s.rr = d + 2 * ld;
    float* f = reinterpret_cast<float*>(base + ld * ld * 4 + 3 * ld * 8);
    s.xh = f;
    s.xl = f + ld;
    s.yh = f + 2 * ld;
    s.yl = f + 3 * ld;
    s.w = f + 4 * ld;
    s.qh = f + 5 * ld;
    s.ql = f + 6 * ld;
    s.ah = f + 7 * ld;
    s.al = f + 8 * ld;
    // then the lattice table (a.lat_cap entries), then ep (its length is mmax, not ld)
    s.tab = reinterpret_cast<float2*>(f + 9 * ld);
    s.ep = reinterpret_cast<double*>(s.tab + a.lat_cap);
    return s;
}

// Shared memory used phase by phase (in the tensor-core kernel it lives in the
// operand ring, which is idle outside the trailing updates).
struct alignas(16) SmemM {
    float rinv[NB];                // reciprocals of the diagonal of L_JJ
    float ph[16][NB], pl[16][NB];  // residual partial sums (double-float)
    float wj[2 * NB];              // solve block (128 entries in the tensor-core kernel)
    double dred[NT / 32];
    double dred2[NT / 32];
    int ired[4][NT / 32];
    float fred[NT / 32];
    int flag;
    float L[NB][NB + 1];           // diagonal block of the FP32 engine (last: the tensor-core
                                   // kernel, which never uses it, puts vectors in its place)
};

// the tensor-core forward solve reduces through ph and pl as one 2 x 8 x 128 buffer
static_assert(offsetof(SmemM, pl) == offsetof(SmemM, ph) + 16 * NB * sizeof(float) && NT / 32 == 8 &&
                  2 * 16 * NB >= 2 * (NT / 32) * (2 * NB) && offsetof(SmemM, ph) % 16 == 0,
              "forward-solve reduction buffers");

// Trailing-update staging of the FP32 engine (read with float4 loads).
struct alignas(16) SmemSimt {
    float Ta[KC][NB + 4];
    float Tb[KC][NB + 4];
};

// Shared memory kept for the whole kernel.
struct alignas(8) SmemKeep {
    float tbl[2 * dfm::kExpTable]; // exp table (copy of c_exp.tbl)
    float fwj[2 * NB];             // w_J of the forward solve fused into the factorisation
    int2 lij[2 * NB];              // lattice indices of the block column's points (update epilogue)
    int task;
};

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ float block_max(SmemM& sm, float v) {
    v = warp_max(v);
    if ((threadIdx.x & 31) == 0) sm.fred[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = sm.fred[0];
#pragma unroll
    for (int i = 1; i < NT / 32; ++i) r = fmaxf(r, sm.fred[i]);
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------- factorisation (FP32)

// C[r0:r0+rb, j0:j0+jb] -= L[r0:r0+rb, 0:j0] * L[j0:j0+jb, 0:j0]^T, register prefetch of the next chunk
__device__ void update_tile32(SmemSimt& sm, float* A, int64_t ld, int r0, int rb, int j0, int jb) {
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    float acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
    float pa[4], pb[4];
    auto load = [&](int p0) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int e = tid + NT * s, r = e & (NB - 1), q = e >> 6;
            pa[s] = r < rb ? A[(int64_t)(r0 + r) + (int64_t)(p0 + q) * ld] : 0.0f;
            pb[s] = r < jb ? A[(int64_t)(j0 + r) + (int64_t)(p0 + q) * ld] : 0.0f;
        }
    };
    load(0);
    for (int p0 = 0; p0 < j0; p0 += KC) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int e = tid + NT * s, r = e & (NB - 1), q = e >> 6;
            sm.Ta[q][r] = pa[s];
            sm.Tb[q][r] = pb[s];
        }
        __syncthreads();
        if (p0 + KC < j0) load(p0 + KC);
#pragma unroll
        for (int q = 0; q < KC; ++q) {
            const float4 ar = *reinterpret_cast<const float4*>(&sm.Ta[q][ty * 4]);
            const float4 bc = *reinterpret_cast<const float4*>(&sm.Tb[q][tx * 4]);
            const float a4[4] = {ar.x, ar.y, ar.z, ar.w}, b4[4] = {bc.x, bc.y, bc.z, bc.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a4[u], b4[v], acc[u][v]);
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

// Left-looking blocked Cholesky of the FP32 matrix in S.L; false if a pivot is not positive.
__device__ bool factor32(SmemM& sm, SmemSimt& st, const SlotM& S, int k, int64_t ld) {
    const int tid = threadIdx.x;
    const int nb = (k + NB - 1) / NB;
    for (int J = 0; J < nb; ++J) {
        const int j0 = J * NB, jb = min(NB, k - j0);
        if (j0 > 0) {
            for (int R = J; R < nb; ++R) update_tile32(st, S.L, ld, R * NB, min(NB, k - R * NB), j0, jb);
            __syncthreads();
        }
        for (int e = tid; e < NB * NB; e += NT) {
            const int r = e & (NB - 1), c = e >> 6;
            if (r < jb && c <= r) sm.L[r][c] = S.L[(j0 + r) + (int64_t)(j0 + c) * ld];
        }
        if (tid == 0) sm.flag = 0;
        __syncthreads();
        for (int c = 0; c < jb; ++c) {
            if (tid == 0) {
                float s = sm.L[c][c];
                for (int p = 0; p < c; ++p) s = fmaf(-sm.L[c][p], sm.L[c][p], s);
                if (!(s > 0.0f)) { sm.flag = 1; s = 1.0f; }
                const float d = sqrtf(s);
                sm.L[c][c] = d;
                sm.rinv[c] = 1.0f / d;
            }
            __syncthreads();
            const float rd = sm.rinv[c];
            for (int r = c + 1 + tid; r < jb; r += NT) {
                float s = sm.L[r][c];
                for (int p = 0; p < c; ++p) s = fmaf(-sm.L[r][p], sm.L[c][p], s);
                sm.L[r][c] = s * rd;
            }
            __syncthreads();
        }
        if (sm.flag) return false;
        for (int e = tid; e < NB * NB; e += NT) {
            const int r = e & (NB - 1), c = e >> 6;
            if (r < jb && c <= r) S.L[(j0 + r) + (int64_t)(j0 + c) * ld] = sm.L[r][c];
        }
        // rows below: x L_JJ^T = row, one row per thread, the row kept in registers
        for (int r = j0 + jb + tid; r < k; r += NT) {
            float x[NB];
#pragma unroll
            for (int c = 0; c < NB; ++c) x[c] = c < jb ? S.L[r + (int64_t)(j0 + c) * ld] : 0.0f;
#pragma unroll
            for (int c = 0; c < NB; ++c) {
                float s = x[c];
#pragma unroll
                for (int p = 0; p < c; ++p) s = fmaf(-x[p], sm.L[c][p], s);
                x[c] = c < jb ? s * sm.rinv[c] : 0.0f;
            }
#pragma unroll
            for (int c = 0; c < NB; ++c)
                if (c < jb) S.L[r + (int64_t)(j0 + c) * ld] = x[c];
        }
        __syncthreads();
    }
    return true;
}

// ---------------------------------------------------------------- factorisation (tensor cores)

constexpr int TB = umma::kTileN;          // 128-wide block columns
constexpr int kTcTilesPerPass = 1;        // one 128-row tile per pass: 256 TMEM columns per CTA
constexpr uint32_t kTcTmemCols = 2 * kTcTilesPerPass * umma::kTileN;
// The operand ring (stages x stage bytes of the scheme) doubles as the shared memory of
// the phases between trailing updates, which need kTcRingMin bytes: 2 stages of the
// three-plane scheme, 3 of the two-plane one.
constexpr int kTcRingMin = 96 * 1024;
// (at least kTcRingMin: schemes with small stages get a ring larger than their stages use)
template <class Sch>
__host__ __device__ constexpr int tc_ring_bytes(int nst) {
    return nst * umma::stage_bytes<Sch>(kTcTilesPerPass) > kTcRingMin ? nst * umma::stage_bytes<Sch>(kTcTilesPerPass)
                                                                       : kTcRingMin;
}
// 16-bit units per term of a scheme (the planes, tensor maps and K chunks count in them)
template <class Sch>
__host__ __device__ constexpr int kw() { return Sch::kElem / 2; }
constexpr int DP = TB + 4;                // row pitch of the diagonal block (rows 16-byte aligned)
static_assert(TB == 2 * NB, "the tensor-core solves use 2 * NB-wide blocks");

struct TcShared {
    umma::Pipe pipe;
    int dead;   // a bounded wait ran out: this CTA stops using the tensor path
};

struct TcCtx {
    TcShared* sh;
    uint8_t* stages;                      // operand ring; between updates also the diagonal block
    umma::Phases ph;
    const CUtensorMap *m0, *m1, *m2;
    uint16_t* p[3];                       // this slot's planes (16-bit terms, tiled, ld x ld)
    int row_base;                         // this slot's first row in the tensor maps
};

// Term (r, c) of a slot's planes, in 16-bit units: 128 x 32-unit tiles (64-byte rows),
// tile (r / 128, u / 32) for u = c * kw (the unit where the term starts), row-major inside
// a tile (the layout the 3-D tensor maps address).
template <class Sch>
__device__ __forceinline__ int64_t plane_off(int r, int c, int64_t ld) {
    const int u = c * kw<Sch>();
    return ((int64_t)(r >> 7) * ((ld * kw<Sch>()) >> 5) + (u >> 5)) * 4096 + (r & 127) * 32 + (u & 31);
}

// Eight consecutive FP32 values (c multiple of 8) split into the scheme's planes.
template <class Sch>
__device__ __forceinline__ void store_planes8(const TcCtx& tc, int64_t off, const float* x) {
    if constexpr (Sch::kElem == 2) {
        __align__(16) uint16_t t[Sch::kPlanes][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint16_t u[Sch::kPlanes];
            umma::split_terms(Sch{}, x[q], u);
#pragma unroll
            for (int pl = 0; pl < Sch::kPlanes; ++pl) t[pl][q] = u[pl];
        }
#pragma unroll
        for (int pl = 0; pl < Sch::kPlanes; ++pl)
            *reinterpret_cast<uint4*>(tc.p[pl] + off) = *reinterpret_cast<const uint4*>(t[pl]);
    } else {
        __align__(16) uint32_t t[Sch::kPlanes][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            uint32_t u[Sch::kPlanes];
            umma::split_terms(Sch{}, x[q], u);
#pragma unroll
            for (int pl = 0; pl < Sch::kPlanes; ++pl) t[pl][q] = u[pl];
        }
#pragma unroll
        for (int pl = 0; pl < Sch::kPlanes; ++pl) {
            uint4* d = reinterpret_cast<uint4*>(tc.p[pl] + off);
            d[0] = *reinterpret_cast<const uint4*>(t[pl]);
            d[1] = *reinterpret_cast<const uint4*>(t[pl] + 4);
        }
    }
}

// Cholesky of the nb x nb (nb <= 32) sub-block of D at (c0, c0) by one warp: lane i
// holds row i in registers; column c is scaled by its pivot, then the later columns
// take the rank-1 update with the scaled entries of the rows they belong to, fetched
// by shuffles.  Every lane runs every update (no divergent branches): entries above a
// lane's diagonal then hold meaningless values, which are never read -- the sub-block's
// upper triangle in D is scratch.  Writes 1 / L[c][c] to rinv; false (the same in all
// lanes) if a pivot is not positive.
__device__ __forceinline__ bool chol32_warp(float (*D)[DP], float* rinv, int c0, int nb, int lane) {
    float a[32];
    const bool live = lane < nb;
#pragma unroll
    for (int j = 0; j < 32; ++j) a[j] = live ? D[c0 + lane][c0 + j] : 0.0f;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        if (c < nb) {
            float piv = __shfl_sync(0xffffffffu, a[c], c);
            if (!(piv > 0.0f)) {
                ok = false;
                piv = 1.0f;
            }
            // the FP32 factor only preconditions the refinement: rsqrtf (2 ulp) in
            // place of an IEEE square root and division on the column's critical path
            const float rd = rsqrtf(piv), d = piv * rd;
            a[c] = lane == c ? d : a[c] * rd;
            rinv[c0 + c] = rd;
#pragma unroll
            for (int j = c + 1; j < 32; ++j) a[j] = fmaf(-a[c], __shfl_sync(0xffffffffu, a[c], j), a[j]);
        }
    }
    if (live) {
#pragma unroll
        for (int j = 0; j < 32; ++j) D[c0 + lane][c0 + j] = a[j];
    }
    return ok;
}

// Rows t0..jb-1 of D, columns c0..c0+31: x L11^T = row with L11 the factored 32 x 32
// sub-block at (c0, c0); one row per thread, four partial sums.
__device__ __forceinline__ void trsm32_rows(float (*D)[DP], const float* rinv, int c0, int t0, int jb) {
    for (int r = t0 + (int)threadIdx.x; r < jb; r += NT) {
        float y[32];
#pragma unroll
        for (int p = 0; p < 32; p += 4) {
            const float4 v = *reinterpret_cast<const float4*>(&D[r][c0 + p]);
            y[p] = v.x;
            y[p + 1] = v.y;
            y[p + 2] = v.z;
            y[p + 3] = v.w;
        }
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            float a0 = y[c], a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
            for (int p = 0; p + 3 < c; p += 4) {
                const float4 d = *reinterpret_cast<const float4*>(&D[c0 + c][c0 + p]);
                a0 = fmaf(-y[p], d.x, a0);
                a1 = fmaf(-y[p + 1], d.y, a1);
                a2 = fmaf(-y[p + 2], d.z, a2);
                a3 = fmaf(-y[p + 3], d.w, a3);
            }
#pragma unroll
            for (int p = (c / 4) * 4; p < c; ++p) a0 = fmaf(-y[p], D[c0 + c][c0 + p], a0);
            y[c] = ((a0 + a1) + (a2 + a3)) * rinv[c0 + c];
        }
#pragma unroll
        for (int p = 0; p < 32; p += 4)
            *reinterpret_cast<float4*>(&D[r][c0 + p]) = make_float4(y[p], y[p + 1], y[p + 2], y[p + 3]);
    }
}

// Trailing update D[r][q] -= sum_c D[r][c0 + c] D[q][c0 + c] for t0 <= q <= r < jb, in 4 x 4
// tiles of (r, q), one tile per thread; rows past jb are read clamped and not written.
__device__ __forceinline__ void syrk32_trailing(float (*D)[DP], int c0, int t0, int jb) {
    const int nt4 = (jb - t0 + 3) / 4;
    const int ntiles = nt4 * (nt4 + 1) / 2;
    for (int e = threadIdx.x; e < ntiles; e += NT) {
        // e -> (bi, bj) with bj <= bi, row-major over the lower triangle of tiles
        int bi = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
        while (bi * (bi + 1) / 2 > e) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= e) ++bi;
        const int bj = e - bi * (bi + 1) / 2;
        const int r0 = t0 + 4 * bi, q0 = t0 + 4 * bj;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
#pragma unroll
        for (int p = 0; p < 32; p += 4) {
            float4 ar[4], br[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ar[u] = *reinterpret_cast<const float4*>(&D[min(r0 + u, TB - 1)][c0 + p]);
                br[u] = *reinterpret_cast<const float4*>(&D[min(q0 + u, TB - 1)][c0 + p]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    acc[u][v] = fmaf(ar[u].x, br[v].x, fmaf(ar[u].y, br[v].y,
                                fmaf(ar[u].z, br[v].z, fmaf(ar[u].w, br[v].w, acc[u][v]))));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int r = r0 + u, q = q0 + v;
                if (r < jb && q <= r) D[r][q] -= acc[u][v];
            }
    }
}

// Column j (= lane) of the inverse of the 32 x 32 lower-triangular block of D at
// (c0, c0), by forward substitution in registers (x_i = 0 above the diagonal), written
// back in place, zeros above the diagonal.  rinv holds the reciprocal diagonal.
__device__ __forceinline__ void inv32_warp(float (*D)[DP], const float* rinv, int c0, int lane) {
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        float s = 0.0f;
#pragma unroll
        for (int p = 0; p < i; ++p) s = fmaf(D[c0 + i][c0 + p], x[p], s);
        const float ri = rinv[c0 + i];
        x[i] = i == lane ? ri : (i > lane ? -s * ri : 0.0f);
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 32; ++i) D[c0 + i][c0 + lane] = x[i];
}

// In-place inverse of the 128 x 128 lower-triangular factor in D, in 32 x 32 blocks:
// the four diagonal blocks first (one warp each), then the column blocks J = 2, 1, 0
// from the identity Linv L = I:
//   Linv[I][J] = -( sum_{K=J+1..I} Linv[I][K] L[K][J] ) Linv[J][J],   I > J,
// whose right-hand side only reads finished inverse blocks and column block J of L,
// which is overwritten last.  Y is 3 x 32 x 32 floats of scratch.
__device__ void trinv128(float (*D)[DP], const float* rinv, float* Y) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp < 4) inv32_warp(D, rinv, 32 * warp, lane);
    __syncthreads();
    for (int J = 2; J >= 0; --J) {
        const int nI = 3 - J;
        for (int e = tid; e < nI * 256; e += NT) {
            const int b = e >> 8, r0 = ((e >> 5) & 7) * 4, c = e & 31, I = J + 1 + b;
            float y[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int K = J + 1; K <= I; ++K) {
#pragma unroll
                for (int p = 0; p < 32; p += 4) {
                    float col[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) col[q] = D[32 * K + p + q][32 * J + c];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 a = *reinterpret_cast<const float4*>(&D[32 * I + r0 + u][32 * K + p]);
                        y[u] = fmaf(a.x, col[0], fmaf(a.y, col[1], fmaf(a.z, col[2], fmaf(a.w, col[3], y[u]))));
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) Y[(b * 32 + r0 + u) * 32 + c] = y[u];
        }
        __syncthreads();
        for (int e = tid; e < nI * 256; e += NT) {
            const int b = e >> 8, r0 = ((e >> 5) & 7) * 4, c = e & 31, I = J + 1 + b;
            float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int p = 0; p < 32; p += 4) {
                float col[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) col[q] = D[32 * J + p + q][32 * J + c];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float4 a = *reinterpret_cast<const float4*>(&Y[(b * 32 + r0 + u) * 32 + p]);
                    z[u] = fmaf(a.x, col[0], fmaf(a.y, col[1], fmaf(a.z, col[2], fmaf(a.w, col[3], z[u]))));
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) D[32 * I + r0 + u][32 * J + c] = -z[u];
        }
        __syncthreads();
    }
}

// Shared-memory use of the factorisation between trailing updates (inside the
// operand ring): diagonal block, reciprocal diagonal, flag, inverse scratch.
constexpr int kDiagRinvOff = TB * DP * 4;
constexpr int kDiagFlagOff = kDiagRinvOff + TB * 4;
constexpr int kDiagYOff = kDiagFlagOff + 16;
constexpr int kDiagRedOff = kDiagYOff + 3 * 32 * 32 * 4;   // per-warp maxima
constexpr int kDiagBytes = kDiagRedOff + (NT / 32) * 4;

// Left-looking blocked Cholesky with 128-wide block columns, all O(k^3) work on the
// tensor cores from the scheme's 16-bit planes.  For block column J:
//   update   C = A[j0:, J] - L[j0:, :j0] L[J, :j0]^T   (tensor cores; the diagonal
//            block's rows stay FP32, the rows below go to the planes only)
//   diagonal L_JJ L_JJ^T = C_JJ in FP32 (blocked, shared memory), then L_JJ^-1
//   panel    L[below, J] = C[below, J] L_JJ^-T          (tensor cores, the inverse's
//            planes in the diagonal block's place, which no later update reads)
// The panel's epilogue writes the FP32 factor (kept in S.L, column-major, for the
// triangular solves) and its planes for the updates of later block columns.  S.L
// keeps L_JJ^-1 (zeros above its diagonal) in place of each diagonal block: the
// solves multiply by it instead of substituting.  False if a pivot is not positive
// or a bounded wait ran out.
// LAT (lattice data): entries of A below the diagonal blocks were not assembled; the
// update epilogue and the first block column take them from the covariance table by
// index offset (the same FP32 values the assembly would have stored).
// With fw (the right-hand side, k floats) the first forward solve w <- L^-1 w runs
// inside the factorisation: after the diagonal block, w_J <- L_JJ^-1 w_J (the panels
// of earlier block columns have already subtracted their part), and the panel's
// epilogue, which holds each row of L[below, J], subtracts L[r, J] w_J from w_r.  The
// factor is then not streamed for that solve.  fwj: 128 floats of shared memory
// outside the operand ring; lij (lattice data): 128 index pairs of shared memory, the
// block column's points for the update epilogue.
struct LatView {
    const float2* tab;   // covariance table (hi, lo) by index offset, rows of length W
    const int* ti;       // lattice indices of the training points
    const int* tj;
    int W;
    __device__ __forceinline__ float a(int ri, int rj, int c) const {
        return tab[abs(ri - ti[c]) * W + abs(rj - tj[c])].x;
    }
};

template <class Sch, bool LAT = false>
__device__ bool factor_tc(TcCtx& tc, const SlotM& S, int k, int64_t ld, unsigned long long* clk,
                          float* fw = nullptr, float* fwj = nullptr, LatView lv = LatView{}, int2* lij = nullptr) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    PhaseTimer tm(clk);
    // the operand ring was written through the generic proxy since the last update
    umma::fence_proxy_async();
    __syncthreads();
    float (*D)[DP] = reinterpret_cast<float (*)[DP]>(tc.stages);
    float* rinv = reinterpret_cast<float*>(tc.stages + kDiagRinvOff);
    int* flag = reinterpret_cast<int*>(tc.stages + kDiagFlagOff);
    float* Y = reinterpret_cast<float*>(tc.stages + kDiagYOff);
    float* L = S.L;
    const int nb = (k + TB - 1) / TB;
    for (int J = 0; J < nb; ++J) {
        const int j0 = J * TB, jb = min(TB, k - j0);
        const bool below = j0 + TB < k;   // rows below the diagonal block (then jb == TB)
        if (j0 > 0) {
            auto epi = [&](int row0, int quad, uint32_t taddr) {
                const int r = row0 + quad * 32 + (threadIdx.x & 31);
                const bool diag_rows = row0 < j0 + TB;
#pragma unroll 1
                for (int c0 = 0; c0 < TB; c0 += 32) {
                    float v[32];
                    umma::tmem_ld32(taddr + c0, v);
                    if (r < k) {
                        float* Lr = L + r + (int64_t)(j0 + c0) * ld;
                        if (diag_rows) {
                            // all 32 loads before the stores (the compiler cannot tell that the
                            // strided stores miss the later loads, and would otherwise wait
                            // for one memory round trip per column)
                            float cur[32];
#pragma unroll
                            for (int j = 0; j < 32; ++j) cur[j] = c0 + j < jb ? Lr[(int64_t)j * ld] : 0.0f;
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (c0 + j < jb) Lr[(int64_t)j * ld] = cur[j] - v[j];
                        } else {
                            if constexpr (LAT) {
                                // the columns' lattice indices from shared memory: one memory
                                // round trip (the table) per group instead of two
                                const int ri = lv.ti[r], rj = lv.tj[r];
                                float av[32];
#pragma unroll
                                for (int j = 0; j < 32; ++j) {
                                    const int2 c = lij[c0 + j];
                                    av[j] = lv.tab[abs(ri - c.x) * lv.W + abs(rj - c.y)].x;
                                }
#pragma unroll
                                for (int j = 0; j < 32; ++j) v[j] = av[j] - v[j];
                            } else {
#pragma unroll
                                for (int j = 0; j < 32; ++j) v[j] = Lr[(int64_t)j * ld] - v[j];
                            }
#pragma unroll
                            for (int g = 0; g < 4; ++g)
                                store_planes8<Sch>(tc, plane_off<Sch>(r, j0 + c0 + 8 * g, ld), v + 8 * g);
                        }
                    }
                }
            };
            if constexpr (LAT) {
                if (tid < TB) {
                    const int c = min(j0 + tid, k - 1);
                    lij[tid] = make_int2(lv.ti[c], lv.tj[c]);
                }
                __syncthreads();
            }
            const bool ok = tc.sh->dead == 0 &&
                            umma::block_column<true, kTcTilesPerPass, Sch>(tc.sh->pipe, tc.ph, tc.stages, tc.m0, tc.m1, tc.m2,
                                                     tc.row_base, j0, k - j0, j0, j0 * kw<Sch>(), epi,
                                                     (int)(ld * kw<Sch>() / 32));
            if (!ok) atomicExch(&tc.sh->dead, 1);
            __syncthreads();
            if (tc.sh->dead) return false;
            tm.lap(kPhUpdate);
        } else if (below) {
            // first block column: the assembled rows below the diagonal block into the planes
            for (int e = tid; e < (k - TB) * (TB / 8); e += NT) {
                const int r = TB + e % (k - TB), g = e / (k - TB);
                float x[8];
                if constexpr (LAT) {
                    const int ri = lv.ti[r], rj = lv.tj[r];
#pragma unroll
                    for (int q = 0; q < 8; ++q) x[q] = lv.a(ri, rj, g * 8 + q);
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) x[q] = L[r + (int64_t)(g * 8 + q) * ld];
                }
                store_planes8<Sch>(tc, plane_off<Sch>(r, g * 8, ld), x);
            }
            tm.lap(kPhDiagIO);
        }
        // diagonal block in shared memory: whole 128 x 128 block, four rows per float4,
        // 16 independent loads per thread.  In the last, partial block everything past jb
        // becomes identity as it is stored (one writer per element), so the factor and
        // its inverse are block diagonal with an identity pad: rows and columns past k
        // never mix in.
        {
            float4 v[TB * TB / 4 / NT];
#pragma unroll
            for (int i = 0; i < TB * TB / 4 / NT; ++i) {
                const int e = tid + i * NT, r4 = (e & (TB / 4 - 1)) * 4, c = e / (TB / 4);
                v[i] = *reinterpret_cast<const float4*>(L + (j0 + r4) + (int64_t)(j0 + c) * ld);
            }
#pragma unroll
            for (int i = 0; i < TB * TB / 4 / NT; ++i) {
                const int e = tid + i * NT, r4 = (e & (TB / 4 - 1)) * 4, c = e / (TB / 4);
                const float x[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = r4 + u;
                    D[r][c] = (r < jb && c < jb) ? x[u] : (r == c ? 1.0f : 0.0f);
                }
            }
        }
        if (tid == 0) *flag = 0;
        __syncthreads();
        tm.lap(kPhDiagIO);
        // blocked right-looking Cholesky, 32 columns per step: the 32 x 32 diagonal
        // sub-block by one warp in registers, the rows below it against that factor, then
        // the symmetric update of the trailing part (three barriers per step)
        for (int c0 = 0; c0 < TB; c0 += 32) {
            if (warp == 0 && !chol32_warp(D, rinv, c0, 32, lane) && lane == 0) *flag = 1;
            __syncthreads();
            const int t0 = c0 + 32;
            if (t0 < TB) {
                trsm32_rows(D, rinv, c0, t0, TB);
                __syncthreads();
                syrk32_trailing(D, c0, t0, TB);
                __syncthreads();
            }
        }
        if (*flag) return false;
        // L_JJ^-1 in place; the FP32 factor keeps the inverse in the diagonal block's
        // place (the triangular solves multiply by it), zeros above its diagonal
        trinv128(D, rinv, Y);
        if (fw) {
            // w_J <- L_JJ^-1 w_J from the inverse in shared memory (two threads per row,
            // 64 columns each, partial sums through the free Y scratch)
            if (tid < TB) fwj[tid] = tid < jb ? fw[j0 + tid] : 0.0f;
            __syncthreads();
            const int r = tid & (TB - 1), h = tid >> 7;
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll 8
            for (int c = 64 * h; c < 64 * h + 64; c += 2) {
                s0 = fmaf(c <= r ? D[r][c] : 0.0f, fwj[c], s0);
                s1 = fmaf(c + 1 <= r ? D[r][c + 1] : 0.0f, fwj[c + 1], s1);
            }
            Y[tid] = s0 + s1;
            __syncthreads();
            if (tid < TB) {
                const float v = Y[tid] + Y[tid + TB];
                fwj[tid] = tid < jb ? v : 0.0f;
                if (tid < jb) fw[j0 + tid] = v;
            }
        }
        tm.lap(kPhDiag);
#pragma unroll
        for (int i = 0; i < TB * TB / 4 / NT; ++i) {
            const int e = tid + i * NT, r4 = (e & (TB / 4 - 1)) * 4, c = e / (TB / 4);
            *reinterpret_cast<float4*>(L + (j0 + r4) + (int64_t)(j0 + c) * ld) =
                make_float4(c <= r4 ? D[r4][c] : 0.0f, c <= r4 + 1 ? D[r4 + 1][c] : 0.0f,
                            c <= r4 + 2 ? D[r4 + 2][c] : 0.0f, c <= r4 + 3 ? D[r4 + 3][c] : 0.0f);
        }
        if (!below) {   // last block column
            __syncthreads();
            tm.lap(kPhDiagIO);
            break;
        }
        // the inverse's planes in the diagonal block's place: the panel's B operand,
        // B[n][q] = 2^-e L_JJ^-1[n][q], with the power of two 2^e >= max |L_JJ^-1| keeping
        // the terms in range of a 16-bit format (the panel's epilogue scales back)
        float amax = 0.0f;
        for (int e = tid; e < TB * TB; e += NT) {
            const int r = e / TB, c = e % TB;
            if (c <= r) amax = fmaxf(amax, fabsf(D[r][c]));
        }
        amax = warp_max(amax);
        float* red = reinterpret_cast<float*>(tc.stages + kDiagRedOff);
        if (lane == 0) red[warp] = amax;
        __syncthreads();
        amax = red[0];
#pragma unroll
        for (int w = 1; w < NT / 32; ++w) amax = fmaxf(amax, red[w]);
        const int ex = amax > 1.0f ? ilogbf(amax) + 1 : 0;   // amax < 2^ex
        const float down = scalbnf(1.0f, -ex), up = scalbnf(1.0f, ex);
        for (int e = tid; e < TB * (TB / 8); e += NT) {
            const int r = e / (TB / 8), g = e % (TB / 8);
            float x[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = g * 8 + q;
                x[q] = c <= r ? D[r][c] * down : 0.0f;
            }
            store_planes8<Sch>(tc, plane_off<Sch>(j0 + r, j0 + g * 8, ld), x);
        }
        // the planes are read next by TMA (async proxy), which also overwrites the
        // diagonal-block buffer
        asm volatile("fence.proxy.async.global;" ::: "memory");
        umma::fence_proxy_async();
        __syncthreads();
        tm.lap(kPhDiagIO);
        {
            auto epi = [&](int row0, int quad, uint32_t taddr) {
                const int r = row0 + quad * 32 + (threadIdx.x & 31);
                float acc = 0.0f;   // L[r, J] w_J of the fused forward solve
#pragma unroll 1
                for (int c0 = 0; c0 < TB; c0 += 32) {
                    float v[32];
                    umma::tmem_ld32(taddr + c0, v);
                    if (r < k) {
                        float* Lr = L + r + (int64_t)(j0 + c0) * ld;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            v[j] *= up;
                            __stcs(Lr + (int64_t)j * ld, v[j]);   // read next by the solves: streaming
                        }
                        if (fw) {
#pragma unroll
                            for (int j = 0; j < 32; ++j) acc = fmaf(v[j], fwj[c0 + j], acc);
                        }
#pragma unroll
                        for (int g = 0; g < 4; ++g)
                            store_planes8<Sch>(tc, plane_off<Sch>(r, j0 + c0 + 8 * g, ld), v + 8 * g);
                    }
                }
                if (fw && r < k) fw[r] -= acc;
            };
            const bool ok = tc.sh->dead == 0 &&
                            umma::block_column<true, kTcTilesPerPass, Sch>(tc.sh->pipe, tc.ph, tc.stages, tc.m0, tc.m1, tc.m2,
                                                     tc.row_base, j0 + TB, k - j0 - TB, j0, TB * kw<Sch>(), epi,
                                                     (int)(ld * kw<Sch>() / 32), j0 * kw<Sch>() / 32);
            if (!ok) atomicExch(&tc.sh->dead, 1);
            // the panel's planes are read by the next update's TMA loads
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncthreads();
            if (tc.sh->dead) return false;
            tm.lap(kPhPanel);
        }
    }
    return true;
}

// ---------------------------------------------------------------- FP32 triangular solves

// The 64 x 64 block of L at (j0, j0) into sm.L: four float4 loads per thread, all in
// flight at once (rows beyond k and the upper part carry stale values that are never used).
__device__ __forceinline__ void load_diag64(SmemM& sm, const float* L, int64_t ld, int j0) {
    const int tid = threadIdx.x;
    float4 v[NB * NB / 4 / NT];
#pragma unroll
    for (int i = 0; i < NB * NB / 4 / NT; ++i) {
        const int e = tid + i * NT, r4 = (e & (NB / 4 - 1)) * 4, c = e / (NB / 4);
        v[i] = *reinterpret_cast<const float4*>(L + (j0 + r4) + (int64_t)(j0 + c) * ld);
    }
#pragma unroll
    for (int i = 0; i < NB * NB / 4 / NT; ++i) {
        const int e = tid + i * NT, r4 = (e & (NB / 4 - 1)) * 4, c = e / (NB / 4);
        sm.L[r4][c] = v[i].x;
        sm.L[r4 + 1][c] = v[i].y;
        sm.L[r4 + 2][c] = v[i].z;
        sm.L[r4 + 3][c] = v[i].w;
    }
}

// w <- L^-1 w (column-oriented: diagonal block by one warp, rows below by all threads,
// one row per thread with 64 independent loads in flight)
__device__ void forward32(SmemM& sm, const float* L, int64_t ld, float* w, int k) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int nb = (k + NB - 1) / NB;
    for (int J = 0; J < nb; ++J) {
        const int j0 = J * NB, jb = min(NB, k - j0);
        load_diag64(sm, L, ld, j0);
        __syncthreads();
        if (tid < 32) {
            float v0 = lane < jb ? w[j0 + lane] : 0.0f;
            float v1 = lane + 32 < jb ? w[j0 + lane + 32] : 0.0f;
            for (int c = 0; c < jb; ++c) {
                const float vc = __shfl_sync(0xffffffffu, c < 32 ? v0 : v1, c & 31);
                const float wc = vc / sm.L[c][c];
                if (lane == (c & 31)) { if (c < 32) v0 = wc; else v1 = wc; }
                if (lane > c && lane < jb) v0 = fmaf(-sm.L[lane][c], wc, v0);
                if (lane + 32 > c && lane + 32 < jb) v1 = fmaf(-sm.L[lane + 32][c], wc, v1);
            }
            if (lane < jb) { w[j0 + lane] = v0; sm.wj[lane] = v0; }
            if (lane + 32 < jb) { w[j0 + lane + 32] = v1; sm.wj[lane + 32] = v1; }
        }
        __syncthreads();
        if (jb == NB) {
            for (int r = j0 + NB + tid; r < k; r += NT) {
                const float* Lr = L + r + (int64_t)j0 * ld;
                float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
                for (int c = 0; c < NB; c += 4) {
                    s0 = fmaf(Lr[(int64_t)c * ld], sm.wj[c], s0);
                    s1 = fmaf(Lr[(int64_t)(c + 1) * ld], sm.wj[c + 1], s1);
                    s2 = fmaf(Lr[(int64_t)(c + 2) * ld], sm.wj[c + 2], s2);
                    s3 = fmaf(Lr[(int64_t)(c + 3) * ld], sm.wj[c + 3], s3);
                }
                w[r] -= (s0 + s1) + (s2 + s3);
            }
        }
        __syncthreads();
    }
}

// w <- L^-T w.  Dot products of the block's columns with the finished part of w:
// warp wp takes columns 8wp .. 8wp+7, its lanes walk the rows (coalesced), eight
// accumulators per thread, then a warp reduction.
__device__ void backward32(SmemM& sm, const float* L, int64_t ld, float* w, int k) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nb = (k + NB - 1) / NB;
    for (int J = nb - 1; J >= 0; --J) {
        const int j0 = J * NB, jb = min(NB, k - j0);
        {
            float s[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) s[q] = 0.0f;
            const int c0 = warp * 8;
            if (jb == NB) {
                int p = j0 + jb + lane;
                for (; p + 96 < k; p += 128) {   // four rows per lane in flight
                    float wv[4], lv[4][8];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        wv[u] = w[p + 32 * u];
#pragma unroll
                        for (int q = 0; q < 8; ++q) lv[u][q] = L[p + 32 * u + (int64_t)(j0 + c0 + q) * ld];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int q = 0; q < 8; ++q) s[q] = fmaf(lv[u][q], wv[u], s[q]);
                }
                for (; p < k; p += 32) {
                    const float wp = w[p];
#pragma unroll
                    for (int q = 0; q < 8; ++q) s[q] = fmaf(L[p + (int64_t)(j0 + c0 + q) * ld], wp, s[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float v = s[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && c0 + q < jb) sm.wj[c0 + q] = w[j0 + c0 + q] - v;
            }
        }
        load_diag64(sm, L, ld, j0);
        __syncthreads();
        if (tid < 32) {
            float v0 = lane < jb ? sm.wj[lane] : 0.0f;
            float v1 = lane + 32 < jb ? sm.wj[lane + 32] : 0.0f;
            for (int c = jb - 1; c >= 0; --c) {
                const float vc = __shfl_sync(0xffffffffu, c < 32 ? v0 : v1, c & 31);
                const float xc = vc / sm.L[c][c];
                if (lane == (c & 31)) { if (c < 32) v0 = xc; else v1 = xc; }
                if (lane < c) v0 = fmaf(-sm.L[c][lane], xc, v0);
                if (lane + 32 < c) v1 = fmaf(-sm.L[c][lane + 32], xc, v1);
            }
            if (lane < jb) w[j0 + lane] = v0;
            if (lane + 32 < jb) w[j0 + lane + 32] = v1;
        }
        __syncthreads();
    }
}

// Triangular solves of the tensor-core kernel, whose FP32 factor holds the inverse
// of every 128 x 128 diagonal block (see factor_tc), with zeros above its diagonal and
// an identity pad past k in the last block.  Both solves stream the factor in chunks
// of 128 rows x 128 columns: warp wp takes columns 16 wp .. 16 wp + 15, lane l rows
// 4 l .. 4 l + 3 of the chunk, one float4 per column (the factor is column-major), all
// sixteen 16-byte loads in flight.  A float4 that starts below k stays inside its
// column (ld is a multiple of 128); rows past k are never written back.  The factor
// is read with streaming (evict-first) loads: one pass per solve, nothing to keep in L2.

// L2 prefetch of 128 rows (512 bytes) of a factor column from p (16-byte aligned: the row
// is a multiple of 128, as is ld), a hint that keeps the next chunks' HBM reads in flight
// without registers; callers stay below k, hence inside the column
__device__ __forceinline__ void l2_prefetch_rows(const float* p) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], 512;" ::"l"(p) : "memory");
}

// Sum of 16 values over the 32 lanes of a warp (transpose-reduce: 16 shuffles instead
// of 80).  Returns in every lane the total of value (lane >> 1) & 15.
__device__ __forceinline__ float warp_sum16(float (&s)[16], int lane) {
    float t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool hi = lane & 16;
        const float keep = hi ? s[i + 8] : s[i], give = hi ? s[i] : s[i + 8];
        t[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 8;
        const float keep = hi ? t[i + 4] : t[i], give = hi ? t[i] : t[i + 4];
        t[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 4;
        const float keep = hi ? t[i + 2] : t[i], give = hi ? t[i] : t[i + 2];
        t[i] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    }
    {
        const bool hi = lane & 2;
        const float keep = hi ? t[1] : t[0], give = hi ? t[0] : t[1];
        t[0] = keep + __shfl_xor_sync(0xffffffffu, give, 2);
    }
    return t[0] + __shfl_xor_sync(0xffffffffu, t[0], 1);
}

// Row-chunk product of the forward solve: acc (rows 4 lane .. 4 lane + 3 of the chunk at
// row r0) = L[r0 .., j0 + c0 .. j0 + c0 + 15] wc
__device__ __forceinline__ float4 chunk_rows(const float* L, int64_t ld, int r0, int jc, const float (&wc)[16]) {
    float4 l4[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) l4[q] = __ldcs(reinterpret_cast<const float4*>(L + r0 + (int64_t)(jc + q) * ld));
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        acc.x = fmaf(l4[q].x, wc[q], acc.x);
        acc.y = fmaf(l4[q].y, wc[q], acc.y);
        acc.z = fmaf(l4[q].z, wc[q], acc.z);
        acc.w = fmaf(l4[q].w, wc[q], acc.w);
    }
    return acc;
}

// w <- L^-1 w, block by block: w_J <- L_JJ^-1 w_J (one chunk: the inverse block), then
// the rows below take w[r] -= L[r, J] w_J.  The warps' partial sums meet in shared
// memory (two buffers, one barrier per chunk).
__device__ void forward_inv(SmemM& sm, const float* L, int64_t ld, float* w, int k) {
    constexpr int TBs = 2 * NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, c0 = warp * 16;
    float* red = &sm.ph[0][0];          // 2 x 8 x 128 floats (ph and pl)
    const int nb = (k + TBs - 1) / TBs;
    int buf = 0;
    for (int J = 0; J < nb; ++J) {
        const int j0 = J * TBs, jb = min(TBs, k - j0);
        // this block's first two chunks below and the next block's inverse, into L2
        if (tid < TBs && j0 + TBs < k) {
            const float* col = L + (int64_t)(j0 + tid) * ld;
            l2_prefetch_rows(col + j0 + TBs);
            if (j0 + 2 * TBs < k) l2_prefetch_rows(col + j0 + 2 * TBs);
            l2_prefetch_rows(L + (j0 + TBs) + (int64_t)(j0 + TBs + tid) * ld);
        }
        if (tid < TBs) sm.wj[tid] = tid < jb ? w[j0 + tid] : 0.0f;
        __syncthreads();
        float wc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) wc[q] = sm.wj[c0 + q];
        *reinterpret_cast<float4*>(red + buf * (8 * TBs) + warp * TBs + 4 * lane) =
            chunk_rows(L, ld, j0 + 4 * lane, j0 + c0, wc);
        __syncthreads();
        if (tid < TBs) {
            const float* rb = red + buf * (8 * TBs) + tid;
            float v = 0.0f;
#pragma unroll
            for (int g = 0; g < 8; ++g) v += rb[g * TBs];
            v = tid < jb ? v : 0.0f;
            sm.wj[tid] = v;
            if (tid < jb) w[j0 + tid] = v;
        }
        buf ^= 1;
        __syncthreads();
        if (jb == TBs && j0 + TBs < k) {
#pragma unroll
            for (int q = 0; q < 16; ++q) wc[q] = sm.wj[c0 + q];
            for (int rc = j0 + TBs; rc < k; rc += TBs, buf ^= 1) {
                if (tid < TBs && rc + 2 * TBs < k) l2_prefetch_rows(L + (rc + 2 * TBs) + (int64_t)(j0 + tid) * ld);
                const int r = rc + 4 * lane;
                const float4 acc = r < k ? chunk_rows(L, ld, r, j0 + c0, wc) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                *reinterpret_cast<float4*>(red + buf * (8 * TBs) + warp * TBs + 4 * lane) = acc;
                __syncthreads();
                if (tid < TBs && rc + tid < k) {
                    const float* rb = red + buf * (8 * TBs) + tid;
                    float v = 0.0f;
#pragma unroll
                    for (int g = 0; g < 8; ++g) v += rb[g * TBs];
                    w[rc + tid] -= v;
                }
            }
            __syncthreads();
        }
    }
}

// w <- L^-T w, blocks from the last: v = w_J - L[below, J]^T w[below] (column dot
// products: the lanes walk the rows, a warp reduction per column), then
// w_J <- L_JJ^-T v (one chunk: the inverse block's columns against v).
__device__ void backward_inv(SmemM& sm, const float* L, int64_t ld, float* w, int k) {
    constexpr int TBs = 2 * NB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, c0 = warp * 16;
    const int nb = (k + TBs - 1) / TBs;
    const int cq = c0 + ((lane >> 1) & 15);   // the column whose total this lane ends with
    for (int J = nb - 1; J >= 0; --J) {
        const int j0 = J * TBs, jb = min(TBs, k - j0);
        float s[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) s[q] = 0.0f;
        // the next block's inverse into L2 (read after this block's rows below)
        if (J > 0 && tid < TBs) l2_prefetch_rows(L + (j0 - TBs) + (int64_t)(j0 - TBs + tid) * ld);
        if (jb == TBs) {
            // whole float4s below k; the last rows (fewer than four) one by one.  Lanes 0-15
            // keep the warp's columns two chunks ahead in L2.
            const int rb = j0 + TBs, nq = (k - rb) >> 2;
            const float* pcol = L + (int64_t)(j0 + c0 + (lane & 15)) * ld;
            if (lane < 16 && rb < k) {
                l2_prefetch_rows(pcol + rb);
                if (rb + TBs < k) l2_prefetch_rows(pcol + rb + TBs);
            }
            for (int ch = lane; ch < nq; ch += 32) {
                const int p = rb + 4 * ch;
                const int pf = rb + 4 * (ch - lane) + 2 * TBs;   // the warp's chunk two ahead
                if (lane < 16 && pf < k) l2_prefetch_rows(pcol + pf);
                const float4 wv = *reinterpret_cast<const float4*>(w + p);
                float4 l4[16];
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    l4[q] = __ldcs(reinterpret_cast<const float4*>(L + p + (int64_t)(j0 + c0 + q) * ld));
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    s[q] = fmaf(l4[q].x, wv.x, fmaf(l4[q].y, wv.y, fmaf(l4[q].z, wv.z, fmaf(l4[q].w, wv.w, s[q]))));
            }
            for (int p = rb + 4 * nq + lane; p < k; p += 32) {
                const float wp = w[p];
#pragma unroll
                for (int q = 0; q < 16; ++q) s[q] = fmaf(L[p + (int64_t)(j0 + c0 + q) * ld], wp, s[q]);
            }
        }
        {
            const float v = warp_sum16(s, lane);
            if ((lane & 1) == 0) sm.wj[cq] = cq < jb ? w[j0 + cq] - v : 0.0f;
        }
        __syncthreads();
        {
            const float4 wv = *reinterpret_cast<const float4*>(sm.wj + 4 * lane);
            float4 l4[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                l4[q] = __ldcs(reinterpret_cast<const float4*>(L + (j0 + 4 * lane) + (int64_t)(j0 + c0 + q) * ld));
#pragma unroll
            for (int q = 0; q < 16; ++q)
                s[q] = fmaf(l4[q].x, wv.x, fmaf(l4[q].y, wv.y, fmaf(l4[q].z, wv.z, l4[q].w * wv.w)));
            const float v = warp_sum16(s, lane);
            if ((lane & 1) == 0 && cq < jb) w[j0 + cq] = v;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- double-float kernel entries

struct Pt {
    float xh, xl, yh, yl;
};

// t = ||p - q|| for coordinates already in units of rho (so t = distance / rho), in
// double-float; the high parts of both points lie on a common power-of-two grid
// chosen so that their differences are exact
__device__ __forceinline__ df t_grid(const Pt& p, const Pt& q) {
    const df dx = dfm::fast_two_sum(p.xh - q.xh, p.xl - q.xl);
    const df dy = dfm::fast_two_sum(p.yh - q.yh, p.yl - q.yl);
    const df sx = dfm::two_prod(dx.h, dx.h), sy = dfm::two_prod(dy.h, dy.h);
    df d2 = dfm::two_sum(sx.h, sy.h);
    d2.l += sx.l + sy.l + 2.0f * (dx.h * dx.l + dy.h * dy.l);
    d2 = dfm::fast_two_sum(d2.h, d2.l);
    return dfm::sqrt_df(d2);
}

// same for arbitrary double-float points (prediction locations)
__device__ __forceinline__ df t_any(const Pt& p, const Pt& q) {
    df dx = dfm::two_sum(p.xh, -q.xh);
    dx = dfm::fast_two_sum(dx.h, dx.l + (p.xl - q.xl));
    df dy = dfm::two_sum(p.yh, -q.yh);
    dy = dfm::fast_two_sum(dy.h, dy.l + (p.yl - q.yl));
    const df sx = dfm::two_prod(dx.h, dx.h), sy = dfm::two_prod(dy.h, dy.h);
    df d2 = dfm::two_sum(sx.h, sy.h);
    d2.l += sx.l + sy.l + 2.0f * (dx.h * dx.l + dy.h * dy.l);
    d2 = dfm::fast_two_sum(d2.h, d2.l);
    return dfm::sqrt_df(d2);
}

__device__ __forceinline__ df exp_neg_sm(const float* tbl, df t) {
    return dfm::exp_neg(t, tbl, c_exp.inv_c, c_exp.c1, c_exp.c2, c_exp.c3);
}

// Lattice data: a point's lattice indices travel in the high-part slots of Pt (xh, yh)
// as integer bits, and the covariance of two points is the task's table entry at their
// index offsets (|di|, |dj|), a (hi, lo) pair of floats.
__device__ __forceinline__ df lat_cov(const float2* tab, int W, const Pt& p, const Pt& q) {
    const int di = abs(__float_as_int(p.xh) - __float_as_int(q.xh));
    const int dj = abs(__float_as_int(p.yh) - __float_as_int(q.yh));
    const float2 e = tab[di * W + dj];   // the table may sit in shared memory
    return df{e.x, e.y};
}

// r = y - A x with A = Sigma + lambda I: double-float entries, one pass over the
// lower triangle in 64 x 64 tiles, each entry feeding its row and its column.
template <bool LAT = false>
__device__ void residual_df(SmemM& sm, const float* tbl, const SlotM& S, int k, double lam, int W = 0) {
    const int tid = threadIdx.x;
    const int rg = tid >> 4, cg = tid & 15;   // 16 x 16 threads, 4 x 4 entries each
    for (int a = tid; a < k; a += NT) { S.ah[a] = 0.0f; S.al[a] = 0.0f; }
    __syncthreads();
    const int nb = (k + NB - 1) / NB;
    for (int I = 0; I < nb; ++I) {
        Pt pa[4];
        df xa[4];
        dfm::acc racc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int a = I * NB + rg * 4 + u;
            const bool ok = a < k;
            pa[u] = ok ? Pt{S.xh[a], LAT ? 0.0f : S.xl[a], S.yh[a], LAT ? 0.0f : S.yl[a]} : Pt{0, 0, 0, 0};
            xa[u] = ok ? df{S.qh[a], S.ql[a]} : df{0, 0};
        }
        for (int J = 0; J <= I; ++J) {
            Pt pb[4];
            df xb[4];
            dfm::acc cacc[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int b = J * NB + cg * 4 + v;
                const bool ok = b < k;
                pb[v] = ok ? Pt{S.xh[b], LAT ? 0.0f : S.xl[b], S.yh[b], LAT ? 0.0f : S.yl[b]} : Pt{0, 0, 0, 0};
                xb[v] = ok ? df{S.qh[b], S.ql[b]} : df{0, 0};
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int a = I * NB + rg * 4 + u, b = J * NB + cg * 4 + v;
                    if (a < k && b < k && (I != J || a > b)) {
                        df e;
                        if constexpr (LAT) e = lat_cov(S.tab, W, pa[u], pb[v]);
                        else e = exp_neg_sm(tbl, t_grid(pa[u], pb[v]));
                        racc[u].add_prod(e, xb[v]);
                        cacc[v].add_prod(e, xa[u]);
                    }
                }
            // column sums of this tile -> columns of block J
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const df c = cacc[v].value();
                sm.ph[rg][cg * 4 + v] = c.h;
                sm.pl[rg][cg * 4 + v] = c.l;
            }
            __syncthreads();
            if (tid < NB) {
                const int b = J * NB + tid;
                if (b < k) {
                    dfm::acc s;
                    s.add_df(df{S.ah[b], S.al[b]});
                    for (int g = 0; g < 16; ++g) s.add_df(df{sm.ph[g][tid], sm.pl[g][tid]});
                    const df v = s.value();
                    S.ah[b] = v.h;
                    S.al[b] = v.l;
                }
            }
            __syncthreads();
        }
        // row sums of block row I
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const df r = racc[u].value();
            sm.ph[cg][rg * 4 + u] = r.h;
            sm.pl[cg][rg * 4 + u] = r.l;
        }
        __syncthreads();
        if (tid < NB) {
            const int a = I * NB + tid;
            if (a < k) {
                dfm::acc s;
                s.add_df(df{S.ah[a], S.al[a]});
                for (int g = 0; g < 16; ++g) s.add_df(df{sm.ph[g][tid], sm.pl[g][tid]});
                const df v = s.value();
                S.ah[a] = v.h;
                S.al[a] = v.l;
            }
        }
        __syncthreads();
    }
    // diagonal (1 + lambda) x and the residual, O(k) FP64 operations
    for (int a = tid; a < k; a += NT)
        S.rr[a] = S.yv[a] - ((double)S.ah[a] + (double)S.al[a] + (1.0 + lam) * S.xs[a]);
    __syncthreads();
}

// Lattice data: r = y - A x over the whole matrix, each row owned by one warp.  A warp
// takes RB rows at a time; its lanes walk the columns (the column's lattice indices and
// solution value loaded once for all RB rows), each entry a table read by index offset
// and one double-float product added to the row's accumulator; a butterfly of
// double-float additions then sums the lanes.  Every entry is read twice (A_ab and
// A_ba) instead of feeding a row and a column sum, which costs one table read more per
// entry but no block-wide reduction or barrier per tile.  The diagonal comes from the
// table's (0, 0) entry, exactly 1, so the sum holds Sigma x and r = y - (sum + lambda x)
// in FP64.
template <int RB>
__device__ void residual_lat(const SlotM& S, int k, double lam, int W) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int* ti = reinterpret_cast<const int*>(S.xh);
    const int* tj = reinterpret_cast<const int*>(S.yh);
    const float2* __restrict__ tab = S.tab;
    for (int a0 = warp * RB; a0 < k; a0 += (NT / 32) * RB) {
        int ia[RB], ja[RB];
        dfm::acc racc[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            const int a = min(a0 + u, k - 1);
            ia[u] = ti[a];
            ja[u] = tj[a];
        }
        for (int b = lane; b < k; b += 32) {
            const int ib = ti[b], jb = tj[b];
            const df xb{S.qh[b], S.ql[b]};
            float2 e[RB];
#pragma unroll
            for (int u = 0; u < RB; ++u) e[u] = tab[abs(ia[u] - ib) * W + abs(ja[u] - jb)];
#pragma unroll
            for (int u = 0; u < RB; ++u) racc[u].add_prod(df{e[u].x, e[u].y}, xb);
        }
        double mine = 0.0;
#pragma unroll
        for (int u = 0; u < RB; ++u) {
            df v = racc[u].value();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const df w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
                v = dfm::add(v, w);
            }
            if (lane == u) mine = (double)v.h + (double)v.l;
        }
        const int a = a0 + lane;
        if (lane < RB && a < k) S.rr[a] = S.yv[a] - (mine + lam * S.xs[a]);
    }
    __syncthreads();
}

// Predictions (Eq. 3) of the task's m points in double-float from the solution in
// (R.qh, R.ql), two points per warp, lanes over the training points; each written to
// yhat (row yrow) when a.yhat is set, its squared error (Eq. 4) to R.ep when a.Pv is.
// With dc (a correction of the solution, FP32, k entries) each point also gets
// u_j = sum_a Sigma_ja dc_a in plain FP32 -- the change dc makes to the prediction, for
// the refinement's stopping rule -- and the block-wide statistics are returned:
// sum (yhat - y)^2, sum yhat^2, sum u^2 and max |u|.  Block-synchronous.
struct PredStats {
    double sse, ysq, usq;
    float umax;
};

template <bool LAT>
__device__ PredStats predict_points(SmemM& sm, const SmemKeep& keep, const TaskArgs& a, const SlotM& R, int k,
                                    int m, int64_t p0, double ox, double oy, double sc, int W, int64_t yrow,
                                    const float* dc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double ysq = 0.0, usq = 0.0;
    float umax = 0.0f;
    for (int j0 = 2 * warp; j0 < m; j0 += 2 * (NT / 32)) {   // two prediction points per warp
        const int j1 = min(j0 + 1, m - 1);
        Pt P0, P1;
        if constexpr (LAT) {
            P0 = Pt{__int_as_float(a.PLX[p0 + j0]), 0.0f, __int_as_float(a.PLY[p0 + j0]), 0.0f};
            P1 = Pt{__int_as_float(a.PLX[p0 + j1]), 0.0f, __int_as_float(a.PLY[p0 + j1]), 0.0f};
        } else {
            const df px0 = dfm::from_double((a.Px[p0 + j0] - ox) * sc), py0 = dfm::from_double((a.Py[p0 + j0] - oy) * sc);
            const df px1 = dfm::from_double((a.Px[p0 + j1] - ox) * sc), py1 = dfm::from_double((a.Py[p0 + j1] - oy) * sc);
            P0 = Pt{px0.h, px0.l, py0.h, py0.l};
            P1 = Pt{px1.h, px1.l, py1.h, py1.l};
        }
        dfm::acc s0, s1;
        float u0 = 0.0f, u1 = 0.0f;
        for (int q = lane; q < k; q += 32) {
            const Pt Q{R.xh[q], LAT ? 0.0f : R.xl[q], R.yh[q], LAT ? 0.0f : R.yl[q]};
            const df xq{R.qh[q], R.ql[q]};
            df e0, e1;
            if constexpr (LAT) {
                e0 = lat_cov(R.tab, W, P0, Q);
                e1 = lat_cov(R.tab, W, P1, Q);
            } else {
                e0 = exp_neg_sm(keep.tbl, t_any(P0, Q));
                e1 = exp_neg_sm(keep.tbl, t_any(P1, Q));
            }
            s0.add_prod(e0, xq);
            s1.add_prod(e1, xq);
            if (dc) {
                const float d = dc[q];
                u0 = fmaf(e0.h, d, u0);
                u1 = fmaf(e1.h, d, u1);
            }
        }
        const double v0 = warp_sum_d((double)s0.h + (double)s0.l);
        const double v1 = warp_sum_d((double)s1.h + (double)s1.l);
        if (dc) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                u0 += __shfl_xor_sync(0xffffffffu, u0, o);
                u1 += __shfl_xor_sync(0xffffffffu, u1, o);
            }
        }
        if (lane < 2 && (lane == 0 || j1 != j0)) {
            const int j = lane == 0 ? j0 : j1;
            const double v = lane == 0 ? v0 : v1;
            const float u = lane == 0 ? u0 : u1;
            if (a.yhat) a.yhat[yrow * a.yhat_stride + p0 + j] = v;
            if (a.Pv) {
                const double e = v - a.Pv[p0 + j];
                R.ep[j] = e * e;
            }
            ysq += v * v;
            usq += (double)u * (double)u;
            umax = fmaxf(umax, fabsf(u));
        }
    }
    __syncthreads();
    PredStats st{0.0, 0.0, 0.0, 0.0f};
    double sse = 0.0;
    if (a.Pv)
        for (int j = tid; j < m; j += NT) sse += R.ep[j];
    sse = warp_sum_d(sse);
    if (dc) {
        ysq = warp_sum_d(ysq);
        usq = warp_sum_d(usq);
        umax = warp_max(umax);
    }
    if (lane == 0) {
        sm.dred[warp] = sse;
        sm.dred2[warp] = ysq;
        sm.fred[warp] = umax;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        st.sse += sm.dred[w];
        st.ysq += sm.dred2[w];
        st.umax = fmaxf(st.umax, sm.fred[w]);
    }
    __syncthreads();
    if (dc) {
        if (lane == 0) sm.dred[warp] = usq;
        __syncthreads();
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) st.usq += sm.dred[w];
        __syncthreads();
    }
    return st;
}

// ---------------------------------------------------------------- one task

template <bool TC, class Sch = umma::SplitBF16x3, bool EXT = false, bool LAT = false>
__device__ void run_task(SmemM& sm, SmemKeep& keep, SmemSimt* simt, TcCtx* tc, const TaskArgs& a, int t, int i,
                         int b) {
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
        return;
    }
    const double lam = tau2 / s2;
    const int64_t t0 = a.T_off[i];
    const int k = (int)(a.T_off[i + 1] - t0);
    const int64_t ld = a.ld;
    const SlotM S = slot_of(a);
    // predictions from kriging weights computed earlier (alpha_in): gather the training
    // points, skip the matrix, its factorisation and the refinement
    const bool pred_only = a.alpha_in != nullptr;
    PhaseTimer tm(a.phase_cycles);
    const long long t_task = a.phase_cycles ? now_cycles() : 0;
    // coordinates become offsets from the subset's first training point in units of
    // rho (so covariance arguments are plain distances); their high parts lie on a
    // power-of-two grid fine enough that differences of high parts are exact floats
    const double sc = 1.0 / rho;
    const double ox = k > 0 ? a.X[a.T_idx[t0]] : 0.0, oy = k > 0 ? a.Y[a.T_idx[t0]] : 0.0;
    int W = 0, H = 0;       // lattice data: row length and rows of the covariance table
    bool lat_ok = true;
    if constexpr (LAT) {
        // lattice indices of the training points, carried as integer bits in the
        // high-part coordinate slots, and the index extents over the training and the
        // prediction points
        int e4[4] = {INT_MAX, INT_MIN, INT_MAX, INT_MIN};
        for (int q = tid; q < k; q += NT) {
            const int g = a.T_idx[t0 + q];
            const int ii = a.LX[g], jj = a.LY[g];
            S.xh[q] = __int_as_float(ii);
            S.yh[q] = __int_as_float(jj);
            S.yv[q] = a.Vals[g];
            S.xs[q] = 0.0;
            S.rr[q] = a.Vals[g];
            e4[0] = min(e4[0], ii); e4[1] = max(e4[1], ii); e4[2] = min(e4[2], jj); e4[3] = max(e4[3], jj);
        }
        for (int j = tid; j < m; j += NT) {
            const int ii = a.PLX[p0 + j], jj = a.PLY[p0 + j];
            e4[0] = min(e4[0], ii); e4[1] = max(e4[1], ii); e4[2] = min(e4[2], jj); e4[3] = max(e4[3], jj);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            e4[0] = min(e4[0], __shfl_xor_sync(0xffffffffu, e4[0], o));
            e4[1] = max(e4[1], __shfl_xor_sync(0xffffffffu, e4[1], o));
            e4[2] = min(e4[2], __shfl_xor_sync(0xffffffffu, e4[2], o));
            e4[3] = max(e4[3], __shfl_xor_sync(0xffffffffu, e4[3], o));
        }
        if (lane == 0)
            for (int u = 0; u < 4; ++u) sm.ired[u][warp] = e4[u];
        __syncthreads();
        for (int w = 0; w < NT / 32; ++w) {
            e4[0] = min(e4[0], sm.ired[0][w]); e4[1] = max(e4[1], sm.ired[1][w]);
            e4[2] = min(e4[2], sm.ired[2][w]); e4[3] = max(e4[3], sm.ired[3][w]);
        }
        H = e4[1] >= e4[0] ? e4[1] - e4[0] + 1 : 1;
        W = e4[3] >= e4[2] ? e4[3] - e4[2] + 1 : 1;
        lat_ok = (int64_t)H * W <= a.lat_cap;
        // the task's covariances by index offset, in FP64 (a few thousand entries)
        if (lat_ok)
            for (int e = tid; e < H * W; e += NT) {
                const double dx = (double)(e / W) * a.lat_hx, dy = (double)(e % W) * a.lat_hy;
                const double v = exp(-sqrt(dx * dx + dy * dy) / rho);
                const float hi = (float)v;
                S.tab[e] = make_float2(hi, (float)(v - (double)hi));
            }
        __syncthreads();
        // FP32 lower triangle of Sigma + lambda I from the table's high parts (indices
        // staged in shared memory: the operand ring is idle before the factorisation);
        // the tensor-core factorisation reads the entries below its 128 x 128 diagonal
        // blocks from the table itself, so only those blocks are stored
        const int* ti = reinterpret_cast<const int*>(S.xh);
        const int* tj = reinterpret_cast<const int*>(S.yh);
        if constexpr (TC) {
            if ((size_t)2 * ld * sizeof(int) <= (size_t)tc_ring_bytes<Sch>(a.tc_stages)) {
                int* f = reinterpret_cast<int*>(tc->stages);
                for (int q = tid; q < k; q += NT) {
                    f[q] = __float_as_int(S.xh[q]);
                    f[ld + q] = __float_as_int(S.yh[q]);
                }
                ti = f;
                tj = f + ld;
                __syncthreads();
            }
        }
        const float lam32 = (float)lam;
        const int nb = (k + NB - 1) / NB;
        const float2* __restrict__ tab = S.tab;
        constexpr int CPT = NB / (NT / NB);     // columns per thread in a 64 x 64 tile
        if (lat_ok && !pred_only)
            for (int bj = 0; bj < nb; ++bj)
                for (int bi = bj; bi < (TC ? min(nb, (bj & ~1) + 2) : nb); ++bi) {
                    const int r = bi * NB + (tid & (NB - 1));
                    if (r >= k) continue;
                    const int ri = ti[r], rj = tj[r];
                    // all of the row's lookups first (independent loads in flight), then the stores
                    float v[CPT];
#pragma unroll
                    for (int u = 0; u < CPT; ++u) {
                        const int c = bj * NB + (tid >> 6) + u * (NT / NB);
                        v[u] = c < r ? tab[abs(ri - ti[c]) * W + abs(rj - tj[c])].x : 1.0f + lam32;
                    }
#pragma unroll
                    for (int u = 0; u < CPT; ++u) {
                        const int c = bj * NB + (tid >> 6) + u * (NT / NB);
                        if (c <= r) S.L[r + (int64_t)c * ld] = v[u];
                    }
                }
        __syncthreads();
    } else {
        float omax = 0.0f;
        for (int q = tid; q < k; q += NT) {
            const int g = a.T_idx[t0 + q];
            omax = fmaxf(omax, (float)fmax(fabs(a.X[g] - ox), fabs(a.Y[g] - oy)));
        }
        omax = block_max(sm, omax) * (float)sc * 1.0001f;
        // |offset| < 2^eb, grid 2^-(21 - eb): high parts and their differences need <= 23 bits
        const int eb = max(0, ilogbf(fmaxf(omax, 1.0f)) + 1);
        const double qscale = exp2((double)(21 - eb)), iqscale = exp2((double)(eb - 21));

        // gather
    #pragma unroll 4
        for (int q = tid; q < k; q += NT) {
            const int g = a.T_idx[t0 + q];
            const double dx = (a.X[g] - ox) * sc, dy = (a.Y[g] - oy) * sc;
            const double hx = rint(dx * qscale) * iqscale, hy = rint(dy * qscale) * iqscale;
            S.xh[q] = (float)hx;
            S.xl[q] = (float)(dx - hx);
            S.yh[q] = (float)hy;
            S.yl[q] = (float)(dy - hy);
            S.yv[q] = a.Vals[g];
            S.xs[q] = 0.0;
            S.rr[q] = a.Vals[g];
        }
        __syncthreads();

        // FP32 lower triangle of Sigma + lambda I (the tensor-core kernel reads the
        // coordinates from shared memory: the operand ring is idle before the factorisation)
        const float *cxh = S.xh, *cxl = S.xl, *cyh = S.yh, *cyl = S.yl;
        if constexpr (TC) {
            if ((size_t)4 * ld * sizeof(float) <= (size_t)tc_ring_bytes<Sch>(a.tc_stages)) {
                float* f = reinterpret_cast<float*>(tc->stages);
                for (int q = tid; q < k; q += NT) {
                    f[q] = S.xh[q];
                    f[ld + q] = S.xl[q];
                    f[2 * ld + q] = S.yh[q];
                    f[3 * ld + q] = S.yl[q];
                }
                cxh = f;
                cxl = f + ld;
                cyh = f + 2 * ld;
                cyl = f + 3 * ld;
                __syncthreads();
            }
        }
        const float lam32 = (float)lam;
        const int nb = pred_only ? 0 : (k + NB - 1) / NB;
        for (int bj = 0; bj < nb; ++bj)
            for (int bi = bj; bi < nb; ++bi) {
                const int r = bi * NB + (tid & (NB - 1));     // fixed row per thread within a tile
                if (r >= k) continue;
                const float rxh = cxh[r], rxl = cxl[r], ryh = cyh[r], ryl = cyl[r];
                for (int cc = tid >> 6; cc < NB; cc += NT / NB) {
                    const int c = bj * NB + cc;
                    if (c > r) break;
                    float v = 1.0f + lam32;
                    if (r != c) {
                        const float dx = (rxh - cxh[c]) + (rxl - cxl[c]);
                        const float dy = (ryh - cyh[c]) + (ryl - cyl[c]);
                        // the FP32 matrix only preconditions the refinement, so the hardware
                        // approximations of the root and the exponential serve (a few ulp)
                        const float d2 = fmaf(dx, dx, dy * dy);
                        v = __expf(-(d2 > 0.0f ? d2 * rsqrtf(d2) : 0.0f));
                    }
                    S.L[r + (int64_t)c * ld] = v;
                }
            }
        __syncthreads();
    }

    tm.lap(kPhGather);
    bool ok = false;
    // the tensor-core factorisation also makes the first forward solve of the data
    // (not of the extended variant's right-hand-side columns)
    const bool fuse_fw = TC && !(EXT && a.rhs);
    if (pred_only) {
        ok = true;
    } else if (lat_ok) {
        if constexpr (TC) {
            if (fuse_fw)
                for (int q = tid; q < k; q += NT) S.w[q] = (float)S.rr[q];
            LatView lv{};
            if constexpr (LAT)
                lv = LatView{S.tab, reinterpret_cast<const int*>(S.xh), reinterpret_cast<const int*>(S.yh), W};
            ok = factor_tc<Sch, LAT>(*tc, S, k, ld, a.phase_cycles, fuse_fw ? S.w : nullptr, keep.fwj, lv, keep.lij);
        }
        else ok = factor32(sm, *simt, S, k, ld);
    }
    tm.t = a.phase_cycles ? now_cycles() : 0;
    if constexpr (!TC) tm.lap(kPhFactorSimt);
    // refinement and prediction work on per-task vectors; in the tensor-core kernel the
    // operand ring is idle from here on, so they move to shared memory when they fit
    if (!ok && a.phase_cycles && tid == 0) atomicAdd(a.phase_cycles + kPhFailFactor, 1ull);
    SlotM R = S;
    if constexpr (TC && LAT) {
        // lattice data: the residual and the prediction read the index vectors, the
        // solution and the task's covariance table (no low coordinate parts); then the
        // solve vector and the accumulators as room allows
        const size_t head = (offsetof(SmemM, L) + 15) / 16 * 16;
        const size_t room = (size_t)tc_ring_bytes<Sch>(a.tc_stages) - head;
        const size_t vec = (size_t)ld * sizeof(float);
        const size_t tabb = ((size_t)H * W * sizeof(float2) + 15) / 16 * 16;
        if (ok && room >= 4 * vec + tabb) {
            float* f = reinterpret_cast<float*>(tc->stages + head);
            R.xh = f;
            R.yh = f + ld;
            R.qh = f + 2 * ld;
            R.ql = f + 3 * ld;
            R.tab = reinterpret_cast<float2*>(f + 4 * ld);
            float* g = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(R.tab) + tabb);
            size_t left = room - 4 * vec - tabb;
            if (left >= vec) {
                R.w = g;
                g += ld;
                left -= vec;
            }
            if (left >= 2 * vec) {
                R.ah = g;
                R.al = g + ld;
            }
            for (int q = tid; q < k; q += NT) {
                R.xh[q] = S.xh[q];
                R.yh[q] = S.yh[q];
            }
            for (int e = tid; e < H * W; e += NT) R.tab[e] = S.tab[e];
            __syncthreads();
        }
    } else if constexpr (TC) {
        // as many of the vectors as fit, most used first: coordinates and solution
        // (residual and prediction), then the solve vector, then the accumulators; the
        // vectors start at SmemM's FP32-engine block, unused by this kernel
        const size_t head = (offsetof(SmemM, L) + 15) / 16 * 16;
        const size_t room = (size_t)tc_ring_bytes<Sch>(a.tc_stages) - head;
        const size_t vec = (size_t)ld * sizeof(float);
        if (ok && room >= 6 * vec) {
            float* f = reinterpret_cast<float*>(tc->stages + head);
            R.xh = f;
            R.xl = f + ld;
            R.yh = f + 2 * ld;
            R.yl = f + 3 * ld;
            R.qh = f + 4 * ld;
            R.ql = f + 5 * ld;
            if (room >= 7 * vec) R.w = f + 6 * ld;
            if (room >= 9 * vec) {
                R.ah = f + 7 * ld;
                R.al = f + 8 * ld;
            }
            for (int q = tid; q < k; q += NT) {
                R.xh[q] = S.xh[q];
                R.xl[q] = S.xl[q];
                R.yh[q] = S.yh[q];
                R.yl[q] = S.yl[q];
            }
            __syncthreads();
        }
    }
    __syncthreads();
    // EXT: the extended variant -- several right-hand sides (one factorisation, each
    // column refined and predicted) and the local log-likelihood; the plain variant
    // keeps the CV path's registers to itself
    const int nrhs = EXT && a.rhs ? a.nrhs : 1;
    for (int rh = 0; rh < nrhs; ++rh) {
        if (EXT && a.rhs) {   // this column's values (the factor stays)
            for (int q = tid; q < k; q += NT) {
                const double yv = a.rhs[rh * a.rhs_stride + a.T_idx[t0 + q]];
                R.yv[q] = yv;
                R.rr[q] = yv;
                R.xs[q] = 0.0;
            }
            __syncthreads();
        }
        // the loss-aware stopping rule serves CV and prediction tasks (not the local
        // log-likelihood's or GLS's, whose results need the solution itself) whose
        // prediction points cost no more than a residual pass
        const bool loss_rule = !a.lik && !a.rhs && a.refine_loss_tol > 0.0 && m <= k;
        bool have_pred = false;       // the predictions of the final solution are done
        if (ok && !pred_only) {
            // iterative refinement: x += L^-T L^-1 r
            ok = false;
            float dprev = 0.0f;
            for (int it = 0; it <= a.refine_max_iter; ++it) {
                const bool fused = fuse_fw && it == 0 && rh == 0;   // L^-1 y came with the factor
                if (fused) {
                    if (R.w != S.w)
                        for (int q = tid; q < k; q += NT) R.w[q] = S.w[q];
                } else {
                    for (int q = tid; q < k; q += NT) R.w[q] = (float)R.rr[q];
                }
                __syncthreads();
                if constexpr (TC) {
                    if (!fused) forward_inv(sm, R.L, ld, R.w, k);
                    backward_inv(sm, R.L, ld, R.w, k);
                } else {
                    forward32(sm, R.L, ld, R.w, k);
                    backward32(sm, R.L, ld, R.w, k);
                }
                tm.lap(kPhSolve);
                float dmax = 0.0f, xmax = 0.0f;
                for (int q = tid; q < k; q += NT) {
                    const double xn = R.xs[q] + (double)R.w[q];
                    R.xs[q] = xn;
                    dmax = fmaxf(dmax, fabsf(R.w[q]));
                    xmax = fmaxf(xmax, fabsf((float)xn));
                }
                dmax = block_max(sm, dmax);
                xmax = block_max(sm, xmax);
                if (!(dmax == dmax) || !(xmax == xmax)) {                 // NaN: give up
                    if (a.phase_cycles && tid == 0) atomicAdd(a.phase_cycles + kPhFailNaN, 1ull);
                    break;
                }
                for (int q = tid; q < k; q += NT) {
                    const df v = dfm::from_double(R.xs[q]);
                    R.qh[q] = v.h;
                    R.ql[q] = v.l;
                }
                __syncthreads();
                if (it >= 1) {
                    if (dmax > 0.5f * dprev) {                             // not contracting
                        if (a.phase_cycles && tid == 0) atomicAdd(a.phase_cycles + kPhFailStall, 1ull);
                        break;
                    }
                    // error left after this correction ~ c |d_i|, c = |d_i| / |d_i-1| the
                    // observed contraction; the solution rule stops when that is small
                    // against |x|
                    const float c = dmax / fmaxf(dprev, 1e-30f);
                    if (c * dmax <= (float)a.refine_tol * xmax) { ok = true; break; }
                    // loss-aware rule, for a solution already within refine_loss_guard times
                    // the solution rule's bound (no guard when that is 0): the predictions of x_i and the change u = K d_i
                    // the last correction made to them; the error left in the predictions is
                    // estimated as g |u|, g = c / (1 - c) (the corrections still to come
                    // shrink geometrically).  Stop when it moves the local SSPE (Eq. 4) by at
                    // most refine_loss_tol relative -- |dz| <= 2 |yhat - y| |dyhat| -- and
                    // every prediction by at most 10 refine_loss_tol of their RMS.  The guard
                    // covers a remaining error whose smooth part K damps less than it damps
                    // the last correction (the estimate alone can then be optimistic).
                    if (loss_rule && (a.refine_loss_guard <= 0.0 ||
                                      c * dmax <= (float)(a.refine_loss_guard * a.refine_tol) * xmax)) {
                        const PredStats ps = predict_points<LAT>(sm, keep, a, R, k, m, p0, ox, oy, sc, W,
                                                                 (int64_t)b, R.w);
                        tm.lap(kPhPredict);
                        const double g = (double)c / (1.0 - (double)c);
                        const double lt = a.refine_loss_tol;
                        const bool loss_ok = !a.Pv || 2.0 * g * sqrt(ps.usq) <= lt * sqrt(ps.sse);
                        const bool pred_ok = g * (double)ps.umax <= 10.0 * lt * sqrt(ps.ysq / (double)max(m, 1));
                        if (loss_ok && pred_ok) {
                            ok = true;
                            have_pred = true;
                            if (a.Pv && tid == 0) a.z[zoff] = ps.sse;
                            break;
                        }
                    }
                }
                dprev = dmax;
                if (it == a.refine_max_iter) break;
                if constexpr (LAT) residual_lat<4>(R, k, lam, W);
                else residual_df<LAT>(sm, keep.tbl, R, k, lam, W);
                tm.lap(kPhResidual);
                if (a.phase_cycles && tid == 0) atomicAdd(a.phase_cycles + kPhResidualPasses, 1ull);
            }
            if (k == 0) ok = true;
        }
        if (!ok) {
            // hand the task to the FP64 kernel
            if (tid == 0) {
                a.tstatus[zoff] = PCV_REFINE_FALLBACK;
                const unsigned pos = atomicAdd(a.fb_count, 1u);
                a.fb_list[pos] = i * a.B + b;   // (subset, configuration), whatever launch order ran it
            }
            __syncthreads();
            return;
        }
        if (pred_only) {
            // the stored kriging weights of this subset and configuration
            const double* al = a.alpha_in + (int64_t)(a.alpha_slot ? a.alpha_slot[b] : 0) * a.alpha_stride + t0;
            for (int q = tid; q < k; q += NT) {
                const double x = al[q];
                R.xs[q] = x;
                const df v = dfm::from_double(x);
                R.qh[q] = v.h;
                R.ql[q] = v.l;
            }
            __syncthreads();
        } else if (a.alpha_out && a.alpha_slot && a.alpha_slot[b] >= 0 && !(EXT && a.rhs)) {
            // keep the refined kriging weights for later predictions at new locations
            double* al = a.alpha_out + (int64_t)a.alpha_slot[b] * a.alpha_stride + t0;
            for (int q = tid; q < k; q += NT) al[q] = R.xs[q];
        }

        // local -2 log-likelihood (Eq. 2) of the training data: the quadratic form from
        // the refined solution, the log-determinant from the FP32 factor's diagonal (the
        // tensor-core engines keep L_JJ^-1 there, whose diagonal is 1 / L_jj)
        if (EXT && a.lik && rh == 0) {
            double ldet = 0.0, quad = 0.0;
            for (int q = tid; q < k; q += NT) {
                const double d = (double)R.L[q + (int64_t)q * ld];
                ldet += TC ? -log(d) : log(d);
                quad += R.yv[q] * R.xs[q];
            }
            ldet = warp_sum_d(ldet);
            quad = warp_sum_d(quad);
            if (lane == 0) {
                sm.dred[warp] = ldet;
                sm.dred2[warp] = quad;
            }
            __syncthreads();
            if (tid == 0) {
                double l = 0.0, qf = 0.0;
                for (int w = 0; w < NT / 32; ++w) {
                    l += sm.dred[w];
                    qf += sm.dred2[w];
                }
                a.lik[zoff] = k * log(2.0 * M_PI) + k * log(s2) + 2.0 * l + qf / s2;
            }
            __syncthreads();
        }

        // predict (Eq. 3) in double-float, squared errors in FP64 (Eq. 4), unless the
        // stopping rule already did so for the final solution
        if (!have_pred) {
            const PredStats ps = predict_points<LAT>(sm, keep, a, R, k, m, p0, ox, oy, sc, W,
                                                     (int64_t)(EXT && a.rhs ? rh : b), nullptr);
            if (a.Pv && tid == 0) a.z[zoff] = ps.sse;
        }
    }
    if (tid == 0) a.tstatus[zoff] = PCV_OK;
    __syncthreads();
    tm.lap(kPhPredict);
    if (a.phase_cycles && tid == 0) {
        atomicAdd(a.phase_cycles + kPhTask, (unsigned long long)(now_cycles() - t_task));
        atomicAdd(a.phase_cycles + kPhTasks, 1ull);
    }
}

__global__ void __launch_bounds__(NT, 2) k_cv_mixed(TaskArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // layout: SmemM, SmemSimt (both 16-byte aligned sizes), then SmemKeep
    SmemM& sm = *reinterpret_cast<SmemM*>(smem_raw);
    SmemSimt& simt = *reinterpret_cast<SmemSimt*>(smem_raw + sizeof(SmemM));
    SmemKeep& keep = *reinterpret_cast<SmemKeep*>(smem_raw + sizeof(SmemM) + sizeof(SmemSimt));
    for (int e = threadIdx.x; e < 2 * dfm::kExpTable; e += NT) keep.tbl[e] = c_exp.tbl[e];
    __syncthreads();
    const int ntask = a.n_order * a.B;
    for (;;) {
        if (threadIdx.x == 0) keep.task = (int)atomicAdd(a.counter, 1u);
        __syncthreads();
        const int t = keep.task;
        __syncthreads();
        if (t >= ntask) break;
        run_task<false, umma::SplitBF16x3, true>(sm, keep, &simt, nullptr, a, t, a.order[t / a.B], t % a.B);
    }
}

constexpr int kSimtSmem = (int)(sizeof(SmemM) + sizeof(SmemKeep) + sizeof(SmemSimt));
static_assert(sizeof(SmemM) % 16 == 0 && sizeof(SmemSimt) % 16 == 0 && alignof(SmemSimt) == 16,
              "SmemSimt must start on a 16-byte boundary after SmemM");
// tensor-core kernel layout (offsets from the 1024-aligned base) for a ring of
// `ring` bytes: operand ring, then the persistent struct, then the pipeline barriers
__host__ __device__ constexpr int tc_keep_off(int ring) { return ring; }
__host__ __device__ constexpr int tc_sh_off(int ring) { return (tc_keep_off(ring) + (int)sizeof(SmemKeep) + 127) / 128 * 128; }
__host__ __device__ constexpr int tc_smem(int ring) { return 1024 + tc_sh_off(ring) + (int)sizeof(TcShared); }
constexpr int kTcRingMax = 144 * 1024;
constexpr int kTcSmem = tc_smem(kTcRingMax);
static_assert(kTcRingMin % 128 == 0 && tc_sh_off(kTcRingMin) % 128 == 0, "shared-memory layout alignment");
static_assert(kTcSmem <= 227 * 1024, "tensor-core kernel exceeds the shared memory of one CTA");
static_assert(sizeof(SmemM) <= (size_t)kTcRingMin && sizeof(SmemM) % 16 == 0,
              "phase scratch must fit in the smallest ring, vectors after it 16-byte aligned");
static_assert(kDiagBytes <= kTcRingMin && kDiagYOff % 16 == 0, "diagonal block must fit in the smallest ring");
static_assert(2 * tc_smem(kTcRingMin) <= 228 * 1024, "two tensor-core CTAs must fit on one SM");
static_assert(tc_ring_bytes<umma::SplitBF16x3>(2) == kTcRingMin && tc_ring_bytes<umma::SplitF16x2>(3) == kTcRingMin,
              "default rings of both schemes");

// Tensor-core variant: two CTAs per SM, 256 TMEM columns each; Sch is the operand scheme,
// EXT the extended variant (several right-hand sides, local log-likelihood), LAT the
// lattice-data variant (covariances from a per-task table by index offset).
template <class Sch, bool EXT = false, bool LAT = false>
__global__ void __launch_bounds__(NT, 2) k_cv_mixed_tc(TaskArgs a, const __grid_constant__ CUtensorMap m0,
                                                       const __grid_constant__ CUtensorMap m1,
                                                       const __grid_constant__ CUtensorMap m2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    TcCtx tc;
    tc.stages = base;
    SmemM& sm = *reinterpret_cast<SmemM*>(base);   // phase scratch shares the operand ring
    const int nst = a.tc_stages;
    const int ring = tc_ring_bytes<Sch>(nst);
    SmemKeep& keep = *reinterpret_cast<SmemKeep*>(base + tc_keep_off(ring));
    tc.sh = reinterpret_cast<TcShared*>(base + tc_sh_off(ring));
    tc.m0 = &m0;
    tc.m1 = &m1;
    tc.m2 = &m2;
    const int64_t slot_elems = (int64_t)a.ld * a.ld * kw<Sch>();   // 16-bit units per slot and plane
    uint16_t* P = reinterpret_cast<uint16_t*>(a.planes);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl)
        tc.p[pl] = pl < Sch::kPlanes ? P + pl * a.plane_elems + blockIdx.x * slot_elems : nullptr;
    tc.row_base = blockIdx.x * a.ld;
    const int warp = threadIdx.x >> 5;
    for (int e = threadIdx.x; e < 2 * dfm::kExpTable; e += NT) keep.tbl[e] = c_exp.tbl[e];
    if (threadIdx.x == 0) {
        umma::pipe_init(tc.sh->pipe, (uint32_t)nst);
        if (a.test_wait_ns) tc.sh->pipe.wait_ns = a.test_wait_ns;
        tc.sh->dead = 0;
        umma::prefetch_map(&m0);
        umma::prefetch_map(&m1);
        if (Sch::kPlanes > 2) umma::prefetch_map(&m2);
    }
    if (warp == 1) umma::tmem_alloc(&tc.sh->pipe.tmem_base, kTcTmemCols);
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const int ntask = a.n_order * a.B;
    for (;;) {
        if (threadIdx.x == 0) {
            keep.task = (int)atomicAdd(a.counter, 1u);
            tc.sh->pipe.withhold = a.test_withhold_task != 0 && keep.task == a.test_withhold_task - 1;
        }
        __syncthreads();
        const int t = keep.task;
        __syncthreads();
        if (t >= ntask) break;
        run_task<true, Sch, EXT, LAT>(sm, keep, nullptr, &tc, a, t, a.order[t / a.B], t % a.B);
    }
    umma::tc_fence_before();
    __syncthreads();
    if (warp == 1) umma::tmem_dealloc(tc.sh->pipe.tmem_base, kTcTmemCols);
}

std::mutex g_prep_mu;
bool g_prepared[64] = {false};

}  // namespace

int64_t slot_bytes_mixed(int32_t ld, int64_t mmax, int64_t lat_cap) {
    const int64_t b = (int64_t)ld * ld * 4 + 3 * (int64_t)ld * 8 + 9 * (int64_t)ld * 4 + lat_cap * 8 + (mmax + 32) * 8;
    return (b + 255) / 256 * 256;
}

int mixed_prepare(int device) {
    std::lock_guard<std::mutex> lk(g_prep_mu);
    if (device < 0 || device >= 64) return (int)cudaErrorInvalidDevice;
    if (g_prepared[device]) return 0;
    dfm::ExpConsts k;
    dfm::exp_constants(k);
    cudaError_t e = cudaMemcpyToSymbol(c_exp, &k, sizeof(k));
    if (e != cudaSuccess) return (int)e;
    e = cudaFuncSetAttribute(k_cv_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, kSimtSmem);
    const void* tc_kernels[] = {
        (const void*)k_cv_mixed_tc<umma::SplitBF16x3>,        (const void*)k_cv_mixed_tc<umma::SplitF16x2>,
        (const void*)k_cv_mixed_tc<umma::SplitF16x2, true>,   (const void*)k_cv_mixed_tc<umma::SplitF16x2, false, true>,
        (const void*)k_cv_mixed_tc<umma::SplitTF32x1>,        (const void*)k_cv_mixed_tc<umma::SplitTF32x1, false, true>,
        (const void*)k_cv_mixed_tc<umma::SplitTF32x3>,        (const void*)k_cv_mixed_tc<umma::SplitTF32x3, false, true>};
    for (const void* f : tc_kernels)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return (int)e;
    g_prepared[device] = true;
    return 0;
}

int mixed_planes(int engine) {
    switch (engine) {
        case kMixedEngineTensor: return umma::SplitF16x2::kPlanes;
        case kMixedEngineTensorBF16: return umma::SplitBF16x3::kPlanes;
        case kMixedEngineTensorTF32: return umma::SplitTF32x1::kPlanes;
        case kMixedEngineTensorTF32x3: return umma::SplitTF32x3::kPlanes;
        default: return 0;
    }
}

int mixed_term_bytes(int engine) {
    return engine == kMixedEngineTensorTF32 || engine == kMixedEngineTensorTF32x3 ? 4 : 2;
}

int mixed_default_stages(int engine) {
    switch (engine) {
        case kMixedEngineTensorBF16: return 2;    // 48 KB stages
        case kMixedEngineTensorTF32: return 4;    // 16 KB stages
        default: return 3;                        // 32 KB stages
    }
}

namespace {
template <class Sch>
int launch_tc(const TaskArgs& a, const CUtensorMap* m, int grid, cudaStream_t st) {
    const int ring = tc_ring_bytes<Sch>(a.tc_stages);
    if (a.tc_stages < 2 || a.tc_stages > umma::kStages || ring < kTcRingMin || ring > kTcRingMax)
        return (int)cudaErrorInvalidValue;
    if (a.rhs || a.lik) {   // the extended variant exists for the default FP16 scheme only
        if constexpr (std::is_same<Sch, umma::SplitF16x2>::value)
            k_cv_mixed_tc<Sch, true><<<grid, NT, tc_smem(ring), st>>>(a, m[0], m[1], m[2]);
        else
            return (int)cudaErrorInvalidValue;
    } else if (a.LX && !std::is_same<Sch, umma::SplitBF16x3>::value) {
        if constexpr (!std::is_same<Sch, umma::SplitBF16x3>::value)
            k_cv_mixed_tc<Sch, false, true><<<grid, NT, tc_smem(ring), st>>>(a, m[0], m[1], m[2]);
    } else {
        k_cv_mixed_tc<Sch><<<grid, NT, tc_smem(ring), st>>>(a, m[0], m[1], m[2]);
    }
    return 0;
}
}  // namespace

int launch_task_mixed(const TaskArgs& a, const void* maps, int engine, int grid, void* stream) {
    const CUtensorMap* m = reinterpret_cast<const CUtensorMap*>(maps);
    const cudaStream_t st = (cudaStream_t)stream;
    int e = 0;
    switch (engine) {
        case kMixedEngineTensor: e = launch_tc<umma::SplitF16x2>(a, m, grid, st); break;
        case kMixedEngineTensorBF16: e = launch_tc<umma::SplitBF16x3>(a, m, grid, st); break;
        case kMixedEngineTensorTF32: e = launch_tc<umma::SplitTF32x1>(a, m, grid, st); break;
        case kMixedEngineTensorTF32x3: e = launch_tc<umma::SplitTF32x3>(a, m, grid, st); break;
        default: k_cv_mixed<<<grid, NT, kSimtSmem, st>>>(a); break;
    }
    if (e) return e;
    count_launch();
    return (int)cudaGetLastError();
}

bool mixed_make_maps(void* planes, int64_t plane_elems, int32_t ld, int grid, int nplanes, int term_bytes,
                     void* maps_out) {
    CUtensorMap* m = reinterpret_cast<CUtensorMap*>(maps_out);
    uint16_t* P = reinterpret_cast<uint16_t*>(planes);
    const uint64_t tiles = (uint64_t)grid * (ld / umma::kTileM) * (ld * (term_bytes / 2) / umma::kChunkK);
    for (int p = 0; p < 3; ++p)   // maps past the scheme's planes repeat the last one (never used)
        if (!umma::make_tiled_map(&m[p], P + std::min(p, nplanes - 1) * plane_elems, tiles)) return false;
    return true;
}

}  // namespace pcv
