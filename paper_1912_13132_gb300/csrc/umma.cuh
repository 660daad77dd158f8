// umma.cuh -- Blackwell (sm_100a family) tensor-core building blocks in inline PTX:
// TMEM allocation, tcgen05.mma (kind::f16, FP32 accumulators), TMA tile loads,
// mbarriers with bounded waits, and the warp-specialised pipeline that computes one
// block-column product
//
//     D[rows r0 .. r0+nr, 0 .. 128) = sum over K of A[r, K] * B[c, K]      (K-major)
//
// with A and B carried as planes of 16-bit terms whose sum is the FP32 value (an
// operand scheme, see SplitBF16x3 and SplitF16x2 below); the scheme's cross products
// of planes, accumulated in FP32, reproduce FP32-accurate products on the 16-bit
// tensor pipe.
//
// Roles (256 threads):  warp 0 lane 0 issues TMA loads into a ring of Pipe::nstages
// stages, warp 1 lane 0 issues the MMAs, warps 4..7 (one per TMEM lane quadrant)
// drain the accumulators through the caller's epilogue.  TPP 128-row tiles (template
// parameter) form one pass; the accumulators of consecutive passes alternate between
// two TMEM buffers so the epilogue of one pass overlaps the MMAs of the next.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace pcv {
namespace umma {

constexpr int kTileM = 128;        // rows per tile (MMA M)
constexpr int kTileN = 128;        // block-column width (MMA N)
constexpr int kChunkK = 32;        // 16-bit elements per TMA box row (64 bytes, 64B swizzle)
constexpr int kTilesPerPass = 2;   // default tiles per pass (template parameter TPP below)
constexpr int kStages = 4;         // maximum ring depth (runtime depth in Pipe::nstages)
constexpr int kTileBytes = kTileM * kChunkK * 2;                    // 8 KB

// Operand schemes.  SplitBF16x3: x = h + m + l, each term the round-to-nearest BF16
// of what the previous ones leave (24 significant bits, representation error
// <= 2^-24 |x|), six products h*h + h*m + m*h + h*l + l*h + m*m (the dropped ones are
// below 2^-24 |a||b|).  SplitF16x2: x = h + l in FP16 (22 significant bits, error
// <= 2^-22 |x| for |x| >= 2^-14, an absolute 2^-25 below that), three products
// h*h + h*l + l*h (the dropped l*l is <= 2^-22 |a||b|): a third fewer bytes per
// element and half the MMAs, for values of magnitude well below 65504.
// kElem: bytes per term; the planes of 4-byte terms are stored as planes of 16-bit
// units twice as wide (a 64-byte TMA box row holds 16 of them), so the tiles, tensor
// maps and K chunks keep their byte layout.  kTF32: the terms are TF32 words, multiplied
// by tcgen05.mma kind::tf32 (K = 8 per instruction: 32 bytes, as K = 16 of kind::f16).
struct SplitBF16x3 {
    static constexpr int kPlanes = 3, kProducts = 6, kElem = 2;
    static constexpr bool kTF32 = false;
    static constexpr uint32_t kFmt = 1;   // instruction-descriptor code of BF16
    __host__ __device__ static constexpr int a(int q) { return q == 2 ? 1 : q == 4 ? 2 : q == 5 ? 1 : 0; }
    __host__ __device__ static constexpr int b(int q) { return q == 1 ? 1 : q == 3 ? 2 : q == 5 ? 1 : 0; }
};
struct SplitF16x2 {
    static constexpr int kPlanes = 2, kProducts = 3, kElem = 2;
    static constexpr bool kTF32 = false;
    static constexpr uint32_t kFmt = 0;   // instruction-descriptor code of FP16
    __host__ __device__ static constexpr int a(int q) { return q == 2 ? 1 : 0; }
    __host__ __device__ static constexpr int b(int q) { return q == 1 ? 1 : 0; }
};
// TF32x1: x rounded to TF32 (11 significant bits), one product: the plain TF32 tensor-core
// factorisation, fast but accurate only for well-conditioned matrices.  TF32x3: x = h + l,
// h = tf32(x), l = tf32(x - h) (22 significant bits), three products h*h + h*l + l*h (the
// split of Ootomo and Yokota, 2022).
struct SplitTF32x1 {
    static constexpr int kPlanes = 1, kProducts = 1, kElem = 4;
    static constexpr bool kTF32 = true;
    static constexpr uint32_t kFmt = 2;   // instruction-descriptor code of TF32
    __host__ __device__ static constexpr int a(int) { return 0; }
    __host__ __device__ static constexpr int b(int) { return 0; }
};
struct SplitTF32x3 {
    static constexpr int kPlanes = 2, kProducts = 3, kElem = 4;
    static constexpr bool kTF32 = true;
    static constexpr uint32_t kFmt = 2;
    __host__ __device__ static constexpr int a(int q) { return q == 2 ? 1 : 0; }
    __host__ __device__ static constexpr int b(int q) { return q == 1 ? 1 : 0; }
};

// one stage: per plane, the B operand's bn / 128 boxes and TPP A tiles
template <class Sch = SplitBF16x3>
__host__ __device__ constexpr int stage_bytes(int tpp, int bn = kTileN) {
    return Sch::kPlanes * (tpp + bn / kTileM) * kTileBytes;
}
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitNs = 2000000000ull;  // bound of every mbarrier wait (2 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------- mbarriers

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete; false once `limit_ns` of wall
// time (default kWaitNs) have passed without it (the caller then reports an error
// instead of hanging).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 64; ++i)
            if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// ---------------------------------------------------------------- TMA

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
// the same with an L2 cache policy (createpolicy) for the loaded lines
__device__ __forceinline__ void tma_load_3d_hint(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                                 uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
// L2 policy: lines are the first candidates for eviction (data read once)
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------- TMEM and MMA

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    __syncwarp();   // .sync.aligned: the whole warp, converged
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand tile written by TMA with 64-byte
// swizzle (rows of 64 bytes, 8-row groups 512 bytes apart).
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);            // start address
    d |= (uint64_t)1 << 16;                           // leading-dimension byte offset (unused here)
    d |= (uint64_t)((512 >> 4) & 0x3FFF) << 32;       // stride-dimension byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)4 << 61;                           // 64-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16, A and B of format `fmt` (0 FP16, 1 BF16), D = FP32,
// both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16kind(int M, int N, uint32_t fmt) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16kind(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// kind::tf32: A and B are FP32 words of which the tensor core uses the TF32 part (8-bit
// exponent, 10 explicit mantissa bits); one instruction covers K = 8 (32 bytes per row,
// the same byte footprint as K = 16 of a 16-bit kind::f16 operand).  Format code 2.
constexpr uint32_t kFmtTF32 = 2;
__device__ __forceinline__ void mma_tf32kind(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                             uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 columns of FP32 from TMEM (one register per column).  The load is a
// .sync.aligned instruction: the whole warp must execute it converged, so the warp is
// reconverged first (callers may have branched per lane since the last one).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    __syncwarp();
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- splitting

// x = hi + mid + lo with each term the round-to-nearest BF16 of what is left; the
// three terms carry 24 significant bits, the representation error is <= 2^-24 |x|.
__device__ __forceinline__ void split3(float x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    l = __float2bfloat16_rn(r2);
}

// The scheme's terms of x as 16-bit patterns, plane by plane.
__device__ __forceinline__ void split_terms(SplitBF16x3, float x, uint16_t* t) {
    __nv_bfloat16 h, m, l;
    split3(x, h, m, l);
    t[0] = __bfloat16_as_ushort(h);
    t[1] = __bfloat16_as_ushort(m);
    t[2] = __bfloat16_as_ushort(l);
}
__device__ __forceinline__ void split_terms(SplitF16x2, float x, uint16_t* t) {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    t[0] = __half_as_ushort(h);
    t[1] = __half_as_ushort(l);
}

// x rounded to TF32 (round to nearest, ties away from zero), as an FP32 word whose low
// 13 mantissa bits are zero
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_terms(SplitTF32x1, float x, uint32_t* t) { t[0] = to_tf32(x); }
__device__ __forceinline__ void split_terms(SplitTF32x3, float x, uint32_t* t) {
    t[0] = to_tf32(x);
    t[1] = to_tf32(x - __uint_as_float(t[0]));
}

// ---------------------------------------------------------------- pipeline state

struct Pipe {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t accf[2];
    uint64_t acce[2];
    uint64_t drain;        // a failed MMA issuer waits here for its issued MMAs to complete
    uint64_t wait_ns;      // bound of the pipeline's waits (kWaitNs unless a test shortens it)
    uint32_t tmem_base;
    uint32_t nstages;      // ring depth in use (1 .. kStages)
    uint32_t drain_phase;
    uint32_t withhold;     // test hook: the producer skips the next stage's loads (its waits run out)
};

// Per-role phase counters; every role walks the same sequence of stages and passes.
struct Phases {
    uint32_t stage = 0;          // stage iterations done (ring position and parity)
    uint32_t nextbuf = 0;        // accumulator buffer of the next pass of a double-buffered call
    uint32_t uses[2] = {0, 0};   // passes that have used each accumulator buffer (barrier parities)
};

__device__ inline void pipe_init(Pipe& p, uint32_t nstages = kStages) {
    p.nstages = nstages;
    p.wait_ns = kWaitNs;
    p.drain_phase = 0;
    p.withhold = 0;
    mbar_init(&p.drain, 1);
    for (int s = 0; s < kStages; ++s) {
        mbar_init(&p.full[s], 1);
        mbar_init(&p.empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
        mbar_init(&p.accf[b], 1);
        mbar_init(&p.acce[b], 4);   // one arrive per epilogue warp
    }
    fence_mbar_init();
}

// One block-column product over all row tiles:
//   rows [r0, r0 + nrows) of A against rows [b0, b0 + BN) of B over the K columns
//   [kc0 * kChunkK, kc0 * kChunkK + K), K a multiple of kChunkK (in 16-bit units).  A and
//   B rows live in the planes' tensor maps at row offset `row_base` (the task's slot).  For
//   each finished 128-row tile the epilogue warps call epi(tile_row0, warp_quadrant,
//   taddr_of_tile) and must read all BN columns of their 32 lanes.  BN = 128 or 256 (the B
//   operand is BN / 128 boxes per plane, one MMA of N = BN per product).  NBUF = 2: the
//   accumulators of consecutive passes alternate between two TMEM buffers of TPP * BN
//   columns, so a pass's epilogue overlaps the next pass's MMAs; NBUF = 1: one buffer, the
//   next pass waits for the epilogue.  Calls of different shapes may follow one another
//   on one Pipe once the previous call has returned in every thread (a barrier): the
//   barrier parities follow each buffer's own use count.  Returns false if a bounded wait
//   ran out.
// Operand layouts in global memory.  Row-major: a plane is a row-major matrix and a
// box is 128 rows x 32 columns of it.  Tiled: a plane is stored as contiguous 8 KB
// tiles of 128 rows x 32 columns (tile (R, kc) at index R * nkc + kc), so that every
// box is one contiguous block of memory; `nkc` = columns / 32.
template <bool TILED>
__device__ __forceinline__ void load_box(void* dst, const CUtensorMap* map, int kc, int row, int nkc, uint64_t* bar) {
    if constexpr (TILED) tma_load_3d(dst, map, 0, 0, (row / kTileM) * nkc + kc, bar);
    else tma_load_2d(dst, map, kc * kChunkK, row, bar);
}
template <bool TILED>
__device__ __forceinline__ void load_box_stream(void* dst, const CUtensorMap* map, int kc, int row, int nkc,
                                                uint64_t* bar, uint64_t policy) {
    if constexpr (TILED) tma_load_3d_hint(dst, map, 0, 0, (row / kTileM) * nkc + kc, bar, policy);
    else tma_load_2d(dst, map, kc * kChunkK, row, bar);
}

template <bool TILED = false, int TPP = kTilesPerPass, class Sch = SplitBF16x3, int BN = kTileN, int NBUF = 2,
          class Epi>
__device__ bool block_column(Pipe& P, Phases& ph, uint8_t* stages, const CUtensorMap* mapA0,
                             const CUtensorMap* mapA1, const CUtensorMap* mapA2, int row_base, int r0,
                             int nrows, int b0, int K, Epi&& epi, int nkc = 0, int kc0 = 0) {
    static_assert(BN % kTileM == 0 && BN <= 256 && (NBUF == 1 || NBUF == 2), "block-column shape");
    constexpr int BB = BN / kTileM;   // B boxes per plane
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (nrows + kTileM - 1) / kTileM;
    const int npass = (ntiles + TPP - 1) / TPP;
    const int nk = K / kChunkK;
    const CUtensorMap* maps[3] = {mapA0, mapA1, mapA2};   // planes beyond the scheme's are unused
    bool ok = true;
    if (warp == 0 && lane == 0) {
        // TMA producer
        uint32_t it = ph.stage;
        int32_t issued[kStages];   // last iteration whose loads went to each ring slot
#pragma unroll
        for (int q = 0; q < kStages; ++q) issued[q] = -1;
        const uint64_t stream = policy_evict_first();
        for (int p = 0; p < npass && ok; ++p) {
            const int t0 = p * TPP;
            const int nt = min(TPP, ntiles - t0);
            // K chunks in ascending order for every tile.  In the left-looking update the first
            // chunks (columns far from the rows updated) carry the smallest terms; reversing the
            // order on alternate tiles, to reuse the B chunks while they are in L2, tripled the
            // refinement passes of the paper-scale workload (1.43 -> 4.4 per task): the
            // accumulation in TMEM is order-sensitive, and small terms go in first.
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = it % P.nstages;
                const uint32_t par = ((it / P.nstages) & 1) ^ 1;
                if (!mbar_wait(&P.empty[s], par, P.wait_ns)) { ok = false; break; }
                if (P.withhold) {   // test hook: this stage is never loaded, its consumers time out
                    P.withhold = 0;
                    continue;
                }
                issued[s] = (int32_t)it;
                uint8_t* st = stages + s * stage_bytes<Sch>(TPP, BN);
                mbar_expect_tx(&P.full[s], (uint32_t)(Sch::kPlanes * (nt + BB) * kTileBytes));
                for (int pl = 0; pl < Sch::kPlanes; ++pl) {
                    for (int h = 0; h < BB; ++h)
                        load_box<TILED>(st + (pl * BB + h) * kTileBytes, maps[pl], kc0 + kc,
                                        row_base + b0 + h * kTileM, nkc, &P.full[s]);
                    for (int t = 0; t < nt; ++t)   // A: read once per block column
                        load_box_stream<TILED>(st + (Sch::kPlanes * BB + t * Sch::kPlanes + pl) * kTileBytes,
                                               maps[pl], kc0 + kc, row_base + r0 + (t0 + t) * kTileM, nkc,
                                               &P.full[s], stream);
                }
            }
        }
        if (!ok) {
            // the shared memory of the ring is reused once this call returns: every load
            // issued must have landed first (a consumed stage's phase is already complete)
            for (int q = 0; q < (int)P.nstages; ++q)
                if (issued[q] >= 0)
                    mbar_wait(&P.full[q], (uint32_t)((issued[q] / P.nstages) & 1), P.wait_ns);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        uint32_t it = ph.stage, nb = ph.nextbuf, u0 = ph.uses[0], u1 = ph.uses[1];   // (scalars: registers)
        const uint32_t idesc = idesc_f16kind(kTileM, BN, Sch::kFmt);
        for (int p = 0; p < npass && ok; ++p) {
            const int t0 = p * TPP;
            const int nt = min(TPP, ntiles - t0);
            const int buf = NBUF == 1 ? 0 : (int)nb;
            const uint32_t ub = buf ? u1 : u0;
            if (!mbar_wait(&P.acce[buf], (ub & 1) ^ 1, P.wait_ns)) { ok = false; break; }
            tc_fence_after();
            for (int kc = 0; kc < nk; ++kc, ++it) {
                const int s = it % P.nstages;
                if (!mbar_wait(&P.full[s], (it / P.nstages) & 1, P.wait_ns)) { ok = false; break; }
                tc_fence_after();
                const uint32_t st = smem_u32(stages + s * stage_bytes<Sch>(TPP, BN));
                for (int t = 0; t < nt; ++t) {
                    const uint32_t d = P.tmem_base + buf * (TPP * BN) + t * BN;
#pragma unroll
                    for (int kk = 0; kk < kChunkK / 16; ++kk)
#pragma unroll
                        for (int q = 0; q < Sch::kProducts; ++q) {
                            const uint32_t a =
                                st + (Sch::kPlanes * BB + t * Sch::kPlanes + Sch::a(q)) * kTileBytes + kk * 32;
                            const uint32_t b = st + Sch::b(q) * BB * kTileBytes + kk * 32;
                            const uint32_t acc = (kc > 0 || kk > 0 || q > 0) ? 1u : 0u;
                            if constexpr (Sch::kTF32) mma_tf32kind(d, smem_desc_sw64(a), smem_desc_sw64(b), idesc, acc);
                            else mma_f16kind(d, smem_desc_sw64(a), smem_desc_sw64(b), idesc, acc);
                        }
                }
                mma_commit(&P.empty[s]);
            }
            if (ok) mma_commit(&P.accf[buf]);
            if (buf) ++u1; else ++u0;
            if (NBUF == 2) nb ^= 1u;
        }
        if (!ok) {
            // the MMAs issued so far read the ring and write TMEM: let them complete
            mma_commit(&P.drain);
            mbar_wait(&P.drain, P.drain_phase, P.wait_ns);
            P.drain_phase ^= 1u;
        }
    } else if (warp >= 4) {
        // epilogue: one warp per TMEM lane quadrant
        const int quad = warp & 3;
        uint32_t nb = ph.nextbuf, u0 = ph.uses[0], u1 = ph.uses[1];
        for (int p = 0; p < npass && ok; ++p) {
            const int t0 = p * TPP;
            const int nt = min(TPP, ntiles - t0);
            const int buf = NBUF == 1 ? 0 : (int)nb;
            // every lane polls the barrier on its own; agree on the outcome (which also
            // reconverges the warp before the aligned TMEM loads of the epilogue)
            const bool got = mbar_wait(&P.accf[buf], (buf ? u1 : u0) & 1, P.wait_ns);
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
            tc_fence_after();
            for (int t = 0; t < nt; ++t) {
                const uint32_t taddr = P.tmem_base + ((uint32_t)(quad * 32) << 16) + buf * (TPP * BN) + t * BN;
                epi(r0 + (t0 + t) * kTileM, quad, taddr);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&P.acce[buf]);
            if (buf) ++u1; else ++u0;
            if (NBUF == 2) nb ^= 1u;
        }
    }
    // every role advances its counters identically (the producer and MMA counts
    // follow from the shape alone)
    ph.stage += (uint32_t)(npass > 0 ? npass * nk : 0);
    if (NBUF == 1) {
        ph.uses[0] += (uint32_t)npass;
    } else {
        ph.uses[ph.nextbuf] += (uint32_t)((npass + 1) / 2);
        ph.uses[ph.nextbuf ^ 1u] += (uint32_t)(npass / 2);
        ph.nextbuf ^= (uint32_t)(npass & 1);
    }
    return ok;
}

// ---------------------------------------------------------------- host: tensor maps

// 2-D tensor map over a row-major BF16 matrix of `rows` rows of `inner` elements
// (inner * 2 bytes a multiple of 16), boxes of kTileM rows x kChunkK elements,
// 64-byte swizzle (the layout the shared-memory descriptors above expect).
inline bool make_plane_map(CUtensorMap* map, void* base, uint64_t inner, uint64_t rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileM};
    cuuint32_t estr[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D tensor map over a tiled BF16 plane (see load_box): dims (32, 128, tiles), box
// (32, 128, 1), 64-byte swizzle.
inline bool make_tiled_map(CUtensorMap* map, void* base, uint64_t tiles) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    cuuint64_t dims[3] = {(cuuint64_t)kChunkK, (cuuint64_t)kTileM, tiles};
    cuuint64_t strides[2] = {(cuuint64_t)kChunkK * 2, (cuuint64_t)kChunkK * kTileM * 2};
    cuuint32_t box[3] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace umma
}  // namespace pcv
