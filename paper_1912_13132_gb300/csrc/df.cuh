// df.cuh -- double-float ("float-float") arithmetic for the refinement residuals.
//
// GB300 runs FP64 at about 1/62 of its FP32 rate, so the accurate residuals and
// predictions of the mixed-precision path are computed with pairs of floats
// (hi + lo, ~48 significant bits) using only FP32 adds, multiplies and FMAs:
//   * error-free transformations: TwoSum (Knuth), Fast2Sum (Dekker), TwoProd via FMA;
//   * exp(-t): Tang's table-driven method (P. T. P. Tang, "Table-driven
//     implementation of the exponential function in IEEE floating-point
//     arithmetic", ACM TOMS 15(2), 1989) carried out in double-float:
//       j = nearest integer to t * 256/ln2,  r = t - j ln2/256 (|r| <= ln2/512),
//       exp(-t) = 2^(-floor(j/256)) * 2^(-(j mod 256)/256) * exp(-r),
//     with 2^(-i/256) from a 256-entry double-float table, ln2/256 split in
//     three floats (the first with 9 significant bits so that j * C1 is exact),
//     and exp(-r) = 1 - r + r^2/2 - r^3/6 + r^4/24 (truncation < 4e-17).
// Every routine is __host__ __device__ so the host can test it against libm.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define PCV_HD __host__ __device__ __forceinline__
#else
#define PCV_HD inline
#endif

namespace pcv {
namespace dfm {

struct df {
    float h, l;
};

constexpr int kExpTable = 256;

PCV_HD df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

PCV_HD df fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}

PCV_HD df two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

PCV_HD df add(df a, df b) {
    const df s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + a.l + b.l);
}

PCV_HD df mul(df a, df b) {
    const df p = two_prod(a.h, b.h);
    return fast_two_sum(p.h, fmaf(a.h, b.l, fmaf(a.l, b.h, p.l)));
}

// a (double-float) from a double, and back
PCV_HD df from_double(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
PCV_HD double to_double(df a) { return (double)a.h + (double)a.l; }

// sqrt of a non-negative double-float: an approximate FP32 root s = a.h / sqrt(a.h)
// from the reciprocal square root, then one correction with the exact residual
// a - s^2 (FMA): s + (a - s^2) / (2 s).  The correction's own relative error (that of
// the approximate reciprocal, ~2^-22) multiplies a term of size ~2^-22 s, so the
// result carries ~44 correct bits.
PCV_HD df sqrt_df(df a) {
    if (!(a.h > 0.0f)) return {0.0f, 0.0f};
#if defined(__CUDA_ARCH__)
    const float r = rsqrtf(a.h);
#else
    const float r = 1.0f / std::sqrt(a.h);
#endif
    const float s = a.h * r;
    const float e = fmaf(-s, s, a.h) + a.l;
    return fast_two_sum(s, e * (0.5f * r));
}

// Accumulator for sums of double-float products (Ogita-Rump-Oishi style: the
// running sum's high part is kept error-free, the errors are summed in `l`).
struct acc {
    float h = 0.0f, l = 0.0f;
    PCV_HD void add_prod(df a, df b) {
        const df p = two_prod(a.h, b.h);
        const df s = two_sum(h, p.h);
        h = s.h;
        l += s.l + fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
    }
    PCV_HD void add_df(df a) {
        const df s = two_sum(h, a.h);
        h = s.h;
        l += s.l + a.l;
    }
    PCV_HD df value() const { return fast_two_sum(h, l); }
};

// 2^-n for 0 <= n <= 126
PCV_HD float pow2_neg(int n) {
#if defined(__CUDA_ARCH__)
    return __int_as_float((127 - n) << 23);
#else
    return std::ldexp(1.0f, -n);
#endif
}

// Constants of the exponential, filled on the host (see exp_constants below).
struct alignas(8) ExpConsts {
    float tbl[2 * kExpTable];  // 2^(-i/256) = tbl[2i] + tbl[2i+1]
    float inv_c;               // 256 / ln2 (rounded)
    float c1, c2, c3;          // ln2/256 = c1 + c2 + c3, c1 with 9 significant bits
};

// exp(-t) for a double-float t >= 0; 0 beyond t = 87 (below FLT_MIN territory).
// `tbl` must be 8-byte aligned on the device.
PCV_HD df exp_neg(df t, const float* tbl, float inv_c, float c1, float c2, float c3) {
    if (!(t.h < 87.0f)) return {0.0f, 0.0f};
    const float jf = rintf(t.h * inv_c);
    const int j = (int)jf;
    const float a = fmaf(-jf, c1, t.h);          // exact: j*c1 has <= 24 bits
    const df p2 = two_prod(jf, c2);              // j*c2 exactly
    df r = two_sum(a, -p2.h);
    r = two_sum(r.h, r.l - p2.l - jf * c3 + t.l);
    // exp(-r) = 1 + q,  q = -r + r^2/2 - r^3/6 + r^4/24
    const df rr = two_prod(r.h, r.h);
    const float q_h2 = 0.5f * rr.h;
    const float q_l2 = 0.5f * rr.l + r.h * r.l;
    const float c34 = r.h * rr.h * fmaf(r.h, 1.0f / 24.0f, -1.0f / 6.0f);
    df q = two_sum(-r.h, q_h2);
    q.l += q_l2 - r.l + c34;
    q = fast_two_sum(q.h, q.l);
    // table value times (1 + q)
    const int i = j & (kExpTable - 1);
    const int n = j >> 8;
#if defined(__CUDA_ARCH__)
    const float2 t2 = reinterpret_cast<const float2*>(tbl)[i];   // one 8-byte load
    const df T = {t2.x, t2.y};
#else
    const df T = {tbl[2 * i], tbl[2 * i + 1]};
#endif
    const df Tq = mul(T, q);
    df res = two_sum(T.h, Tq.h);
    res = fast_two_sum(res.h, res.l + T.l + Tq.l);
    // scale by 2^-n (n <= 125 here, so 2^-n is a normal float)
    const float sc = pow2_neg(n);
    return {res.h * sc, res.l * sc};
}

PCV_HD df exp_neg(df t, const ExpConsts& k) { return exp_neg(t, k.tbl, k.inv_c, k.c1, k.c2, k.c3); }

// Host-side constants: table by libm exp2 in double, ln2/256 split from a long
// double value of ln 2.
inline void exp_constants(ExpConsts& k) {
    for (int i = 0; i < kExpTable; ++i) {
        const double v = std::exp2(-(double)i / kExpTable);
        k.tbl[2 * i] = (float)v;
        k.tbl[2 * i + 1] = (float)(v - (double)k.tbl[2 * i]);
    }
    const long double ln2 = 0.693147180559945309417232121458176568L;
    const long double c = ln2 / kExpTable;
    const long double c1 = std::nearbyint(c * 131072.0L) / 131072.0L;   // 9 significant bits
    const long double rest = c - c1;
    k.c1 = (float)c1;
    k.c2 = (float)rest;
    k.c3 = (float)(rest - (long double)k.c2);
    k.inv_c = (float)(1.0L / c);
}

}  // namespace dfm
}  // namespace pcv
