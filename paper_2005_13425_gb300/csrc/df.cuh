// Double-float ("float-float") arithmetic on the FP32 pipes.
//
// A value is an unevaluated pair (h, l) of floats, |l| <= ulp(h)/2, giving a
// 48-bit significand.  The building blocks are the classical error-free
// transformations: Knuth's TwoSum (the exact rounding error of a + b) and the
// FMA-based TwoProd (the exact rounding error of a * b), as used by Dekker
// (1971) and by Ogita, Rump and Oishi's compensated dot product Dot2 (2005).
// Every operation uses the explicit round-to-nearest intrinsics so the
// compiler can neither contract nor reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace nekgb {
namespace dfa {

// Compensated dot-product accumulator: s is the running FP32 sum, c the
// running sum of every rounding error (of the products and of the sums).
struct Acc {
    float s, c;
};

// TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float aa = __fsub_rn(s, bb);
    e = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
}

// acc = (xh + xl) * (yh + yl): exact product of the high parts plus the
// first-order cross terms (the xl*yl term is below the 48-bit precision).
__device__ __forceinline__ Acc first(float xh, float xl, float yh, float yl) {
    Acc a;
    a.s = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -a.s);
    e = __fmaf_rn(xh, yl, e);
    a.c = __fmaf_rn(xl, yh, e);
    return a;
}

// acc += (xh + xl) * (yh + yl)   (Dot2 step: TwoProd + TwoSum)
__device__ __forceinline__ void fma(Acc &a, float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    float s, err;
    two_sum(a.s, p, s, err);
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(err, e));
}

// Normalise (Fast2Sum, valid because |c| << |s|): returns (h, l).
__device__ __forceinline__ float2 norm(const Acc &a) {
    const float h = __fadd_rn(a.s, a.c);
    const float l = __fsub_rn(a.c, __fsub_rn(h, a.s));
    return make_float2(h, l);
}

// a + b for normalised pairs (accurate: TwoSum on the high parts).
__device__ __forceinline__ float2 add(float2 a, float2 b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, e);
    const float l = __fsub_rn(e, __fsub_rn(h, s));
    return make_float2(h, l);
}

// (P.s + P.c) + sgn*(Q.s + Q.c) as a normalised pair (sgn = +1 or -1;
// TwoSum on the leading parts, the compensations added after).
__device__ __forceinline__ float2 add_acc(const Acc &P, const Acc &Q, float sgn) {
    float s, e;
    two_sum(P.s, sgn * Q.s, s, e);
    e = __fadd_rn(e, __fadd_rn(P.c, sgn * Q.c));
    const float h = __fadd_rn(s, e);
    const float l = __fsub_rn(e, __fsub_rn(h, s));
    return make_float2(h, l);
}

// (P.s + P.c) + sgn*(Q.s + Q.c) as an unnormalised pair (s, e): the
// leading parts added by TwoSum, the compensations folded into e, without
// the final Fast2Sum.  |e| stays within a few ulps of s, which is all the
// consumers need (the cross terms of the next products, pair additions and
// the FP64 reassembly s + e are exact or accurate for such pairs); it saves
// three operations per value.
__device__ __forceinline__ float2 add_acc_raw(const Acc &P, const Acc &Q, float sgn) {
    float s, e;
    two_sum(P.s, sgn * Q.s, s, e);
    return make_float2(s, __fadd_rn(e, __fadd_rn(P.c, sgn * Q.c)));
}

// The accumulator (s, c) itself as an unnormalised pair (|c| is a few ulps
// of s at most), for the same consumers as add_acc_raw.
__device__ __forceinline__ float2 raw(const Acc &a) { return make_float2(a.s, a.c); }

// Compensated FP32 accumulation of products of floats (Dot2 on single
// values): s + c carries sum(a*b) to about 2^-47 relative, with FP32
// instructions only.  value() returns the FP64 total.
struct Acc32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);
        float t, err;
        two_sum(s, p, t, err);
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, e));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Compensated FP32 accumulation of weighted squares cw (h + l)^2 of pairs
// (cw a power of two): the product h^2 is exact (TwoProd), the cross term
// 2hl rides with its error, l^2 (below 2^-46 relative) is dropped.  Each
// term is accurate to about 2^-45 relative, the sum adds compensated; used
// for <r,r>_c on the FP32 pipes, where the FP64 pipe is the bottleneck.
struct SqAcc32 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add_sq(float h, float l, float cw) {
        const float hc = __fmul_rn(h, cw);                 // exact: cw = 2^-k
        const float p = __fmul_rn(hc, h);
        const float e = __fmaf_rn(hc, h, -p);              // exact rounding error of hc h
        const float x = __fmaf_rn(__fmul_rn(2.f, hc), l, e);
        float t, err;
        two_sum(s, p, t, err);
        s = t;
        c = __fadd_rn(c, __fadd_rn(err, x));
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Split a double into a normalised pair: h = fl32(x), l = fl32(x - h).
// x - h is exact in FP64, so h + l carries 48 bits of x.
__device__ __forceinline__ float2 split(double x) {
    const float h = __double2float_rn(x);
    const float l = __double2float_rn(x - (double)h);
    return make_float2(h, l);
}

// h + l is exact in FP64 for a normalised pair (at most 48 significant bits).
__device__ __forceinline__ double join(float2 v) { return (double)v.x + (double)v.y; }

// Pair of x * 2^sh built with integer operations only (no FP64 pipe): h
// holds the leading 24 significant bits of x (truncated), l the next 23
// (truncated), both with x's sign; |x*2^sh - (h + l)| < 2^-46 |x*2^sh|.
// Values whose scaled magnitude falls below 2^-126 become (0, 0): callers
// scale so that the data's maximum is in [1, 2), which makes that an
// absolute error below 2^-126 of the maximum.  With SAT, magnitudes at or
// above 2^128 after scaling become (+-inf, 0) (callers whose scale is an
// estimate); without it the caller guarantees they do not occur.
template <bool SAT = false>
__device__ __forceinline__ float2 split_scaled(double x, int sh) {
    const long long b = __double_as_longlong(x);
    const unsigned hi32 = (unsigned)((unsigned long long)b >> 32), lo32 = (unsigned)b;
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7ffu);
    const int ef = e - 1023 + sh + 127;                  // float exponent field of h
    if (e == 0 || ef < 1) return make_float2(0.f, 0.f);
    if (SAT && ef > 254) return make_float2(__uint_as_float(sign | 0x7f800000u), 0.f);
    const unsigned mh = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
    const float h = __uint_as_float(sign | ((unsigned)ef << 23) | mh);
    const int el = ef - 46;                              // exponent field of the unit 2^(e-1069+sh)
    float l = 0.f;
    if (el >= 1) {
        const unsigned k = (lo32 >> 6) & 0x7fffffu;      // next 23 bits as an integer
        const float kf = __fsub_rn(__uint_as_float(0x4b000000u | k), 8388608.0f);   // exactly k
        l = __uint_as_float(__float_as_uint(__fmul_rn(kf, __uint_as_float((unsigned)el << 23))) | sign);
    }
    return make_float2(h, l);
}

// f * 2^so as a double, built with integer operations (f normal or zero).
__device__ __forceinline__ double to_double_scaled(float f, int so) {
    const unsigned b = __float_as_uint(f);
    const int ef = (int)((b >> 23) & 0xffu);
    if (ef == 0) return 0.0;
    const long long ed = (long long)(ef - 127 + 1023 + so);
    if (ed <= 0) return 0.0;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if (ed >= 2047) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull));
    return __longlong_as_double(
        (long long)(sign | ((unsigned long long)ed << 52) | ((unsigned long long)(b & 0x7fffffu) << 29)));
}

// (h + l) * 2^so in FP64: one FP64 add (exact: the pair has <= 48 bits).
__device__ __forceinline__ double join_scaled(float2 v, int so) {
    return __dadd_rn(to_double_scaled(v.x, so), to_double_scaled(v.y, so));
}

}  // namespace dfa
}  // namespace nekgb
