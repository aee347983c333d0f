// Float-float arithmetic on the FP32 pipes.  This GPU's FP64 pipe issues at a
// small fraction of its FP32 rate, so the FP64 vector kernels keep their data
// in FP64 in memory but compute in pairs of floats (hi + lo, ~48 significant
// bits): doubles are split, and results recombined, with integer operations
// only, and products and sums carry their rounding errors (TwoProd, TwoSum).
#pragma once

#include <cstdint>

#include "helm_internal.h"

namespace helm {
namespace ffa {

struct ff {
    float hi, lo;
};

// x = hi + lo exactly up to the 5 lowest mantissa bits of x (48 of 53 bits
// kept); values below 2^-126 (and the low part below 2^-75) read as 0, which
// is far under anything these vectors hold.
__device__ __forceinline__ ff split_d(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hw = (unsigned int)(b >> 32);
    const unsigned int sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FF);
    const int ef = e - 1023 + 127;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e == 0x7FF) return {__uint_as_float(m ? 0x7FC00000u : (sign | 0x7F800000u)), 0.f};
    if (ef <= 0) return {0.f, 0.f};
    if (ef >= 255) return {__uint_as_float(sign | 0x7F800000u), 0.f};
    const float hi = __uint_as_float(sign | ((unsigned int)ef << 23) | (unsigned int)(m >> 29));
    const int es = e - 948;  // float exponent field of 2^(e - 1075), the weight of the low 29 bits
    float lo = 0.f;
    if (es > 0) lo = __uint2float_rn((unsigned int)(m & 0x1FFFFFFFull)) * __uint_as_float((unsigned int)es << 23);
    return {hi, sign ? -lo : lo};
}

// double -> float rounded to nearest (up to one unit where the low part's own
// rounding meets a tie), without the FP64 pipe
__device__ __forceinline__ float d2f(double x) {
    const ff s = split_d(x);
    return s.hi + s.lo;
}

// exact float -> double through the bits (zero and values below 2^-126 give
// a signed zero)
__device__ __forceinline__ double f2d(float f) {
    const unsigned int u = __float_as_uint(f);
    const unsigned int e = (u >> 23) & 0xFF;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if (e == 0) return __longlong_as_double((long long)sign);
    const unsigned long long ex = e == 0xFF ? 0x7FFull : (unsigned long long)(e - 127 + 1023);
    return __longlong_as_double((long long)(sign | (ex << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// hi + lo as a double, within one unit in the last place: TwoSum gives
// s = RN(hi + lo) and the exact rest e (|e| <= half an FP32 unit of s); e,
// counted in FP64 units of s (half units where s is a power of two and e
// points toward zero, where the binade below begins), is added to or taken
// from the bits of s, whose 29 low mantissa bits are zero, so that no carry or
// borrow leaves the binade except in that one case, which the half units
// account for.
__device__ __forceinline__ double join_d(ff a) {
    const float s = a.hi + a.lo;
    const float v = s - a.hi;
    const float e = (a.hi - (s - v)) + (a.lo - v);
    const unsigned int us = __float_as_uint(s), ue = __float_as_uint(e);
    const int es = (int)((us >> 23) & 0xFF), ee = (int)((ue >> 23) & 0xFF);
    if (es == 0 || es == 0xFF || ee == 0) return f2d(s);
    const bool toward0 = ((us ^ ue) & 0x80000000u) != 0;
    const bool pow2 = (us & 0x7FFFFFu) == 0;
    // |e| = me 2^(ee - 150); an FP64 unit of s is 2^(es - 179) (2^(es - 180) below a power of two)
    const int sh = ee - es + 29 + ((toward0 && pow2) ? 1 : 0);
    const unsigned int me = (ue & 0x7FFFFFu) | 0x800000u;
    const unsigned long long k =
        sh >= 0 ? ((unsigned long long)me << sh) : (sh > -32 ? (unsigned long long)(me >> (-sh)) : 0ull);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(f2d(s));
    return __longlong_as_double((long long)(toward0 ? bits - k : bits + k));
}

// s += p with p's rounding error carried into the low word (Knuth's TwoSum)
__device__ __forceinline__ void acc_add(ff& s, float p) {
    const float t = s.hi + p;
    const float v = t - s.hi;
    const float e = (s.hi - (t - v)) + (p - v);
    s.hi = t;
    s.lo += e;
}
// s += a * b for a, b float-float: the head product exactly (TwoProd), the
// cross terms and the tail into the low word
__device__ __forceinline__ void acc_mul(ff& s, ff a, ff b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    acc_add(s, p);
    s.lo += fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// a + b of two accumulators (tree reductions)
__device__ __forceinline__ ff ff_sum(ff a, ff b) {
    ff s = a;
    acc_add(s, b.hi);
    s.lo += b.lo;
    return s;
}
__device__ __forceinline__ ff shfl_down_ff(ff a, int o) {
    return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

// ---- complex vectors of the FP64 solver in two storage forms: complex128
// (the caller's arrays) and float-float (one float4 per entry: re.hi, re.lo,
// im.hi, im.lo; the Krylov work vectors), read and written as pairs of ff
struct cff {
    ff re, im;
};
__device__ __forceinline__ cff ld_c(const cplx<double>* p) {
    const cplx<double> v = *p;
    return {split_d(v.re), split_d(v.im)};
}
__device__ __forceinline__ cff ld_c(const float4* p) {
    const float4 v = *p;
    return {{v.x, v.y}, {v.z, v.w}};
}
// hi + lo renormalised (TwoSum): |lo| <= half a unit of hi, so that a later
// product may drop lo * lo
__device__ __forceinline__ ff ff_norm(ff a) {
    const float s = a.hi + a.lo;
    const float v = s - a.hi;
    return {s, (a.hi - (s - v)) + (a.lo - v)};
}
__device__ __forceinline__ void st_c(cplx<double>* p, cff v) { *p = mk<double>(join_d(v.re), join_d(v.im)); }
__device__ __forceinline__ void st_c(float4* p, cff v) {
    const ff r = ff_norm(v.re), i = ff_norm(v.im);
    *p = make_float4(r.hi, r.lo, i.hi, i.lo);
}

}  // namespace ffa
}  // namespace helm
