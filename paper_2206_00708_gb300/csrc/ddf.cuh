// Double-float arithmetic on the FP32 pipe for the FP64 Arnoldi of the solvers: GB300's
// FP64 pipe runs at 1/64 of its FP32 pipe, so inner products and basis updates of FP64
// vectors run faster as exact FP32 transformations (the two-sum of Knuth, the
// two-product by FMA) on 24 + 24-bit splits of the FP64 values, with 2^-48 relative
// accuracy per product instead of 2^-53.  The vectors stay FP64 in memory.
#pragma once

#include <cuda_runtime.h>

namespace bem {
namespace ddf {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a double as hi + lo floats with integer operations only (no FP64 instruction):
// hi = its leading 24 significand bits (truncated), lo = the next 29 rounded to FP32,
// |a - hi - lo| <= 2^-48 |a|.  Magnitudes below 2^-100 or above 2^127 give 0 (vector
// entries of the Krylov process are far inside that range).
__device__ __forceinline__ void split(double a, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (e < -100 || e > 127) {
        hi = 0.0f;
        lo = 0.0f;
        return;
    }
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
    const unsigned rest = (unsigned)(m & 0x1FFFFFFFull);
    const float r = __uint2float_rn(rest) * 1.8626451492309570e-9f;  // 2^-29, exact
    const float sc = __uint_as_float((unsigned)(e - 23 + 127) << 23);
    lo = __uint_as_float(__float_as_uint(r * sc) | sign);
}

// the double of a float from its bits (zero and FP32 subnormals give 0)
__device__ __forceinline__ double widen(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    if (e == 0) return 0.0;
    const unsigned long long de = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | (de << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// (s, c) += (ah + al)(bh + bl): the leading product exactly, its cross terms rounded, al bl
// dropped (2^-48); the running error c collects every rounding error (the sum of Ogita,
// Rump and Oishi, "Accurate sum and dot product", 2005, in double-float form)
__device__ __forceinline__ void mac(float& s, float& c, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    float t;
    two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
}

// complex double-float value: (re_h, re_l, im_h, im_l)
__device__ __forceinline__ float4 split2(double2 a) {
    float4 r;
    split(a.x, r.x, r.y);
    split(a.y, r.z, r.w);
    return r;
}

// (S.x, S.y) re, (S.z, S.w) im accumulators += conj(a) b, or += a b
template <bool CONJ>
__device__ __forceinline__ void cmac(float4& S, const float4& a, const float4& b) {
    // re += ar br + (CONJ ? ai bi : -ai bi);  im += ar bi + (CONJ ? -ai br : ai br)
    mac(S.x, S.y, a.x, a.y, b.x, b.y);
    if (CONJ) mac(S.x, S.y, a.z, a.w, b.z, b.w);
    else mac(S.x, S.y, -a.z, -a.w, b.z, b.w);
    mac(S.z, S.w, a.x, a.y, b.z, b.w);
    if (CONJ) mac(S.z, S.w, -a.z, -a.w, b.x, b.y);
    else mac(S.z, S.w, a.z, a.w, b.x, b.y);
}

// (S) += (T): two double-float complex accumulators added (the running errors summed)
__device__ __forceinline__ void add(float4& S, const float4& T) {
    float t;
    two_sum(S.x, T.x, S.x, t);
    S.y = __fadd_rn(S.y, __fadd_rn(T.y, t));
    two_sum(S.z, T.z, S.z, t);
    S.w = __fadd_rn(S.w, __fadd_rn(T.w, t));
}

// the double2 value of an accumulator
__device__ __forceinline__ double2 value(const float4& S) {
    return make_double2(widen(S.x) + widen(S.y), widen(S.z) + widen(S.w));
}

}  // namespace ddf
}  // namespace bem
