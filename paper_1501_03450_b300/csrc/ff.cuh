// Compensated FP32 arithmetic: a value is an unevaluated sum hi + lo of two
// floats, about 48 significant bits.  Sums use the error-free two-sum,
// products the error-free FMA product (Dekker/Knuth transformations), so
// every operation is a short fixed sequence of FP32 instructions.
//
// Sums return a renormalised pair (|lo| <= ulp(hi)/2).  Products return the
// pair unrenormalised: hi = fl(a.hi b.hi) and lo = its exact rounding error
// plus the cross terms, |lo| <= about 2 ulp(hi).  Every operation here reads
// lo in full (two-sum of the high parts, then the low parts added before one
// renormalisation), so such a pair is as good an input as a renormalised one,
// and skipping the renormalisation saves three instructions per product.
#pragma once

#include <cuda_runtime.h>

namespace st {

struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_make(double x) {
    const float hi = (float)x;
    return FF{hi, (float)(x - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(const FF& a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// s + e = a + b exactly, for |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ FF ff_add(const FF& a, const FF& b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    FF r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ FF ff_add_f(const FF& a, float b) {
    float s, e;
    two_sum(a.hi, b, s, e);
    e += a.lo;
    FF r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ FF ff_neg(const FF& a) { return FF{-a.hi, -a.lo}; }

// Lazy sum for results that feed straight into ff_mul / ff_add (which read lo
// in full and renormalise): the rounding error goes into lo unnormalised.
__device__ __forceinline__ FF ff_add_lazy(const FF& a, const FF& b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return FF{s, e + (a.lo + b.lo)};
}
// a + b for a b proportional to a and much smaller (a relative correction):
// folded into lo; hi keeps carrying the value
__device__ __forceinline__ FF ff_addlo(const FF& a, float b) { return FF{a.hi, a.lo + b}; }
// a + b for a b small against ulp-scale of a.hi, or possibly larger when a
// nearly vanishes: folded into lo and renormalised, so that hi carries the
// value in every case (exact when |a.hi| >= |a.lo + b|)
__device__ __forceinline__ FF ff_addn(const FF& a, float b) {
    FF r;
    fast_two_sum(a.hi, a.lo + b, r.hi, r.lo);
    return r;
}
// a + b + c, c a small float term, renormalised once
__device__ __forceinline__ FF ff_add3(const FF& a, const FF& b, float c) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += (a.lo + b.lo) + c;
    FF r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

// a * b, unrenormalised (see the header)
__device__ __forceinline__ FF ff_mul(const FF& a, const FF& b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return FF{p, e};
}

__device__ __forceinline__ FF ff_mul_f(const FF& a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return FF{p, e};
}

// renormalised copy (|lo| <= ulp(hi)/2) of a pair whose lo is small against hi
__device__ __forceinline__ FF ff_norm(const FF& a) {
    FF r;
    fast_two_sum(a.hi, a.lo, r.hi, r.lo);
    return r;
}

// ---- two compensated values side by side, in Blackwell's packed FP32x2
// instructions (one instruction per pair of lanes' worth of work; the same
// rounding per component as the scalar operations) --------------------------
struct FF2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a - b, rounded once (the FMA by -1 is exact before its rounding)
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = __fadd2_rn(a, b);
    const float2 bp = f2_sub(s, a);
    e = __fadd2_rn(f2_sub(a, f2_sub(s, bp)), f2_sub(b, bp));
}

__device__ __forceinline__ FF2 ff2_add(const FF2& a, const FF2& b) {
    float2 s, e;
    two_sum2(a.hi, b.hi, s, e);
    e = __fadd2_rn(e, __fadd2_rn(a.lo, b.lo));
    FF2 r;
    r.hi = __fadd2_rn(s, e);
    r.lo = f2_sub(e, f2_sub(r.hi, s));
    return r;
}

// a * b, unrenormalised like ff_mul
__device__ __forceinline__ FF2 ff2_mul(const FF2& a, const FF2& b) {
    const float2 p = __fmul2_rn(a.hi, b.hi);
    float2 e = __ffma2_rn(a.hi, b.hi, f2_neg(p));
    e = __ffma2_rn(a.hi, b.lo, e);
    e = __ffma2_rn(a.lo, b.hi, e);
    return FF2{p, e};
}

__device__ __forceinline__ FF2 ff2_pack(const FF& x, const FF& y) {
    return FF2{make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)};
}
__device__ __forceinline__ FF ff2_first(const FF2& a) { return FF{a.hi.x, a.lo.x}; }
__device__ __forceinline__ FF ff2_second(const FF2& a) { return FF{a.hi.y, a.lo.y}; }

// a * b + c with a small float correction folded into the compensation word
__device__ __forceinline__ FF ff_fma(const FF& a, const FF& b, const FF& c) { return ff_add(ff_mul(a, b), c); }

}  // namespace st
