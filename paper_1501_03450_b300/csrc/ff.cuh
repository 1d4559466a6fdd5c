// Compensated FP32 arithmetic: a value is an unevaluated sum hi + lo of two
// floats (|lo| <= ulp(hi)/2), about 48 significant bits.  Sums use the
// error-free two-sum, products the error-free FMA product (Dekker/Knuth
// transformations), so every operation is a short fixed sequence of FP32
// instructions.
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

__device__ __forceinline__ FF ff_mul(const FF& a, const FF& b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    FF r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ FF ff_mul_f(const FF& a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    FF r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// a * b + c with a small float correction folded into the compensation word
__device__ __forceinline__ FF ff_fma(const FF& a, const FF& b, const FF& c) { return ff_add(ff_mul(a, b), c); }

}  // namespace st
