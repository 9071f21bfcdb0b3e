// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// float32 numbers with |lo| <= ulp(hi)/2, about 48 significand bits.  The
// operations are the error-free transformations of Knuth (TwoSum), Dekker
// (FastTwoSum) and the fused multiply-add product error (TwoProd), as in
// Dekker (1971) and the double-double libraries built on them.  Additions
// use the "sloppy" variant (the errors of the two low parts are not summed
// separately): its error is bounded relative to |a| + |b|, which is the
// norm-wise bound an FFT needs.  Used by the TC_PREC_DF64 form, where the
// transforms and products run on the float32 pipe, which GB300 issues at 58x
// its float64 rate.
#pragma once
#include <cuda_runtime.h>

struct dfloat {
    float hi, lo;
    __host__ __device__ dfloat() : hi(0.0f), lo(0.0f) {}
    __host__ __device__ dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ dfloat(double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __host__ __device__ dfloat(int x) : dfloat((double)x) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

struct dcomplex {
    dfloat x, y;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly, for |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    float s, e, h, l;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    fast_two_sum(s, e, h, l);
    return dfloat(h, l);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);           // exact error of the leading product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float h, l;
    fast_two_sum(p, e, h, l);
    return dfloat(h, l);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { a = a + b; return a; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { a = a * b; return a; }

// a*b + sign*(c*d) with one renormalisation (complex products); sign = +-1
__device__ __forceinline__ dfloat df_dot2(dfloat a, dfloat b, dfloat c, dfloat d, float sign) {
    const float p = a.hi * b.hi;
    const float ep = fmaf(a.hi, b.hi, -p);     // a.hi b.hi = p + ep exactly
    const float q0 = c.hi * d.hi;
    const float eq0 = fmaf(c.hi, d.hi, -q0);   // c.hi d.hi = q0 + eq0 exactly
    float s, e;
    two_sum(p, sign * q0, s, e);
    e += ep + sign * eq0;
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    e = fmaf(sign * c.hi, d.lo, e);
    e = fmaf(sign * c.lo, d.hi, e);
    float h, l;
    fast_two_sum(s, e, h, l);
    return dfloat(h, l);
}
