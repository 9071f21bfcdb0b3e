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

// a + s*b with one renormalisation
__device__ __forceinline__ dfloat df_fma(dfloat a, dfloat s, dfloat b) {
    const float ph = s.hi * b.hi;
    float pe = fmaf(s.hi, b.hi, -ph);
    pe = fmaf(s.hi, b.lo, pe);
    pe = fmaf(s.lo, b.hi, pe);
    float t, f;
    two_sum(a.hi, ph, t, f);
    f += pe + a.lo;
    float h, l;
    fast_two_sum(t, f, h, l);
    return dfloat(h, l);
}

// ---- float64 <-> float32 / double-float by integer operations ---------------
// GB300's float64 pipe also executes the float64 <-> float32 conversions, so
// the float32 and double-float kernels move values in and out of float64
// storage with bit manipulation (integer selects only):
//   f_bits:  the leading 24 significand bits of x as a float (truncated);
//   df_bits: hi = f_bits(x), lo = the next 23 bits, made a float exactly as
//            (2^23 + n) - 2^23 and scaled (x = hi + lo to 2^-46 relative);
//   d_bits:  exact widening of a float,
//   d_of:    d_bits(hi) + d_bits(lo), one exact float64 add.
// |x| < 2^-126 gives 0 (subnormal floats become 0), |x| >= 2^128 infinity,
// NaN stays NaN.
__device__ __forceinline__ unsigned f_bits_u(unsigned h32, unsigned l32) {
    const unsigned sgn = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu);
    const int fe = e - 1023 + 127;
    const unsigned hm = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    return fe >= 1 && fe <= 254 ? (sgn | ((unsigned)fe << 23) | hm)
         : fe <= 0 ? sgn
         : (sgn | 0x7f800000u | (e == 0x7ff && (hm | (l32 & 0x1fffffffu)) ? 0x400000u : 0u));
}
__device__ __forceinline__ float f_bits(double x) {
    return __uint_as_float(f_bits_u((unsigned)__double2hiint(x), (unsigned)__double2loint(x)));
}
__device__ __forceinline__ dfloat df_bits(double x) {
    const unsigned h32 = (unsigned)__double2hiint(x), l32 = (unsigned)__double2loint(x);
    const unsigned sgn = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu);
    const int fe = e - 1023 + 127;
    const float n = __uint_as_float(0x4b000000u | ((l32 & 0x1fffffffu) >> 6)) - 8388608.0f;
    const int le = e - 1069 + 127;                     // exponent of 2^(e - 1069)
    const float sc = __uint_as_float(le >= 1 ? (unsigned)le << 23 : 0u);
    const unsigned lb = fe >= 1 && fe <= 254 ? (__float_as_uint(n * sc) | sgn) : sgn;
    return dfloat(__uint_as_float(f_bits_u(h32, l32)), __uint_as_float(lb));
}
__device__ __forceinline__ double d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned sgn = u & 0x80000000u;
    const unsigned fe = (u >> 23) & 0xffu, fm = u & 0x7fffffu;
    const unsigned hi = fe == 0 ? sgn
                      : fe == 0xff ? (sgn | 0x7ff00000u | (fm ? 0x80000u : 0u))
                      : (sgn | ((fe + 1023 - 127) << 20) | (fm >> 3));
    const unsigned lo = (fe == 0 || fe == 0xff) ? 0u : (fm << 29);
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double d_of(dfloat a) { return d_bits(a.hi) + d_bits(a.lo); }
