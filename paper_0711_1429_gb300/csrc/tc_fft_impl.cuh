// Templates of the plane phase (z transforms, theta rows and products),
// instantiated per arithmetic type by tc_fft_f64.cu, tc_fft_f32.cu and
// tc_fft_df.cu, which compile in parallel.
#pragma once
// Plane phase: pseudo-spectral products of the velocity with the 3/2 rule.
//
// Paper: Fourier expansion in theta and z; the non-linear terms are those of
// the primitive-variable equations (Appendix, below Eq. 3), i.e. the six
// products uu, uv, uw, vv, vw, ww of the velocity.  They are formed in
// physical space on an Mt x Mz = (3 Ntheta/2) x (3 Nz/2) grid, which makes
// the quadratic products free of aliasing on the retained modes.
//
// Three kernels per substep:
//   k_zinv  : per (field, r, tile of C azimuthal columns): complex inverse
//             FFT in z, Nz retained slots zero-padded to Mz.
//   k_rows  : per (r, z-row): inverse real FFT in theta of u, v, w (packed as
//             u + i v and w), the products, forward real FFTs of the
//             products packed in pairs, truncation to the Nh retained columns.
//             The five transformed products are uu - vv, uv, uw, vw, ww - vv:
//             the isotropic part vv of the momentum flux is a pressure
//             gradient, which the pressure-free v and eta rows annihilate.
//   k_zfwd  : per (product, r, tile): forward complex FFT in z, truncation to
//             the Nz slots and scaling by 1/(Mt Mz).
// All transforms are mixed-radix Stockham FFTs in shared memory.  Float64:
// radix 3, then 4, then 2, with the stage twiddles in tangent form (fewer
// float64 instructions); float32 and double-float z columns: radix 3, 16,
// then 8, 4 or 2; axial lengths with odd prime factors add paired prime
// stages (5..17).
// Template parameter T is the arithmetic type: double, float (mixed form) or
// dfloat (double-float form).
#include "tc_internal.h"
#include "tc_dfloat.h"
#include <type_traits>

// threads per block of the paired theta rows (k_rows2)
#ifndef TC_ROWS2_THREADS
#define TC_ROWS2_THREADS 256
#endif

// float64 state -> arithmetic type of the transform; float and double-float
// through integer bit operations (the float64 pipe also does conversions)
template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return f_bits(x); }
template <> __device__ __forceinline__ dfloat from_f64<dfloat>(double x) { return df_bits(x); }

template <typename T> struct V2;
template <> struct V2<double> { typedef double2 t; };
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<dfloat> { typedef dcomplex t; };

// The threads of a block that work on one transform group (a z tile, or one
// theta row of a block that holds several): tid = 0 .. nth-1 within the group.
struct TG { int tid, nth; };
__device__ __forceinline__ TG tg_block() { return TG{(int)threadIdx.x, (int)blockDim.x}; }

template <typename C> __device__ __forceinline__ C c_add(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

// a * w (SIGN < 0) or a * conj(w) (SIGN > 0); w is a forward twiddle.
template <int SIGN, typename C> __device__ __forceinline__ C c_tw(C a, C w) {
    C r;
    if (SIGN < 0) { r.x = a.x * w.x - a.y * w.y; r.y = a.x * w.y + a.y * w.x; }
    else          { r.x = a.x * w.x + a.y * w.y; r.y = a.y * w.x - a.x * w.y; }
    return r;
}
// double-float complex products: one renormalisation per component
template <> __device__ __forceinline__ dcomplex c_tw<-1, dcomplex>(dcomplex a, dcomplex w) {
    dcomplex r;
    r.x = df_dot2(a.x, w.x, a.y, w.y, -1.0f);
    r.y = df_dot2(a.x, w.y, a.y, w.x, 1.0f);
    return r;
}
template <> __device__ __forceinline__ dcomplex c_tw<1, dcomplex>(dcomplex a, dcomplex w) {
    dcomplex r;
    r.x = df_dot2(a.x, w.x, a.y, w.y, 1.0f);
    r.y = df_dot2(a.y, w.x, a.x, w.y, -1.0f);
    return r;
}
// multiply by SIGN * i
template <int SIGN, typename C> __device__ __forceinline__ C c_si(C a) {
    C r;
    if (SIGN < 0) { r.x = a.y; r.y = -a.x; } else { r.x = -a.y; r.y = a.x; }
    return r;
}

// ---- butterflies ------------------------------------------------------------
// x * (re + i im) for a constant
template <typename C, typename T> __device__ __forceinline__ C c_mulc(C a, T re, T im) {
    C r;
    r.x = a.x * re - a.y * im;
    r.y = a.x * im + a.y * re;
    return r;
}
template <int SIGN, typename C> __device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
    C a0 = c_add(v0, v2), a1 = c_sub(v0, v2), a2 = c_add(v1, v3), a3 = c_si<SIGN>(c_sub(v1, v3));
    v0 = c_add(a0, a2); v1 = c_add(a1, a3); v2 = c_sub(a0, a2); v3 = c_sub(a1, a3);
}
// In-place R-point DFT X_k = sum_r v_r exp(SIGN 2 pi i r k/R); output k lands
// in v[dft_slot<R>(k)].
template <int R> __host__ __device__ constexpr int dft_slot(int k) { return R == 16 ? 4 * (k % 4) + k / 4 : k; }
template <int R, int SIGN, typename T, typename C> __device__ __forceinline__ void dft(C* v) {
    if constexpr (R == 2) {
        C a = c_add(v[0], v[1]), b = c_sub(v[0], v[1]);
        v[0] = a; v[1] = b;
    } else if constexpr (R == 3) {
        const T h = (T)0.5;
        const T s3 = (T)0.86602540378443864676;   // sin(2 pi/3)
        C sm = c_add(v[1], v[2]), df = c_sub(v[1], v[2]);
        C t0; t0.x = v[0].x - h * sm.x; t0.y = v[0].y - h * sm.y;
        C id = c_si<SIGN>(df); id.x *= s3; id.y *= s3;
        v[0] = c_add(v[0], sm);
        v[1] = c_add(t0, id);
        v[2] = c_sub(t0, id);
    } else if constexpr (R == 4) {
        dft4<SIGN>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        // even and odd halves, then X_k = E_k + w^k O_k, X_{k+4} = E_k - w^k O_k
        dft4<SIGN>(v[0], v[2], v[4], v[6]);
        dft4<SIGN>(v[1], v[3], v[5], v[7]);
        const T c = (T)0.70710678118654752440;   // cos(pi/4)
        const T sc = SIGN > 0 ? c : -c;
        C o1 = c_mulc(v[3], c, sc);              // w = exp(SIGN i pi/4)
        C o2 = c_si<SIGN>(v[5]);                 // w^2 = SIGN i
        C o3 = c_mulc(v[7], -c, sc);             // w^3
        C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
        v[0] = c_add(e0, o0); v[4] = c_sub(e0, o0);
        v[1] = c_add(e1, o1); v[5] = c_sub(e1, o1);
        v[2] = c_add(e2, o2); v[6] = c_sub(e2, o2);
        v[3] = c_add(e3, o3); v[7] = c_sub(e3, o3);
    } else {   // R == 16: 4 x 4 with internal twiddles exp(SIGN 2 pi i j k/16)
        #pragma unroll
        for (int j = 0; j < 4; ++j) dft4<SIGN>(v[j], v[j + 4], v[j + 8], v[j + 12]);
        const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;   // pi/8
        const T c2 = (T)0.70710678118654752440;
        const T sg = SIGN > 0 ? (T)1 : (T)-1;
        // element j + 4 k1 holds Y_j[k1]; multiply by w16^(j k1)
        v[5] = c_mulc(v[5], c1, sg * s1);            // j=1,k1=1: e=1
        v[9] = c_mulc(v[9], c2, sg * c2);            // j=1,k1=2: e=2
        v[13] = c_mulc(v[13], s1, sg * c1);          // j=1,k1=3: e=3
        v[6] = c_mulc(v[6], c2, sg * c2);            // j=2,k1=1: e=2
        v[10] = c_si<SIGN>(v[10]);                   // j=2,k1=2: e=4
        v[14] = c_mulc(v[14], -c2, sg * c2);         // j=2,k1=3: e=6
        v[7] = c_mulc(v[7], s1, sg * c1);            // j=3,k1=1: e=3
        v[11] = c_mulc(v[11], -c2, sg * c2);         // j=3,k1=2: e=6
        v[15] = c_mulc(v[15], -c1, -sg * s1);        // j=3,k1=3: e=9
        #pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    }
}

// One Stockham butterfly: reads src[j + r M/R], twiddles by
// exp(SIGN 2 pi i r (j mod Ns)/(Ns R)), R-point DFT, writes
// dst[(j/Ns) Ns R + (j mod Ns) + r Ns].
// sh: element stride 2^sh (interleaved columns of the z tiles; 0 for a
// contiguous column).
template <int R, int SIGN, typename T, typename C>
__device__ __forceinline__ void stockham_bfly(const C* sc, C* dcol, int j, int nb, int Ns, const C* tws, int sh = 0) {
    C v[R];
    const int jm = j % Ns;
    #pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sc[(j + r * nb) << sh];
    if (Ns > 1) {
        const C* t = tws + jm * (R - 1);
        #pragma unroll
        for (int r = 1; r < R; ++r) v[r] = c_tw<SIGN>(v[r], t[r - 1]);
    }
    dft<R, SIGN, T>(v);
    C* dc = dcol + (((j / Ns) * Ns * R + jm) << sh);
    #pragma unroll
    for (int r = 0; r < R; ++r) dc[(r * Ns) << sh] = v[dft_slot<R>(r)];
}

// Float64 Stockham butterfly of radix 2, 3 or 4 with the stage twiddles in
// tangent form: w_r = k_r (1 + i tau_r), so v_r w_r = k_r u_r with
// u_r = v_r (1 + i tau_r) (conjugate for the inverse), two fused
// multiply-adds, and the factors k_r are carried by the multiply-adds of the
// butterfly itself (k_3 = rho k_1 for radix 4, k_2 = rho k_1 for radix 3).
// Radix 4 then takes 22 multiply-adds instead of 6 multiplies, 6
// multiply-adds and 16 adds; radix 3 takes 16 instead of 22.  Table layout
// per jm as built on the host (tangent_twiddles).
template <int R> __host__ __device__ constexpr int tan_entries() { return R == 2 ? 2 : 6; }
// With SKIP1 (radix 3 only) output r = 1 is not written: the last stage of a
// transform whose middle band of outputs is never read.
template <int R, int SIGN, bool SKIP1 = false>
__device__ __forceinline__ void stockham_bfly_tan(const double2* sc, double2* dcol, int j, int nb, int Ns,
                                                  const double* __restrict__ tw, int sh = 0) {
    static_assert(!SKIP1 || R == 3, "only the radix-3 butterfly skips an output");
    const int jm = j % Ns;
    double2 v[R];
    #pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sc[(j + r * nb) << sh];
    const double* t = tw + jm * tan_entries<R>();
    auto tang = [](double2 a, double tau) {
        const double s = SIGN < 0 ? tau : -tau;
        return make_double2(fma(-s, a.y, a.x), fma(s, a.x, a.y));
    };
    double2* dc = dcol + (((j / Ns) * Ns * R + jm) << sh);
    const int o1 = Ns << sh, o2 = (2 * Ns) << sh, o3 = (3 * Ns) << sh;
    if constexpr (R == 2) {
        const double2 u1 = tang(v[1], t[0]);
        const double k1 = t[1];
        dc[0] = make_double2(fma(k1, u1.x, v[0].x), fma(k1, u1.y, v[0].y));
        dc[o1] = make_double2(fma(-k1, u1.x, v[0].x), fma(-k1, u1.y, v[0].y));
    } else if constexpr (R == 3) {
        const double2 u1 = tang(v[1], t[0]), u2 = tang(v[2], t[1]);
        const double rho = t[2], k1 = t[3], hk = t[4], sk = SIGN < 0 ? t[5] : -t[5];
        const double2 b = make_double2(fma(rho, u2.x, u1.x), fma(rho, u2.y, u1.y));
        const double2 bm = make_double2(fma(-rho, u2.x, u1.x), fma(-rho, u2.y, u1.y));
        const double2 t0 = make_double2(fma(-hk, b.x, v[0].x), fma(-hk, b.y, v[0].y));
        dc[0] = make_double2(fma(k1, b.x, v[0].x), fma(k1, b.y, v[0].y));
        if constexpr (!SKIP1) dc[o1] = make_double2(fma(sk, bm.y, t0.x), fma(-sk, bm.x, t0.y));
        dc[o2] = make_double2(fma(-sk, bm.y, t0.x), fma(sk, bm.x, t0.y));
    } else {
        const double2 u1 = tang(v[1], t[0]), u2 = tang(v[2], t[1]), u3 = tang(v[3], t[2]);
        const double k1 = t[3], k2 = t[4], rho = t[5];
        const double ks = SIGN < 0 ? k1 : -k1;
        const double2 a0 = make_double2(fma(k2, u2.x, v[0].x), fma(k2, u2.y, v[0].y));
        const double2 a1 = make_double2(fma(-k2, u2.x, v[0].x), fma(-k2, u2.y, v[0].y));
        const double2 b = make_double2(fma(rho, u3.x, u1.x), fma(rho, u3.y, u1.y));
        const double2 bm = make_double2(fma(-rho, u3.x, u1.x), fma(-rho, u3.y, u1.y));
        dc[0] = make_double2(fma(k1, b.x, a0.x), fma(k1, b.y, a0.y));
        dc[o2] = make_double2(fma(-k1, b.x, a0.x), fma(-k1, b.y, a0.y));
        dc[o1] = make_double2(fma(ks, bm.y, a1.x), fma(-ks, bm.x, a1.y));
        dc[o3] = make_double2(fma(-ks, bm.y, a1.x), fma(ks, bm.x, a1.y));
    }
}

// Odd prime radix R (5, 7, 11, 13, 17).  With w = exp(SIGN 2 pi i/R) and
// h = (R-1)/2, the inputs pair up as a_j = v_j + v_(R-j), b_j = v_j - v_(R-j)
// (j = 1..h), and for k = 1..h
//   X_k     = v_0 + sum_j a_j cos(2 pi j k/R) + SIGN i sum_j b_j sin(2 pi j k/R),
//   X_(R-k) = the same with the sine sum subtracted,
// since v_j w^(jk) + v_(R-j) w^(-jk) = a_j cos + SIGN i b_j sin.  That takes
// about 4 h^2 real multiply-adds per butterfly instead of 4 (R-1)^2 for the
// direct sum.  The roots (cos, -sin)(2 pi e/R) follow the stage's twiddles.
template <typename C, typename T> __device__ __forceinline__ C c_axpy_r(C acc, T s, C a) {
    acc.x = acc.x + s * a.x;
    acc.y = acc.y + s * a.y;
    return acc;
}
template <int R, int SIGN, typename T, typename C>
__device__ __noinline__ void stockham_bfly_odd(const C* sc, C* dcol, int j, int nb, int Ns, const C* tws, int sh) {
    constexpr int H = (R - 1) / 2;
    C v[R];
    const int jm = j % Ns;
    #pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sc[(j + r * nb) << sh];
    if (Ns > 1) {
        const C* t = tws + jm * (R - 1);
        #pragma unroll
        for (int r = 1; r < R; ++r) v[r] = c_tw<SIGN>(v[r], t[r - 1]);
    }
    const C* roots = tws + Ns * (R - 1);
    C x0 = v[0];
    #pragma unroll
    for (int q = 1; q <= H; ++q) {
        const C a = c_add(v[q], v[R - q]), b = c_sub(v[q], v[R - q]);
        v[q] = a;
        v[R - q] = b;
        x0 = c_add(x0, a);
    }
    C* dc = dcol + (((j / Ns) * Ns * R + jm) << sh);
    dc[0] = x0;
    #pragma unroll
    for (int k = 1; k <= H; ++k) {
        C p = v[0], s;
        #pragma unroll
        for (int q = 1; q <= H; ++q) {
            const C w = roots[(q * k) % R];          // (cos, -sin)(2 pi q k/R)
            p = c_axpy_r(p, w.x, v[q]);
            if (q == 1) { s.x = -w.y * v[R - q].x; s.y = -w.y * v[R - q].y; }
            else        s = c_axpy_r(s, -w.y, v[R - q]);
        }
        const C is = c_si<SIGN>(s);
        dc[(k * Ns) << sh] = c_add(p, is);
        dc[((R - k) * Ns) << sh] = c_sub(p, is);
    }
}
template <int SIGN, typename T, typename C>
__device__ __forceinline__ void stockham_bfly_prime(const C* sc, C* dcol, int j, int nb, int Ns, int R, const C* tws,
                                                    int sh) {
    switch (R) {
        case 5: stockham_bfly_odd<5, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh); break;
        case 7: stockham_bfly_odd<7, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh); break;
        case 11: stockham_bfly_odd<11, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh); break;
        case 13: stockham_bfly_odd<13, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh); break;
        default: stockham_bfly_odd<17, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh); break;
    }
}

// ncols transforms of length pl.M stored contiguously in buf0 (column c at
// c*M), with the plan chosen at run time.  Returns the buffer holding the
// result (buf0 or buf1).
// IL: the ncols columns are interleaved (element i of column c at
// i ncols + c, ncols a power of two), else contiguous (column c at c M).
template <typename T, int SIGN, int F = 1, bool IL = false>
__device__ typename V2<T>::t* fft_stockham(const TG tg, typename V2<T>::t* buf0, typename V2<T>::t* buf1,
                                           int ncols, const FftPlan& pl,
                                           const typename V2<T>::t* __restrict__ tw) {
    typedef typename V2<T>::t C;
    C* src = buf0;
    C* dst = buf1;
    const int M = pl.M;
    const int sh = IL ? __ffs(ncols) - 1 : 0;
    for (int s = 0; s < pl.nst; ++s) {
        const int R = pl.R[s], Ns = pl.Ns[s];
        const int nb = M / R;
        const C* tws = tw + pl.twoff[s];
        for (int b = tg.tid; b < ncols * nb; b += tg.nth) {
            int col, j;
            if constexpr (IL) { col = b & (ncols - 1); j = b >> sh; }
            else { col = b / nb; j = b - col * nb; }
            const C* sc = src + (IL ? col : col * M);
            C* dcol = dst + (IL ? col : col * M);
            // family 0 plans use radices 2, 3, 4 only: instantiating only
            // those keeps the register demand of the theta kernels low
            if (R == 3) stockham_bfly<3, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh);
            else if (R == 4) stockham_bfly<4, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh);
            else if (R == 2) stockham_bfly<2, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh);
            else if (F >= 1 && R == 8) {
                if constexpr (F >= 1) stockham_bfly<8, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh);
            } else if (F >= 1 && R == 16) {
                if constexpr (F >= 1) stockham_bfly<16, SIGN, T>(sc, dcol, j, nb, Ns, tws, sh);
            } else if constexpr (F == 2) {
                // odd prime stages: only in the kernels instantiated for axial
                // lengths with factors 5..17 (their register demand is higher)
                stockham_bfly_prime<SIGN, T>(sc, dcol, j, nb, Ns, R, tws, sh);
            }
        }
        __syncthreads();
        C* t = src; src = dst; dst = t;
    }
    return src;
}

// ---- compile-time plans ------------------------------------------------------
// The same mixed-radix plans as on the host (families below; twiddle offsets
// as on the host) with the length known at compile time: every division by
// the stage constants becomes a multiply-shift and the stage loop unrolls.
// Family 0 (theta rows, few columns per block: many small butterflies):
// radix-3 stages, then 4, then 2.  Family 1 (z columns, many columns per
// block): radix-3 stages, then 16, then one stage of 8, 4 or 2.  Family 3
// (float64 forward z transforms): radix 4, then 2, then the radix-3 stages
// last, so that the last stage writes the outputs in three bands of M/3 and
// a truncated transform can skip the middle band (see k_zfwd).
__host__ __device__ constexpr int plan_radix_f(int M, int s, int F) {
    int i = 0;
    if (F == 3) {
        while (M % 4 == 0) { if (i == s) return 4; M /= 4; ++i; }
        while (M % 2 == 0) { if (i == s) return 2; M /= 2; ++i; }
        while (M % 3 == 0) { if (i == s) return 3; M /= 3; ++i; }
        return 1;
    }
    while (M % 3 == 0) { if (i == s) return 3; M /= 3; ++i; }
    if (F == 0) {
        while (M % 4 == 0) { if (i == s) return 4; M /= 4; ++i; }
        while (M % 2 == 0) { if (i == s) return 2; M /= 2; ++i; }
        return 1;
    }
    while (M % 16 == 0) { if (i == s) return 16; M /= 16; ++i; }
    return (i == s) ? M : 1;     // the one remainder stage (8, 4, 2), or none
}
__host__ __device__ constexpr int plan_nst_f(int M, int F) {
    int n = 0;
    while (plan_radix_f(M, n, F) > 1) ++n;
    return n;
}
__host__ __device__ constexpr int plan_ns_f(int M, int s, int F) {
    int ns = 1;
    for (int i = 0; i < s; ++i) ns *= plan_radix_f(M, i, F);
    return ns;
}
__host__ __device__ constexpr int plan_off_f(int M, int s, int F) {
    int o = 0;
    for (int i = 0; i < s; ++i) o += plan_ns_f(M, i, F) * (plan_radix_f(M, i, F) - 1);
    return o;
}

__host__ __device__ constexpr int plan_tan_off(int M, int s, int F = 0) {
    int o = 0;
    for (int i = 0; i < s; ++i) o += plan_ns_f(M, i, F) * (plan_radix_f(M, i, F) == 2 ? 2 : 6);
    return o;
}

// First radix-3 stage (Ns = 1, no twiddles) of an inverse transform whose
// input is a spectrum zero-padded by the 3/2 rule: input j + M/3 lies in the
// zero band for every j < M/3, so the butterfly skips it.  With v1 = 0 the
// radix-3 sums are bit for bit those of the full butterfly.
template <int SIGN, typename T, typename C>
__device__ __forceinline__ void stockham_bfly3_zero_mid(const C* sc, C* dcol, int j, int nb, int sh = 0) {
    const T h = (T)0.5;
    const T s3 = (T)0.86602540378443864676;   // sin(2 pi/3)
    const C v0 = sc[j << sh], v2 = sc[(j + 2 * nb) << sh];
    C t0; t0.x = v0.x - h * v2.x; t0.y = v0.y - h * v2.y;
    C id = c_si<SIGN>(v2); id.x *= s3; id.y *= s3;   // SIGN i s3 v2 = -(SIGN i s3 (0 - v2))
    C* dc = dcol + ((3 * j) << sh);
    dc[0] = c_add(v0, v2);
    dc[1 << sh] = c_sub(t0, id);
    dc[2 << sh] = c_add(t0, id);
}

template <typename T, int SIGN, int M, int F, int S, bool Z0 = false, bool IL = false>
__device__ __forceinline__ typename V2<T>::t* fft_fixed_stage(const TG tg, typename V2<T>::t* src, typename V2<T>::t* dst,
                                                              int ncols, const typename V2<T>::t* __restrict__ tw,
                                                              const double* __restrict__ twtan) {
    typedef typename V2<T>::t C;
    static_assert(F != 3 || std::is_same<T, double>::value, "family 3 has float64 tangent twiddles only");
    if constexpr (S == plan_nst_f(M, F)) {
        return src;
    } else {
        constexpr int R = plan_radix_f(M, S, F);
        constexpr int Ns = plan_ns_f(M, S, F);
        constexpr int nb = M / R;
        const C* tws = tw + plan_off_f(M, S, F);
        const int sh = IL ? __ffs(ncols) - 1 : 0;
        for (int b = tg.tid; b < ncols * nb; b += tg.nth) {
            int col, j;
            if constexpr (IL) { col = b & (ncols - 1); j = b >> sh; }
            else { col = b / nb; j = b - col * nb; }
            const C* sc = src + (IL ? col : col * M);
            C* dc = dst + (IL ? col : col * M);
            if constexpr (Z0 && S == 0 && R == 3)
                stockham_bfly3_zero_mid<SIGN, T>(sc, dc, j, nb, sh);
            else if constexpr (F == 3 && S + 1 == plan_nst_f(M, F))   // last stage, radix 3: skip band 1
                stockham_bfly_tan<R, SIGN, true>(sc, dc, j, nb, Ns, twtan + plan_tan_off(M, S, F), sh);
            else if constexpr (std::is_same<T, double>::value && (F == 0 || F == 3) && Ns > 1)
                stockham_bfly_tan<R, SIGN>(sc, dc, j, nb, Ns, twtan + plan_tan_off(M, S, F), sh);
            else
                stockham_bfly<R, SIGN, T>(sc, dc, j, nb, Ns, tws, sh);
        }
        __syncthreads();
        return fft_fixed_stage<T, SIGN, M, F, S + 1, Z0, IL>(tg, dst, src, ncols, tw, twtan);
    }
}


// Dispatch on the transform length: compile-time plans for the lengths of
// the supported grids (those of tc_fft_fixed_length), the run-time plan
// otherwise (same arithmetic).
// Z0: the input is a 3/2-padded spectrum (middle third zero), which the
// first stage of the compile-time plans skips.  Families 0 and 3 of the
// float64 z transforms are launched only for lengths with a compile-time
// plan (the host checks tc_fft_fixed_length).
template <typename T, int SIGN, int F, bool Z0 = false, bool IL = false>
__device__ typename V2<T>::t* fft(const TG tg, typename V2<T>::t* buf0, typename V2<T>::t* buf1, int ncols,
                                  const FftPlan& pl, const typename V2<T>::t* __restrict__ tw,
                                  const double* __restrict__ twtan = nullptr) {
#define TC_FFT_CASE(MM) case MM: return fft_fixed_stage<T, SIGN, MM, F, 0, Z0, IL>(tg, buf0, buf1, ncols, tw, twtan);
    if constexpr (F == 2) {
        return fft_stockham<T, SIGN, 2, IL>(tg, buf0, buf1, ncols, pl, tw);
    } else {
        switch (pl.M) {
            TC_FFT_CASE(12) TC_FFT_CASE(18) TC_FFT_CASE(24) TC_FFT_CASE(36) TC_FFT_CASE(48)
            TC_FFT_CASE(72) TC_FFT_CASE(96) TC_FFT_CASE(144) TC_FFT_CASE(192) TC_FFT_CASE(288)
            TC_FFT_CASE(384) TC_FFT_CASE(576) TC_FFT_CASE(768) TC_FFT_CASE(1152) TC_FFT_CASE(1536)
            default: return fft_stockham<T, SIGN, (F == 3 ? 0 : F), IL>(tg, buf0, buf1, ncols, pl, tw);
        }
    }
#undef TC_FFT_CASE
}

// Two transforms of one plan family (theta rows: the full length M1 and the
// half length M2) advanced stage by stage in one loop, one barrier per
// stage for both; each keeps its own plan, twiddles and ping-pong pair.  On
// return a_res / b_res hold the buffers with the results.
// F: plan family of this transform (0, or 3 for a float64 full-length
// forward transform whose middle band of outputs is not read).
template <typename T, int SIGN, int M, int S, bool Z0 = false, int F = 0>
__device__ __forceinline__ void pair_bfly(typename V2<T>::t* src, typename V2<T>::t* dst, int j,
                                          const typename V2<T>::t* __restrict__ tw,
                                          const double* __restrict__ twtan) {
    static_assert(F == 0 || (F == 3 && std::is_same<T, double>::value), "family 3 is float64 only");
    constexpr int R = plan_radix_f(M, S, F);
    constexpr int Ns = plan_ns_f(M, S, F);
    constexpr int nb = M / R;
    if constexpr (Z0 && S == 0 && R == 3)
        stockham_bfly3_zero_mid<SIGN, T>(src, dst, j, nb);
    else if constexpr (F == 3 && S + 1 == plan_nst_f(M, F))   // last stage, radix 3: skip band 1
        stockham_bfly_tan<R, SIGN, true>(src, dst, j, nb, Ns, twtan + plan_tan_off(M, S, F));
    else if constexpr (std::is_same<T, double>::value && Ns > 1)
        stockham_bfly_tan<R, SIGN>(src, dst, j, nb, Ns, twtan + plan_tan_off(M, S, F));
    else
        stockham_bfly<R, SIGN, T>(src, dst, j, nb, Ns, tw + plan_off_f(M, S, F));
}
template <typename T, int SIGN, int M1, int M2, int S, bool Z0A = false, int FA = 0>
__device__ __forceinline__ void fft_pair_stage(const TG tg, typename V2<T>::t* a0, typename V2<T>::t* a1,
                                               typename V2<T>::t* b0, typename V2<T>::t* b1,
                                               typename V2<T>::t*& a_res, typename V2<T>::t*& b_res, int na,
                                               const typename V2<T>::t* __restrict__ tw1, const double* __restrict__ tt1,
                                               const typename V2<T>::t* __restrict__ tw2, const double* __restrict__ tt2) {
    constexpr int n1 = plan_nst_f(M1, FA), n2 = plan_nst_f(M2, 0);
    if constexpr (S >= n1 && S >= n2) {
        a_res = a0;
        b_res = b0;
    } else {
        constexpr bool A = S < n1, B = S < n2;
        constexpr int nb1 = A ? M1 / plan_radix_f(M1, S, FA) : 0;
        constexpr int nb2 = B ? M2 / plan_radix_f(M2, S, 0) : 0;
        const int nA = A ? na * nb1 : 0;
        for (int b = tg.tid; b < nA + nb2; b += tg.nth) {
            if constexpr (A) {
                if (b < nA) {
                    const int col = b / nb1;
                    pair_bfly<T, SIGN, M1, (A ? S : 0), Z0A, FA>(a0 + col * M1, a1 + col * M1, b - col * nb1, tw1, tt1);
                    continue;
                }
            }
            if constexpr (B) pair_bfly<T, SIGN, M2, (B ? S : 0)>(b0, b1, b - nA, tw2, tt2);
        }
        __syncthreads();
        fft_pair_stage<T, SIGN, M1, M2, S + 1, Z0A, FA>(tg, A ? a1 : a0, A ? a0 : a1, B ? b1 : b0, B ? b0 : b1,
                                                        a_res, b_res, na, tw1, tt1, tw2, tt2);
    }
}
// Full-length (plan p1, na contiguous columns) and half-length (plan p2,
// one column) transforms together when FUSE is set and both lengths have
// compile-time plans, else one after the other.  FA: plan family of the
// full-length transform (tt1 then holds that family's tangent twiddles;
// p1 and tw1 stay the family-0 plan, used only where a length has no
// compile-time plan).
template <typename T, int SIGN, bool FUSE, bool Z0A = false, int FA = 0>
__device__ void fft_pair(const TG tg, typename V2<T>::t* a0, typename V2<T>::t* a1, typename V2<T>::t* b0, typename V2<T>::t* b1,
                         typename V2<T>::t*& a_res, typename V2<T>::t*& b_res, int na,
                         const FftPlan& p1, const typename V2<T>::t* __restrict__ tw1, const double* __restrict__ tt1,
                         const FftPlan& p2, const typename V2<T>::t* __restrict__ tw2, const double* __restrict__ tt2) {
#define TC_PAIR_CASE(MM) case MM: if (p2.M == MM / 2) { fft_pair_stage<T, SIGN, MM, MM / 2, 0, Z0A, FA>(tg, a0, a1, b0, b1, a_res, b_res, na, tw1, tt1, tw2, tt2); return; } break;
    if constexpr (FUSE) {
        switch (p1.M) {
            TC_PAIR_CASE(24) TC_PAIR_CASE(36) TC_PAIR_CASE(48) TC_PAIR_CASE(72) TC_PAIR_CASE(96)
            TC_PAIR_CASE(144) TC_PAIR_CASE(192) TC_PAIR_CASE(288) TC_PAIR_CASE(384) TC_PAIR_CASE(576)
            TC_PAIR_CASE(768) TC_PAIR_CASE(1152) TC_PAIR_CASE(1536)
            default: break;
        }
    }
#undef TC_PAIR_CASE
    a_res = fft<T, SIGN, FA, Z0A>(tg, a0, a1, na, p1, tw1, tt1);
    b_res = fft<T, SIGN, 0>(tg, b0, b1, 1, p2, tw2, tt2);
}

// z twiddles of the plan the kernel runs: pz (family 1) or pz0 (family 0).
// Float64 kernels of families 0 and 3 read their tangent tables (twz_tan,
// twz3_tan) instead, and never the table returned here.
template <typename T, int ZF> __device__ __forceinline__ const typename V2<T>::t* twz_of(const TcDev& d);
template <typename T> __device__ __forceinline__ const typename V2<T>::t* twz(const TcDev& d);
template <> __device__ __forceinline__ const dcomplex* twz<dfloat>(const TcDev& d) { return reinterpret_cast<const dcomplex*>(d.twz_x); }
template <> __device__ __forceinline__ const double2* twz<double>(const TcDev& d) { return d.twz_d; }
template <> __device__ __forceinline__ const float2* twz<float>(const TcDev& d) { return d.twz_f; }
template <typename T, int ZF> __device__ __forceinline__ const typename V2<T>::t* twz_of(const TcDev& d) {
    if constexpr (ZF != 0) return twz<T>(d);
    else if constexpr (std::is_same<T, float>::value) return d.twz0_f;
    else if constexpr (std::is_same<T, dfloat>::value) return reinterpret_cast<const dcomplex*>(d.twz0_x);
    else return twz<T>(d);
}
template <typename T> __device__ __forceinline__ const typename V2<T>::t* twt(const TcDev& d);
template <> __device__ __forceinline__ const dcomplex* twt<dfloat>(const TcDev& d) { return reinterpret_cast<const dcomplex*>(d.twt_x); }
template <> __device__ __forceinline__ const double2* twt<double>(const TcDev& d) { return d.twt_d; }
template <> __device__ __forceinline__ const float2* twt<float>(const TcDev& d) { return d.twt_f; }
template <typename T> __device__ __forceinline__ const typename V2<T>::t* twh(const TcDev& d);
template <> __device__ __forceinline__ const dcomplex* twh<dfloat>(const TcDev& d) { return reinterpret_cast<const dcomplex*>(d.twh_x); }
template <> __device__ __forceinline__ const double2* twh<double>(const TcDev& d) { return d.twh_d; }
template <> __device__ __forceinline__ const float2* twh<float>(const TcDev& d) { return d.twh_f; }
template <typename T> __device__ __forceinline__ const typename V2<T>::t* twr(const TcDev& d);
template <> __device__ __forceinline__ const dcomplex* twr<dfloat>(const TcDev& d) { return reinterpret_cast<const dcomplex*>(d.twr_x); }
template <> __device__ __forceinline__ const double2* twr<double>(const TcDev& d) { return d.twr_d; }
template <> __device__ __forceinline__ const float2* twr<float>(const TcDev& d) { return d.twr_f; }


// ---- k_zinv: spectral (u, v, w) -> zbuf[f][r][q][j] ---------------------------
// ZF = 0: float64 with the radix-3/4/2 plan pz0 and tangent-form twiddles
// (compile-time lengths only); ZF = 1: axial lengths 2^a 3^b; ZF = 2:
// lengths with odd prime factors.
// Block (bx, r, f): z tile bx + tile0 of radial plane r, field f.
template <typename T, int ZF>
__device__ __forceinline__ void zinv_body(const TcDev& d, const double2* __restrict__ f0,
                                          const double2* __restrict__ f1, const double2* __restrict__ f2,
                                          int tile0, int bx, int r, int f) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    const int ct = d.ztile;
    const int lct = __ffs(ct) - 1;          // the z tile is 1, 2, 4 or 8 columns
    C* buf1 = buf0 + ct * d.Mz;
    const int j0 = (bx + tile0) * ct;
    const double2* src = f == 0 ? f0 : (f == 1 ? f1 : f2);
    const int Mz = d.Mz, Nz = d.Nz, Nh = d.Nh;
    // the ct columns interleaved in shared memory (element q of column c at
    // q ct + c = idx): the global rows and the shared tile are both read and
    // written in order, without bank conflicts
    for (int idx = threadIdx.x; idx < ct * Mz; idx += blockDim.x) {
        const int q = idx >> lct, c = idx & (ct - 1);
        int s = -1;
        if (q < Nz / 2) s = q;
        else if (q > Mz - Nz / 2) s = Nz - (Mz - q);
        C val; val.x = 0; val.y = 0;
        if (s >= 0) {
            double2 x = src[((size_t)r * Nz + s) * Nh + j0 + c];
            val.x = from_f64<T>(x.x); val.y = from_f64<T>(x.y);
        }
        buf0[idx] = val;
    }
    __syncthreads();
    C* res = fft<T, +1, ZF, (ZF == 0), true>(tg_block(), buf0, buf1, ct, ZF == 0 ? d.pz0 : d.pz, twz_of<T, ZF>(d),
                                             d.twz_tan);
    C* out = reinterpret_cast<C*>(d.zbuf) + ((size_t)f * d.Nr + r) * Mz * Nh;
    for (int idx = threadIdx.x; idx < ct * Mz; idx += blockDim.x) {
        const int q = idx >> lct, c = idx & (ct - 1);
        out[(size_t)q * Nh + j0 + c] = res[idx];
    }
}
template <typename T, int ZF>
__global__ void __launch_bounds__(256) k_zinv(TcDev d, const double2* __restrict__ f0,
                                              const double2* __restrict__ f1,
                                              const double2* __restrict__ f2, int tile0) {
    zinv_body<T, ZF>(d, f0, f1, f2, tile0, blockIdx.x, blockIdx.y, blockIdx.z);
}
// Many cases of one shape class (the same Ntheta, Nz, z tile and form) in
// one launch: grid y runs over the radial planes of every case, ymap[y] =
// (case, plane); the case's descriptor holds its own fields and tables.
template <typename T, int ZF>
__global__ void __launch_bounds__(256) k_zinv_b(const TcDev* __restrict__ ds, const int2* __restrict__ ymap) {
    const int2 m = ymap[blockIdx.y];
    const TcDev& d = ds[m.x];
    zinv_body<T, ZF>(d, d.u, d.v, d.w, 0, blockIdx.x, m.y, blockIdx.z);
}

// ---- k_rows: theta transforms and products for one (r, q) row --------------
// Inverse: u + i v in one complex transform of length Mt (Hermitian
// extension), w through the half-length real transform: with H = Mt/2,
// Z_k = (X_k + conj X_{H-k}) + i (X_k - conj X_{H-k}) exp(2 pi i k/Mt),
// z = inverse FFT_H(Z), w_{2m} = Re z_m, w_{2m+1} = Im z_m.
// Forward: (uu - vv) + i uv and uw + i vw in two complex transforms of
// length Mt, ww - vv through the half-length real transform:
// z_m = b_{2m} + i b_{2m+1}, Z = FFT_H(z),
// X_k = (Z_k + conj Z_{H-k})/2 + exp(-2 pi i k/Mt) (Z_k - conj Z_{H-k})/(2i).
// Shared-memory layouts (LAYOUT 5 or 4, in units of Mt complex values):
//   5: two full and one half column per ping-pong side; the forward pass
//      transforms (uu - vv) + i uv and (uw + i vw) as one 2-column transform
//      together with (ww - vv): 10 barrier stages per row for 768 = 3 4^4.
//   4: three full and two half columns; (uw + i vw) is transformed after the
//      other two have been written: 15 barrier stages, but 20% less shared
//      memory, which buys a fourth resident block where 5 Mt does not fit
//      four (float64 rows with Mt = 768).
// The launcher picks 5 unless 5 Mt of float64 / float32 values exceeds the
// four-block budget; the double-float rows always use 5.  With FUSE the full
// and half-length transforms advance together (one barrier per stage for
// both); the double-float rows, latency-bound and at a higher register count
// when fused, run them one after the other.
template <typename T, int LAYOUT, bool FUSE>
__device__ __forceinline__ void rows_body(const TcDev& d, const int q, const int r, const TG tg, const int sub) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Mt = d.Mt, Nh = d.Nh, Mz = d.Mz, Nr = d.Nr;
    const int H = Mt / 2;
    // row group `sub` of the block owns LAYOUT Mt complex values of shared
    // memory; a group past the last row computes on zeros and stores nothing
    const bool valid = q < Mz;
    C* F1 = reinterpret_cast<C*>(smem_raw) + (size_t)sub * LAYOUT * Mt;
    C *F2, *F3, *H1, *H2;
    if constexpr (LAYOUT == 5) {            // [F1 (2 Mt) | H1 | F2 (2 Mt) | H2]
        H1 = F1 + 2 * Mt;
        F2 = H1 + H;
        H2 = F2 + 2 * Mt;
        F3 = nullptr;
    } else {                                // [F1 | F2 | F3 | H1 | H2]
        F2 = F1 + Mt;
        F3 = F2 + Mt;
        H1 = F3 + Mt;
        H2 = H1 + H;
    }
    const C* zb = reinterpret_cast<const C*>(d.zbuf);
    const int qv = valid ? q : 0;
    const C* ur = zb + (((size_t)0 * Nr + r) * Mz + qv) * Nh;
    const C* vr = zb + (((size_t)1 * Nr + r) * Mz + qv) * Nh;
    const C* wr = zb + (((size_t)2 * Nr + r) * Mz + qv) * Nh;
    const C* tr = twr<T>(d);
    for (int p = tg.tid; p < Mt; p += tg.nth) {
        C a;
        a.x = 0; a.y = 0;
        if (!valid) {
        } else if (p == 0) {
            a.x = ur[0].x; a.y = vr[0].x;
        } else if (p < Nh) {
            C U = ur[p], V = vr[p];
            a.x = U.x - V.y; a.y = U.y + V.x;
        } else if (p > Mt - Nh) {
            const int j = Mt - p;
            C U = ur[j], V = vr[j];
            a.x = U.x + V.y; a.y = V.x - U.y;
        }
        F1[p] = a;
    }
    for (int k = tg.tid; k < H; k += tg.nth) {
        C xk, xm;
        xk.x = 0; xk.y = 0; xm.x = 0; xm.y = 0;
        if (valid && k < Nh) { xk = wr[k]; if (k == 0) xk.y = 0; }
        const int kk = H - k;
        if (valid && k > 0 && kk < Nh) xm = wr[kk];
        // E = xk + conj(xm), O = (xk - conj(xm)) exp(+2 pi i k/Mt)
        C E, Dd, O, z;
        E.x = xk.x + xm.x; E.y = xk.y - xm.y;
        Dd.x = xk.x - xm.x; Dd.y = xk.y + xm.y;
        const C t = tr[k];                     // exp(-2 pi i k/Mt)
        O.x = Dd.x * t.x + Dd.y * t.y; O.y = Dd.y * t.x - Dd.x * t.y;
        z.x = E.x - O.y; z.y = E.y + O.x;      // E + i O
        H1[k] = z;
    }
    __syncthreads();
    C *r1, *r2;
    fft_pair<T, +1, FUSE, true>(tg, F1, F2, H1, H2, r1, r2, 1, d.pt, twt<T>(d), d.twt_tan, d.ph, twh<T>(d), d.twh_tan);
    C* o1 = (r1 == F1) ? F2 : F1;              // free full buffer(s)
    C* o2 = (r2 == H1) ? H2 : H1;              // free half buffer
    C* p2 = (LAYOUT == 5) ? o1 + Mt : F3;      // where uw + i vw goes
    // Float64: the forward factor 1/(Mt Mz) and the 1/2 of the real-pair
    // unpacking below are applied here, as s = 1/(2 Mt Mz) on one factor of
    // every product (three multiplies per point), instead of two multiplies
    // per output value in the unpacking and two more in k_zfwd.
    constexpr bool PRE = std::is_same<T, double>::value;
    const T s = PRE ? (T)(0.5 * d.fscale) : (T)1;
    for (int m = tg.tid; m < H; m += tg.nth) {
        const C w2 = r2[m];
        T bb[2];
        for (int e = 0; e < 2; ++e) {
            const int p = 2 * m + e;
            const T u = r1[p].x, v = r1[p].y, w = e ? w2.y : w2.x;
            C b0, b1;
            if constexpr (PRE) {
                const T us = s * u, vs = s * v, ws = s * w;
                const T vv = vs * v;
                b0.x = us * u - vv; b0.y = us * v;   // s (uu - vv), s uv
                b1.x = us * w; b1.y = vs * w;        // s uw, s vw
                bb[e] = ws * w - vv;                 // s (ww - vv)
            } else {
                const T vv = v * v;
                b0.x = u * u - vv; b0.y = u * v;     // uu - vv, uv
                b1.x = u * w; b1.y = v * w;          // uw, vw
                bb[e] = w * w - vv;                  // ww - vv
            }
            o1[p] = b0; p2[p] = b1;
        }
        C z; z.x = bb[0]; z.y = bb[1];
        o2[m] = z;
    }
    __syncthreads();
    // float64 forward full-length transforms in plan family 3: the unpacking
    // below reads outputs j < Nh and Mt - j only, never the band Nh .. 2 Nh - 1
    constexpr int FA = PRE ? 3 : 0;
    const double* tta = PRE ? d.twt3_tan : d.twt_tan;
    C *s1, *s3;
    fft_pair<T, -1, FUSE, false, FA>(tg, o1, r1, o2, r2, s1, s3, LAYOUT == 5 ? 2 : 1, d.pt, twt<T>(d), tta, d.ph, twh<T>(d), d.twh_tan);
    C* pb = reinterpret_cast<C*>(d.pbuf);
    // unpack two real transforms from one complex transform of length Mt
    auto half = [](T x) -> T {                 // the unpacking's 1/2 (already in s for float64)
        if constexpr (PRE) return x;
        else return (T)0.5 * x;
    };
    auto mhalf = [](T x) -> T {
        if constexpr (PRE) return -x;
        else return (T)-0.5 * x;
    };
    auto unpack_full = [&](const C* out, int j, int slot) {
        const C cj = out[j];
        const C cm = out[j == 0 ? 0 : Mt - j];
        C x1, x2;
        x1.x = half(cj.x + cm.x); x1.y = half(cj.y - cm.y);
        x2.x = half(cj.y + cm.y); x2.y = mhalf(cj.x - cm.x);
        pb[(((size_t)slot * Nr + r) * Mz + q) * Nh + j] = x1;
        pb[(((size_t)(slot + 1) * Nr + r) * Mz + q) * Nh + j] = x2;
    };
    constexpr int NF = (LAYOUT == 5) ? 2 : 1;   // full columns written now
    for (int idx = valid ? tg.tid : (NF + 1) * Nh; idx < (NF + 1) * Nh; idx += tg.nth) {
        const int c = idx / Nh, j = idx - c * Nh;
        if (c < NF) {
            unpack_full(s1 + c * Mt, j, 2 * c);     // uu - vv, uv (and uw, vw)
        } else {
            const C zk = s3[j];
            const C zm = s3[j == 0 ? 0 : H - j];
            C ev, od, x;
            ev.x = half(zk.x + zm.x); ev.y = half(zk.y - zm.y);
            // (Z_k - conj Z_{H-k})/(2i)
            od.x = half(zk.y + zm.y); od.y = mhalf(zk.x - zm.x);
            const C t = tr[j];
            x.x = ev.x + od.x * t.x - od.y * t.y;
            x.y = ev.y + od.x * t.y + od.y * t.x;
            pb[(((size_t)4 * Nr + r) * Mz + q) * Nh + j] = x;   // ww - vv
        }
    }
    if constexpr (LAYOUT == 4) {
        // uw + i vw: its ping-pong partner is the full buffer not holding s1
        C* s2 = fft<T, -1, FA>(tg, F3, (s1 == o1) ? r1 : o1, 1, d.pt, twt<T>(d), tta);
        for (int j = valid ? tg.tid : Nh; j < Nh; j += tg.nth) unpack_full(s2, j, 2);   // uw, vw
    }
}
// ---- k_rows2: two theta rows at once, every transform of full length -------
// The rows q0 = 2 qp and q1 = q0 + 1 of plane r (a row past Mz computes on
// zeros and stores nothing).  Each real signal pairs with another of the same
// two rows in one complex transform of length Mt:
//   inverse: u + i v of q0, u + i v of q1, w(q0) + i w(q1)   (3 columns)
//   forward: (uu - vv) + i uv and uw + i vw of q0, the same of q1, and
//            (ww - vv)(q0) + i (ww - vv)(q1)                   (5 columns)
// A real signal's spectrum is Hermitian, so the input of column a + i b is
// A_p + i B_p for p < Nh and conj(A_(Mt-p)) + i conj(B_(Mt-p)) for
// p > Mt - Nh; the outputs split as A_j = (Z_j + conj Z_(Mt-j))/2 and
// B_j = (Z_j - conj Z_(Mt-j))/(2i).  With all columns of one length, every
// stage is one loop over the butterflies of all columns (no half-length
// transform with its pre- and post-twiddles, and no second butterfly shape
// in the stage loop).  Shared memory: two sides of 5 columns of Mt.  Used for
// the float32 rows of the mixed form.
template <typename T>
__device__ __forceinline__ void rows2_body(const TcDev& d, const int qp, const int r, const TG tg, const int sub) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Mt = d.Mt, Nh = d.Nh, Mz = d.Mz, Nr = d.Nr;
    C* A = reinterpret_cast<C*>(smem_raw) + (size_t)sub * 10 * Mt;
    C* B = A + 5 * Mt;
    const int q0 = 2 * qp;
    const bool v0 = q0 < Mz, v1 = q0 + 1 < Mz;
    const C* zb = reinterpret_cast<const C*>(d.zbuf);
    const size_t fs = (size_t)Nr * Mz * Nh;                        // field stride of zbuf
    const C* row0 = zb + ((size_t)r * Mz + (v0 ? q0 : 0)) * Nh;     // u of row q0
    const C* row1 = zb + ((size_t)r * Mz + (v1 ? q0 + 1 : 0)) * Nh; // u of row q1
    // column input from the spectra a, b of two real signals
    auto herm = [&](const C* a, const C* b, bool va, bool vb, int p) -> C {
        C z;
        z.x = 0; z.y = 0;
        if (p == 0) {
            if (va) z.x = a[0].x;
            if (vb) z.y = b[0].x;
        } else if (p < Nh) {
            C U, V;
            U.x = 0; U.y = 0; V.x = 0; V.y = 0;
            if (va) U = a[p];
            if (vb) V = b[p];
            z.x = U.x - V.y; z.y = U.y + V.x;
        } else if (p > Mt - Nh) {
            const int j = Mt - p;
            C U, V;
            U.x = 0; U.y = 0; V.x = 0; V.y = 0;
            if (va) U = a[j];
            if (vb) V = b[j];
            z.x = U.x + V.y; z.y = V.x - U.y;
        }
        return z;
    };
    for (int p = tg.tid; p < Mt; p += tg.nth) {
        A[p] = herm(row0, row0 + fs, v0, v0, p);                    // u + i v of q0
        A[Mt + p] = herm(row1, row1 + fs, v1, v1, p);               // u + i v of q1
        A[2 * Mt + p] = herm(row0 + 2 * fs, row1 + 2 * fs, v0, v1, p);   // w(q0) + i w(q1)
    }
    __syncthreads();
    C* R = fft<T, +1, 0, true>(tg, A, B, 3, d.pt, twt<T>(d), d.twt_tan);
    C* O = (R == A) ? B : A;
    for (int p = tg.tid; p < Mt; p += tg.nth) {
        const C a0 = R[p], a1 = R[Mt + p], ww = R[2 * Mt + p];
        T bb[2];
        #pragma unroll
        for (int e = 0; e < 2; ++e) {
            const C uv = e ? a1 : a0;
            const T u = uv.x, v = uv.y, w = e ? ww.y : ww.x;
            const T vv = v * v;
            C b0, b1;
            b0.x = u * u - vv; b0.y = u * v;         // uu - vv, uv
            b1.x = u * w; b1.y = v * w;              // uw, vw
            bb[e] = w * w - vv;                      // ww - vv
            O[(2 * e) * Mt + p] = b0;
            O[(2 * e + 1) * Mt + p] = b1;
        }
        C z; z.x = bb[0]; z.y = bb[1];
        O[4 * Mt + p] = z;
    }
    __syncthreads();
    const C* S = fft<T, -1, 0>(tg, O, R, 5, d.pt, twt<T>(d), d.twt_tan);
    C* pb = reinterpret_cast<C*>(d.pbuf);
    const size_t ps = (size_t)Nr * Mz * Nh;                        // product stride of pbuf
    C* out0 = pb + ((size_t)r * Mz + q0) * Nh;
    const T h = (T)0.5;
    for (int j = tg.tid; j < Nh; j += tg.nth) {
        const int jm = j == 0 ? 0 : Mt - j;
        #pragma unroll
        for (int c = 0; c < 5; ++c) {
            const C cj = S[c * Mt + j], cm = S[c * Mt + jm];
            C x1, x2;
            x1.x = h * (cj.x + cm.x); x1.y = h * (cj.y - cm.y);
            x2.x = h * (cj.y + cm.y); x2.y = -h * (cj.x - cm.x);
            if (c < 4) {                             // two products of one row
                const int e = c >> 1, slot = 2 * (c & 1);
                if (e ? v1 : v0) {
                    C* o = out0 + (size_t)e * Nh + j;
                    o[slot * ps] = x1;
                    o[(slot + 1) * ps] = x2;
                }
            } else {                                 // ww - vv of both rows
                if (v0) out0[4 * ps + j] = x1;
                if (v1) out0[4 * ps + Nh + j] = x2;
            }
        }
    }
}

// rpb rows per block (short rows: more rows per block keep the threads of a
// block busy), blockDim.x / rpb threads per row.
__device__ __forceinline__ TG row_group(int rpb, int& sub) {
    const int nth = (int)blockDim.x / rpb;
    sub = (int)threadIdx.x / nth;
    return TG{(int)threadIdx.x - sub * nth, nth};
}
template <typename T, int LAYOUT, bool FUSE>
__global__ void __launch_bounds__(256) k_rows(TcDev d, int rpb) {
    int sub;
    const TG tg = row_group(rpb, sub);
    rows_body<T, LAYOUT, FUSE>(d, blockIdx.x * rpb + sub, blockIdx.y, tg, sub);
}
template <typename T, int LAYOUT, bool FUSE>
__global__ void __launch_bounds__(256) k_rows_b(const TcDev* __restrict__ ds, const int2* __restrict__ ymap, int rpb) {
    const int2 m = ymap[blockIdx.y];
    int sub;
    const TG tg = row_group(rpb, sub);
    rows_body<T, LAYOUT, FUSE>(ds[m.x], blockIdx.x * rpb + sub, m.y, tg, sub);
}
// gpb row pairs per block, blockDim.x / gpb threads per pair
template <typename T>
__global__ void __launch_bounds__(TC_ROWS2_THREADS) k_rows2(TcDev d, int gpb) {
    int sub;
    const TG tg = row_group(gpb, sub);
    rows2_body<T>(d, blockIdx.x * gpb + sub, blockIdx.y, tg, sub);
}
template <typename T>
__global__ void __launch_bounds__(TC_ROWS2_THREADS) k_rows2_b(const TcDev* __restrict__ ds, const int2* __restrict__ ymap,
                                                              int gpb) {
    const int2 m = ymap[blockIdx.y];
    int sub;
    const TG tg = row_group(gpb, sub);
    rows2_body<T>(ds[m.x], blockIdx.x * gpb + sub, m.y, tg, sub);
}

// ---- k_zfwd: pbuf -> spectral products, scaled by 1/(Mt Mz) (float64: already in pbuf) ----
template <typename T, int ZF>
__device__ __forceinline__ void zfwd_body(const TcDev& d, int tile0, int bx, int r, int p) {
    typedef typename V2<T>::t C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    const int ct = d.ztile;
    const int lct = __ffs(ct) - 1;          // the z tile is 1, 2, 4 or 8 columns
    C* buf1 = buf0 + ct * d.Mz;
    const int j0 = (bx + tile0) * ct;
    const int Mz = d.Mz, Nz = d.Nz, Nh = d.Nh, Nr = d.Nr;
    const C* in = reinterpret_cast<const C*>(d.pbuf) + ((size_t)p * Nr + r) * Mz * Nh;
    for (int idx = threadIdx.x; idx < ct * Mz; idx += blockDim.x) {     // interleaved columns, as in zinv_body
        const int q = idx >> lct, c = idx & (ct - 1);
        buf0[idx] = in[(size_t)q * Nh + j0 + c];
    }
    __syncthreads();
    // family 3 (float64): the last stage skips outputs M/3 .. 2M/3 - 1, i.e.
    // q = Nz/2 .. Nz - 1, which the truncation below never reads
    C* res = fft<T, -1, ZF, false, true>(tg_block(), buf0, buf1, ct, (ZF == 0 || ZF == 3) ? d.pz0 : d.pz,
                                         twz_of<T, ZF>(d), ZF == 3 ? d.twz3_tan : d.twz_tan);
    T scale;
    if constexpr (std::is_same<T, double>::value) scale = 1.0;     // applied in k_rows
    else if constexpr (std::is_same<T, float>::value) scale = d.fscale_f;
    else scale = dfloat(d.fscale_f, d.fscale_lo);
    // products: double2 for float64, float2 for the mixed form, double-float
    // pairs for the double-float form (read as such by the line kernel)
    typedef typename std::conditional<std::is_same<T, double>::value, double2, C>::type PO;
    PO* outp = reinterpret_cast<PO*>(d.prod) + ((size_t)p * Nr + r) * Nz * Nh;
    for (int idx = threadIdx.x; idx < ct * Nz; idx += blockDim.x) {
        const int s = idx >> lct, c = idx & (ct - 1);
        C val; val.x = 0; val.y = 0;
        if (s != Nz / 2) {
            const int n = s < Nz / 2 ? s : s - Nz;
            const int qq = n >= 0 ? n : Mz + n;
            val = res[(qq << lct) + c];
            if constexpr (!std::is_same<T, double>::value) { val.x *= scale; val.y *= scale; }
        }
        outp[(size_t)s * Nh + j0 + c] = val;
    }
}
template <typename T, int ZF>
__global__ void __launch_bounds__(256) k_zfwd(TcDev d, int tile0) {
    zfwd_body<T, ZF>(d, tile0, blockIdx.x, blockIdx.y, blockIdx.z);
}
template <typename T, int ZF>
__global__ void __launch_bounds__(256) k_zfwd_b(const TcDev* __restrict__ ds, const int2* __restrict__ ymap) {
    const int2 m = ymap[blockIdx.y];
    zfwd_body<T, ZF>(ds[m.x], 0, blockIdx.x, m.y, blockIdx.z);
}

// ---- host launchers --------------------------------------------------------------
static inline bool z_has_odd_primes(const TcDev& d) {
    for (int i = 0; i < d.pz.nst; ++i)
        if (d.pz.R[i] % 2 && d.pz.R[i] != 3) return true;
    return false;
}

// Shared-memory layout of the theta rows (see k_rows): 5 Mt unless that
// exceeds the budget of four resident blocks (57 KB each) for float64 or
// float32 values.
template <typename T>
static int rows_layout(const TcDev& d) {
    typedef typename V2<T>::t C;
    if (std::is_same<T, dfloat>::value) return 5;
    return 5 * (size_t)d.Mt * sizeof(C) <= 57 * 1024 ? 5 : 4;
}
// Theta rows per block: about 384 points per block (one row from Mt = 288 up,
// up to 8 rows of 48 or fewer points), so that the 256 threads of a block
// have butterflies to work on in every stage.
static int rows_per_block(const TcDev& d) {
    int rpb = 1;
    while (rpb < 8 && (rpb * 2) * d.Mt <= 384) rpb *= 2;
    return rpb;
}
// Float32 theta rows in pairs (k_rows2) where two sides of 5 columns fit the
// 200 KB of one block; row pairs per block: about 768 points per block, up
// to 8 pairs.
template <typename T>
static bool rows_paired(const TcDev& d) {
    return std::is_same<T, float>::value && 10 * (size_t)d.Mt * sizeof(typename V2<T>::t) <= 200 * 1024;
}
static int row_pairs_per_block(const TcDev& d) {
    int gpb = 1;
    while (gpb < 8 && (gpb * 2) * 2 * d.Mt <= 768) gpb *= 2;
    return gpb;
}

template <typename T>
static void plane_kernel_t(const TcDev& d, int which, cudaStream_t s, int tile0, int ntiles) {
    typedef typename V2<T>::t C;
    const int ct = d.ztile;
    const size_t smz = 2 * (size_t)ct * d.Mz * sizeof(C);
    const int layout = rows_layout<T>(d);
    const size_t smr = (size_t)layout * d.Mt * sizeof(C);
    const bool odd = z_has_odd_primes(d);
    // the radix-3/4/2 plan pz0 (tangent twiddles in float64) when the axial
    // length has a compile-time plan, else radix 16 or the prime stages
    const bool fam0 = d.zfam0 != 0;
    if (which == 0) {
        const dim3 g(ntiles, d.Nr, 3);
        if (odd) k_zinv<T, 2><<<g, 256, smz, s>>>(d, d.u, d.v, d.w, tile0);
        else if (fam0) k_zinv<T, 0><<<g, 256, smz, s>>>(d, d.u, d.v, d.w, tile0);
        else k_zinv<T, 1><<<g, 256, smz, s>>>(d, d.u, d.v, d.w, tile0);
    } else if (which == 1) {
        constexpr bool fuse = !std::is_same<T, dfloat>::value;
        if (rows_paired<T>(d)) {
            const int gpb = row_pairs_per_block(d);
            const dim3 g(((d.Mz + 1) / 2 + gpb - 1) / gpb, d.Nr);
            k_rows2<T><<<g, TC_ROWS2_THREADS, gpb * 10 * (size_t)d.Mt * sizeof(C), s>>>(d, gpb);
            return;
        }
        const int rpb = rows_per_block(d);
        const dim3 g((d.Mz + rpb - 1) / rpb, d.Nr);
        if (layout == 5) k_rows<T, 5, fuse><<<g, 256, rpb * smr, s>>>(d, rpb);
        else k_rows<T, 4, fuse><<<g, 256, rpb * smr, s>>>(d, rpb);
    } else {
        const dim3 g(ntiles, d.Nr, TC_NPROD);
        if (odd) k_zfwd<T, 2><<<g, 256, smz, s>>>(d, tile0);
        else if (fam0) {
            if constexpr (std::is_same<T, double>::value) k_zfwd<T, 3><<<g, 256, smz, s>>>(d, tile0);
            else k_zfwd<T, 0><<<g, 256, smz, s>>>(d, tile0);
        } else k_zfwd<T, 1><<<g, 256, smz, s>>>(d, tile0);
    }
}


// One plane kernel for every case of a shape class: d0 is the class's
// representative descriptor (shapes, z tile, plans), ds the descriptors of
// all its cases on the device, ymap (case, plane) for each of the nplanes
// radial planes.  The kernels and launch shapes are those of the single case.
template <typename T>
static void plane_kernel_batch_t(const TcDev& d0, const TcDev* ds, const int2* ymap, int nplanes, int which,
                                 cudaStream_t s) {
    typedef typename V2<T>::t C;
    const int ct = d0.ztile;
    const size_t smz = 2 * (size_t)ct * d0.Mz * sizeof(C);
    const int layout = rows_layout<T>(d0);
    const size_t smr = (size_t)layout * d0.Mt * sizeof(C);
    const bool odd = z_has_odd_primes(d0);
    const bool fam0 = d0.zfam0 != 0;
    const int ntiles = d0.Nh / ct;
    if (which == 0) {
        const dim3 g(ntiles, nplanes, 3);
        if (odd) k_zinv_b<T, 2><<<g, 256, smz, s>>>(ds, ymap);
        else if (fam0) k_zinv_b<T, 0><<<g, 256, smz, s>>>(ds, ymap);
        else k_zinv_b<T, 1><<<g, 256, smz, s>>>(ds, ymap);
    } else if (which == 1) {
        constexpr bool fuse = !std::is_same<T, dfloat>::value;
        if (rows_paired<T>(d0)) {
            const int gpb = row_pairs_per_block(d0);
            const dim3 g(((d0.Mz + 1) / 2 + gpb - 1) / gpb, nplanes);
            k_rows2_b<T><<<g, TC_ROWS2_THREADS, gpb * 10 * (size_t)d0.Mt * sizeof(C), s>>>(ds, ymap, gpb);
            return;
        }
        const int rpb = rows_per_block(d0);
        const dim3 g((d0.Mz + rpb - 1) / rpb, nplanes);
        if (layout == 5) k_rows_b<T, 5, fuse><<<g, 256, rpb * smr, s>>>(ds, ymap, rpb);
        else k_rows_b<T, 4, fuse><<<g, 256, rpb * smr, s>>>(ds, ymap, rpb);
    } else {
        const dim3 g(ntiles, nplanes, TC_NPROD);
        if (odd) k_zfwd_b<T, 2><<<g, 256, smz, s>>>(ds, ymap);
        else if (fam0) {
            if constexpr (std::is_same<T, double>::value) k_zfwd_b<T, 3><<<g, 256, smz, s>>>(ds, ymap);
            else k_zfwd_b<T, 0><<<g, 256, smz, s>>>(ds, ymap);
        } else k_zfwd_b<T, 1><<<g, 256, smz, s>>>(ds, ymap);
    }
}

// Shared-memory opt-in of every plane kernel of one arithmetic type.
template <typename T>
static cudaError_t plane_attributes_t() {
    const int lim = 200 * 1024;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
        cudaError_t r = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r != cudaSuccess) e = r;
    };
    constexpr bool fuse = !std::is_same<T, dfloat>::value;
    set((const void*)k_zinv<T, 0>); set((const void*)k_zinv<T, 1>); set((const void*)k_zinv<T, 2>);
    set((const void*)k_zfwd<T, 0>); set((const void*)k_zfwd<T, 1>); set((const void*)k_zfwd<T, 2>);
    if constexpr (std::is_same<T, double>::value) set((const void*)k_zfwd<T, 3>);
    set((const void*)k_rows<T, 5, fuse>); set((const void*)k_rows<T, 4, fuse>);
    set((const void*)k_zinv_b<T, 0>); set((const void*)k_zinv_b<T, 1>); set((const void*)k_zinv_b<T, 2>);
    set((const void*)k_zfwd_b<T, 0>); set((const void*)k_zfwd_b<T, 1>); set((const void*)k_zfwd_b<T, 2>);
    if constexpr (std::is_same<T, double>::value) set((const void*)k_zfwd_b<T, 3>);
    set((const void*)k_rows_b<T, 5, fuse>); set((const void*)k_rows_b<T, 4, fuse>);
    if constexpr (std::is_same<T, float>::value) { set((const void*)k_rows2<T>); set((const void*)k_rows2_b<T>); }
    return e;
}
