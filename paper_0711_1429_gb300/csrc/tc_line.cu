// Line phase: for every Fourier pair (m, alpha) the radial rows of Eq. 6 (v)
// and Eq. 7 (eta), the banded radial solves, the Runge-Kutta memory and the
// reconstruction of u, w from continuity; plus the mean flow (m = alpha = 0).
//
// One thread owns one pair and walks its radial line; the 32 threads of a
// warp hold 32 consecutive azimuthal indices at one axial slot, so every
// radial point is one coalesced 512-byte access per field.
//
// Notation (Appendix): D f = f', D_* f = f' + f/r, k^2 = alpha^2 + m^2/r^2,
// c = 1/k^2, c1..c3 its r-derivatives, nu = 2/Re.  On row j a chain operator
// applied to (coefficient x field) is the row stencil (d0, l1, l2, l4 for
// I, D, D D_*, D D_* D D_*) applied to the pointwise product; D D g is
// written D D_* g - D(g/r).
//
// Runge-Kutta (3 substeps, explicit third order + Crank-Nicolson): substep k
// solves (M - beta_k dt L) x^k = H_k + gamma_k dt E(x^(k-1)) with the stored
//   H_k = (M + alpha_k dt L) x^(k-1) + zeta_k dt E(x^(k-2)),
// and prepares H_(k+1) = RHS_k + zeta_(k+1) dt E(x^(k-1)) + (beta_k +
// alpha_(k+1)) dt L x^k, using M x^k = RHS_k + beta_k dt L x^k.
#include "tc_internal.h"
#include "tc_dfloat.h"
#include <type_traits>

__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }

namespace {

struct Coef { double k2, c, c1, c2, c3; };

// k^2, c = 1/k^2 = r^2/g and its r-derivatives, g = alpha^2 r^2 + m^2:
// c1 = 2 r m^2/g^2, c2 = 2 m^2 (m^2 - 3 alpha^2 r^2)/g^3,
// c3 = -24 m^2 alpha^2 r (m^2 - alpha^2 r^2)/g^4.
__device__ __forceinline__ Coef coef_at(double r, double rinv, double m, double al) {
    const double m2 = m * m, a2 = al * al, r2 = r * r;
    Coef o;
    o.k2 = a2 + m2 * rinv * rinv;
    const double g = a2 * r2 + m2;
    const double gi = 1.0 / g;
    const double gi2 = gi * gi;
    o.c = r2 * gi;
    o.c1 = 2.0 * r * m2 * gi2;
    o.c2 = 2.0 * m2 * (m2 - 3.0 * a2 * r2) * gi2 * gi;
    o.c3 = -24.0 * m2 * a2 * r * (m2 - a2 * r2) * gi2 * gi2;
    return o;
}

__device__ __forceinline__ double2 cz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// (i s) * a
__device__ __forceinline__ double2 cimag(double s, double2 a) { return make_double2(-s * a.y, s * a.x); }
// i * a
__device__ __forceinline__ double2 ci(double2 a) { return make_double2(-a.y, a.x); }
// a + s * b
__device__ __forceinline__ double2 caxpy(double2 a, double s, double2 b) { return make_double2(fma(s, b.x, a.x), fma(s, b.y, a.y)); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// finiteness from the exponent bits (integer pipe, no float64 compare)
__device__ __forceinline__ bool dfinite(double x) { return (__double2hiint(x) & 0x7ff00000) != 0x7ff00000; }
__device__ __forceinline__ bool cfinite(double2 a) { return dfinite(a.x) && dfinite(a.y); }

__device__ __forceinline__ double2 ld_prod(const double2* p, size_t o) { return p[o]; }
__device__ __forceinline__ double2 ld_prod(const float2* p, size_t o) { float2 f = p[o]; return make_double2(d_bits(f.x), d_bits(f.y)); }

// generic complex helpers for float2 / double2
template <typename CT> __device__ __forceinline__ CT tz() { CT r; r.x = 0; r.y = 0; return r; }
template <typename CT, typename T> __device__ __forceinline__ CT timag(T s, CT a) { CT r; r.x = -s * a.y; r.y = s * a.x; return r; }
template <typename CT> __device__ __forceinline__ CT tadd(CT a, CT b) { CT r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename CT, typename T> __device__ __forceinline__ CT taxpy(CT a, T s, CT b) { CT r; r.x = fma(s, b.x, a.x); r.y = fma(s, b.y, a.y); return r; }
template <typename CT, typename T> __device__ __forceinline__ CT tscale(T s, CT a) { CT r; r.x = s * a.x; r.y = s * a.y; return r; }
__device__ __forceinline__ double2 to_d2(double2 a) { return a; }
// float32 <-> float64 through the integer conversions of tc_dfloat.h (the
// float64 pipe is the mixed line kernel's bottleneck); the double-float form
// converts with float64 instructions, which measured faster there (fewer
// registers in a kernel that is already at its register budget)
__device__ __forceinline__ double2 to_d2(float2 a) { return make_double2(d_bits(a.x), d_bits(a.y)); }
__device__ __forceinline__ double2 to_d2(dcomplex a) { return make_double2((double)a.x, (double)a.y); }
// the same exact widening by bit operations and one float64 add (d_of), for
// the mixed form's continuity term
__device__ __forceinline__ double2 to_d2_bits(dcomplex a) { return make_double2(d_of(a.x), d_of(a.y)); }
template <typename CT> __device__ __forceinline__ CT from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) { return make_float2(f_bits(a.x), f_bits(a.y)); }
template <> __device__ __forceinline__ dcomplex from_d2<dcomplex>(double2 a) { dcomplex r; r.x = dfloat(a.x); r.y = dfloat(a.y); return r; }
__device__ __forceinline__ dcomplex dc_bits(double2 a) { dcomplex r; r.x = df_bits(a.x); r.y = df_bits(a.y); return r; }
__device__ __forceinline__ dcomplex dc_fma(const dcomplex& a, dfloat s, const dcomplex& b) {
    dcomplex r;
    r.x = df_fma(a.x, s, b.x);
    r.y = df_fma(a.y, s, b.y);
    return r;
}
__device__ __forceinline__ dcomplex dc_scale(dfloat s, const dcomplex& a) {
    dcomplex r;
    r.x = s * a.x;
    r.y = s * a.y;
    return r;
}
__device__ __forceinline__ dcomplex dc_i(const dcomplex& a) {   // i a
    dcomplex r;
    r.x = -a.y;
    r.y = a.x;
    return r;
}
__device__ __forceinline__ dcomplex dc_of(float2 a) { dcomplex r; r.x = dfloat(a.x, 0.0f); r.y = dfloat(a.y, 0.0f); return r; }
__device__ __forceinline__ double2 ld_prod(const dcomplex* p, size_t o) { return to_d2(p[o]); }
__device__ __forceinline__ dfloat as_df(float2 v) { return dfloat(v.x, v.y); }

// element types of the three forms: 0 float64, 1 mixed (float32 explicit
// rows), 2 double-float explicit rows
template <int MODE> struct LineTypes;
template <> struct LineTypes<0> { typedef double T; typedef double2 CT; };
template <> struct LineTypes<1> { typedef float T; typedef float2 CT; };
template <> struct LineTypes<2> { typedef dfloat T; typedef dcomplex CT; };

// Pair index -> (n slot, j); returns false for pairs that are not evolved:
// the axial Nyquist slot, (0,0) (mean flow) and (0, n<0) (conjugates).
__device__ __forceinline__ bool pair_info(const TcDev& d, int pair, double& m, double& al, long long& partner) {
    const int s = pair / d.Nh, j = pair - s * d.Nh;
    if (s == d.Nz / 2) return false;
    if (j == 0 && (s == 0 || s > d.Nz / 2)) return false;
    const int n = s < d.Nz / 2 ? s : s - d.Nz;
    m = j * d.m0;
    al = n * d.alpha0;
    partner = (j == 0) ? (long long)(d.Nz - s) * d.Nh : -1;
    return true;
}

#define TAB(base, k, row, comp) (base)[((size_t)((k) * d.Nr + (row)) * 5 + (comp)) * d.npairs + pair]

// Reduced band row on the unknowns 1..Nr-2: entries on columns j-2..j+2.
struct Row5 { double a, b, dd, c, e; };

}  // namespace

// ---------------------------------------------------------------------------
// Band of the v rows (interior j = 2..Nr-3), entry s multiplies v_{j-2+s}:
//   mass      M = d0 - l2 c + l1 c1
//   implicit  L = nu [2 l2 - l4 c + l1 (c2/r + c3 - c1/r^2 - 2 m^2 c/r^3)
//                     - 2 l2 c1/r - d0 k^2]
// (Eq. 6 with D_1 read as D and D[(1/r) DD(1/k^2) v] read as D[(c2/r) v]).
__device__ void v_band(const TcDev& d, int j, double m, double al, double* M5, double* L5) {
    for (int s = 0; s < 5; ++s) {
        const int i = j - 2 + s;
        const double r = d.r[i], ri = d.rinv[i];
        const Coef q = coef_at(r, ri, m, al);
        const double w0 = d.d0[j * 5 + s], w1 = d.l1[j * 5 + s], w2 = d.l2[j * 5 + s], w4 = d.l4[j * 5 + s];
        M5[s] = w0 - w2 * q.c + w1 * q.c1;
        L5[s] = d.nu * (2.0 * w2 - w4 * q.c
                        + w1 * (q.c2 * ri + q.c3 - q.c1 * ri * ri - 2.0 * m * m * q.c * ri * ri * ri)
                        - 2.0 * w2 * q.c1 * ri - w0 * q.k2);
    }
}

// eta rows j = 1..Nr-2: mass d0, implicit nu (l2 - d0 k^2), from start[j].
__device__ void eta_band(const TcDev& d, int j, double m, double al, double* L5) {
    const int st = d.start[j];
    for (int s = 0; s < 5; ++s) {
        const int i = st + s;
        const double ri = d.rinv[i];
        const double k2 = al * al + m * m * ri * ri;
        L5[s] = d.nu * (d.l2[j * 5 + s] - d.d0[j * 5 + s] * k2);
    }
}

// Pentadiagonal LU without pivoting of the reduced system on unknowns
// 1..Nr-2, rows produced by `row(i)`; stores per row (m2, m1, 1/diag, c', e)
// and returns false on a vanishing pivot.
template <typename RowFn>
__device__ bool band_lu(const TcDev& d, double* tab, int k, int pair, RowFn row) {
    double p2d = 1, p2c = 0, p2e = 0, p1d = 1, p1c = 0, p1e = 0;
    bool ok = true;
    for (int i = 1; i <= d.Nr - 2; ++i) {
        Row5 R = row(i);
        const double scale = fabs(R.a) + fabs(R.b) + fabs(R.dd) + fabs(R.c) + fabs(R.e);
        const double m2 = (i >= 3) ? R.a / p2d : 0.0;
        double b = R.b - m2 * p2c;
        double dd = R.dd - m2 * p2e;
        const double m1 = (i >= 2) ? b / p1d : 0.0;
        dd = dd - m1 * p1c;
        const double cc = R.c - m1 * p1e;
        if (!(fabs(dd) > 1e-13 * scale)) ok = false;
        TAB(tab, k, i, 0) = m2;
        TAB(tab, k, i, 1) = m1;
        TAB(tab, k, i, 2) = 1.0 / dd;
        TAB(tab, k, i, 3) = cc;
        TAB(tab, k, i, 4) = R.e;
        p2d = p1d; p2c = p1c; p2e = p1e;
        p1d = dd; p1c = cc; p1e = R.e;
    }
    return ok;
}

// Per-pair tables: LU factors of (M - beta_k dt L) for v and eta, k = 0..2,
// with the boundary rows folded in, and the implicit band L of the v rows.
__global__ void __launch_bounds__(128) k_setup(TcDev d) {
    const int pair = blockIdx.x * blockDim.x + threadIdx.x;
    if (pair >= d.npairs) return;
    double m, al;
    long long partner;
    if (!pair_info(d, pair, m, al, partner)) return;
    const int N = d.Nr;
    const double* e0 = d.dwall;       // D at r_0 on points 0..4
    const double* e1 = d.dwall + 5;   // D at r_{N-1} on points N-5..N-1
    bool ok = true;
    for (int i = 0; i < N; ++i) {
        const Coef q = coef_at(d.r[i], d.rinv[i], m, al);
        d.tab_c[(size_t)i * d.npairs + pair] = q.c;
        d.tab_c1[(size_t)i * d.npairs + pair] = q.c1;
        if (d.tab_cx) {
            const dfloat a(q.c), b(q.c1);
            d.tab_cx[(size_t)i * d.npairs + pair] = make_float2(a.hi, a.lo);
            d.tab_c1x[(size_t)i * d.npairs + pair] = make_float2(b.hi, b.lo);
        }
    }
    // implicit band of the v rows (substep independent)
    for (int j = 2; j <= N - 3; ++j) {
        double M5[5], L5[5];
        v_band(d, j, m, al, M5, L5);
        for (int s = 0; s < 5; ++s) TAB(d.tab_lv, 0, j, s) = L5[s];
    }
    for (int k = 0; k < 3; ++k) {
        const double bdt = d.rk_beta[k] * d.dt;
        // ---- v system ----
        auto vrow_full = [&](int j, double* A) {
            double M5[5], L5[5];
            v_band(d, j, m, al, M5, L5);
            for (int s = 0; s < 5; ++s) A[s] = M5[s] - bdt * L5[s];
        };
        double A2[5], A3[5];
        vrow_full(2, A2);
        vrow_full(N - 3, A3);
        // row 1 (Dv(r_0) = 0 on v_1..v_4) minus f * row 2 eliminates v_4
        const double fv = e0[4] / A2[4];
        const Row5 v1r = {0.0, 0.0, e0[1] - fv * A2[1], e0[2] - fv * A2[2], e0[3] - fv * A2[3]};
        // row N-2 (Dv(r_{N-1}) = 0 on v_{N-5}..v_{N-2}) minus g * row N-3
        const double gv = e1[0] / A3[0];
        const Row5 vNr = {e1[1] - gv * A3[1], e1[2] - gv * A3[2], e1[3] - gv * A3[3], 0.0, 0.0};
        ok &= band_lu(d, d.tab_luv, k, pair, [&](int i) -> Row5 {
            if (i == 1) return v1r;
            if (i == N - 2) return vNr;
            double A[5];
            vrow_full(i, A);
            Row5 R = {A[0], A[1], A[2], A[3], A[4]};
            if (i == 2) R.a = 0.0;          // column 0: v_0 = 0
            if (i == N - 3) R.e = 0.0;      // column N-1: v_{N-1} = 0
            return R;
        });
        TAB(d.tab_luv, k, 0, 0) = fv;
        TAB(d.tab_luv, k, N - 1, 0) = gv;
        // ---- eta system ----
        auto erow_full = [&](int j, double* A) {
            double L5[5];
            eta_band(d, j, m, al, L5);
            for (int s = 0; s < 5; ++s) A[s] = d.d0[j * 5 + s] - bdt * L5[s];
        };
        double B1[5], B2[5], B3[5], BN[5];
        erow_full(1, B1);          // start 0: columns 0..4
        erow_full(2, B2);
        erow_full(N - 3, B3);
        erow_full(N - 2, BN);      // start N-5
        const double fe = B1[4] / B2[4];
        const Row5 e1r = {0.0, 0.0, B1[1] - fe * B2[1], B1[2] - fe * B2[2], B1[3] - fe * B2[3]};
        const double ge = BN[0] / B3[0];
        const Row5 eNr = {BN[1] - ge * B3[1], BN[2] - ge * B3[2], BN[3] - ge * B3[3], 0.0, 0.0};
        ok &= band_lu(d, d.tab_lue, k, pair, [&](int i) -> Row5 {
            if (i == 1) return e1r;
            if (i == N - 2) return eNr;
            double A[5];
            erow_full(i, A);
            Row5 R = {A[0], A[1], A[2], A[3], A[4]};
            if (i == 2) R.a = 0.0;
            if (i == N - 3) R.e = 0.0;
            return R;
        });
        TAB(d.tab_lue, k, 0, 0) = fe;
        TAB(d.tab_lue, k, N - 1, 0) = ge;
    }
    if (!ok) atomicOr(d.flag + 1, 1);
}

// ---------------------------------------------------------------------------
// u, w from v, eta (continuity and the definition of eta):
//   Dv: 0 on rows 0, Nr-1; explicit one-sided rows 1, Nr-2; compact rows
//       d0 . Dv = l1 . v on rows 2..Nr-3 (solved with the reversed
//       factorisation dsol, the elimination running from the outer wall in);
//   u = (i alpha D_*v - (i m/r) eta)/k^2,   w = ((i m/r) D_*v + i alpha eta)/k^2.
// z_j of the elimination is kept in u[j] until the ascending pass.
__device__ void reconstruct_pair(const TcDev& d, int pair, double m, double al, long long partner) {
    const int N = d.Nr;
    const size_t P = d.npairs;
    double2 xw[5];
    for (int s = 0; s < 5; ++s) xw[s] = cz();
    double2 Dv1 = cz(), DvN = cz();
    double2 z1 = cz(), z2 = cz();     // z_{jr+1}, z_{jr+2}
    double2 r3 = cz(), r2 = cz();
    auto known = [&](int jr, double2 rhs) -> double2 {
        const double* w0 = d.d0 + jr * 5;
        if (jr + 1 == N - 2) rhs = caxpy(rhs, -w0[3], DvN);
        if (jr + 2 == N - 2) rhs = caxpy(rhs, -w0[4], DvN);
        if (jr - 1 == 1) rhs = caxpy(rhs, -w0[1], Dv1);
        if (jr - 2 == 1) rhs = caxpy(rhs, -w0[0], Dv1);
        return rhs;
    };
    auto elim = [&](int jr, double2 rhs) {
        const double* q = d.dsol + jr * 5;
        double2 z = caxpy(caxpy(known(jr, rhs), -q[0], z2), -q[1], z1);
        d.u[(size_t)jr * P + pair] = z;
        z2 = z1;
        z1 = z;
    };
    for (int i = N - 1; i >= 0; --i) {
        for (int s = 4; s > 0; --s) xw[s] = xw[s - 1];
        xw[0] = d.v[(size_t)i * P + pair];
        if (i > N - 5) continue;
        if (i == N - 5) {                       // one-sided row N-2
            const double* w = d.l1 + (N - 2) * 5;
            double2 acc = cz();
            for (int s = 0; s < 5; ++s) acc = caxpy(acc, w[s], xw[s]);
            DvN = acc;
        }
        const int jr = i + 2;
        if (jr >= 2 && jr <= N - 3) {
            const double* w = d.l1 + jr * 5;
            double2 acc = cz();
            for (int s = 0; s < 5; ++s) acc = caxpy(acc, w[s], xw[s]);
            if (jr >= 4) elim(jr, acc);
            else if (jr == 3) r3 = acc;
            else r2 = acc;
        }
        if (i == 0) {                           // one-sided row 1
            const double* w = d.l1 + 1 * 5;
            double2 acc = cz();
            for (int s = 0; s < 5; ++s) acc = caxpy(acc, w[s], xw[s]);
            Dv1 = acc;
        }
    }
    if (N - 3 >= 3) elim(3, r3);
    elim(2, r2);
    // ascending: back substitution and u, w
    double2 p1 = cz(), p2 = cz();               // Dv_{i-1}, Dv_{i-2} among unknowns 2..N-3
    for (int i = 0; i < N; ++i) {
        double2 Dv;
        if (i == 0 || i == N - 1) Dv = cz();
        else if (i == 1) Dv = Dv1;
        else if (i == N - 2) Dv = DvN;
        else {
            const double* q = d.dsol + i * 5;
            const double2 z = d.u[(size_t)i * P + pair];
            Dv = cscale(q[2], caxpy(caxpy(z, -q[3], p1), -q[4], p2));
            p2 = p1;
            p1 = Dv;
        }
        const double ri = d.rinv[i];
        const double c = d.tab_c[(size_t)i * P + pair];
        const double2 V = d.v[(size_t)i * P + pair];
        const double2 E = d.eta[(size_t)i * P + pair];
        const double2 Dsv = caxpy(Dv, ri, V);
        // u = i (c alpha Dsv - c m/r eta), w = i (c m/r Dsv + c alpha eta)
        const double ca = c * al, cm = c * m * ri;
        const double2 uu = ci(make_double2(fma(ca, Dsv.x, -cm * E.x), fma(ca, Dsv.y, -cm * E.y)));
        const double2 ww = ci(make_double2(fma(cm, Dsv.x, ca * E.x), fma(cm, Dsv.y, ca * E.y)));
        d.u[(size_t)i * P + pair] = uu;
        d.w[(size_t)i * P + pair] = ww;
        if (partner >= 0) {
            d.u[(size_t)i * P + partner] = cconj(uu);
            d.w[(size_t)i * P + partner] = cconj(ww);
        }
    }
}

// ---------------------------------------------------------------------------
// One substep of the line phase, one thread per Fourier pair, for the pairs
// of the azimuthal columns ja .. ja + jw - 1 in every axial slot (all pairs
// when ja = 0, jw = Ntheta/2).
//
// Explicit rows E (Eq. 6 rows 2..Nr-3, Eq. 7 rows 1..Nr-2) are sums over the
// 5 stencil points of d0 . A + l1 . B (+ l2 . C for v), where A, B, C are
// pointwise "inner" functions of the products and of u, v, w at that point.
// With the five products a = uu - vv, uv, uw, vw, b = ww - vv:
//   v:   A = -i alpha uv - i m/r vw + b/r                 - 2 i nu m w/r^2
//        B = i alpha c1 uv - i m (2c/r^2 - c1/r) vw + c alpha^2 a
//            + 2 c alpha m/r uw + c m^2/r^2 b             - 2 i nu m c1 w/r^2
//        C = -i alpha c uv - i m c/r vw                   + 2 i nu m c w/r^2
//            - 3 nu c1 (i alpha u + i m/r w)              [continuity term]
//   eta: A = m alpha a/r - 2 i m uv/r^2 + (m^2/r^2 - alpha^2) uw - alpha m b/r
//            + 2 i alpha vw/r + 4 i nu m u/r^3 + 2 nu m alpha v/r^2
//        B = -i m uv/r + i alpha vw + 2 i nu m u/r^2
// (the terms of Eqs. 6-7 regrouped per stencil; the vv parts cancel because
// c k^2 = 1).  In the mixed form everything except the continuity term is
// formed in float32 from the float32 products, and the continuity term in
// double-float arithmetic; in the double-float form all explicit rows are
// formed in double-float arithmetic (float32 pipe) from the double-float
// products; the right sides, the solves, the RK memory and the
// reconstruction are float64 in every form.
//
// Inner functions of the explicit rows at one radial point, from the five
// products and u, v, w: A, B, C of the v rows (C without the continuity
// term) and A, B of the eta rows, as listed above.
template <typename T, typename CT>
__device__ __forceinline__ void inner_terms(const CT& pa, const CT& uv, const CT& uw, const CT& vw, const CT& pb,
                                            const CT& U, const CT& V, const CT& W, T ri, T c, T c1,
                                            T mt, T at, T nut, CT& a, CT& b, CT& cc, CT& ae, CT& be) {
    const T ri2 = ri * ri;
    // v rows
    a = timag(-at, uv);
    a = tadd(a, timag(-mt * ri, vw));
    a = taxpy(a, ri, pb);
    a = tadd(a, timag((T)-2 * nut * mt * ri2, W));
    b = timag(at * c1, uv);
    b = tadd(b, timag(-mt * ((T)2 * c * ri2 - c1 * ri), vw));
    b = taxpy(b, c * at * at, pa);
    b = taxpy(b, c * (T)2 * at * mt * ri, uw);
    b = taxpy(b, c * mt * mt * ri2, pb);
    b = tadd(b, timag((T)-2 * nut * mt * c1 * ri2, W));
    cc = timag(-at * c, uv);
    cc = tadd(cc, timag(-mt * c * ri, vw));
    cc = tadd(cc, timag((T)2 * nut * mt * c * ri2, W));
    // eta rows
    ae = tscale(mt * at * ri, pa);
    ae = tadd(ae, timag((T)-2 * mt * ri2, uv));
    ae = taxpy(ae, mt * mt * ri2 - at * at, uw);
    ae = taxpy(ae, -at * mt * ri, pb);
    ae = tadd(ae, timag((T)2 * at * ri, vw));
    ae = tadd(ae, timag((T)4 * nut * mt * ri2 * ri, U));
    ae = taxpy(ae, (T)2 * nut * mt * at * ri2, V);
    be = timag(-mt * ri, uv);
    be = tadd(be, timag(at, vw));
    be = tadd(be, timag((T)2 * nut * mt * ri2, U));
}

// k^2 = alpha^2 + m^2/r^2 of the implicit eta band, rounded the same way in
// every kernel that forms it
__device__ __forceinline__ double k2_at(double m, double al, double ri) {
    return __fma_rn(__dmul_rn(m, m), __dmul_rn(ri, ri), __dmul_rn(al, al));
}

// Implicit part of the next RK memory on row jr (SMR91 low storage):
// H_(k+1) += (beta_k + alpha_(k+1)) dt L x^(k+1), with L the v band of row jr
// (the per-pair table) or nu (l2 - d0 k^2) of the eta row, applied to the
// window xw / ew of x^(k+1) on the row's five stencil points (k2w: k^2 at
// those points).  The line kernel calls it during its back substitution; the
// deferred form (k_rk_memory) calls it after a line kernel that left it out,
// with the same operands, so both give the same bits.
__device__ __forceinline__ void rk_memory_row(const TcDev& d, int pair, int jr, const double2* xw, const double2* ew,
                                              const double* k2w, double hdt, double hdtnu, bool do_v, bool do_e) {
    const size_t o = (size_t)jr * d.npairs + pair;
    if (do_v) {
        double2 acc = cz();
        for (int s = 0; s < 5; ++s) acc = caxpy(acc, TAB(d.tab_lv, 0, jr, s), xw[s]);
        d.Hv[o] = caxpy(d.Hv[o], hdt, acc);
    }
    if (do_e) {
        double2 acc = cz();
        for (int s = 0; s < 5; ++s)
            acc = caxpy(acc, fma(-d.d0[jr * 5 + s], k2w[s], d.l2[jr * 5 + s]), ew[s]);
        d.He[o] = caxpy(d.He[o], hdtnu, acc);
    }
}

// The sweeps of one pair (ROLE 0: v and eta; 1: v only; 2: eta only, for the
// kernel in which one thread advances v and another eta of the same pair);
// returns false for a thread without a pair to evolve.  The arithmetic of
// each field is the same in every role.  With NOH the implicit part of the
// next RK memory is left to k_rk_memory (launched after this kernel, before
// the next substep's line kernel).
// Roles 1 and 2 run in two warps of one block and keep step: the eta thread
// reads v of the old state at row i while the v thread overwrites row i - 2
// with its elimination, so a block barrier opens every iteration of the
// forward sweep and closes the sweep.  Every thread of such a block runs the
// same loop: a thread without a pair works on a stand-in pair (n = 0,
// j = 1, always evolved) and stores nothing.
template <int MODE, int ROLE, bool NOH = false>
__device__ __forceinline__ bool line_sweeps(const TcDev& d, int k, int ja, int jw, const int idx, int& pair_out,
                                            double& m_out, double& al_out, long long& partner_out) {
    constexpr bool MIXED = (MODE == 1);
    constexpr bool DV = ROLE != 2, DE = ROLE != 1;
    typedef typename LineTypes<MODE>::T T;
    typedef typename LineTypes<MODE>::CT CT;
    constexpr bool SYNC = ROLE != 0;
    // thread idx -> pair among the columns ja .. ja + jw - 1 of every axial slot
    bool act = idx < d.Nz * jw;
    int pair = act ? (idx / jw) * d.Nh + ja + idx % jw : 0;
    double m = 0.0, al = 0.0;
    long long partner = -1;
    if (act) act = pair_info(d, pair, m, al, partner);
    if (!act) {
        if constexpr (!SYNC) return false;
        pair = 1;                                   // stand-in: loads only
        pair_info(d, pair, m, al, partner);
        partner = -1;
    }
    pair_out = pair; m_out = m; al_out = al; partner_out = partner;
    const int N = d.Nr;
    const size_t P = d.npairs;
    const CT* prod = reinterpret_cast<const CT*>(d.prod);
    const size_t PS = (size_t)N * P;            // product stride
    const int kn = (k + 1) % 3;
    const double gdt = d.rk_gamma[k] * d.dt;
    const double zdt = d.rk_zeta[kn] * d.dt;
    const double hdt = (d.rk_beta[k] + d.rk_alpha[kn]) * d.dt;
    const double nu = d.nu;
    const T mt = (T)m, at = (T)al, nut = (T)nu;
    // double-float constants of the mixed form's continuity term
    const dfloat mD(m), alD(al), m3nu(-3.0 * nu);
    const dfloat* l2x = reinterpret_cast<const dfloat*>(d.l2x);
    const dfloat* rinvx = reinterpret_cast<const dfloat*>(d.rinvx);
    const T* w0s;
    const T* w1s;
    const T* w2s;
    if constexpr (MODE == 1) { w0s = d.d0f; w1s = d.l1f; w2s = d.l2f; }
    else if constexpr (MODE == 2) {
        w0s = reinterpret_cast<const dfloat*>(d.d0x);
        w1s = reinterpret_cast<const dfloat*>(d.l1x);
        w2s = reinterpret_cast<const dfloat*>(d.l2x);
    } else { w0s = d.d0; w1s = d.l1; w2s = d.l2; }

    // ---- forward sweep: explicit rows, right sides, forward elimination ----
    CT Av[5], Bv[5], Cv[5], Ae[5], Be[5];
    dcomplex Cp[5];                             // continuity inner function (mixed form)
    for (int s = 0; s < 5; ++s) Av[s] = Bv[s] = Cv[s] = Ae[s] = Be[s] = tz<CT>();
    double2 yv1 = cz(), yv2 = cz(), ye1 = cz(), ye2 = cz();   // y_{j-1}, y_{j-2}
    double2 rv_prev = cz(), re_prev = cz(), re_row1 = cz();
    const double fv = TAB(d.tab_luv, k, 0, 0), gv = TAB(d.tab_luv, k, N - 1, 0);
    const double fe = TAB(d.tab_lue, k, 0, 0), ge = TAB(d.tab_lue, k, N - 1, 0);

    auto erow = [&](int j) -> double2 {          // explicit eta row j (start = i-4)
        CT acc = tz<CT>();
        for (int s = 0; s < 5; ++s) {
            acc = taxpy(acc, w0s[j * 5 + s], Ae[s]);
            acc = taxpy(acc, w1s[j * 5 + s], Be[s]);
        }
        return to_d2(acc);
    };
    auto vrow = [&](int j) -> double2 {
        CT acc = tz<CT>();
        for (int s = 0; s < 5; ++s) {
            acc = taxpy(acc, w0s[j * 5 + s], Av[s]);
            acc = taxpy(acc, w1s[j * 5 + s], Bv[s]);
            acc = taxpy(acc, w2s[j * 5 + s], Cv[s]);
        }
        double2 r;
        if constexpr (MIXED) {
            // float32 rows plus the continuity term -3 nu l2 . (c' phi) in
            // double-float, then widened to float64
            dcomplex cc;
            for (int s = 0; s < 5; ++s) cc = dc_fma(cc, l2x[j * 5 + s], Cp[s]);
            r = to_d2_bits(dc_fma(dc_of(acc), m3nu, cc));
        } else {
            r = to_d2(acc);
        }
        return r;
    };
    // right side of row j and the partial H_(k+1) (without the L x^k term)
    auto rhs_v = [&](int j, double2 E) -> double2 {
        const size_t o = (size_t)j * P + pair;
        const double2 r = caxpy(d.Hv[o], gdt, E);
        if (act) d.Hv[o] = caxpy(r, zdt, E);
        return r;
    };
    auto rhs_e = [&](int j, double2 E) -> double2 {
        const size_t o = (size_t)j * P + pair;
        const double2 r = caxpy(d.He[o], gdt, E);
        if (act) d.He[o] = caxpy(r, zdt, E);
        return r;
    };
    auto fwd_v = [&](int j, double2 r) {
        const double m2 = TAB(d.tab_luv, k, j, 0), m1 = TAB(d.tab_luv, k, j, 1);
        const double2 y = caxpy(caxpy(r, -m2, yv2), -m1, yv1);
        if (act) d.v[(size_t)j * P + pair] = y;
        yv2 = yv1; yv1 = y;
    };
    auto fwd_e = [&](int j, double2 r) {
        const double m2 = TAB(d.tab_lue, k, j, 0), m1 = TAB(d.tab_lue, k, j, 1);
        const double2 y = caxpy(caxpy(r, -m2, ye2), -m1, ye1);
        if (act) d.eta[(size_t)j * P + pair] = y;
        ye2 = ye1; ye1 = y;
    };

    for (int i = 0; i < N; ++i) {
        if constexpr (SYNC) __syncthreads();    // the two roles within one row of each other
        for (int s = 0; s < 4; ++s) {
            if constexpr (DV) { Av[s] = Av[s + 1]; Bv[s] = Bv[s + 1]; Cv[s] = Cv[s + 1]; Cp[s] = Cp[s + 1]; }
            if constexpr (DE) { Ae[s] = Ae[s + 1]; Be[s] = Be[s + 1]; }
        }
        {
            const size_t o = (size_t)i * P + pair;
            const CT pa = prod[o], uv = prod[o + PS], uw = prod[o + 2 * PS], vw = prod[o + 3 * PS], pb = prod[o + 4 * PS];
            const double2 Ud = d.u[o], Vd = d.v[o], Wd = d.w[o];
            const CT U = from_d2<CT>(Ud), V = from_d2<CT>(Vd), W = from_d2<CT>(Wd);
            T ri, c, c1;
            double c1d = 0.0;
            if constexpr (MODE == 1) { ri = d.rinvf[i]; c = d.tab_cx[o].x; c1 = d.tab_c1x[o].x; }
            else if constexpr (MODE == 2) { ri = as_df(d.rinvx[i]); c = as_df(d.tab_cx[o]); c1 = as_df(d.tab_c1x[o]); }
            else { ri = d.rinv[i]; c = d.tab_c[o]; c1d = d.tab_c1[o]; c1 = c1d; }
            CT a, b, cc, ae, be;
            inner_terms(pa, uv, uw, vw, pb, U, V, W, ri, c, c1, mt, at, nut, a, b, cc, ae, be);
            if constexpr (DV) {
                if constexpr (MODE == 1) {
                    // phi = i alpha u + (i m/r) w, times c', in double-float
                    const dcomplex phi = dc_i(dc_fma(dc_scale(alD, dc_bits(Ud)), mD * rinvx[i], dc_bits(Wd)));
                    Cp[4] = dc_scale(as_df(d.tab_c1x[o]), phi);
                } else if constexpr (MODE == 2) {
                    const CT phi = tadd(timag(at, U), timag(mt * ri, W));
                    cc = taxpy(cc, (T)(-3.0 * nu) * c1, phi);
                } else {
                    const double2 phi = cadd(cimag(al, Ud), cimag(m * d.rinv[i], Wd));
                    cc = caxpy(cc, -3.0 * nu * c1d, phi);
                }
                Av[4] = a; Bv[4] = b; Cv[4] = cc;
            }
            if constexpr (DE) { Ae[4] = ae; Be[4] = be; }
        }
        if (i < 4) continue;
        const int j = i - 2;
        if (i == 4) {
            if constexpr (DE) re_row1 = rhs_e(1, erow(1));
            if constexpr (DV) {
                const double2 rv2 = rhs_v(2, vrow(2));
                fwd_v(1, cscale(-fv, rv2));
                fwd_v(2, rv2);
                rv_prev = rv2;
            }
            if constexpr (DE) {
                const double2 re2 = rhs_e(2, erow(2));
                fwd_e(1, caxpy(re_row1, -fe, re2));
                fwd_e(2, re2);
                re_prev = re2;
            }
        } else if (j <= N - 3) {
            if constexpr (DV) {
                const double2 rv = rhs_v(j, vrow(j));
                fwd_v(j, rv);
                rv_prev = rv;
            }
            if constexpr (DE) {
                const double2 re = rhs_e(j, erow(j));
                fwd_e(j, re);
                re_prev = re;
            }
        }
        if (i == N - 1) {
            if constexpr (DV) fwd_v(N - 2, cscale(-gv, rv_prev));
            if constexpr (DE) {
                const double2 reN = rhs_e(N - 2, erow(N - 2));
                fwd_e(N - 2, caxpy(reN, -ge, re_prev));
            }
        }
    }

    if constexpr (SYNC) __syncthreads();        // the forward reads of both roles are done
    // ---- backward sweep: back substitution, H_(k+1) += (beta+alpha') dt L x ----
    double2 xw[5], ew[5];
    double k2w[5];
    for (int s = 0; s < 5; ++s) { xw[s] = cz(); ew[s] = cz(); k2w[s] = 0.0; }
    bool bad = false;
    if constexpr (!NOH) k2w[0] = k2_at(m, al, d.rinv[N - 1]);
    if (act) {
        if constexpr (DV) d.v[(size_t)(N - 1) * P + pair] = cz();
        if constexpr (DE) d.eta[(size_t)(N - 1) * P + pair] = cz();
    }
    const double hdtnu = hdt * nu;
    auto h_update = [&](int jr, bool do_v, bool do_e) {
        if constexpr (!NOH) rk_memory_row(d, pair, jr, xw, ew, k2w, hdt, hdtnu, do_v && DV && act, do_e && DE && act);
    };
    for (int i = N - 2; i >= 0; --i) {
        for (int s = 4; s > 0; --s) { xw[s] = xw[s - 1]; ew[s] = ew[s - 1]; k2w[s] = k2w[s - 1]; }
        if constexpr (!NOH) k2w[0] = k2_at(m, al, d.rinv[i]);
        if (i >= 1) {
            const size_t o = (size_t)i * P + pair;
            if constexpr (DV) {
                const double2 yv = d.v[o];
                const double2 xv = cscale(TAB(d.tab_luv, k, i, 2),
                                          caxpy(caxpy(yv, -TAB(d.tab_luv, k, i, 3), xw[1]), -TAB(d.tab_luv, k, i, 4), xw[2]));
                bad |= !cfinite(xv);
                xw[0] = xv;
                if (act) {
                    d.v[o] = xv;
                    if (partner >= 0) d.v[(size_t)i * P + partner] = cconj(xv);
                }
            }
            if constexpr (DE) {
                const double2 ye = d.eta[o];
                const double2 xe = cscale(TAB(d.tab_lue, k, i, 2),
                                          caxpy(caxpy(ye, -TAB(d.tab_lue, k, i, 3), ew[1]), -TAB(d.tab_lue, k, i, 4), ew[2]));
                bad |= !cfinite(xe);
                ew[0] = xe;
                if (act) {
                    d.eta[o] = xe;
                    if (partner >= 0) d.eta[(size_t)i * P + partner] = cconj(xe);
                }
            }
        } else {
            xw[0] = cz(); ew[0] = cz();
            if (act) {
                if constexpr (DV) d.v[pair] = cz();
                if constexpr (DE) d.eta[pair] = cz();
            }
        }
        if (i == N - 5) h_update(N - 2, false, true);          // one-sided eta row N-2
        const int jr = i + 2;
        if (i <= N - 5 && jr >= 2) h_update(jr, true, true);
        if (i == 0) h_update(1, false, true);                  // one-sided eta row 1
    }
    if (bad && act) atomicOr(d.flag, 1);
    if (act && partner >= 0) {
        if constexpr (DV) { d.v[(size_t)(N - 1) * P + partner] = cz(); d.v[partner] = cz(); }
        if constexpr (DE) { d.eta[(size_t)(N - 1) * P + partner] = cz(); d.eta[partner] = cz(); }
    }
    return act;
}

template <int MODE, bool NOH = false>
__device__ __forceinline__ void line_body(const TcDev& d, int k, int ja, int jw, const int idx) {
    int pair;
    double m, al;
    long long partner;
    if (line_sweeps<MODE, 0, NOH>(d, k, ja, jw, idx, pair, m, al, partner)) reconstruct_pair(d, pair, m, al, partner);
}

// Kernel variants: a register budget from launch bounds (threads per block,
// resident blocks per SM), or an explicit register cap.
template <int MODE, int MAXT, int MINB, bool NOH = false>
__global__ void __launch_bounds__(MAXT, MINB) k_line(TcDev d, int k, int ja, int jw) {
    line_body<MODE, NOH>(d, k, ja, jw, blockIdx.x * blockDim.x + threadIdx.x);
}
template <int MODE, int NREG, bool NOH = false>
__global__ void __maxnreg__(NREG) k_line_r(TcDev d, int k, int ja, int jw) {
    line_body<MODE, NOH>(d, k, ja, jw, blockIdx.x * blockDim.x + threadIdx.x);
}
// Split variant for few pairs (a short line phase is bound by the latency
// of one thread's radial recurrences): blocks of 64 threads, the first warp
// advances v and the second eta of the same 32 pairs, then, after the block
// barrier, the first warp rebuilds u and w.  The same arithmetic per field
// as k_line.
template <int MODE, bool NOH = false>
__global__ void __launch_bounds__(64) k_line_s(TcDev d, int k, int ja, int jw) {
    const int lane = threadIdx.x & 31;
    const bool vrole = threadIdx.x < 32;
    const int idx = blockIdx.x * 32 + lane;
    int pair = 0;
    double m = 0.0, al = 0.0;
    long long partner = -1;
    bool act;
    if (vrole) act = line_sweeps<MODE, 1, NOH>(d, k, ja, jw, idx, pair, m, al, partner);
    else act = line_sweeps<MODE, 2, NOH>(d, k, ja, jw, idx, pair, m, al, partner);
    __syncthreads();
    if (vrole && act) reconstruct_pair(d, pair, m, al, partner);
}

// The implicit part of the next RK memory (rk_memory_row) for the pairs of
// the columns ja .. ja + jw - 1, after a line kernel of substep k launched
// with NOH: one thread per pair walks its radial line downwards like the
// back substitution, reading x^(k+1) (v, eta) instead of computing it.  It
// needs only the results of that line kernel, so it can run beside the next
// substep's plane phase.
// Grid-stride over the pairs: launched beside the theta rows it runs in few
// blocks (four per SM), so that it takes mostly what the rows leave free.
__global__ void __launch_bounds__(128) k_rk_memory(TcDev d, int k, int ja, int jw) {
    const int N = d.Nr;
    const size_t P = d.npairs;
    const int kn = (k + 1) % 3;
    const double hdt = (d.rk_beta[k] + d.rk_alpha[kn]) * d.dt;
    const double hdtnu = hdt * d.nu;
    const int n = d.Nz * jw;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        const int pair = (idx / jw) * d.Nh + ja + idx % jw;
        double m, al;
        long long partner;
        if (!pair_info(d, pair, m, al, partner)) continue;
        double2 xw[5], ew[5];
        double k2w[5];
        for (int s = 0; s < 5; ++s) { xw[s] = cz(); ew[s] = cz(); k2w[s] = 0.0; }
        k2w[0] = k2_at(m, al, d.rinv[N - 1]);
        for (int i = N - 2; i >= 0; --i) {
            for (int s = 4; s > 0; --s) { xw[s] = xw[s - 1]; ew[s] = ew[s - 1]; k2w[s] = k2w[s - 1]; }
            k2w[0] = k2_at(m, al, d.rinv[i]);
            if (i >= 1) {
                xw[0] = d.v[(size_t)i * P + pair];
                ew[0] = d.eta[(size_t)i * P + pair];
            } else {
                xw[0] = cz(); ew[0] = cz();
            }
            if (i == N - 5) rk_memory_row(d, pair, N - 2, xw, ew, k2w, hdt, hdtnu, false, true);
            const int jr = i + 2;
            if (i <= N - 5 && jr >= 2) rk_memory_row(d, pair, jr, xw, ew, k2w, hdt, hdtnu, true, true);
            if (i == 0) rk_memory_row(d, pair, 1, xw, ew, k2w, hdt, hdtnu, false, true);
        }
    }
}

// Many cases in one launch: blocks of 128 threads, bmap[block] = (case,
// block within the case), the case's descriptor from ds.
template <int MODE>
__global__ void __launch_bounds__(128, 4) k_line_b(const TcDev* __restrict__ ds, const int2* __restrict__ bmap, int k) {
    const int2 m = bmap[blockIdx.x];
    const TcDev& d = ds[m.x];
    line_body<MODE>(d, k, 0, d.Nh, m.y * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Initial RK memory H_1 = (M + alpha_1 dt L) x for v and eta, and u, w.
__global__ void __launch_bounds__(128) k_init(TcDev d) {
    const int pair = blockIdx.x * blockDim.x + threadIdx.x;
    if (pair >= d.npairs) return;
    double m, al;
    long long partner;
    if (!pair_info(d, pair, m, al, partner)) return;
    const int N = d.Nr;
    const size_t P = d.npairs;
    const double adt = d.rk_alpha[0] * d.dt;
    for (int j = 0; j < N; ++j) {
        const size_t o = (size_t)j * P + pair;
        double2 hv = cz(), he = cz();
        if (j >= 2 && j <= N - 3) {
            // mass band M = d0 - l2 c + l1 c' from the c, c' tables, implicit
            // band L from the table of k_setup
            for (int s = 0; s < 5; ++s) {
                const size_t oi = (size_t)(j - 2 + s) * P + pair;
                const double M5 = d.d0[j * 5 + s] - d.l2[j * 5 + s] * d.tab_c[oi] + d.l1[j * 5 + s] * d.tab_c1[oi];
                hv = caxpy(hv, M5 + adt * TAB(d.tab_lv, 0, j, s), d.v[oi]);
            }
        }
        if (j >= 1 && j <= N - 2) {
            const int st = d.start[j];
            for (int s = 0; s < 5; ++s) {
                const double ri = d.rinv[st + s];
                const double L5 = d.nu * (d.l2[j * 5 + s] - d.d0[j * 5 + s] * (al * al + m * m * ri * ri));
                const double2 x = d.eta[(size_t)(st + s) * P + pair];
                he = caxpy(he, d.d0[j * 5 + s] + adt * L5, x);
            }
        }
        d.Hv[o] = hv;
        d.He[o] = he;
    }
    reconstruct_pair(d, pair, m, al, partner);
}

// ---------------------------------------------------------------------------
// Mean flow (m = alpha = 0), zero mean pressure gradient (Sec. 4):
//   dW/dt = nu D D_* W - D(vw) - 2 vw/r,   dU/dt = nu (D D_* U + U/r^2) - D(uv) - uv/r,
// rows 1..Nr-2 with Dirichlet values W(R_i) = 1, W(R_o) = Re_o/Re_i, U = 0.
// One block: rows are assembled in parallel into shared memory, then two
// threads run the banded eliminations (U and W) serially.
template <typename PT>
__device__ __forceinline__ void mean_body(const TcDev& d, int k, int init) {
    extern __shared__ double sm[];
    const int N = d.Nr;
    double* A = sm;                    // [2][N][5] system rows
    double* Lb = A + 2 * N * 5;        // [2][N][5] implicit rows
    double* rhs = Lb + 2 * N * 5;      // [2][N]
    double* x = rhs + 2 * N;           // [2][N]
    double* Ex = x + 2 * N;            // [2][N] explicit rows
    const PT* prod = reinterpret_cast<const PT*>(d.prod);
    const size_t PS = (size_t)N * d.npairs;
    const int kn = (k + 1) % 3;
    const double bdt = d.rk_beta[k] * d.dt;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        x[j] = d.U[j];
        x[N + j] = d.W[j];
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        if (j < 1 || j > N - 2) continue;
        const int st = d.start[j];
        double eu = 0.0, ew = 0.0;
        for (int s = 0; s < 5; ++s) {
            const int i = st + s;
            const double w0 = d.d0[j * 5 + s], w1 = d.l1[j * 5 + s], w2 = d.l2[j * 5 + s];
            const double ri = d.rinv[i];
            Lb[(0 * N + j) * 5 + s] = d.nu * (w2 + w0 * ri * ri);   // U
            Lb[(1 * N + j) * 5 + s] = d.nu * w2;                    // W
            if (!init) {
                const double uv = ld_prod(prod, (size_t)i * d.npairs + PS).x;
                const double vw = ld_prod(prod, (size_t)i * d.npairs + 3 * PS).x;
                eu += -w1 * uv - w0 * uv * ri;
                ew += -w1 * vw - 2.0 * w0 * vw * ri;
            }
        }
        Ex[j] = eu;
        Ex[N + j] = ew;
    }
    __syncthreads();
    if (init) {
        // H_1 = (M + alpha_1 dt L) x, and u(0,0) = U, w(0,0) = W
        const double adt = d.rk_alpha[0] * d.dt;
        for (int j = threadIdx.x; j < N; j += blockDim.x) {
            double hu = 0.0, hw = 0.0;
            if (j >= 1 && j <= N - 2) {
                const int st = d.start[j];
                for (int s = 0; s < 5; ++s) {
                    hu += (d.d0[j * 5 + s] + adt * Lb[j * 5 + s]) * x[st + s];
                    hw += (d.d0[j * 5 + s] + adt * Lb[(N + j) * 5 + s]) * x[N + st + s];
                }
            }
            d.HU[j] = hu;
            d.HW[j] = hw;
            d.u[(size_t)j * d.npairs] = make_double2(x[j], 0.0);
            d.w[(size_t)j * d.npairs] = make_double2(x[N + j], 0.0);
        }
        return;
    }
    // right sides and system rows
    const double gdt = d.rk_gamma[k] * d.dt, zdt = d.rk_zeta[kn] * d.dt;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        for (int p = 0; p < 2; ++p) {
            double* H = p == 0 ? d.HU : d.HW;
            if (j >= 1 && j <= N - 2) {
                const double rr = H[j] + gdt * Ex[p * N + j];
                rhs[p * N + j] = rr;
                H[j] = rr + zdt * Ex[p * N + j];
                for (int s = 0; s < 5; ++s)
                    A[(p * N + j) * 5 + s] = d.d0[j * 5 + s] - bdt * Lb[(p * N + j) * 5 + s];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int p = threadIdx.x;
        const double b0 = p == 0 ? 0.0 : 1.0;                 // value at r_0
        const double bN = p == 0 ? 0.0 : d.W_outer;           // value at r_{N-1}
        double* Ap = A + p * N * 5;
        double* rp = rhs + p * N;
        double* xp = x + p * N;
        // move the Dirichlet columns to the right side
        for (int j = 1; j <= N - 2; ++j) {
            const int st = d.start[j];
            if (st == 0) { rp[j] -= Ap[j * 5 + 0] * b0; Ap[j * 5 + 0] = 0.0; }
            if (st + 4 == N - 1) { rp[j] -= Ap[j * 5 + 4] * bN; Ap[j * 5 + 4] = 0.0; }
        }
        // reduced rows on unknowns 1..N-2: (a, b, d, c, e) about the diagonal
        auto reduced = [&](int j, double* R) {
            const int off = d.start[j] - (j - 2);   // 0 for centred rows
            for (int t = 0; t < 5; ++t) R[t] = 0.0;
            for (int s = 0; s < 5; ++s) {
                const int t = s + off;
                if (t >= 0 && t < 5) R[t] = Ap[j * 5 + s];
            }
        };
        // row 1 reaches column 4 (t = 5) and row N-2 column N-5 (t = -1):
        // fold them with rows 2 and N-3
        double R1[5], R2[5], R3[5], RN[5];
        reduced(2, R2);
        reduced(N - 3, R3);
        {
            const double f = Ap[1 * 5 + 4] / R2[4];
            for (int t = 0; t < 5; ++t) R1[t] = 0.0;
            R1[2] = Ap[1 * 5 + 1] - f * R2[1];
            R1[3] = Ap[1 * 5 + 2] - f * R2[2];
            R1[4] = Ap[1 * 5 + 3] - f * R2[3];
            rp[1] -= f * rp[2];
            const double g = Ap[(N - 2) * 5 + 0] / R3[0];
            for (int t = 0; t < 5; ++t) RN[t] = 0.0;
            RN[0] = Ap[(N - 2) * 5 + 1] - g * R3[1];
            RN[1] = Ap[(N - 2) * 5 + 2] - g * R3[2];
            RN[2] = Ap[(N - 2) * 5 + 3] - g * R3[3];
            rp[N - 2] -= g * rp[N - 3];
        }
        // forward elimination (multipliers in place of the row)
        double p2d = 1, p2c = 0, p2e = 0, p1d = 1, p1c = 0, p1e = 0;
        double y1 = 0, y2 = 0;
        double* U3 = Lb + p * N * 5;                     // reuse: (1/d, c, e)
        for (int i = 1; i <= N - 2; ++i) {
            double R[5];
            if (i == 1) for (int t = 0; t < 5; ++t) R[t] = R1[t];
            else if (i == N - 2) for (int t = 0; t < 5; ++t) R[t] = RN[t];
            else reduced(i, R);
            const double m2 = (i >= 3) ? R[0] / p2d : 0.0;
            double b = R[1] - m2 * p2c, dd = R[2] - m2 * p2e;
            const double m1 = (i >= 2) ? b / p1d : 0.0;
            dd -= m1 * p1c;
            const double cc = R[3] - m1 * p1e;
            const double y = rp[i] - m2 * y2 - m1 * y1;
            U3[i * 5 + 0] = 1.0 / dd; U3[i * 5 + 1] = cc; U3[i * 5 + 2] = R[4];
            rp[i] = y;
            y2 = y1; y1 = y;
            p2d = p1d; p2c = p1c; p2e = p1e;
            p1d = dd; p1c = cc; p1e = R[4];
        }
        double x1 = 0, x2 = 0;
        for (int i = N - 2; i >= 1; --i) {
            const double xi = (rp[i] - U3[i * 5 + 1] * x1 - U3[i * 5 + 2] * x2) * U3[i * 5 + 0];
            xp[i] = xi;
            x2 = x1; x1 = xi;
        }
        xp[0] = b0;
        xp[N - 1] = bN;
    }
    __syncthreads();
    // H_(k+1) += (beta_k + alpha_(k+1)) dt L x, write the profiles
    const double hdt = (d.rk_beta[k] + d.rk_alpha[kn]) * d.dt;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        if (j >= 1 && j <= N - 2) {
            const int st = d.start[j];
            double lu = 0.0, lw = 0.0;
            for (int s = 0; s < 5; ++s) {
                const int i = st + s;
                const double w0 = d.d0[j * 5 + s], w2 = d.l2[j * 5 + s], ri = d.rinv[i];
                lu += d.nu * (w2 + w0 * ri * ri) * x[i];
                lw += d.nu * w2 * x[N + i];
            }
            d.HU[j] += hdt * lu;
            d.HW[j] += hdt * lw;
        }
        d.U[j] = x[j];
        d.W[j] = x[N + j];
        d.u[(size_t)j * d.npairs] = make_double2(x[j], 0.0);
        d.w[(size_t)j * d.npairs] = make_double2(x[N + j], 0.0);
    }
}
template <typename PT>
__global__ void __launch_bounds__(256) k_mean(TcDev d, int k, int init) { mean_body<PT>(d, k, init); }
// one block per case of a shape class
template <typename PT>
__global__ void __launch_bounds__(256) k_mean_b(const TcDev* __restrict__ ds, int k) { mean_body<PT>(ds[blockIdx.x], k, 0); }

// ---------------------------------------------------------------------------
// Diagnostics: strain-rate density for the viscous dissipation.
//
// compact_D: first radial derivative of one Fourier slot of a field, the
// operator of the energy budget: explicit one-sided 5-point D on the walls
// (dwall) and on rows 1, Nr-2 (l1 rows with d0 = 1), compact rows
// d0 . Df = l1 . f on 2..Nr-3 solved with the reversed factorisation dsol
// (descending elimination, z kept in Df, then ascending substitution).
__device__ void compact_D(const TcDev& d, const double2* __restrict__ f, double2* Df, int pair) {
    const int N = d.Nr;
    const size_t P = d.npairs;
    auto F = [&](int i) { return f[(size_t)i * P + pair]; };
    double2 D0 = cz(), D1 = cz(), DN2 = cz(), DN1 = cz();
    for (int s = 0; s < 5; ++s) {
        D0 = caxpy(D0, d.dwall[s], F(s));
        DN1 = caxpy(DN1, d.dwall[5 + s], F(N - 5 + s));
        D1 = caxpy(D1, d.l1[5 + s], F(d.start[1] + s));
        DN2 = caxpy(DN2, d.l1[(N - 2) * 5 + s], F(d.start[N - 2] + s));
    }
    double2 z1 = cz(), z2 = cz();               // z_(jr+1), z_(jr+2)
    for (int jr = N - 3; jr >= 2; --jr) {
        const double* w0 = d.d0 + jr * 5;
        const double* w1 = d.l1 + jr * 5;
        double2 rhs = cz();
        for (int s = 0; s < 5; ++s) {
            const int c = jr - 2 + s;
            rhs = caxpy(rhs, w1[s], F(c));
            if (c == 0) rhs = caxpy(rhs, -w0[s], D0);
            else if (c == 1) rhs = caxpy(rhs, -w0[s], D1);
            else if (c == N - 2) rhs = caxpy(rhs, -w0[s], DN2);
            else if (c == N - 1) rhs = caxpy(rhs, -w0[s], DN1);
        }
        const double* q = d.dsol + jr * 5;
        const double2 z = caxpy(caxpy(rhs, -q[0], z2), -q[1], z1);
        Df[(size_t)jr * P + pair] = z;
        z2 = z1;
        z1 = z;
    }
    double2 p1 = cz(), p2 = cz();               // Df_(i-1), Df_(i-2) among 2..Nr-3
    for (int i = 2; i <= N - 3; ++i) {
        const double* q = d.dsol + i * 5;
        const double2 x = cscale(q[2], caxpy(caxpy(Df[(size_t)i * P + pair], -q[3], p1), -q[4], p2));
        Df[(size_t)i * P + pair] = x;
        p2 = p1;
        p1 = x;
    }
    Df[pair] = D0;
    Df[P + pair] = D1;
    Df[(size_t)(N - 2) * P + pair] = DN2;
    Df[(size_t)(N - 1) * P + pair] = DN1;
}

__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// One thread per Fourier slot (every slot; the (0,0) slot holds the mean
// flow U, W): 2 S:S with the cylindrical strain components
//   S_rr = Dv, S_tt = (i m/r) w + v/r, S_zz = i alpha u,
//   S_rt = (Dw - w/r + (i m/r) v)/2, S_rz = (i alpha v + Du)/2,
//   S_tz = ((i m/r) u + i alpha w)/2,
// times the Parseval weight (1 for m = 0, 2 otherwise), into dens[r][slot].
__global__ void __launch_bounds__(128) k_strain(TcDev d, double2* Du, double2* Dv, double2* Dw, double* dens) {
    const int pair = blockIdx.x * blockDim.x + threadIdx.x;
    if (pair >= d.npairs) return;
    const int sl = pair / d.Nh, j = pair - sl * d.Nh;
    const int n = sl < d.Nz / 2 ? sl : (sl == d.Nz / 2 ? 0 : sl - d.Nz);
    const double m = j * d.m0, al = n * d.alpha0;
    const double wgt = j == 0 ? 1.0 : 2.0;
    compact_D(d, d.u, Du, pair);
    compact_D(d, d.v, Dv, pair);
    compact_D(d, d.w, Dw, pair);
    const size_t P = d.npairs;
    for (int i = 0; i < d.Nr; ++i) {
        const size_t o = (size_t)i * P + pair;
        const double ri = d.rinv[i];
        const double2 U = d.u[o], V = d.v[o], W = d.w[o];
        const double2 srr = Dv[o];
        const double2 stt = caxpy(cimag(m * ri, W), ri, V);
        const double2 szz = cimag(al, U);
        const double2 srt = cscale(0.5, cadd(caxpy(Dw[o], -ri, W), cimag(m * ri, V)));
        const double2 srz = cscale(0.5, cadd(cimag(al, V), Du[o]));
        const double2 stz = cscale(0.5, cadd(cimag(m * ri, U), cimag(al, W)));
        dens[o] = wgt * (2.0 * (cabs2(srr) + cabs2(stt) + cabs2(szz)) +
                         4.0 * (cabs2(srt) + cabs2(srz) + cabs2(stz)));
    }
}

// dprof[r] = sum over slots of dens[r][slot] (fixed order: reproducible)
__global__ void __launch_bounds__(256) k_slot_sum(TcDev d, const double* __restrict__ dens) {
    const int r = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < d.npairs; i += blockDim.x) acc += dens[(size_t)r * d.npairs + i];
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) d.dprof[r] = red[0];
}

void tc_launch_strain(const TcDev& d, cudaStream_t s) {
    const size_t P1 = (size_t)d.Nr * d.npairs;   // <= Nr Mz Nh: fits the scratch
    double2* D = reinterpret_cast<double2*>(d.pbuf);
    double* dens = reinterpret_cast<double*>(d.zbuf);
    k_strain<<<(d.npairs + 127) / 128, 128, 0, s>>>(d, D, D + P1, D + 2 * P1, dens);
    k_slot_sum<<<d.Nr, 256, 0, s>>>(d, dens);
}

// ---------------------------------------------------------------------------
// After a field is set: zero the (0,0) slot and the axial Nyquist slot, and
// make the m = 0 column Hermitian (slot Nz - n = conj(slot n)), so that the
// field is real.  One thread per (r, element) of the j = 0 column and of the
// Nyquist slot.
__global__ void __launch_bounds__(256) k_realify(TcDev d, double2* f) {
    const int r = blockIdx.y;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int Nz = d.Nz, Nh = d.Nh;
    if (r >= d.Nr || idx >= Nz + Nh) return;
    double2* pl = f + (size_t)r * d.npairs;
    if (idx < Nz) {
        const int s = idx;                               // slot of the j = 0 column
        if (s == 0) pl[0] = cz();
        else if (s > Nz / 2) pl[(size_t)s * Nh] = cconj(pl[(size_t)(Nz - s) * Nh]);
    } else {
        pl[(size_t)(Nz / 2) * Nh + (idx - Nz)] = cz();   // Nyquist slot, every j
    }
}

void tc_launch_realify(const TcDev& d, double2* field, cudaStream_t s) {
    k_realify<<<dim3((d.Nz + d.Nh + 255) / 256, d.Nr), 256, 0, s>>>(d, field);
}

void tc_launch_setup_tables(const TcDev& d, cudaStream_t s) {
    k_setup<<<(d.npairs + 127) / 128, 128, 0, s>>>(d);
}

void tc_launch_line_phase(const TcDev& d, int k, cudaStream_t s) { tc_launch_line_chunk(d, k, s, 0, d.Nh); }

// line_block encodes the variant: 64/128/256 threads with the register
// budget of one 256-thread block per SM; 128 threads with a budget for 3
// (1003) or 4 (1004) resident blocks per SM; 64 threads capped at 144
// registers (2007: 7 resident blocks, 448 threads per SM, which splits 131 k
// pairs into 1.9 waves instead of 1.7); 3001: the split variant.  NOH
// (double-float and mixed forms only): without the implicit RK-memory term.
template <int MODE, bool NOH>
static void line_chunk_t(const TcDev& d, int k, cudaStream_t s, int ja, int jw) {
    const int v = d.line_block > 0 ? d.line_block : 128;
    if (v == 3001) {                    // split: 32 pairs per 64-thread block
        k_line_s<MODE, NOH><<<(d.Nz * jw + 31) / 32, 64, 0, s>>>(d, k, ja, jw);
        return;
    }
    const int bs = v == 2007 ? 64 : (v > 1000 ? 128 : v);
    const int grid = (d.Nz * jw + bs - 1) / bs;
    if (v == 1003) k_line<MODE, 128, 3, NOH><<<grid, bs, 0, s>>>(d, k, ja, jw);
    else if (v == 1004) k_line<MODE, 128, 4, NOH><<<grid, bs, 0, s>>>(d, k, ja, jw);
    else if (v == 2007) k_line_r<MODE, 144, NOH><<<grid, bs, 0, s>>>(d, k, ja, jw);
    else k_line<MODE, 256, 1, NOH><<<grid, bs, 0, s>>>(d, k, ja, jw);
}

void tc_launch_line_chunk(const TcDev& d, int k, cudaStream_t s, int ja, int jw) {
    if (d.prec == 1) line_chunk_t<1, false>(d, k, s, ja, jw);
    else if (d.prec == 2) line_chunk_t<2, false>(d, k, s, ja, jw);
    else line_chunk_t<0, false>(d, k, s, ja, jw);
}

void tc_launch_line_chunk_deferred(const TcDev& d, int k, cudaStream_t s, int ja, int jw) {
    if (d.prec == 1) line_chunk_t<1, true>(d, k, s, ja, jw);
    else if (d.prec == 2) line_chunk_t<2, true>(d, k, s, ja, jw);
    else line_chunk_t<0, false>(d, k, s, ja, jw);   // float64: never deferred
}

void tc_launch_rk_memory(const TcDev& d, int k, cudaStream_t s, int ja, int jw, bool background) {
    int blocks = (d.Nz * jw + 127) / 128;
    if (background) {
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
        }
        blocks = blocks < 4 * sms ? blocks : 4 * sms;
    }
    k_rk_memory<<<blocks, 128, 0, s>>>(d, k, ja, jw);
}

const void* tc_rk_memory_kernel() { return (const void*)k_rk_memory; }

static size_t mean_smem(const TcDev& d) { return (size_t)(2 * d.Nr * 5 * 2 + 2 * d.Nr * 3) * sizeof(double); }

void tc_launch_mean_phase(const TcDev& d, int k, cudaStream_t s) {
    if (d.prec == 1) k_mean<float2><<<1, 256, mean_smem(d), s>>>(d, k, 0);
    else if (d.prec == 2) k_mean<dcomplex><<<1, 256, mean_smem(d), s>>>(d, k, 0);
    else k_mean<double2><<<1, 256, mean_smem(d), s>>>(d, k, 0);
}

void tc_launch_line_batch(int prec, const TcDev* ds, const int2* bmap, int nblocks, int k, cudaStream_t s) {
    if (prec == 1) k_line_b<1><<<nblocks, 128, 0, s>>>(ds, bmap, k);
    else if (prec == 2) k_line_b<2><<<nblocks, 128, 0, s>>>(ds, bmap, k);
    else k_line_b<0><<<nblocks, 128, 0, s>>>(ds, bmap, k);
}

int tc_line_batch_block() { return 128; }

void tc_launch_mean_batch(int prec, const TcDev* ds, int ncases, int maxNr, int k, cudaStream_t s) {
    TcDev dm;
    dm.Nr = maxNr;
    if (prec == 1) k_mean_b<float2><<<ncases, 256, mean_smem(dm), s>>>(ds, k);
    else if (prec == 2) k_mean_b<dcomplex><<<ncases, 256, mean_smem(dm), s>>>(ds, k);
    else k_mean_b<double2><<<ncases, 256, mean_smem(dm), s>>>(ds, k);
}

cudaError_t tc_set_line_kernel_attributes() {
    const int lim = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute((const void*)k_mean<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute((const void*)k_mean<dcomplex>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    for (const void* f : {(const void*)k_mean_b<double2>, (const void*)k_mean_b<dcomplex>, (const void*)k_mean_b<float2>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute((const void*)k_mean<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

void tc_launch_init_state(const TcDev& d, cudaStream_t s) {
    k_init<<<(d.npairs + 127) / 128, 128, 0, s>>>(d);
    k_mean<double2><<<1, 256, mean_smem(d), s>>>(d, 0, 1);
}
