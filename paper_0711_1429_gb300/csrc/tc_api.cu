// C ABI of libtc: handle life cycle, host-side tables (radial grid, compact
// stencils, FFT plans and twiddles, the reversed factorisation of the
// averaging stencil), the captured Runge-Kutta step, field I/O and
// diagnostics.  See include/tc.h for the contract of every entry point.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <array>
#include <map>
#include <mutex>

#include "tc_host.h"

namespace {

thread_local std::string g_err;

#define CK(call)                                                                  \
    do {                                                                          \
        cudaError_t _e = (call);                                                  \
        if (_e != cudaSuccess) {                                                  \
            set_err(std::string(#call) + ": " + cudaGetErrorString(_e));          \
            return TC_ERR_CUDA;                                                   \
        }                                                                         \
    } while (0)

typedef long double ld;

// ---- exact-order dense solve in long double (partial pivoting) --------------
bool solve_ld(int n, std::vector<ld>& A, std::vector<ld>& b) {
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabsl(A[i * n + col]) > fabsl(A[piv * n + col])) piv = i;
        if (A[piv * n + col] == 0.0L) return false;
        if (piv != col) {
            for (int k = 0; k < n; ++k) std::swap(A[col * n + k], A[piv * n + k]);
            std::swap(b[col], b[piv]);
        }
        for (int i = col + 1; i < n; ++i) {
            const ld f = A[i * n + col] / A[col * n + col];
            if (f == 0.0L) continue;
            for (int k = col; k < n; ++k) A[i * n + k] -= f * A[col * n + k];
            b[i] -= f * b[col];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        ld s = b[i];
        for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * b[k];
        b[i] = s / A[i * n + i];
    }
    return true;
}

// Scaled monomial p_q(x) = ((x - xc)/h)^q and its derivatives times h^k:
// h^k D^k p_q = q!/(q-k)! ((x - xc)/h)^(q-k).
ld hder(int q, int k, ld x, ld xc, ld h) {
    if (k > q) return 0.0L;
    ld f = 1.0L;
    for (int t = 0; t < k; ++t) f *= (ld)(q - t);
    return f * powl((x - xc) / h, (ld)(q - k));
}
// h^n times the chain operators D, D D_*, D D_* D D_* applied to p_q at x
ld hop(int which, int q, ld x, ld xc, ld h) {
    const ld y = h / x;   // h/r
    switch (which) {
        case 0: return hder(q, 0, x, xc, h);
        case 1: return hder(q, 1, x, xc, h);
        case 2: return hder(q, 2, x, xc, h) + y * hder(q, 1, x, xc, h) - y * y * hder(q, 0, x, xc, h);
        default:
            return hder(q, 4, x, xc, h) + 2 * y * hder(q, 3, x, xc, h) - 3 * y * y * hder(q, 2, x, xc, h)
                   + 3 * y * y * y * hder(q, 1, x, xc, h) - 3 * y * y * y * y * hder(q, 0, x, xc, h);
    }
}



// Stencils of the 5-point compact explicit scheme (Sec. 2.1: five points,
// order at least 4, coefficients by polynomial matching; the paper leaves the
// construction open, and this is the reading used): interior rows make
// D D_* D D_* exact to degree 8 jointly with d0 (sum d0 = 1), then D D_* and
// D exact to degree 4 against that d0; near-wall rows 1, Nr-2 explicit
// one-sided to degree 4; wall derivative rows for the Neumann condition and
// the wall shear.
bool build_stencils(const std::vector<double>& r, HostStencils& S) {
    const int N = (int)r.size();
    S.start.assign(N, 0);
    S.d0.assign(N * 5, 0.0); S.l1.assign(N * 5, 0.0); S.l2.assign(N * 5, 0.0); S.l4.assign(N * 5, 0.0);
    S.dwall.assign(10, 0.0);
    for (int j = 2; j <= N - 3; ++j) {
        const int st = j - 2;
        S.start[j] = st;
        const ld xc = r[j], h = ((ld)r[st + 4] - (ld)r[st]) / 4.0L;
        std::vector<ld> A(100, 0.0L), b(10, 0.0L);
        for (int q = 0; q < 9; ++q) {
            for (int s = 0; s < 5; ++s) {
                A[q * 10 + s] = -hop(3, q, r[st + s], xc, h);       // d0 unknowns
                A[q * 10 + 5 + s] = hop(0, q, r[st + s], xc, h);    // h^4 l4 unknowns
            }
        }
        for (int s = 0; s < 5; ++s) A[9 * 10 + s] = 1.0L;
        b[9] = 1.0L;
        if (!solve_ld(10, A, b)) return false;
        ld d0[5];
        for (int s = 0; s < 5; ++s) {
            d0[s] = b[s];
            S.d0[j * 5 + s] = (double)b[s];
            S.l4[j * 5 + s] = (double)(b[5 + s] / (h * h * h * h));
        }
        for (int which = 1; which <= 2; ++which) {
            std::vector<ld> M(25), rhs(5);
            for (int q = 0; q < 5; ++q) {
                ld acc = 0.0L;
                for (int s = 0; s < 5; ++s) {
                    M[q * 5 + s] = hop(0, q, r[st + s], xc, h);
                    acc += d0[s] * hop(which, q, r[st + s], xc, h);
                }
                rhs[q] = acc;
            }
            if (!solve_ld(5, M, rhs)) return false;
            const ld hp = which == 1 ? h : h * h;
            for (int s = 0; s < 5; ++s) (which == 1 ? S.l1 : S.l2)[j * 5 + s] = (double)(rhs[s] / hp);
        }
    }
    auto one_sided = [&](int st, ld xe, int which, double* out) -> bool {
        const ld h = ((ld)r[st + 4] - (ld)r[st]) / 4.0L;
        std::vector<ld> M(25), rhs(5);
        for (int q = 0; q < 5; ++q) {
            for (int s = 0; s < 5; ++s) M[q * 5 + s] = hop(0, q, r[st + s], xe, h);
            rhs[q] = hop(which, q, xe, xe, h);
        }
        if (!solve_ld(5, M, rhs)) return false;
        const ld hp = which == 1 ? h : h * h;
        for (int s = 0; s < 5; ++s) out[s] = (double)(rhs[s] / hp);
        return true;
    };
    const int rows[2] = {1, N - 2}, starts[2] = {0, N - 5};
    for (int t = 0; t < 2; ++t) {
        const int j = rows[t], st = starts[t];
        S.start[j] = st;
        S.d0[j * 5 + (j - st)] = 1.0;
        if (!one_sided(st, r[j], 1, &S.l1[j * 5])) return false;
        if (!one_sided(st, r[j], 2, &S.l2[j * 5])) return false;
    }
    S.start[N - 1] = N - 5;
    if (!one_sided(0, r[0], 1, &S.dwall[0])) return false;
    if (!one_sided(N - 5, r[N - 1], 1, &S.dwall[5])) return false;

    // Factorisation of the d0 rows 2..N-3 on the unknowns Dv_2..Dv_{N-3},
    // eliminated from the outer wall inwards (row order N-3, N-4, ..., 2):
    // per row (m2, m1, 1/diag, c, e) with m2, m1 referring to rows j+2, j+1
    // and c, e to columns j-1, j-2.
    S.dsol.assign(N * 5, 0.0);
    std::vector<ld> Ud(N, 1.0L), Uc(N, 0.0L), Ue(N, 0.0L);
    for (int j = N - 3; j >= 2; --j) {
        const double* w = &S.d0[j * 5];
        const ld m2 = (j + 2 <= N - 3) ? w[4] / Ud[j + 2] : 0.0L;
        const ld t3 = (j + 1 <= N - 3) ? (ld)w[3] - m2 * Uc[j + 2] : 0.0L;
        const ld t2 = (ld)w[2] - m2 * ((j + 2 <= N - 3) ? Ue[j + 2] : 0.0L);
        const ld m1 = (j + 1 <= N - 3) ? t3 / Ud[j + 1] : 0.0L;
        Ud[j] = t2 - m1 * ((j + 1 <= N - 3) ? Uc[j + 1] : 0.0L);
        Uc[j] = (j - 1 >= 2) ? (ld)w[1] - m1 * ((j + 1 <= N - 3) ? Ue[j + 1] : 0.0L) : 0.0L;
        Ue[j] = (j - 2 >= 2) ? (ld)w[0] : 0.0L;
        if (Ud[j] == 0.0L) return false;
        S.dsol[j * 5 + 0] = (double)m2;
        S.dsol[j * 5 + 1] = (double)m1;
        S.dsol[j * 5 + 2] = (double)(1.0L / Ud[j]);
        S.dsol[j * 5 + 3] = (double)Uc[j];
        S.dsol[j * 5 + 4] = (double)Ue[j];
    }
    return true;
}

// Mixed-radix Stockham plans.  Family 0 (theta rows): radix-3 stages first,
// then 4, then 2.  Family 1 (z columns): radix-3 stages, then 16, then one
// stage of 8, 4 or 2.  Family 3 (float64 forward z): radix 4, then 2, then
// the radix-3 stages last.
bool make_plan(int M, FftPlan& p, std::vector<ld>& twre, std::vector<ld>& twim, int family) {
    p.M = M;
    p.nst = 0;
    int m = M, Ns = 1, off = 0;
    std::vector<int> radices;
    if (family == 3) {                          // radix 4, 2, then 3 last
        while (m % 4 == 0) { radices.push_back(4); m /= 4; }
        while (m % 2 == 0) { radices.push_back(2); m /= 2; }
    }
    while (m % 3 == 0) { radices.push_back(3); m /= 3; }
    if (family == 3) {
    } else if (family == 0) {
        while (m % 4 == 0) { radices.push_back(4); m /= 4; }
        while (m % 2 == 0) { radices.push_back(2); m /= 2; }
    } else {
        while (m % 16 == 0) { radices.push_back(16); m /= 16; }
        if (m % 8 == 0) { radices.push_back(8); m /= 8; }
        else if (m % 4 == 0) { radices.push_back(4); m /= 4; }
        else if (m % 2 == 0) { radices.push_back(2); m /= 2; }
    }
    for (int pr : {5, 7, 11, 13, 17})          // prime stages (direct sums)
        while (m % pr == 0) { radices.push_back(pr); m /= pr; }
    if (m != 1 || (int)radices.size() > TC_MAX_STAGES) return false;
    const ld twopi = 6.283185307179586476925286766559005768L;
    for (int R : radices) {
        p.R[p.nst] = R;
        p.Ns[p.nst] = Ns;
        p.twoff[p.nst] = off;
        for (int jm = 0; jm < Ns; ++jm)
            for (int r = 1; r < R; ++r) {
                const ld a = -twopi * (ld)(r * jm) / (ld)(Ns * R);
                twre.push_back(cosl(a));
                twim.push_back(sinl(a));
            }
        off += Ns * (R - 1);
        if (R != 2 && R != 3 && R != 4 && R != 8 && R != 16) {   // R-th roots of a prime stage
            for (int e = 0; e < R; ++e) {
                const ld a = -twopi * (ld)e / (ld)R;
                twre.push_back(cosl(a));
                twim.push_back(sinl(a));
            }
            off += R;
        }
        Ns *= R;
        p.nst++;
    }
    p.ntw = off;
    return true;
}

// Tangent-form twiddles of a family-0 plan, per stage and jm: the twiddle
// w_r = cos a + i sin a (a = -2 pi r jm/(Ns R)) is written k_r (1 + i tau_r)
// with k_r = cos a, tau_r = sin a/cos a.  Entries per jm: R = 4: tau1 tau2
// tau3 k1 k2 k3/k1; R = 3: tau1 tau2 k2/k1 k1 k1/2 k1 sin(2 pi/3);
// R = 2: tau1 k1.  A cosine that vanishes is replaced by 1e-200 (the
// products k_r u_r stay exact to rounding; |tau| <= 1e200).
std::vector<double> tangent_twiddles(const FftPlan& p) {
    const ld twopi = 6.283185307179586476925286766559005768L;
    const ld s3 = 0.866025403784438646763723170752936183L;
    std::vector<double> t;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.R[s], Ns = p.Ns[s];
        for (int jm = 0; jm < Ns; ++jm) {
            ld k[4] = {1, 1, 1, 1}, tau[4] = {0, 0, 0, 0};
            for (int r = 1; r < R; ++r) {
                const ld a = -twopi * (ld)(r * jm) / (ld)(Ns * R);
                ld c = cosl(a);
                if (fabsl(c) < 1e-200L) c = 1e-200L;
                k[r] = c;
                tau[r] = sinl(a) / c;
            }
            if (R == 4) {
                for (ld x : {tau[1], tau[2], tau[3], k[1], k[2], k[3] / k[1]}) t.push_back((double)x);
            } else if (R == 3) {
                for (ld x : {tau[1], tau[2], k[2] / k[1], k[1], k[1] / 2, k[1] * s3}) t.push_back((double)x);
            } else if (R == 2) {
                for (ld x : {tau[1], k[1]}) t.push_back((double)x);
            } else {
                return {};   // family-0 plans have radices 2, 3, 4 only
            }
        }
    }
    return t;
}

bool is_2a3b(int n) {
    if (n < 1) return false;
    while (n % 2 == 0) n /= 2;
    while (n % 3 == 0) n /= 3;
    return n == 1;
}

// axial sizes: factors 2, 3, 5, 7, 11, 13, 17 (the paper's Nz = 170 = 2 5 17)
bool is_smooth(int n) {
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7, 11, 13, 17})
        while (n % p == 0) n /= p;
    return n == 1;
}

}  // namespace

namespace tcx {
void set_err(const std::string& s) { g_err = s; }
}  // namespace tcx
using tcx::set_err;

// Used by the allocation-free transform entry point (tc_noalloc.cu).
bool tc_build_fft_plan(int M, FftPlan& p, std::vector<long double>& re, std::vector<long double>& im, int family) {
    return make_plan(M, p, re, im, family);
}
void tc_set_error_message(const std::string& s) { set_err(s); }



namespace {

template <typename T>
int dalloc(tc_handle* h, T*& p, size_t count) {
    void* q = nullptr;
    const size_t bytes = count * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_err(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
        return TC_ERR_CUDA;
    }
    h->allocs.push_back(q);
    h->dev_bytes += bytes;
    p = static_cast<T*>(q);
    return TC_OK;
}

template <typename T>
int upload(tc_handle* h, const T*& dst, const std::vector<T>& src) {
    T* p = nullptr;
    int rc = dalloc(h, p, src.size());
    if (rc) return rc;
    CK(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    dst = p;
    return TC_OK;
}

void free_all(tc_handle* h) {
    tcx::drop_graphs(h);
    tcx::release_pipeline(h);
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
}

// Tile autotuner: candidate azimuthal tiles of the z kernels and block sizes
// of the line kernel are timed on the (zero) initial state, which they leave
// unchanged, and the fastest pair is kept for the shape class (Nr, Ntheta,
// Nz, precision).  The choice changes no arithmetic.
std::mutex g_tune_mu;
std::map<std::array<int, 4>, std::pair<int, int>> g_tune;

int autotune(tc_handle* h) {
    TcDev& d = h->d;
    const std::array<int, 4> key = {d.Nr, 2 * d.Nh, d.Nz, d.prec};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) { d.ztile = it->second.first; d.line_block = it->second.second; return TC_OK; }
    }
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    auto timed = [&](auto fn) -> float {
        fn();                                  // warm-up
        cudaEventRecord(a, h->stream);
        for (int rep = 0; rep < 3; ++rep) fn();
        cudaEventRecord(b, h->stream);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    };
    // a narrower z tile must be at least 1% faster: near ties go to the wider
    // tile, whose column groups are coarser in the overlapped step
    float best = 1e30f;
    int best_t = d.ztile;
    for (int t : {8, 4, 2, 1}) {
        if (d.Nh % t) continue;
        if (2 * (size_t)t * d.Mz * sizeof(double2) > 200 * 1024) continue;
        d.ztile = t;
        const float ms = timed([&] { tc_launch_plane_kernel(d, 0, h->stream); tc_launch_plane_kernel(d, 2, h->stream); });
        if (ms < 0.99f * best) { best = ms; best_t = t; }
    }
    d.ztile = best_t;
    best = 1e30f;
    int best_b = d.line_block;
    for (int bs : {64, 128, 256, 1003, 1004, 2007, 3001}) {
        d.line_block = bs;
        const float ms = timed([&] { tc_launch_line_phase(d, 0, h->stream); });
        if (ms < best) { best = ms; best_b = bs; }
    }
    d.line_block = best_b;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    CK(cudaGetLastError());
    CK(cudaMemset(d.flag, 0, 4 * sizeof(int)));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {d.ztile, d.line_block};
    return TC_OK;
}

int init_handle(tc_handle* h) {
    const tc_params& P = h->prm;
    TcDev& d = h->d;
    std::memset(&d, 0, sizeof(d));
    d.Nr = P.Nr;
    d.Nz = P.Nz;
    d.Nh = P.Ntheta / 2;
    d.Mt = 3 * P.Ntheta / 2;
    d.Mz = 3 * P.Nz / 2;
    d.npairs = d.Nz * d.Nh;
    d.mixed = P.precision == TC_PREC_MIXED ? 1 : 0;
    d.prec = P.precision;
    // widest z tile (azimuthal columns per block) that divides Ntheta/2 and
    // whose two Mz-long complex columns per tile fit the 200 KB of shared
    // memory a block may use
    d.ztile = 1;
    for (int t : {8, 4, 2}) {
        if (d.Nh % t == 0 && 2 * (size_t)t * d.Mz * sizeof(double2) <= 200 * 1024) { d.ztile = t; break; }
    }
    d.line_block = 128;
    d.fscale = 1.0 / ((double)d.Mt * (double)d.Mz);
    d.fscale_f = (float)d.fscale;
    d.fscale_lo = (float)(d.fscale - (double)d.fscale_f);
    d.dt = P.dt;
    d.nu = 2.0 / P.Re_inner;
    d.W_outer = P.Re_outer / P.Re_inner;
    // grid: R_i = 2 zeta/(1 - zeta), r_j = R_i + (2 j)/(Nr - 1)
    const double Ri = 2.0 * P.radius_ratio / (1.0 - P.radius_ratio);
    h->r.resize(P.Nr);
    h->jac.assign(P.Nr, 1.0);
    if (P.stretch == 0.0) {
        for (int j = 0; j < P.Nr; ++j) h->r[j] = Ri + (2.0 * (double)j) / (double)(P.Nr - 1);
    } else {
        // tanh map, denser at both walls
        const double ta = std::tanh(P.stretch);
        for (int j = 0; j < P.Nr; ++j) {
            const double sj = -1.0 + (2.0 * (double)j) / (double)(P.Nr - 1);
            const double t = std::tanh(P.stretch * sj);
            h->r[j] = (Ri + 1.0) + t / ta;
            h->jac[j] = P.stretch * (1.0 - t * t) / ta;
        }
    }
    h->Ri = Ri;
    h->Ro = h->r[P.Nr - 1];
    const double rc = Ri + 1.0;
    const double Theta = P.Theta > 0 ? P.Theta : 10.0 * M_PI / rc;
    const double Lz = P.Lz > 0 ? P.Lz : 5.0;
    d.m0 = 2.0 * M_PI / Theta;
    d.alpha0 = 2.0 * M_PI / Lz;
    // Runge-Kutta (Spalart, Moser & Rogers 1991, Crank-Nicolson per substep)
    const double ga[3] = {8.0 / 15.0, 5.0 / 12.0, 3.0 / 4.0};
    const double ze[3] = {0.0, -17.0 / 60.0, -5.0 / 12.0};
    const double ab[3] = {4.0 / 15.0, 1.0 / 15.0, 1.0 / 6.0};
    for (int k = 0; k < 3; ++k) {
        d.rk_gamma[k] = ga[k]; d.rk_zeta[k] = ze[k]; d.rk_alpha[k] = ab[k]; d.rk_beta[k] = ab[k];
    }
    if (!build_stencils(h->r, h->S)) { set_err("stencil construction failed"); return TC_ERR_STATE; }
    int rc_ = TC_OK;
    std::vector<double> rinv(P.Nr);
    for (int j = 0; j < P.Nr; ++j) rinv[j] = 1.0 / h->r[j];
    if ((rc_ = upload(h, d.r, h->r))) return rc_;
    if ((rc_ = upload(h, d.rinv, rinv))) return rc_;
    if ((rc_ = upload(h, d.start, h->S.start))) return rc_;
    if ((rc_ = upload(h, d.d0, h->S.d0))) return rc_;
    if ((rc_ = upload(h, d.l1, h->S.l1))) return rc_;
    if ((rc_ = upload(h, d.l2, h->S.l2))) return rc_;
    if ((rc_ = upload(h, d.l4, h->S.l4))) return rc_;
    if ((rc_ = upload(h, d.dwall, h->S.dwall))) return rc_;
    if ((rc_ = upload(h, d.dsol, h->S.dsol))) return rc_;
    {
        std::vector<float> f0(h->S.d0.begin(), h->S.d0.end()), f1(h->S.l1.begin(), h->S.l1.end()),
            f2(h->S.l2.begin(), h->S.l2.end()), fr(rinv.begin(), rinv.end());
        if ((rc_ = upload(h, d.d0f, f0))) return rc_;
        if ((rc_ = upload(h, d.l1f, f1))) return rc_;
        if ((rc_ = upload(h, d.l2f, f2))) return rc_;
        if ((rc_ = upload(h, d.rinvf, fr))) return rc_;
        auto dsplit = [](const std::vector<double>& v) {
            std::vector<float2> o(v.size());
            for (size_t i = 0; i < v.size(); ++i) {
                const float hh = (float)v[i];
                o[i] = make_float2(hh, (float)(v[i] - (double)hh));
            }
            return o;
        };
        if ((rc_ = upload(h, d.d0x, dsplit(h->S.d0)))) return rc_;
        if ((rc_ = upload(h, d.l1x, dsplit(h->S.l1)))) return rc_;
        if ((rc_ = upload(h, d.l2x, dsplit(h->S.l2)))) return rc_;
        if ((rc_ = upload(h, d.rinvx, dsplit(rinv)))) return rc_;
    }
    // FFT plans
    std::vector<ld> zr, zi, tr, ti, hr, hi;
    if (!make_plan(d.Mz, d.pz, zr, zi, 1) || !make_plan(d.Mt, d.pt, tr, ti, 0) || !make_plan(d.Mt / 2, d.ph, hr, hi, 0)) {
        set_err("FFT length is not of the form 2^a 3^b");
        return TC_ERR_ARG;
    }
    std::vector<double2> twz_d(zr.size()), twt_d(tr.size());
    std::vector<float2> twz_f(zr.size()), twt_f(tr.size());
    for (size_t i = 0; i < zr.size(); ++i) { twz_d[i] = make_double2((double)zr[i], (double)zi[i]); twz_f[i] = make_float2((float)zr[i], (float)zi[i]); }
    for (size_t i = 0; i < tr.size(); ++i) { twt_d[i] = make_double2((double)tr[i], (double)ti[i]); twt_f[i] = make_float2((float)tr[i], (float)ti[i]); }
    std::vector<double2> twh_d(hr.size()), twr_d(d.Mt / 2);
    std::vector<float2> twh_f(hr.size()), twr_f(d.Mt / 2);
    for (size_t i = 0; i < hr.size(); ++i) { twh_d[i] = make_double2((double)hr[i], (double)hi[i]); twh_f[i] = make_float2((float)hr[i], (float)hi[i]); }
    for (int k = 0; k < d.Mt / 2; ++k) {
        const ld a = -6.283185307179586476925286766559005768L * (ld)k / (ld)d.Mt;
        twr_d[k] = make_double2((double)cosl(a), (double)sinl(a));
        twr_f[k] = make_float2((float)cosl(a), (float)sinl(a));
    }
    if (twh_d.empty()) { twh_d.push_back(make_double2(1, 0)); twh_f.push_back(make_float2(1, 0)); }
    {   // double-float tables: hi = nearest float, lo = nearest float of the rest
        auto split = [](const std::vector<ld>& re, const std::vector<ld>& im, size_t n) {
            std::vector<float4> o(n > 0 ? n : 1, make_float4(1.0f, 0.0f, 0.0f, 0.0f));
            for (size_t i = 0; i < n; ++i) {
                const float rh = (float)re[i], ih = (float)im[i];
                o[i] = make_float4(rh, (float)(re[i] - (ld)rh), ih, (float)(im[i] - (ld)ih));
            }
            return o;
        };
        std::vector<ld> rr(d.Mt / 2), ri(d.Mt / 2);
        for (int k = 0; k < d.Mt / 2; ++k) {
            const ld a = -6.283185307179586476925286766559005768L * (ld)k / (ld)d.Mt;
            rr[k] = cosl(a); ri[k] = sinl(a);
        }
        if ((rc_ = upload(h, d.twz_x, split(zr, zi, zr.size())))) return rc_;
        if ((rc_ = upload(h, d.twt_x, split(tr, ti, tr.size())))) return rc_;
        if ((rc_ = upload(h, d.twh_x, split(hr, hi, hr.size())))) return rc_;
        if ((rc_ = upload(h, d.twr_x, split(rr, ri, rr.size())))) return rc_;
    }
    if ((rc_ = upload(h, d.twh_d, twh_d))) return rc_;
    if ((rc_ = upload(h, d.twh_f, twh_f))) return rc_;
    if ((rc_ = upload(h, d.twr_d, twr_d))) return rc_;
    if ((rc_ = upload(h, d.twr_f, twr_f))) return rc_;
    if (twz_d.empty()) { twz_d.push_back(make_double2(1, 0)); twz_f.push_back(make_float2(1, 0)); }
    if (twt_d.empty()) { twt_d.push_back(make_double2(1, 0)); twt_f.push_back(make_float2(1, 0)); }
    if ((rc_ = upload(h, d.twz_d, twz_d))) return rc_;
    if ((rc_ = upload(h, d.twt_d, twt_d))) return rc_;
    // float64 z transforms in the radix-3/4/2 plan with tangent twiddles
    // when the padded axial length has a compile-time plan
    d.zfam0 = 0;
    if (tc_fft_fixed_length(d.Mz) && is_2a3b(d.Mz)) {
        std::vector<ld> r0, i0;
        if (make_plan(d.Mz, d.pz0, r0, i0, 0)) {
            std::vector<double> c = tangent_twiddles(d.pz0);
            if (!c.empty()) {
                if ((rc_ = upload(h, d.twz_tan, c))) return rc_;
                FftPlan p3;
                std::vector<ld> r3, i3;
                if (!make_plan(d.Mz, p3, r3, i3, 3) || p3.R[p3.nst - 1] != 3) {
                    set_err("axial plan of family 3 does not end in a radix-3 stage");
                    return TC_ERR_ARG;
                }
                std::vector<double> c3 = tangent_twiddles(p3);
                if (c3.empty()) { set_err("axial plan of family 3 with a radix other than 2, 3, 4"); return TC_ERR_ARG; }
                if ((rc_ = upload(h, d.twz3_tan, c3))) return rc_;
                std::vector<float2> f0(r0.size() ? r0.size() : 1, make_float2(1.0f, 0.0f));
                std::vector<float4> x0(r0.size() ? r0.size() : 1, make_float4(1.0f, 0.0f, 0.0f, 0.0f));
                for (size_t i = 0; i < r0.size(); ++i) {
                    const float rh = (float)r0[i], ih = (float)i0[i];
                    f0[i] = make_float2(rh, ih);
                    x0[i] = make_float4(rh, (float)(r0[i] - (ld)rh), ih, (float)(i0[i] - (ld)ih));
                }
                if ((rc_ = upload(h, d.twz0_f, f0))) return rc_;
                if ((rc_ = upload(h, d.twz0_x, x0))) return rc_;
                d.zfam0 = 1;
            }
        }
    }
    {
        std::vector<double> a = tangent_twiddles(d.pt), b = tangent_twiddles(d.ph);
        if (a.empty() || b.empty()) { set_err("theta plan with a radix other than 2, 3, 4"); return TC_ERR_ARG; }
        if ((rc_ = upload(h, d.twt_tan, a))) return rc_;
        if ((rc_ = upload(h, d.twh_tan, b))) return rc_;
        FftPlan p3;
        std::vector<ld> r3, i3;
        if (!make_plan(d.Mt, p3, r3, i3, 3) || p3.R[p3.nst - 1] != 3) {
            set_err("theta plan of family 3 does not end in a radix-3 stage");
            return TC_ERR_ARG;
        }
        std::vector<double> c3 = tangent_twiddles(p3);
        if (c3.empty()) { set_err("theta plan of family 3 with a radix other than 2, 3, 4"); return TC_ERR_ARG; }
        if ((rc_ = upload(h, d.twt3_tan, c3))) return rc_;
    }
    if ((rc_ = upload(h, d.twz_f, twz_f))) return rc_;
    if ((rc_ = upload(h, d.twt_f, twt_f))) return rc_;
    // fields
    const size_t P1 = (size_t)d.Nr * d.npairs;
    double2* f[6];
    for (int i = 0; i < 6; ++i) if ((rc_ = dalloc(h, f[i], P1))) return rc_;
    d.v = f[0]; d.eta = f[1]; d.u = f[2]; d.w = f[3]; d.Hv = f[4]; d.He = f[5];
    for (int i = 0; i < 6; ++i) CK(cudaMemset(f[i], 0, P1 * sizeof(double2)));
    double2* pr;
    if ((rc_ = dalloc(h, pr, TC_NPROD * P1))) return rc_;
    CK(cudaMemset(pr, 0, TC_NPROD * P1 * sizeof(double2)));
    d.prod = pr;
    const size_t Z1 = (size_t)d.Nr * d.Mz * d.Nh;
    double2 *zb, *pb;
    if ((rc_ = dalloc(h, zb, 3 * Z1))) return rc_;
    if ((rc_ = dalloc(h, pb, TC_NPROD * Z1))) return rc_;
    d.zbuf = zb; d.pbuf = pb;
    double* mean;
    if ((rc_ = dalloc(h, mean, 6 * (size_t)d.Nr))) return rc_;
    d.U = mean; d.W = mean + d.Nr; d.HU = mean + 2 * d.Nr; d.HW = mean + 3 * d.Nr; d.eprof = mean + 4 * d.Nr;
    d.dprof = mean + 5 * d.Nr;
    CK(cudaMemset(mean, 0, 6 * (size_t)d.Nr * sizeof(double)));
    // circular Couette flow W = A r + B/r, W(R_i) = 1, W(R_o) = Re_o/Re_i
    {
        const double Ro = h->Ro, Wo = d.W_outer;
        const double A = (Wo * Ro - Ri) / (Ro * Ro - Ri * Ri);
        const double B = Ri - A * Ri * Ri;
        std::vector<double> W(P.Nr);
        for (int j = 0; j < P.Nr; ++j) W[j] = A * h->r[j] + B / h->r[j];
        CK(cudaMemcpy(d.W, W.data(), P.Nr * sizeof(double), cudaMemcpyHostToDevice));
    }
    // per-pair tables
    if ((rc_ = dalloc(h, d.tab_luv, 3 * (size_t)d.Nr * 5 * d.npairs))) return rc_;
    if ((rc_ = dalloc(h, d.tab_lue, 3 * (size_t)d.Nr * 5 * d.npairs))) return rc_;
    if ((rc_ = dalloc(h, d.tab_lv, (size_t)d.Nr * 5 * d.npairs))) return rc_;
    if ((rc_ = dalloc(h, d.tab_c, (size_t)d.Nr * d.npairs))) return rc_;
    if ((rc_ = dalloc(h, d.tab_c1, (size_t)d.Nr * d.npairs))) return rc_;
    if (d.prec != TC_PREC_FP64) {     // float (hi, lo) copies of c and c'
        if ((rc_ = dalloc(h, d.tab_cx, (size_t)d.Nr * d.npairs))) return rc_;
        if ((rc_ = dalloc(h, d.tab_c1x, (size_t)d.Nr * d.npairs))) return rc_;
    }
    int* flag;
    if ((rc_ = dalloc(h, flag, 4))) return rc_;
    CK(cudaMemset(flag, 0, 4 * sizeof(int)));
    d.flag = flag;
    CK(tc_set_kernel_attributes());
    CK(tc_set_line_kernel_attributes());
    tc_launch_setup_tables(d, h->stream);
    CK(cudaGetLastError());
    int hf[4];
    CK(cudaMemcpy(hf, d.flag, sizeof(hf), cudaMemcpyDeviceToHost));
    if (hf[1]) { set_err("a radial system has a vanishing pivot (LU without pivoting)"); return TC_ERR_STATE; }
    if (P.autotune) {
        if ((rc_ = autotune(h))) return rc_;
    }
    h->need_init = true;
    return TC_OK;
}

}  // namespace

namespace tcx {

int ensure_init(tc_handle* h) {
    if (!h->need_init) return TC_OK;
    tc_launch_init_state(h->d, h->stream);
    CK(cudaGetLastError());
    h->need_init = false;
    return TC_OK;
}

int prepare_pipeline(tc_handle* h) {
    if (h->pipe_ready) return TC_OK;
    // on a failure, whatever was created is released again
    cudaError_t e = cudaSuccess;
    for (auto& st : h->aux)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (int c = 0; c < TC_MAX_CHUNKS; ++c) {
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->evz[c], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->evl[c], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->evm, cudaEventDisableTiming);
    for (auto& ev : h->evj)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->srk, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->evrk0, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->evrk1, cudaEventDisableTiming);
    h->pipe_ready = true;                // lets release_pipeline free what exists
    if (e != cudaSuccess) {
        release_pipeline(h);
        set_err(std::string("pipeline streams and events: ") + cudaGetErrorString(e));
        return TC_ERR_CUDA;
    }
    return TC_OK;
}

void release_pipeline(tc_handle* h) {
    if (!h->pipe_ready) return;
    for (auto& st : h->aux) { if (st) cudaStreamDestroy(st); st = nullptr; }
    for (int c = 0; c < TC_MAX_CHUNKS; ++c) {
        if (h->evz[c]) cudaEventDestroy(h->evz[c]);
        if (h->evl[c]) cudaEventDestroy(h->evl[c]);
        h->evz[c] = h->evl[c] = nullptr;
    }
    if (h->evm) cudaEventDestroy(h->evm);
    h->evm = nullptr;
    for (auto& ev : h->evj) { if (ev) cudaEventDestroy(ev); ev = nullptr; }
    if (h->srk) cudaStreamDestroy(h->srk);
    if (h->evrk0) cudaEventDestroy(h->evrk0);
    if (h->evrk1) cudaEventDestroy(h->evrk1);
    h->srk = nullptr;
    h->evrk0 = h->evrk1 = nullptr;
    h->pipe_ready = false;
}

bool chunks_valid(const tc_handle* h, int c) {
    const TcDev& d = h->d;
    return c >= 1 && c <= TC_MAX_CHUNKS && (d.Nh / d.ztile) % c == 0;
}

// Column groups of the overlapped step: the value set by tc_set_tiles, else
// the one chosen by timing (tc_step with the autotuner on), else none.
int pipeline_chunks(const tc_handle* h) {
    const int c = h->chunks > 0 ? h->chunks : h->chunks_auto;
    return chunks_valid(h, c) ? c : 1;
}

// One step.  Without column groups: the 15 kernels in order.  With C groups
// the plane and line phases overlap: the z-forward transform of group c is
// followed at once by the line kernel of group c (its pairs need only that
// group's products), whose output feeds the next substep's z-inverse
// transform of group c; the mean flow needs the j = 0 column (group 0) and
// must precede the z inverse of group 0 (its (0,0) slot holds U, W).  The
// theta rows of each substep wait for every group.  The line kernels of
// alternate groups use two streams so that they overlap too.
// Deferred RK memory (double-float and mixed forms, inside a captured step):
// the line kernels leave out the implicit part of the next RK memory, and
// k_rk_memory adds it for substep k - 1 on its own stream beside the theta
// rows of substep k, whose float32 work leaves the float64 pipe idle; the
// line kernel of substep k waits for it.  The last substep's memory is
// completed at the end of the step.  Same bits as the full line kernel.
bool defer_rk(const tc_handle* h) {
    const int m = h->rk_defer >= 0 ? h->rk_defer : h->rk_defer_auto;
    return h->pipe_ready && h->d.prec != TC_PREC_FP64 && m == 1;
}
void drop_graphs(tc_handle* h) {
    for (cudaGraphExec_t* g : {&h->graph, &h->graph_first, &h->graph_next}) {
        if (*g) cudaGraphExecDestroy(*g);
        *g = nullptr;
    }
}
static void rk_fork(tc_handle* h, int kprev, cudaStream_t s) {
    cudaEventRecord(h->evrk0, s);
    cudaStreamWaitEvent(h->srk, h->evrk0, 0);
    tc_launch_rk_memory(h->d, kprev, h->srk, 0, h->d.Nh, true);
    cudaEventRecord(h->evrk1, h->srk);
}
static void line_chunk(const tc_handle* h, int k, cudaStream_t s, int ja, int jw) {
    if (defer_rk(h)) tc_launch_line_chunk_deferred(h->d, k, s, ja, jw);
    else tc_launch_line_chunk(h->d, k, s, ja, jw);
}

// With the deferred RK memory, `lead` starts the step with the previous
// step's last RK memory (beside the first theta rows) and `trail` ends it with
// this step's own; the self-contained step has trail only.
void launch_step(tc_handle* h, cudaStream_t s, bool lead, bool trail) {
    TcDev& d = h->d;
    const int C = h->pipe_ready ? pipeline_chunks(h) : 1;
    const bool defer = defer_rk(h);
    auto pending = [&](int k) { return defer && (k > 0 || lead); };   // an RK memory to add before line k
    if (C <= 1) {
        // the mean flow (one block) runs beside the line kernel, which does
        // not touch U, W or the (0,0) slot; the next z inverse waits for it
        const bool side = h->pipe_ready;
        for (int k = 0; k < 3; ++k) {
            if (side && k > 0) cudaStreamWaitEvent(s, h->evm, 0);
            tc_launch_plane_kernel(d, 0, s);
            if (pending(k)) rk_fork(h, k > 0 ? k - 1 : 2, s);
            tc_launch_plane_kernel(d, 1, s);
            tc_launch_plane_kernel(d, 2, s);
            if (pending(k)) cudaStreamWaitEvent(s, h->evrk1, 0);
            if (side) {
                cudaEventRecord(h->evz[0], s);
                cudaStreamWaitEvent(h->aux[2], h->evz[0], 0);
                tc_launch_mean_phase(d, k, h->aux[2]);
                cudaEventRecord(h->evm, h->aux[2]);
                line_chunk(h, k, s, 0, d.Nh);
            } else {
                line_chunk(h, k, s, 0, d.Nh);
                tc_launch_mean_phase(d, k, s);
            }
        }
        if (side) cudaStreamWaitEvent(s, h->evm, 0);
        if (defer && trail) tc_launch_rk_memory(d, 2, s, 0, d.Nh, false);
        return;
    }
    const int tpc = (d.Nh / d.ztile) / C;      // z tiles per group
    const int cw = tpc * d.ztile;              // columns per group
    cudaStream_t sM = h->aux[2], sZ = h->aux[3];
    tc_launch_plane_kernel(d, 0, s);           // z inverse of the first substep
    for (int k = 0; k < 3; ++k) {
        if (pending(k)) rk_fork(h, k > 0 ? k - 1 : 2, s);
        tc_launch_plane_kernel(d, 1, s);       // theta rows and products
        for (int c = 0; c < C; ++c) {
            tc_launch_plane_kernel_tiles(d, 2, s, c * tpc, tpc);
            cudaEventRecord(h->evz[c], s);
        }
        cudaStreamWaitEvent(sM, h->evz[0], 0);
        tc_launch_mean_phase(d, k, sM);
        cudaEventRecord(h->evm, sM);
        for (int c = 0; c < C; ++c) {
            cudaStream_t sL = h->aux[c & 1];
            cudaStreamWaitEvent(sL, h->evz[c], 0);
            if (pending(k)) cudaStreamWaitEvent(sL, h->evrk1, 0);
            line_chunk(h, k, sL, c * cw, cw);
            cudaEventRecord(h->evl[c], sL);
            if (k < 2) {
                cudaStreamWaitEvent(sZ, h->evl[c], 0);
                if (c == 0) cudaStreamWaitEvent(sZ, h->evm, 0);
                tc_launch_plane_kernel_tiles(d, 0, sZ, c * tpc, tpc);
            }
        }
        for (int a = 0; a < (k < 2 ? 4 : 3); ++a) {
            cudaEventRecord(h->evj[a], h->aux[a]);
            cudaStreamWaitEvent(s, h->evj[a], 0);
        }
    }
    if (defer && trail) tc_launch_rk_memory(d, 2, s, 0, d.Nh, false);
}

static int capture_step(tc_handle* h, bool lead, bool trail, cudaGraphExec_t* out) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    launch_step(h, cs, lead, trail);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (e != cudaSuccess) { cudaStreamDestroy(cs); set_err(std::string("graph capture: ") + cudaGetErrorString(e)); return TC_ERR_CUDA; }
    unsigned long long flags = 0;
    if (defer_rk(h)) {
        // the deferred RK memory fills what the theta rows leave free: every
        // other kernel node gets the highest priority, so that its blocks are
        // dispatched first
        int least = 0, greatest = 0;
        size_t n = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
            cudaGraphGetNodes(g, nullptr, &n) == cudaSuccess) {
            std::vector<cudaGraphNode_t> nodes(n);
            if (cudaGraphGetNodes(g, nodes.data(), &n) == cudaSuccess) {
                const void* rk = tc_rk_memory_kernel();
                for (cudaGraphNode_t nd : nodes) {
                    cudaGraphNodeType t;
                    cudaKernelNodeParams kp;
                    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
                    if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
                    cudaLaunchAttributeValue v{};
                    v.priority = kp.func == rk ? least : greatest;
                    cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v);
                }
                flags = cudaGraphInstantiateFlagUseNodePriority;
            }
        }
        cudaGetLastError();
    }
    e = cudaGraphInstantiateWithFlags(out, g, flags);
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) { *out = nullptr; set_err(std::string("graph instantiate: ") + cudaGetErrorString(e)); return TC_ERR_CUDA; }
    return TC_OK;
}

// The self-contained step graph, and with the deferred RK memory the first
// and following steps of a tc_step call.
int ensure_graph(tc_handle* h) {
    int rc_;
    if ((rc_ = prepare_pipeline(h))) return rc_;
    if (!h->graph && (rc_ = capture_step(h, false, true, &h->graph))) return rc_;
    if (defer_rk(h)) {
        if (!h->graph_first && (rc_ = capture_step(h, false, false, &h->graph_first))) return rc_;
        if (!h->graph_next && (rc_ = capture_step(h, true, false, &h->graph_next))) return rc_;
    }
    return TC_OK;
}

int validate(const tc_params* p) {
    if (!p) { set_err("null parameters"); return TC_ERR_ARG; }
    if (p->Nr < 9) { set_err("Nr must be >= 9"); return TC_ERR_ARG; }
    if (p->Ntheta < 4 || p->Ntheta % 4 || !is_2a3b(p->Ntheta)) { set_err("Ntheta must be a multiple of 4 and of the form 2^a 3^b"); return TC_ERR_ARG; }
    if (p->Nz < 4 || p->Nz % 2 || !is_smooth(p->Nz)) { set_err("Nz must be even, >= 4, with prime factors in {2, 3, 5, 7, 11, 13, 17}"); return TC_ERR_ARG; }
    if (!(p->radius_ratio > 0.0 && p->radius_ratio < 1.0)) { set_err("radius ratio must lie in (0, 1)"); return TC_ERR_ARG; }
    if (!(p->Re_inner > 0.0) || !std::isfinite(p->Re_outer)) { set_err("Re_inner must be > 0 and Re_outer finite"); return TC_ERR_ARG; }
    if (!(p->dt > 0.0) || !std::isfinite(p->dt)) { set_err("dt must be > 0"); return TC_ERR_ARG; }
    if (!(p->stretch >= 0.0 && p->stretch <= 8.0)) { set_err("stretch must lie in [0, 8]"); return TC_ERR_ARG; }
    if (p->precision != TC_PREC_FP64 && p->precision != TC_PREC_MIXED && p->precision != TC_PREC_DF64) { set_err("unknown precision"); return TC_ERR_ARG; }
    // shared memory of one block (at most 200 KB): a z transform holds two
    // complex columns of 3 Nz/2 values (16 bytes each in the float64 and
    // double-float forms), a theta row 4 (double-float: 5) complex rows of
    // 3 Ntheta/2 values
    const size_t Mz = 3 * (size_t)p->Nz / 2, Mt = 3 * (size_t)p->Ntheta / 2, lim = 200 * 1024;
    const size_t row_bytes = (p->precision == TC_PREC_DF64 ? 5 : 4) * Mt * (p->precision == TC_PREC_MIXED ? 8 : 16);
    if (2 * Mz * 16 > lim || row_bytes > lim || 2 * Mt * 16 > lim) {
        set_err("grid too large for the shared memory of one transform block: Nz <= 4266, Ntheta <= " +
                std::string(p->precision == TC_PREC_DF64 ? "1706" : p->precision == TC_PREC_MIXED ? "4266" : "2133"));
        return TC_ERR_SIZE;
    }
    return TC_OK;
}

// Sum of the allocations of init_handle (plus the physical-space buffer of
// tc_get_field and a per-allocation rounding allowance of 2 MiB).
size_t estimate_device_bytes(const tc_params& p) {
    const size_t Nr = p.Nr, Nh = p.Ntheta / 2, Nz = p.Nz, Mt = 3 * (size_t)p.Ntheta / 2, Mz = 3 * Nz / 2;
    const size_t np = Nz * Nh, P1 = Nr * np, Z1 = Nr * Mz * Nh;
    size_t b = 0;
    b += (6 + TC_NPROD) * P1 * sizeof(double2);                 // fields, products
    b += (3 + TC_NPROD) * Z1 * sizeof(double2);                 // zbuf, pbuf
    b += (3 + 3) * Nr * 5 * np * sizeof(double);                // LU tables
    b += Nr * 5 * np * sizeof(double) + 4 * Nr * np * sizeof(double);   // L band, c, c1 (+ double-float copies)
    b += Nr * Mz * Mt * sizeof(double);                         // physical output (on demand)
    b += 64 * Nr * sizeof(double) + 4 * (Mz + 2 * Mt) * sizeof(double2);  // radial tables, twiddles
    return b + 40 * (2u << 20);
}

}  // namespace tcx
using tcx::ensure_init;
using tcx::launch_step;
using tcx::ensure_graph;
using tcx::validate;

extern "C" {

const char* tc_last_error(void) { return g_err.c_str(); }

tc_handle* tc_create_ex(const tc_params* params) {
    if (validate(params)) return nullptr;
    if (params->device >= 0) {
        cudaError_t e = cudaSetDevice(params->device);
        if (e != cudaSuccess) { set_err(std::string("cudaSetDevice: ") + cudaGetErrorString(e)); return nullptr; }
    }
    tc_handle* h = new tc_handle();
    h->prm = *params;
    int rc = init_handle(h);
    if (rc) {
        std::string msg = g_err;
        free_all(h);
        delete h;
        set_err(msg);
        return nullptr;
    }
    g_err.clear();
    return h;
}

tc_handle* tc_create(int Nr, int Ntheta, int Nz, double radius_ratio, double Re_inner,
                     double Re_outer, double dt) {
    tc_params p;
    std::memset(&p, 0, sizeof(p));
    p.Nr = Nr; p.Ntheta = Ntheta; p.Nz = Nz; p.radius_ratio = radius_ratio;
    p.Re_inner = Re_inner; p.Re_outer = Re_outer; p.dt = dt;
    p.Theta = 0.0; p.Lz = 0.0; p.precision = TC_PREC_FP64; p.device = -1; p.autotune = 1; p.stretch = 0.0;
    return tc_create_ex(&p);
}

void tc_destroy(tc_handle* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int tc_set_stream(tc_handle* h, void* s) {
    if (!h) { set_err("null handle"); return TC_ERR_ARG; }
    h->stream = (cudaStream_t)s;
    return TC_OK;
}

int tc_get_tiles(const tc_handle* h, int* ztile, int* line_variant, int* chunks) {
    if (!h) { set_err("null handle"); return TC_ERR_ARG; }
    if (ztile) *ztile = h->d.ztile;
    if (line_variant) *line_variant = h->d.line_block > 0 ? h->d.line_block : 128;
    if (chunks) *chunks = tcx::pipeline_chunks(h);
    return TC_OK;
}

int tc_set_rk_deferral(tc_handle* h, int mode) {
    if (!h) { set_err("null handle"); return TC_ERR_ARG; }
    if (mode < -1 || mode > 1) { set_err("mode must be -1 (chosen by timing), 0 or 1"); return TC_ERR_ARG; }
    h->rk_defer = mode;
    if (mode < 0) h->rk_defer_auto = -1;
    tcx::drop_graphs(h);
    return TC_OK;
}

int tc_get_rk_deferral(const tc_handle* h, int* on) {
    if (!h || !on) { set_err("null handle or output"); return TC_ERR_ARG; }
    const int m = h->rk_defer >= 0 ? h->rk_defer : h->rk_defer_auto;
    *on = (h->d.prec != TC_PREC_FP64 && m == 1) ? 1 : 0;
    return TC_OK;
}

int tc_set_tiles(tc_handle* h, int ztile, int line_variant, int chunks) {
    if (!h) { set_err("null handle"); return TC_ERR_ARG; }
    TcDev& d = h->d;
    if (ztile != 0) {
        if ((ztile != 1 && ztile != 2 && ztile != 4 && ztile != 8) || d.Nh % ztile ||
            2 * (size_t)ztile * d.Mz * sizeof(double2) > 200 * 1024) {
            set_err("ztile must be 1, 2, 4 or 8, divide Ntheta/2 and fit the shared memory");
            return TC_ERR_ARG;
        }
    }
    if (line_variant != 0 && line_variant != 64 && line_variant != 128 && line_variant != 256 &&
        line_variant != 1003 && line_variant != 1004 && line_variant != 2007 && line_variant != 3001) {
        set_err("line_variant must be 64, 128, 256, 1003, 1004, 2007 or 3001");
        return TC_ERR_ARG;
    }
    if (chunks != 0 && chunks != 1 && chunks != 2 && chunks != 4 && chunks != 8) {
        set_err("chunks must be 1, 2, 4 or 8");
        return TC_ERR_ARG;
    }
    if (ztile) d.ztile = ztile;
    if (line_variant) d.line_block = line_variant;
    if (chunks) h->chunks = chunks;
    tcx::drop_graphs(h);
    return TC_OK;
}

}  // extern "C"

int tcx::check_flags(tc_handle* h) {
    int hf[4];
    CK(cudaMemcpy(hf, h->d.flag, sizeof(hf), cudaMemcpyDeviceToHost));
    if (hf[0]) { set_err("non-finite value in v or eta"); return TC_ERR_NONFINITE; }
    return TC_OK;
}
using tcx::check_flags;

namespace {
// With the autotuner on, the first tc_step of three or more steps runs one
// self-contained step with each candidate launch plan not pinned by the
// caller: 1 and 2 column groups and, in the double-float and mixed forms,
// the RK memory's implicit part in the line kernel or deferred beside the
// theta rows.  Each is timed with events; the fastest is kept for this
// handle and the shape class.  Every plan gives the same bits, so the tuning
// steps are ordinary steps.
std::map<std::array<int, 4>, std::pair<int, int>> g_tune_plan;   // (column groups, deferral)

int tune_chunks(tc_handle* h, int nsteps, int* done) {
    *done = 0;
    TcDev& d = h->d;
    const bool tune_c = h->chunks <= 0 && h->chunks_auto <= 0;
    const bool tune_d = d.prec != TC_PREC_FP64 && h->rk_defer < 0 && h->rk_defer_auto < 0;
    if (!h->prm.autotune) {
        if (h->rk_defer_auto < 0) h->rk_defer_auto = 0;
        return TC_OK;
    }
    if (!tune_c && !tune_d) return TC_OK;
    const std::array<int, 4> key = {d.Nr, 2 * d.Nh, d.Nz, d.prec};
    if (h->chunks <= 0 && h->rk_defer < 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_plan.find(key);
        if (it != g_tune_plan.end()) {
            h->chunks_auto = it->second.first;
            h->rk_defer_auto = it->second.second;
            tcx::drop_graphs(h);
            return TC_OK;
        }
    }
    std::vector<int> cs, ds;
    if (tune_c) { cs.push_back(1); if (tcx::chunks_valid(h, 2)) cs.push_back(2); }
    else cs.push_back(h->chunks > 0 ? h->chunks : h->chunks_auto);
    if (tune_d) { ds.push_back(0); ds.push_back(1); }
    else ds.push_back(d.prec == TC_PREC_FP64 ? 0 : (h->rk_defer >= 0 ? h->rk_defer : h->rk_defer_auto));
    if (cs.size() * ds.size() == 1) {
        h->chunks_auto = cs[0];
        h->rk_defer_auto = ds[0];
        tcx::drop_graphs(h);
        return TC_OK;
    }
    if (nsteps < (int)(cs.size() * ds.size()) + 1) return TC_OK;   // decide on a later, longer call
    cudaEvent_t a = nullptr, b = nullptr;
    struct Events {                      // destroyed on every exit
        cudaEvent_t *a, *b;
        ~Events() { if (*a) cudaEventDestroy(*a); if (*b) cudaEventDestroy(*b); }
    } guard{&a, &b};
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    float best = 1e30f;
    int bestc = cs[0], bestd = ds[0];
    for (int c : cs) {
        for (int df : ds) {
            h->chunks_auto = c;
            h->rk_defer_auto = df;
            tcx::drop_graphs(h);
            int rc = ensure_graph(h);
            if (rc) return rc;
            CK(cudaGraphUpload(h->graph, h->stream));
            CK(cudaEventRecord(a, h->stream));
            CK(cudaGraphLaunch(h->graph, h->stream));
            CK(cudaEventRecord(b, h->stream));
            CK(cudaEventSynchronize(b));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, a, b));
            if (ms < best) { best = ms; bestc = c; bestd = df; }
            ++*done;
        }
    }
    h->chunks_auto = bestc;
    h->rk_defer_auto = bestd;
    tcx::drop_graphs(h);
    if (h->chunks <= 0 && h->rk_defer < 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_plan[key] = {bestc, bestd};
    }
    return TC_OK;
}
}  // namespace

extern "C" {

int tc_advance_substeps(tc_handle* h, int nsub) {
    tcx::Range nvtx_range("tc_advance_substeps");
    if (!h || nsub < 0) { set_err("invalid handle or substep count"); return TC_ERR_ARG; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    for (int n = 0; n < nsub; ++n) {
        const int k = h->phase;
        tc_launch_plane_phase(h->d, h->stream);
        tc_launch_line_phase(h->d, k, h->stream);
        tc_launch_mean_phase(h->d, k, h->stream);
        CK(cudaGetLastError());
        h->phase = (k + 1) % 3;
        if (h->phase == 0) { h->t += h->d.dt; h->step += 1; }
    }
    CK(cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

// ---- one case split across ranks (transpose form) ------------------------
int tc_split_set(tc_handle* h, int r0, int r1, int j0, int j1) {
    tcx::Range nvtx_range("tc_split_set");
    if (!h) { set_err("null handle"); return TC_ERR_ARG; }
    const TcDev& d = h->d;
    if (r0 < 0 || r1 > d.Nr || r0 >= r1 || j0 < 0 || j1 > d.Nh || j0 >= j1) {
        set_err("tc_split_set: need 0 <= r0 < r1 <= Nr and 0 <= j0 < j1 <= Ntheta/2");
        return TC_ERR_ARG;
    }
    if (h->phase != 0) { set_err("tc_split_set: inside a step"); return TC_ERR_ARG; }
    if (!h->prod_slab || r1 - r0 > h->split_r1 - h->split_r0) {
        double2* p = nullptr;
        if (int rc = dalloc(h, p, (size_t)TC_NPROD * (r1 - r0) * d.npairs)) return rc;
        h->prod_slab = p;
    }
    h->split = true;
    h->split_r0 = r0; h->split_r1 = r1; h->split_j0 = j0; h->split_j1 = j1;
    return TC_OK;
}

int tc_split_planes(tc_handle* h) {
    tcx::Range nvtx_range("tc_split_planes");
    if (!h || !h->split) { set_err("tc_split_planes: no split set"); return TC_ERR_ARG; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    // the plane kernels on the slab: its planes of u, v, w, the scratch
    // buffers from their start, the products into the slab buffer
    TcDev ds = h->d;
    const size_t off = (size_t)h->split_r0 * ds.npairs;
    ds.Nr = h->split_r1 - h->split_r0;
    ds.u += off; ds.v += off; ds.w += off;
    ds.prod = h->prod_slab;
    tc_launch_plane_phase(ds, h->stream);
    CK(cudaGetLastError());
    return TC_OK;
}

int tc_split_pairs(tc_handle* h) {
    tcx::Range nvtx_range("tc_split_pairs");
    if (!h || !h->split) { set_err("tc_split_pairs: no split set"); return TC_ERR_ARG; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    const int k = h->phase;
    tc_launch_line_chunk(h->d, k, h->stream, h->split_j0, h->split_j1 - h->split_j0);
    if (h->split_j0 == 0) tc_launch_mean_phase(h->d, k, h->stream);
    CK(cudaGetLastError());
    h->phase = (k + 1) % 3;
    if (h->phase == 0) { h->t += h->d.dt; h->step += 1; }
    return TC_OK;
}

int tc_split_finish(tc_handle* h) {
    if (!h) { set_err("null handle"); return TC_ERR_ARG; }
    CK(cudaStreamSynchronize(h->stream));
    return check_flags(h);
}

void* tc_device_array(tc_handle* h, int which) {
    if (!h) { set_err("null handle"); return nullptr; }
    const TcDev& d = h->d;
    switch (which) {
        case TC_ARRAY_U: return d.u;
        case TC_ARRAY_V: return d.v;
        case TC_ARRAY_W: return d.w;
        case TC_ARRAY_ETA: return d.eta;
        case TC_ARRAY_PROD: return d.prod;
        case TC_ARRAY_PROD_SLAB: return h->prod_slab;
        default: set_err("unknown array"); return nullptr;
    }
}

int tc_step(tc_handle* h, int nsteps) {
    tcx::Range nvtx_range("tc_step");
    if (!h || nsteps < 0) { set_err("invalid handle or step count"); return TC_ERR_ARG; }
    if (h->phase != 0) { set_err("tc_step called inside a step; finish it with tc_advance_substeps"); return TC_ERR_ARG; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    int done = 0;
    if ((rc = tune_chunks(h, nsteps, &done))) return rc;
    if ((rc = ensure_graph(h))) return rc;
    if (tcx::defer_rk(h) && nsteps > done) {
        // the previous step's last RK memory runs beside the next step's
        // first theta rows; the last one is completed after the final step
        CK(cudaGraphLaunch(h->graph_first, h->stream));
        for (int n = done + 1; n < nsteps; ++n) CK(cudaGraphLaunch(h->graph_next, h->stream));
        tc_launch_rk_memory(h->d, 2, h->stream, 0, h->d.Nh, false);
        CK(cudaGetLastError());
    } else {
        for (int n = done; n < nsteps; ++n) CK(cudaGraphLaunch(h->graph, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    h->t += nsteps * h->d.dt;
    h->step += nsteps;
    return check_flags(h);
}

// State image: header, then v, eta, u, w, Hv, He (Nr * npairs complex128
// each), then U, W, HU, HW (Nr float64 each).
namespace {
struct StateHeader {
    char magic[8];                 // "TCSTATE1"
    int Nr, Ntheta, Nz, phase;
    long long step;
    double t;
};
}  // namespace

size_t tc_state_bytes(const tc_handle* h) {
    if (!h) return 0;
    const size_t P1 = (size_t)h->d.Nr * h->d.npairs;
    return sizeof(StateHeader) + 6 * P1 * sizeof(double2) + 4 * (size_t)h->d.Nr * sizeof(double);
}

int tc_save_state(tc_handle* h, void* buf, size_t bytes) {
    tcx::Range nvtx_range("tc_save_state");
    if (!h || !buf) { set_err("null handle or buffer"); return TC_ERR_ARG; }
    if (bytes != tc_state_bytes(h)) { set_err("state buffer size " + std::to_string(bytes) + " != " + std::to_string(tc_state_bytes(h))); return TC_ERR_SIZE; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    TcDev& d = h->d;
    StateHeader hd;
    std::memcpy(hd.magic, "TCSTATE1", 8);
    hd.Nr = d.Nr; hd.Ntheta = 2 * d.Nh; hd.Nz = d.Nz; hd.phase = h->phase;
    hd.step = h->step; hd.t = h->t;
    unsigned char* p = static_cast<unsigned char*>(buf);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    const size_t F = (size_t)d.Nr * d.npairs * sizeof(double2);
    for (const double2* f : {d.v, d.eta, d.u, d.w, d.Hv, d.He}) {
        CK(cudaMemcpyAsync(p, f, F, cudaMemcpyDeviceToHost, h->stream));
        p += F;
    }
    const size_t M = (size_t)d.Nr * sizeof(double);
    for (const double* f : {d.U, d.W, d.HU, d.HW}) {
        CK(cudaMemcpyAsync(p, f, M, cudaMemcpyDeviceToHost, h->stream));
        p += M;
    }
    CK(cudaStreamSynchronize(h->stream));
    return TC_OK;
}

int tc_load_state(tc_handle* h, const void* buf, size_t bytes) {
    tcx::Range nvtx_range("tc_load_state");
    if (!h || !buf) { set_err("null handle or buffer"); return TC_ERR_ARG; }
    if (bytes != tc_state_bytes(h)) { set_err("state buffer size " + std::to_string(bytes) + " != " + std::to_string(tc_state_bytes(h))); return TC_ERR_SIZE; }
    TcDev& d = h->d;
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "TCSTATE1", 8) != 0 || hd.Nr != d.Nr || hd.Ntheta != 2 * d.Nh || hd.Nz != d.Nz ||
        hd.phase < 0 || hd.phase > 2) {
        set_err("state image of another shape, or a damaged header");
        return TC_ERR_ARG;
    }
    const unsigned char* p = static_cast<const unsigned char*>(buf) + sizeof(hd);
    const size_t F = (size_t)d.Nr * d.npairs * sizeof(double2);
    for (double2* f : {d.v, d.eta, d.u, d.w, d.Hv, d.He}) {
        CK(cudaMemcpyAsync(f, p, F, cudaMemcpyHostToDevice, h->stream));
        p += F;
    }
    const size_t M = (size_t)d.Nr * sizeof(double);
    for (double* f : {d.U, d.W, d.HU, d.HW}) {
        CK(cudaMemcpyAsync(f, p, M, cudaMemcpyHostToDevice, h->stream));
        p += M;
    }
    CK(cudaStreamSynchronize(h->stream));
    h->need_init = false;            // the image holds the RK memories and u, w
    h->phase = hd.phase;
    h->step = hd.step;
    h->t = hd.t;
    return TC_OK;
}

size_t tc_field_bytes(const tc_handle* h, int which, int space) {
    if (!h) return 0;
    const TcDev& d = h->d;
    if (which == TC_FIELD_MEAN_U || which == TC_FIELD_MEAN_W) return (size_t)d.Nr * sizeof(double);
    if (which < 0 || which > TC_FIELD_ETA) return 0;
    if (space == TC_PHYSICAL) return (size_t)d.Nr * d.Mz * d.Mt * sizeof(double);
    return (size_t)d.Nr * d.npairs * sizeof(double2);
}

int tc_get_field(tc_handle* h, int which, int space, void* buf, size_t bytes) {
    tcx::Range nvtx_range("tc_get_field");
    if (!h || !buf) { set_err("null handle or buffer"); return TC_ERR_ARG; }
    if (which < 0 || which > TC_FIELD_MEAN_W || (space != TC_SPECTRAL && space != TC_PHYSICAL)) {
        set_err("unknown field or space");
        return TC_ERR_ARG;
    }
    const size_t need = tc_field_bytes(h, which, space);
    if (bytes != need) { set_err("buffer size " + std::to_string(bytes) + " != " + std::to_string(need)); return TC_ERR_SIZE; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    TcDev& d = h->d;
    if (which == TC_FIELD_MEAN_U || which == TC_FIELD_MEAN_W) {
        CK(cudaMemcpyAsync(buf, which == TC_FIELD_MEAN_U ? d.U : d.W, bytes, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return TC_OK;
    }
    const double2* src = which == TC_FIELD_U ? d.u : which == TC_FIELD_V ? d.v : which == TC_FIELD_W ? d.w : d.eta;
    if (space == TC_SPECTRAL) {
        CK(cudaMemcpyAsync(buf, src, bytes, cudaMemcpyDeviceToHost, h->stream));
    } else {
        if (!d.phys) {
            double* p;
            if ((rc = dalloc(h, p, (size_t)d.Nr * d.Mz * d.Mt))) return rc;
            d.phys = p;
            tcx::drop_graphs(h);
        }
        tc_launch_to_physical(d, src, h->stream);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(buf, d.phys, bytes, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return TC_OK;
}

// Shared by tc_set_field and tc_set_field_async: the copy and the Hermitian
// fix-up are queued on the handle's stream; sync waits for them.
static int set_field_impl(tc_handle* h, int which, const void* buf, size_t bytes, bool sync) {
    if (!h || !buf) { set_err("null handle or buffer"); return TC_ERR_ARG; }
    TcDev& d = h->d;
    if (which == TC_FIELD_MEAN_U || which == TC_FIELD_MEAN_W) {
        if (bytes != (size_t)d.Nr * sizeof(double)) { set_err("mean profile needs Nr float64"); return TC_ERR_SIZE; }
        CK(cudaMemcpyAsync(which == TC_FIELD_MEAN_U ? d.U : d.W, buf, bytes, cudaMemcpyDefault, h->stream));
        if (sync) CK(cudaStreamSynchronize(h->stream));
        h->need_init = true;
        h->phase = 0;
        return TC_OK;
    }
    if (which != TC_FIELD_V && which != TC_FIELD_ETA) { set_err("only V, ETA, MEAN_U and MEAN_W can be set"); return TC_ERR_ARG; }
    const size_t need = (size_t)d.Nr * d.npairs * sizeof(double2);
    if (bytes != need) { set_err("buffer size " + std::to_string(bytes) + " != " + std::to_string(need)); return TC_ERR_SIZE; }
    double2* dst = which == TC_FIELD_V ? d.v : d.eta;
    CK(cudaMemcpyAsync(dst, buf, bytes, cudaMemcpyDefault, h->stream));   // host or device source
    // Hermitian m = 0 column, zero Nyquist slot and (0,0), on the device
    tc_launch_realify(d, dst, h->stream);
    CK(cudaGetLastError());
    if (sync) CK(cudaStreamSynchronize(h->stream));
    h->need_init = true;
    h->phase = 0;
    return TC_OK;
}

int tc_set_field(tc_handle* h, int which, const void* buf, size_t bytes) {
    tcx::Range nvtx_range("tc_set_field");
    return set_field_impl(h, which, buf, bytes, true);
}

int tc_set_field_async(tc_handle* h, int which, const void* buf, size_t bytes) {
    tcx::Range nvtx_range("tc_set_field_async");
    return set_field_impl(h, which, buf, bytes, false);
}

int tc_get_field_async(tc_handle* h, int which, void* buf, size_t bytes, void* stream) {
    tcx::Range nvtx_range("tc_get_field_async");
    if (!h || !buf) { set_err("null handle or buffer"); return TC_ERR_ARG; }
    if (which < 0 || which > TC_FIELD_MEAN_W) { set_err("unknown field"); return TC_ERR_ARG; }
    const size_t need = tc_field_bytes(h, which, TC_SPECTRAL);
    if (bytes != need) { set_err("buffer size " + std::to_string(bytes) + " != " + std::to_string(need)); return TC_ERR_SIZE; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    const TcDev& d = h->d;
    const void* src = which == TC_FIELD_MEAN_U ? (const void*)d.U : which == TC_FIELD_MEAN_W ? (const void*)d.W
                    : which == TC_FIELD_U ? (const void*)d.u : which == TC_FIELD_V ? (const void*)d.v
                    : which == TC_FIELD_W ? (const void*)d.w : (const void*)d.eta;
    cudaStream_t s = stream ? (cudaStream_t)stream : h->stream;
    if (s != h->stream) {
        // ordered after everything queued so far on the handle's stream
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
        cudaEventDestroy(ev);
        CK(e);
    }
    CK(cudaMemcpyAsync(buf, src, bytes, cudaMemcpyDefault, s));   // host or device destination
    return TC_OK;
}

int tc_torque_stats(tc_handle* h, tc_stats* out) {
    tcx::Range nvtx_range("tc_torque_stats");
    if (!h || !out) { set_err("null handle or output"); return TC_ERR_ARG; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    TcDev& d = h->d;
    const int N = d.Nr;
    std::vector<double> W(N), ep(N), dp(N);
    tc_launch_energy(d, h->stream);
    tc_launch_strain(d, h->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(W.data(), d.W, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(ep.data(), d.eprof, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(dp.data(), d.dprof, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const double* e0 = &h->S.dwall[0];
    const double* e1 = &h->S.dwall[5];
    double dWi = 0, dWo = 0;
    for (int s = 0; s < 5; ++s) { dWi += e0[s] * W[s]; dWo += e1[s] * W[N - 5 + s]; }
    const double si = std::fabs(dWi - W[0] / h->r[0]);
    const double so = std::fabs(dWo - W[N - 1] / h->r[N - 1]);
    out->t = h->t;
    out->step = h->step;
    out->G_inner = 2.0 * M_PI * h->Ri * si;
    out->G_outer = 2.0 * M_PI * h->Ro * h->Ro / h->Ri * so;
    out->Re_tau_inner = std::sqrt(d.nu * si) / d.nu;
    out->Re_tau_outer = std::sqrt(d.nu * so) / d.nu;
    // fourth-order radial quadrature with weight r (uniform grid):
    // trapezoid with end weights 3/8, 7/6, 23/24
    double num = 0, dnum = 0, den = 0;
    const double hh = h->prm.stretch != 0.0 ? 2.0 / (N - 1) : (h->r[N - 1] - h->r[0]) / (N - 1);
    for (int j = 0; j < N; ++j) {
        double w = 1.0;
        if (j == 0 || j == N - 1) w = 3.0 / 8.0;
        else if (j == 1 || j == N - 2) w = 7.0 / 6.0;
        else if (j == 2 || j == N - 3) w = 23.0 / 24.0;
        w *= hh * h->jac[j] * h->r[j];
        num += w * ep[j];
        dnum += w * dp[j];
        den += w;
    }
    out->energy = 0.5 * num / den;
    out->dissipation = d.nu * dnum / den;
    // wall power: signed wall shear of the mean azimuthal flow times the
    // wall velocity, over the volume per unit box area (R_o^2 - R_i^2)/2
    const double Ri = h->r[0], Ro = h->r[N - 1];
    const double ti = dWi - W[0] / Ri, to = dWo - W[N - 1] / Ro;
    out->power_in = d.nu * (Ro * W[N - 1] * to - Ri * W[0] * ti) / (0.5 * (Ro * Ro - Ri * Ri));
    return TC_OK;
}

size_t tc_device_bytes(const tc_handle* h) { return h ? h->dev_bytes : 0; }

int tc_phase_times(tc_handle* h, int nsteps, double* ms, int nphases) {
    tcx::Range nvtx_range("tc_phase_times");
    if (!h || nsteps < 1 || !ms || nphases < TC_NPHASES) { set_err("invalid arguments"); return TC_ERR_ARG; }
    if (h->phase != 0) { set_err("tc_phase_times called inside a step"); return TC_ERR_ARG; }
    int rc;
    if ((rc = ensure_init(h))) return rc;
    cudaEvent_t ev[TC_NPHASES + 1];
    for (int i = 0; i <= TC_NPHASES; ++i) CK(cudaEventCreate(&ev[i]));
    double acc[TC_NPHASES] = {0, 0, 0, 0, 0};
    for (int n = 0; n < nsteps; ++n) {
        for (int k = 0; k < 3; ++k) {
            CK(cudaEventRecord(ev[0], h->stream));
            for (int w = 0; w < 3; ++w) {
                tc_launch_plane_kernel(h->d, w, h->stream);
                CK(cudaEventRecord(ev[w + 1], h->stream));
            }
            tc_launch_line_phase(h->d, k, h->stream);
            CK(cudaEventRecord(ev[4], h->stream));
            tc_launch_mean_phase(h->d, k, h->stream);
            CK(cudaEventRecord(ev[5], h->stream));
            CK(cudaEventSynchronize(ev[5]));
            for (int i = 0; i < TC_NPHASES; ++i) {
                float t = 0;
                CK(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
                acc[i] += t;
            }
        }
        h->t += h->d.dt;
        h->step += 1;
    }
    for (int i = 0; i <= TC_NPHASES; ++i) cudaEventDestroy(ev[i]);
    for (int i = 0; i < TC_NPHASES; ++i) ms[i] = acc[i] / (3.0 * nsteps);
    return check_flags(h);
}

int tc_fma_peak(int device, double* fp64_tflops, double* fp32_tflops) {
    if (!fp64_tflops || !fp32_tflops) { set_err("null output"); return TC_ERR_ARG; }
    if (device >= 0) CK(cudaSetDevice(device));
    CK(tc_probe_fma(fp64_tflops, fp32_tflops));
    return TC_OK;
}

}  // extern "C"
