"""Linearised operator of one Fourier mode about circular Couette flow.

Sec. 3 validates the code through the critical Reynolds number Re_c of
the first Taylor-vortex instability (68.2 < Re_c < 68.4 at zeta = 0.5,
184 < Re_c < 186 at zeta = 0.95, on the straight-vortex box of Table 1).
This module assembles, from the oracle's own rows, the semi-discrete system
of one pair (m, alpha)

    B dx/dt = A x,     x = (v, eta) on the radial grid,

where the boundary rows of v and eta are algebraic (zero rows of B) and the
non-linear terms are linearised about the base flow (U = 0, W(r)): with
primes for the perturbation, the spectral products of this pair are
uw = W u', vw = W v', ww = 2 W w', uu = uv = vv = 0.  The growth rate is the
largest real part of the finite generalised eigenvalues.
"""
import numpy as np
from scipy.linalg import eig

from . import operators as op
from .rk import couette_profile


def linear_system(case, S, m, alpha, W=None):
    Nr = case.Nr
    r = case.r.reshape(-1, 1)
    mm = np.array([[m]], dtype=np.float64)
    aa = np.array([[alpha]], dtype=np.float64)
    coef = op.coefficients(r, mm, aa)
    Mv, Lv = op.v_operators(S, r, mm, aa, case.nu, coef)
    Me, Le = op.eta_operators(S, r, mm, aa, case.nu, coef)
    Wb = (couette_profile(case) if W is None else W).reshape(-1, 1)
    n = 2 * Nr
    A = np.zeros((n, n), dtype=np.complex128)
    B = np.zeros((n, n), dtype=np.complex128)
    vrows = np.arange(2, Nr - 2)
    erows = np.arange(1, Nr - 1)
    for i in range(n):
        x = np.zeros((n, 1), dtype=np.complex128)
        x[i] = 1.0
        v, eta = x[:Nr], x[Nr:]
        u, w = op.reconstruct_uw(S, r, mm, aa, coef[0], v, eta)
        zero = np.zeros_like(v)
        P = {"uu": zero, "uv": zero, "uw": Wb * u, "vv": zero, "vw": Wb * v, "ww": 2.0 * Wb * w}
        rv = op.band_apply(S, Lv, v) + op.v_explicit(S, r, mm, aa, case.nu, coef, u, v, w, P)
        re = op.band_apply(S, Le, eta) + op.eta_explicit(S, r, mm, aa, case.nu, u, v, w, P)
        A[vrows, i] = rv[vrows, 0]
        A[Nr + erows, i] = re[erows, 0]
        B[vrows, i] = op.band_apply(S, Mv, v)[vrows, 0]
        B[Nr + erows, i] = op.band_apply(S, Me, eta)[erows, 0]
        # boundary rows: v_0 = 0, Dv(r_0) = 0, Dv(r_N-1) = 0, v_N-1 = 0, eta_0 = eta_N-1 = 0
        A[0, i] = v[0, 0]
        A[1, i] = S.dwall[0] @ v[0:5, 0]
        A[Nr - 2, i] = S.dwall[1] @ v[Nr - 5:Nr, 0]
        A[Nr - 1, i] = v[Nr - 1, 0]
        A[Nr, i] = eta[0, 0]
        A[2 * Nr - 1, i] = eta[Nr - 1, 0]
    return A, B


def growth_rate(case, S, m, alpha, W=None):
    A, B = linear_system(case, S, m, alpha, W)
    lam = eig(A, B, right=False)
    # the six algebraic boundary rows give infinite eigenvalues, which the
    # QZ algorithm returns as inf or as values near 1/eps: keep |lambda| < 1e8
    # (physical decay rates here are below nu k_max^2 ~ 1e5)
    lam = lam[np.isfinite(lam)]
    lam = lam[np.abs(lam) < 1e8]
    return float(np.max(lam.real))
