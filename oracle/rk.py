"""The 3-substep implicit/explicit Runge-Kutta step (Sec. 2.1 and Sec. 3.1).

The paper: explicit third-order Runge-Kutta for the non-linear and the
curvature-related viscous terms, Crank-Nicolson for the remaining viscous
terms, 3 substeps per step; the coefficients are not printed.  Reading used:
the low-storage scheme of Spalart, Moser & Rogers (1991), whose explicit part
is the third-order scheme with gamma = (8/15, 5/12, 3/4),
zeta = (0, -17/60, -5/12) and whose implicit part is Crank-Nicolson within
each substep, alpha_k = beta_k = (gamma_k + zeta_k)/2 = (4/15, 1/15, 1/6).

Substep k, written for the rows of each equation (M mass, L implicit,
E explicit):

  (M - beta_k dt L) x^k = (M + alpha_k dt L) x^(k-1)
                          + dt (gamma_k E(x^(k-1)) + zeta_k E(x^(k-2))).

This module stores E of the previous substep explicitly (the plain form).
"""
from fractions import Fraction
import numpy as np
from scipy.linalg import solve_banded

from .stencils import build_stencils
from .fourier import products
from . import operators as op


class SMR91:
    gamma = (Fraction(8, 15), Fraction(5, 12), Fraction(3, 4))
    zeta = (Fraction(0), Fraction(-17, 60), Fraction(-5, 12))
    alpha = (Fraction(4, 15), Fraction(1, 15), Fraction(1, 6))
    beta = (Fraction(4, 15), Fraction(1, 15), Fraction(1, 6))

    @classmethod
    def floats(cls):
        f = lambda t: tuple(float(x) for x in t)
        return f(cls.alpha), f(cls.beta), f(cls.gamma), f(cls.zeta)


class OracleSolver:
    """One Taylor-Couette case advanced by the plain FP64 method.

    State: v, eta spectral (Nr, Nz, Nh) complex128; mean profiles U (axial)
    and W (azimuthal), (Nr,) float64.  Starts from circular Couette flow
    W = A r + B/r (Eq. 1 with W(R_i) = 1, W(R_o) = Re_o/Re_i) and zero
    perturbation."""

    def __init__(self, case, stencils=None, pairs=None):
        """pairs: optional boolean (Nz, Nh) mask restricting the evolved pairs
        (the others stay zero); used to check sampled pairs of large cases."""
        self.case = case
        self.S = stencils if stencils is not None else build_stencils(case.r)
        cs = case
        self.r_col = cs.r.reshape(-1, 1)
        mask = cs.active_mask()
        if pairs is not None:
            mask = mask & pairs
        self.act = np.nonzero(mask)          # (n-slot, j) of active pairs
        m_full = np.broadcast_to(cs.m_of()[0], (cs.Nz, cs.Nh))
        a_full = np.broadcast_to(cs.alpha_of()[0], (cs.Nz, cs.Nh))
        self.m = m_full[self.act].reshape(1, -1)
        self.alpha = a_full[self.act].reshape(1, -1)
        self.coef = op.coefficients(self.r_col, self.m, self.alpha)
        self.Mv, self.Lv = op.v_operators(self.S, self.r_col, self.m, self.alpha, cs.nu, self.coef)
        self.Me, self.Le = op.eta_operators(self.S, self.r_col, self.m, self.alpha, cs.nu, self.coef)
        self.MW, self.LW, self.MU, self.LU = op.mean_operators(self.S, cs.r, cs.nu)
        # conjugate partners of the m = 0, n < 0 slots
        n = np.fft.fftfreq(cs.Nz, d=1.0 / cs.Nz).astype(int)
        self.conj_dst = [s for s in range(cs.Nz) if n[s] < 0 and s != cs.Nz // 2]
        self.conj_src = [int(np.mod(-n[s], cs.Nz)) for s in self.conj_dst]
        self.v = np.zeros((cs.Nr, cs.Nz, cs.Nh), dtype=np.complex128)
        self.eta = np.zeros_like(self.v)
        self.U = np.zeros(cs.Nr)
        self.W = couette_profile(cs)
        self.E_prev = None
        self.t = 0.0
        self.steps = 0

    # ---- field access -------------------------------------------------------
    def set_fields(self, v=None, eta=None, U=None, W=None):
        if v is not None:
            self.v = np.array(v, dtype=np.complex128)
        if eta is not None:
            self.eta = np.array(eta, dtype=np.complex128)
        if U is not None:
            self.U = np.array(U, dtype=np.float64)
        if W is not None:
            self.W = np.array(W, dtype=np.float64)
        self._hermitian(self.v)
        self._hermitian(self.eta)
        self.E_prev = None

    def _gather(self, F):
        return F[:, self.act[0], self.act[1]]

    def _scatter(self, a):
        cs = self.case
        F = np.zeros((cs.Nr, cs.Nz, cs.Nh), dtype=np.complex128)
        F[:, self.act[0], self.act[1]] = a
        self._hermitian(F)
        return F

    def _hermitian(self, F):
        """m = 0 column: slot n < 0 holds the conjugate of slot -n; the axial
        Nyquist slot and (0, 0) of v, eta are zero."""
        F[:, self.conj_dst, 0] = np.conj(F[:, self.conj_src, 0])
        F[:, self.case.Nz // 2, :] = 0.0
        F[:, 0, 0] = 0.0

    def velocity(self):
        """Spectral u (axial), v (radial), w (azimuthal); (0,0) holds U, 0, W."""
        va, ea = self._gather(self.v), self._gather(self.eta)
        ua, wa = op.reconstruct_uw(self.S, self.r_col, self.m, self.alpha, self.coef[0], va, ea)
        u, w = self._scatter(ua), self._scatter(wa)
        u[:, 0, 0] = self.U
        w[:, 0, 0] = self.W
        v = self.v.copy()
        v[:, 0, 0] = 0.0
        return u, v, w

    # ---- one substep ----------------------------------------------------------
    def explicit_terms(self, P=None):
        """E(x) for v, eta (active pairs) and for U, W; the products P (dict of
        spectral arrays) are formed from the current velocity unless given."""
        cs = self.case
        u, v, w = self.velocity()
        if P is None:
            P = products(cs, u, v, w)
        Pa = {k: self._gather(P[k]) for k in P}
        ua, va, wa = self._gather(u), self._gather(v), self._gather(w)
        Ev = op.v_explicit(self.S, self.r_col, self.m, self.alpha, cs.nu, self.coef, ua, va, wa, Pa)
        Ee = op.eta_explicit(self.S, self.r_col, self.m, self.alpha, cs.nu, ua, va, wa, Pa)
        EU, EW = op.mean_explicit(self.S, cs.r, P["uv"][:, 0, 0].real, P["vw"][:, 0, 0].real)
        return {"v": Ev, "eta": Ee, "U": EU, "W": EW}

    def substep(self, k):
        self.advance(k, self.explicit_terms())

    def advance(self, k, E):
        """Right sides and banded solves of substep k, given E(x^(k-1))."""
        cs = self.case
        al, be, ga, ze = SMR91.floats()
        dt = cs.dt
        Nr = cs.Nr
        Ep = self.E_prev if self.E_prev is not None else {key: 0.0 * val for key, val in E.items()}
        ex = lambda key: dt * (ga[k] * E[key] + ze[k] * Ep[key])

        # v: rows 2..Nr-3, boundary rows 0, 1, Nr-2, Nr-1 have zero right side
        va = self._gather(self.v)
        rhs = (op.band_apply(self.S, self.Mv, va) + al[k] * dt * op.band_apply(self.S, self.Lv, va)
               + ex("v"))
        rhs[[0, 1, Nr - 2, Nr - 1]] = 0.0
        A = (self.Mv - be[k] * dt * self.Lv).real
        v_new = op.solve_rows(op.v_system(self.S, A), rhs)

        # eta: rows 1..Nr-2, eta = 0 on rows 0, Nr-1
        ea = self._gather(self.eta)
        rhs = (op.band_apply(self.S, self.Me, ea) + al[k] * dt * op.band_apply(self.S, self.Le, ea)
               + ex("eta"))
        rhs[[0, Nr - 1]] = 0.0
        A = (self.Me - be[k] * dt * self.Le).real
        e_new = op.solve_rows(op.eta_system(self.S, A), rhs)

        # mean flow
        rW = (op.band_apply(self.S, self.MW, self.W) + al[k] * dt * op.band_apply(self.S, self.LW, self.W)
              + ex("W"))
        rW[0], rW[Nr - 1] = 1.0, cs.W_outer
        W_new = solve_banded((3, 3), op.eta_system(self.S, self.MW - be[k] * dt * self.LW), rW)
        rU = (op.band_apply(self.S, self.MU, self.U) + al[k] * dt * op.band_apply(self.S, self.LU, self.U)
              + ex("U"))
        rU[0], rU[Nr - 1] = 0.0, 0.0
        U_new = solve_banded((3, 3), op.eta_system(self.S, self.MU - be[k] * dt * self.LU), rU)

        self.v = self._scatter(v_new)
        self.eta = self._scatter(e_new)
        self.W, self.U = W_new, U_new
        self.E_prev = E

    def step(self, nsteps=1):
        for _ in range(nsteps):
            for k in range(3):
                self.substep(k)
            self.E_prev = None      # zeta_1 = 0: nothing carries over a step
            self.t += self.case.dt
            self.steps += 1


def couette_profile(case, r=None):
    """Circular Couette flow W = A r + B/r with W(R_i) = 1 and
    W(R_o) = Re_o/Re_i (Eq. 1 is the case Re_o = 0)."""
    r = case.r if r is None else r
    Ri, Ro, Wo = case.Ri, case.r[-1], case.W_outer
    A = (Wo * Ro - Ri) / (Ro ** 2 - Ri ** 2)
    B = (Ri - A * Ri ** 2)
    return A * r + B / r
