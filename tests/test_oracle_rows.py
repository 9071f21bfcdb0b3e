"""Manufactured-solution pin of the rows of Eq. 6 and Eq. 7.

The continuum reference is built WITHOUT Eqs. 6-7: from the textbook
primitive-variable cylindrical Navier-Stokes equations (vector Laplacian,
conservative non-linear terms), combined the way the v-eta formulation
eliminates the pressure (Appendix):

    v equation:   d/dt [v + D(c (i alpha u + i m/r w))]
                  = nu {visc_v + D[c (i alpha visc_u + i m/r visc_w)]}
                    + HV + D[c (i alpha HU + i m/r HW)]
    eta equation: d/dt eta = nu {(i m/r) visc_u - i alpha visc_w}
                  + (i m/r) HU - i alpha HW

with u, w rebuilt from continuity.  The oracle's discrete rows (mass,
implicit + explicit viscous, non-linear) must approach d0 . (continuum) at
fourth order; a dropped term, a wrong sign or a wrong reading of a garbled
term in Eq. 6 stops the convergence.
"""
import math

import numpy as np
import pytest

from oracle.grid import radial_grid
from oracle.stencils import build_stencils
from oracle import operators as op

sp = pytest.importorskip("sympy")

r = sp.symbols("r", positive=True)
M_, AL_ = sp.Rational(23, 10), sp.Rational(13, 10)      # m and alpha of the mode
I = sp.I
D = lambda f: sp.diff(f, r)
Ds = lambda f: sp.diff(f, r) + f / r
k2 = AL_ ** 2 + M_ ** 2 / r ** 2
c = 1 / k2

v_s = (sp.sin(2 * r) + I * sp.cos(r)) * sp.exp(r / 10)
eta_s = sp.cos(3 * r / 2) + I * sp.sin(r) / 2
u_s = (I * AL_ * Ds(v_s) - I * M_ / r * eta_s) / k2
w_s = (I * M_ / r * Ds(v_s) + I * AL_ * eta_s) / k2
PROD = {"uu": sp.cos(r), "uv": sp.sin(13 * r / 10) + I * r / 5, "uw": sp.exp(-r / 3) * (1 + I),
        "vv": r ** 2 / 10, "vw": I * sp.cos(7 * r / 10), "ww": sp.sin(r) * sp.cos(r) - I / 3}


def lap(f):
    return sp.diff(f, r, 2) + D(f) / r - k2 * f


visc_u = lap(u_s)
visc_v = lap(v_s) - v_s / r ** 2 - 2 * I * M_ / r ** 2 * w_s
visc_w = lap(w_s) - w_s / r ** 2 + 2 * I * M_ / r ** 2 * v_s
uu, uv, uw, vv, vw, ww = (PROD[k] for k in ("uu", "uv", "uw", "vv", "vw", "ww"))
HU = -(I * AL_ * uu + Ds(uv) + I * M_ / r * uw)
HV = -(I * AL_ * uv + Ds(vv) + I * M_ / r * vw - ww / r)
HW = -(I * AL_ * uw + D(vw) + 2 * vw / r + I * M_ / r * ww)

CONT = {
    "v_mass": v_s + D(c * (I * AL_ * u_s + I * M_ / r * w_s)),
    "v_visc": visc_v + D(c * (I * AL_ * visc_u + I * M_ / r * visc_w)),
    "v_nl": HV + D(c * (I * AL_ * HU + I * M_ / r * HW)),
    "eta_visc": I * M_ / r * visc_u - I * AL_ * visc_w,
    "eta_nl": I * M_ / r * HU - I * AL_ * HW,
}
FN = {k: sp.lambdify(r, e, "numpy") for k, e in CONT.items()}
FIELDS = {k: sp.lambdify(r, e, "numpy") for k, e in
          dict(v=v_s, eta=eta_s, u=u_s, w=w_s, **PROD).items()}


def _ev(f, x):
    return np.asarray(f(x), dtype=np.complex128) * np.ones_like(x)


def _residuals(N, zeta=0.5):
    x = radial_grid(zeta, N)
    S = build_stencils(x)
    rc = x.reshape(-1, 1)
    m = np.array([[float(M_)]])
    al = np.array([[float(AL_)]])
    coef = op.coefficients(rc, m, al)
    g = {k: _ev(f, x).reshape(-1, 1) for k, f in FIELDS.items()}
    zero = np.zeros_like(g["v"])
    P = {k: g[k] for k in ("uu", "uv", "uw", "vv", "vw", "ww")}
    P0 = {k: zero for k in P}
    Mv, Lv = op.v_operators(S, rc, m, al, 1.0, coef)
    Me, Le = op.eta_operators(S, rc, m, al, 1.0, coef)
    disc = {
        "v_mass": op.band_apply(S, Mv, g["v"]),
        "v_visc": op.band_apply(S, Lv, g["v"])
        + op.v_explicit(S, rc, m, al, 1.0, coef, g["u"], g["v"], g["w"], P0),
        "v_nl": op.v_explicit(S, rc, m, al, 1.0, coef, zero, zero, zero, P),
        "eta_visc": op.band_apply(S, Le, g["eta"])
        + op.eta_explicit(S, rc, m, al, 1.0, g["u"], g["v"], g["w"], P0),
        "eta_nl": op.eta_explicit(S, rc, m, al, 1.0, zero, zero, zero, P),
    }
    out = {}
    for k, dv in disc.items():
        ref = S.apply(S.d0, _ev(FN[k], x))
        rows = slice(2, N - 2)
        out[k] = np.max(np.abs(dv[rows, 0] - ref[rows])) / np.max(np.abs(ref[rows]))
        if k.startswith("eta"):
            # explicit one-sided near-wall rows: lower (third) order
            out[k + "_wall"] = max(abs(dv[j, 0] - _ev(FN[k], x)[j]) for j in (1, N - 2)) / np.max(np.abs(ref[rows]))
    return out


def test_rows_converge_to_primitive_equations():
    Ns = (17, 33, 65)
    res = [_residuals(N) for N in Ns]
    for k in res[0]:
        e = [rr[k] for rr in res]
        orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        need = 2.5 if k.endswith("_wall") else 3.7
        assert min(orders) > need, (k, e, orders)
    # absolute accuracy at N = 65: every row family within 1e-5 relative
    for k, e in res[-1].items():
        if not k.endswith("_wall"):
            assert e < 1e-5, (k, e)


def test_pin_catches_a_dropped_term(monkeypatch):
    """Plant a mistake in the oracle (drop D[c3 v] from the implicit v rows):
    the manufactured-solution residual stops converging."""
    orig = op.v_operators

    def broken(S, r, m, alpha, nu, coef):
        k2, c, c1, c2, c3 = coef
        return orig(S, r, m, alpha, nu, (k2, c, c1, c2, 0.0 * c3))
    monkeypatch.setattr(op, "v_operators", broken)
    e = [_residuals(N)["v_visc"] for N in (17, 33, 65)]
    assert e[-1] > 1e-4 and e[-1] / e[0] > 0.1


def test_reconstruction_is_divergence_free_and_matches_eta():
    """u, w rebuilt from v, eta satisfy continuity with the compact D and the
    definition of eta to round-off."""
    N = 33
    x = radial_grid(0.883, N)
    S = build_stencils(x)
    rc = x.reshape(-1, 1)
    rng = np.random.default_rng(0)
    m = np.array([[0.0, 3.2, 6.4, 3.2]])
    al = np.array([[1.25, 0.0, -2.5, 3.75]])
    k2 = op.coefficients(rc, m, al)[0]
    v = rng.standard_normal((N, 4)) + 1j * rng.standard_normal((N, 4))
    v[[0, -1]] = 0
    eta = rng.standard_normal((N, 4)) + 1j * rng.standard_normal((N, 4))
    u, w = op.reconstruct_uw(S, rc, m, al, k2, v, eta)
    Dsv = op.radial_derivative(S, v) + v / rc
    div = 1j * al * u + 1j * m / rc * w + Dsv
    assert np.max(np.abs(div)) < 1e-12 * np.max(np.abs(Dsv))
    assert np.max(np.abs(1j * m / rc * u - 1j * al * w - eta)) < 1e-12 * np.max(np.abs(eta))


def test_isotropic_flux_changes_no_row():
    """Adding q to uu, vv and ww adds the gradient of q to the non-linear term,
    which the pressure-free v and eta rows must annihilate (Appendix: pressure
    is eliminated).  The GPU path relies on it to transform 5 products
    (uu - vv, uv, uw, vw, ww - vv) instead of 6."""
    N = 33
    x = radial_grid(0.883, N)
    S = build_stencils(x)
    rc = x.reshape(-1, 1)
    rng = np.random.default_rng(1)
    m = np.array([[0.0, 3.2, 6.4, 9.6]])
    al = np.array([[1.25, 0.0, -2.5, 3.75]])
    coef = op.coefficients(rc, m, al)
    P = {k: rng.standard_normal((N, 4)) + 1j * rng.standard_normal((N, 4))
         for k in ("uu", "uv", "uw", "vv", "vw", "ww")}
    z = np.zeros((N, 4), complex)
    q = rng.standard_normal((N, 4)) + 1j * rng.standard_normal((N, 4))
    P2 = dict(P, uu=P["uu"] + q, vv=P["vv"] + q, ww=P["ww"] + q)
    for f, rows in ((lambda PP: op.v_explicit(S, rc, m, al, 1.0, coef, z, z, z, PP), slice(2, N - 2)),
                    (lambda PP: op.eta_explicit(S, rc, m, al, 1.0, z, z, z, PP), slice(1, N - 1))):
        a, b = f(P)[rows], f(P2)[rows]
        assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))
    # while a non-isotropic change is not annihilated
    P3 = dict(P, uu=P["uu"] + q)
    a, b = op.v_explicit(S, rc, m, al, 1.0, coef, z, z, z, P), op.v_explicit(S, rc, m, al, 1.0, coef, z, z, z, P3)
    assert np.max(np.abs(a - b)[2:N - 2]) > 1e-3 * np.max(np.abs(a))
