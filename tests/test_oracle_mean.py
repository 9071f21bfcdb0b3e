"""Pins of the oracle's mean-flow rows (m = alpha = 0), the axial row U in
particular.

The paper gives the mean-flow equations only through their ingredients: the
primitive-variable momentum equations of the Appendix, averaged over theta and
z, with zero mean pressure gradient (Sec. 4).  Averaged, the axial and the
azimuthal momentum equations read

    dU/dt = nu (U'' + U'/r)        - (1/r)   d(r   <uv>)/dr
    dW/dt = nu (W'' + W'/r - W/r^2) - (1/r^2) d(r^2 <vw>)/dr

(u axial, v radial, w azimuthal).  The references below are built from these
textbook forms, not from the oracle's row forms, so a dropped curvature term
(U/r^2 in the axial viscous row, uv/r or 2 vw/r in the forcing) or a wrong
sign fails one of them:

* the steady sliding-inner-cylinder flow, U = ln(r/R_o)/ln(R_i/R_o), solves
  U'' + U'/r = 0 with U(R_i) = 1, U(R_o) = 0; the discrete steady U rows
  reproduce it at fourth order in N_r (the axial counterpart of Fig. 2);
* manufactured profiles U, W, <uv>, <vw>: the discrete rows applied to them
  approach d0 . (continuum right side) at fourth order, viscous and forcing
  parts separately.
"""
import math

import numpy as np
import pytest
from scipy.linalg import solve_banded

from oracle.grid import Case, radial_grid
from oracle.stencils import build_stencils
from oracle import operators as op

sp = pytest.importorskip("sympy")


def steady_U_sliding(N, zeta):
    """nu (U'' + U'/r) = 0 through the oracle's U rows, U(R_i) = 1, U(R_o) = 0."""
    cs = Case(N, 4, 4, zeta, 100.0, 0.0, 1e-3)
    S = build_stencils(cs.r)
    MW, LW, MU, LU = op.mean_operators(S, cs.r, cs.nu)
    rhs = np.zeros(N)
    rhs[0] = 1.0
    U = solve_banded((3, 3), op.eta_system(S, LU), rhs)
    exact = np.log(cs.r / cs.Ro) / math.log(cs.Ri / cs.Ro)
    return np.max(np.abs(U - exact))


@pytest.mark.parametrize("zeta", [0.5, 0.883])
def test_sliding_cylinder_fourth_order(zeta):
    Ns = (17, 33, 65, 129)
    errs = [steady_U_sliding(N, zeta) for N in Ns]
    slope = -np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert 3.6 < slope < 5.5, (slope, errs)
    assert errs[1] < 1e-5, errs


# ---- manufactured profiles ------------------------------------------------------

r = sp.symbols("r", positive=True)
U_s = sp.sin(3 * r / 2) * sp.exp(-r / 7) + r / 3
W_s = sp.cos(r) + 1 / r
uv_s = sp.cos(6 * r / 5) * r / 4 + sp.Rational(1, 5)
vw_s = sp.sin(r / 2) ** 2 - sp.exp(-r / 3)
CONT = {
    "U_visc": sp.diff(U_s, r, 2) + sp.diff(U_s, r) / r,
    "W_visc": sp.diff(W_s, r, 2) + sp.diff(W_s, r) / r - W_s / r ** 2,
    "U_nl": -sp.diff(r * uv_s, r) / r,
    "W_nl": -sp.diff(r ** 2 * vw_s, r) / r ** 2,
}
FN = {k: sp.lambdify(r, e, "numpy") for k, e in CONT.items()}
FLD = {k: sp.lambdify(r, e, "numpy") for k, e in dict(U=U_s, W=W_s, uv=uv_s, vw=vw_s).items()}


def _residuals(N, zeta):
    x = radial_grid(zeta, N)
    S = build_stencils(x)
    g = {k: np.asarray(f(x), dtype=np.float64) * np.ones_like(x) for k, f in FLD.items()}
    MW, LW, MU, LU = op.mean_operators(S, x, 1.0)
    EU, EW = op.mean_explicit(S, x, g["uv"], g["vw"])
    disc = {"U_visc": op.band_apply(S, LU, g["U"]), "W_visc": op.band_apply(S, LW, g["W"]),
            "U_nl": EU, "W_nl": EW}
    out = {}
    for k, dv in disc.items():
        cont = np.asarray(FN[k](x), dtype=np.float64) * np.ones_like(x)
        ref = S.apply(S.d0, cont)
        rows = slice(2, N - 2)
        scale = np.max(np.abs(ref[rows]))
        out[k] = np.max(np.abs(dv[rows] - ref[rows])) / scale
        # explicit one-sided near-wall rows 1 and N-2 (d0 = delta)
        out[k + "_wall"] = max(abs(dv[j] - cont[j]) for j in (1, N - 2)) / scale
    return out


@pytest.mark.parametrize("zeta", [0.5, 0.883])
def test_mean_rows_converge_to_averaged_momentum_equations(zeta):
    Ns = (17, 33, 65)
    res = [_residuals(N, zeta) for N in Ns]
    for k in res[0]:
        e = [rr[k] for rr in res]
        orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        need = 2.5 if k.endswith("_wall") else 3.7
        assert min(orders) > need, (k, e, orders)
    for k, e in res[-1].items():
        if not k.endswith("_wall"):
            assert e < 1e-5, (k, e)


# ---- planted mistakes: each plausible slip in the mean rows fails a pin ---------

def _drop_curvature_of_U(S, r, nu):
    MW, LW, MU, LU = ORIG_OPS(S, r, nu)
    return MW, LW, MU, nu * op.band(S, [(S.l2, 1.0)], ())


def _drop_uv_over_r(S, r, uv00, vw00):
    EU, EW = ORIG_EXPL(S, r, uv00, vw00)
    return -S.apply(S.l1, uv00), EW


def _halve_vw_over_r(S, r, uv00, vw00):
    EU, EW = ORIG_EXPL(S, r, uv00, vw00)
    return EU, -S.apply(S.l1, vw00) - S.apply(S.d0, vw00 / r.reshape(-1))


ORIG_OPS = op.mean_operators
ORIG_EXPL = op.mean_explicit


def test_dropped_U_over_r2_fails_the_sliding_cylinder(monkeypatch):
    monkeypatch.setattr(op, "mean_operators", _drop_curvature_of_U)
    errs = [steady_U_sliding(N, 0.5) for N in (33, 65)]
    assert errs[-1] > 1e-3 and errs[-1] / errs[0] > 0.5, errs


@pytest.mark.parametrize("planted, key", [(_drop_uv_over_r, "U_nl"), (_halve_vw_over_r, "W_nl")])
def test_dropped_forcing_term_fails_the_manufactured_pin(monkeypatch, planted, key):
    monkeypatch.setattr(op, "mean_explicit", planted)
    e = [_residuals(N, 0.5)[key] for N in (17, 33, 65)]
    assert e[-1] > 1e-3 and e[-1] / e[0] > 0.5, e


def test_dropped_U_over_r2_fails_the_manufactured_pin(monkeypatch):
    monkeypatch.setattr(op, "mean_operators", _drop_curvature_of_U)
    e = [_residuals(N, 0.5)["U_visc"] for N in (17, 33, 65)]
    assert e[-1] > 1e-3 and e[-1] / e[0] > 0.5, e
