"""Pins of the oracle on the smoothly stretched radial grid (Sec. 2.1: 5
arbitrarily spaced, smoothly stretched points, order >= 4): stencil order,
Couette N_r^-4 and the laminar torque of Table 2 on a tanh grid, the
manufactured-solution rows of Eqs. 6-7, and the radial quadrature."""
import math

import numpy as np

from oracle.grid import Case, radial_grid
from oracle.stencils import build_stencils
from oracle import operators as op
from oracle import diagnostics as dg
from scipy.linalg import solve_banded

A = 1.5   # tanh stretching


def _steady_W(cs, S):
    MW, LW, MU, LU = op.mean_operators(S, cs.r, cs.nu)
    rhs = np.zeros(cs.Nr)
    rhs[0], rhs[-1] = 1.0, cs.W_outer
    return solve_banded((3, 3), op.eta_system(S, LW), rhs)


def test_grid_is_denser_at_the_walls():
    r = radial_grid(0.5, 33, A)
    d = np.diff(r)
    assert d[0] < 0.5 * d[16] and d[-1] < 0.5 * d[16]
    assert abs(r[-1] - r[0] - 2.0) < 1e-14 and np.all(d > 0)


def test_couette_fourth_order_on_stretched_grid():
    errs, Ns = [], (17, 33, 65, 129)
    for N in Ns:
        cs = Case(N, 4, 4, 0.5, 60.0, 0.0, 1e-3, stretch=A)
        S = build_stencils(cs.r)
        z, r, Ri = cs.zeta, cs.r, cs.Ri
        exact = 1.0 / (1.0 - z * z) * (Ri / r - z * z * r / Ri)
        errs.append(np.max(np.abs(_steady_W(cs, S) - exact)))
    slope = -np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert slope > 3.5, (slope, errs)
    cs = Case(65, 4, 4, 0.5, 60.0, 0.0, 1e-3, stretch=A)
    S = build_stencils(cs.r)
    Gi, Go = dg.torque(cs, S, _steady_W(cs, S))
    assert abs(Gi - 4 * math.pi / 0.75) < 1e-4 and abs(Go - Gi) < 1e-4


def test_rows_converge_on_stretched_grid():
    import pytest
    pytest.importorskip("sympy")
    import test_oracle_rows as rows
    orig = rows.radial_grid
    try:
        rows.radial_grid = lambda zeta, N: orig(zeta, N, A)
        res = [rows._residuals(N) for N in (17, 33, 65)]
    finally:
        rows.radial_grid = orig
    for k in res[0]:
        e = [x[k] for x in res]
        orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
        assert min(orders) > (2.5 if k.endswith("_wall") else 3.5), (k, e, orders)


def test_quadrature_is_fourth_order_with_the_jacobian():
    errs = []
    for N in (17, 33, 65):
        cs = Case(N, 4, 4, 0.7, 100.0, 0.0, 1e-3, stretch=A)
        w = dg.radial_weights(cs.r, A)
        f = np.exp(0.3 * cs.r) * cs.r
        a, b = cs.r[0], cs.r[-1]
        F = lambda x: np.exp(0.3 * x) * (x / 0.3 - 1 / 0.09)
        errs.append(abs(np.dot(w, f) - (F(b) - F(a))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 3.5, (errs, orders)
