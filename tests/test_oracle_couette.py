"""Pins of the oracle's mean-flow rows, torque and Re_tau against the closed
form of circular Couette flow (Eq. 1), Fig. 2 (N_r^-4 convergence) and
Table 2 (laminar torque)."""
import json
import math
import os

import numpy as np
from scipy.linalg import solve_banded

from oracle.grid import Case
from oracle.stencils import build_stencils
from oracle import operators as op
from oracle import diagnostics as dg
from oracle.rk import OracleSolver, couette_profile

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def steady_W(case, S):
    """Discrete steady azimuthal mean flow: nu D D_* W = 0 on rows 1..Nr-2
    with W(R_i) = 1, W(R_o) = Re_o/Re_i, through the oracle's mean rows."""
    MW, LW, MU, LU = op.mean_operators(S, case.r, case.nu)
    rhs = np.zeros(case.Nr)
    rhs[0], rhs[-1] = 1.0, case.W_outer
    return solve_banded((3, 3), op.eta_system(S, LW), rhs)


def exact_eq1(case):
    """Eq. 1: w = W_i/(1 - zeta^2) [R_i/r - zeta^2 r/R_i]  (outer wall at rest)."""
    z = case.zeta
    r, Ri = case.r, case.Ri
    return 1.0 / (1.0 - z * z) * (Ri / r - z * z * r / Ri)


def test_couette_fourth_order_convergence():
    """Fig. 2: ||E||_inf ~ N_r^-4 at zeta = 0.5."""
    errs, Ns = [], (17, 33, 65, 129)
    for N in Ns:
        cs = Case(N, 4, 4, 0.5, 60.0, 0.0, 1e-3)
        S = build_stencils(cs.r)
        errs.append(np.max(np.abs(steady_W(cs, S) - exact_eq1(cs))))
    slope = -np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert GOLD["couette_error_order"]["value"] == 4
    assert 3.7 < slope < 5.0, (slope, errs)
    # and the profile itself is the one of Eq. 1 at N_r = 33
    assert errs[1] < 1e-5


def test_laminar_torque_table2():
    """Table 2 laminar rows: 16.7551 at zeta = 0.5 (Re = 60, 68); the
    closed form is 4 pi/(1 - zeta^2); inner and outer torques agree."""
    g = GOLD["laminar_torque_zeta_0.5"]
    cs = Case(65, 4, 4, 0.5, 60.0, 0.0, 1e-3)
    S = build_stencils(cs.r)
    Gi, Go = dg.torque(cs, S, steady_W(cs, S))
    assert abs(Gi - g["value"]) < 10 ** -g["digits"]
    assert abs(Gi - 4 * math.pi / (1 - 0.25)) < 1e-4
    assert abs(Gi - Go) / Gi < 1e-5          # equal up to the O(h^4) error
    # the Re dependence vanishes in the laminar regime (rows 60 and 68 equal)
    cs68 = Case(65, 4, 4, 0.5, 68.0, 0.0, 1e-3)
    Gi68, _ = dg.torque(cs68, S, steady_W(cs68, S))
    assert abs(Gi68 - Gi) < 1e-12 * Gi


def test_re_tau_ratio_is_zeta_in_laminar_flow():
    """Sec. 5: Re_tau(outer)/Re_tau(inner) = zeta (exact for laminar flow)."""
    cs = Case(65, 4, 4, 0.883, 3000.0, 0.0, 1e-3)
    S = build_stencils(cs.r)
    ti, to = dg.re_tau(cs, S, steady_W(cs, S))
    assert abs(to / ti - 0.883) < 1e-6


def test_counter_rotating_profile():
    """W = A r + B/r with W(R_o) = Re_o/Re_i is annihilated by D D_*."""
    cs = Case(65, 4, 4, 0.5, 250.0, -55.0, 1e-3)
    S = build_stencils(cs.r)
    W = steady_W(cs, S)
    assert np.max(np.abs(W - couette_profile(cs))) < 1e-6
    assert abs(W[-1] + 55.0 / 250.0) < 1e-15


def test_time_marching_reaches_couette():
    """The RK mean-flow path relaxes a wrong profile to the discrete steady
    state (zero perturbation, large dt; the implicit part is A-stable)."""
    cs = Case(33, 4, 4, 0.5, 20.0, 0.0, 0.5)
    s = OracleSolver(cs)
    s.set_fields(W=np.linspace(1.0, 0.0, cs.Nr))
    s.step(200)
    S = s.S
    assert np.max(np.abs(s.W - steady_W(cs, S))) < 1e-10
    assert np.max(np.abs(s.U)) == 0.0


def test_laminar_state_is_a_fixed_point():
    """With no perturbation the discrete laminar state is left unchanged."""
    cs = Case(33, 8, 8, 0.883, 200.0, 0.0, 1e-3)
    s = OracleSolver(cs)
    W0 = steady_W(cs, s.S)
    s.set_fields(W=W0)
    s.step(3)
    assert np.max(np.abs(s.W - W0)) < 1e-14
    assert np.max(np.abs(s.v)) == 0.0 and np.max(np.abs(s.eta)) == 0.0
