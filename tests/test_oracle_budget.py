"""Pins of the energy-budget diagnostics of the oracle: the compact radial
derivative, the dissipation eps = nu <2 S:S> and the wall power P_in.

  * radial_D is exact on polynomials of degree <= 4 (every row of the
    compact scheme and the wall stencils are), and fourth-order on a smooth
    non-polynomial profile;
  * circular Couette flow W = A r + B/r: 2 S:S = (W' - W/r)^2 = 4 B^2/r^4, so
    eps = P_in = 2 nu B^2 (1/R_i^2 - 1/R_o^2) / ((R_o^2 - R_i^2)/2) in closed
    form (the wall power balances the dissipation in the steady state);
  * for a solenoidal field with no-slip walls, int 2 S:S = int |omega|^2 +
    2 (W_i^2 - W_o^2) per unit box area: the strain form and an independent
    vorticity form must agree to truncation order (a wrong sign or factor in
    any strain component leaves an O(1) gap);
  * along a non-linear run, E(T) - E(0) = int_0^T (P_in - eps) dt to the
    accuracy of the discretisation, improving with Nr.
"""
import numpy as np
import pytest

from oracle.grid import Case
from oracle.stencils import build_stencils
from oracle.rk import OracleSolver
from oracle import diagnostics as dg
from helpers import inputs


@pytest.mark.parametrize("stretch", [0.0, 1.5])
def test_radial_D_exact_on_quartics(stretch):
    c = Case(33, 8, 8, 0.5, 100.0, 0.0, 1e-3, stretch=stretch)
    S = build_stencils(c.r)
    for p in range(5):
        f = c.r ** p
        exact = p * c.r ** (p - 1) if p else np.zeros_like(c.r)
        assert np.abs(dg.radial_D(S, f) - exact).max() <= 1e-11 * max(1.0, np.abs(f).max())


def test_radial_D_fourth_order():
    errs = []
    for Nr in (33, 65, 129):
        c = Case(Nr, 8, 8, 0.5, 100.0, 0.0, 1e-3)
        S = build_stencils(c.r)
        errs.append(np.abs(dg.radial_D(S, np.sin(2.0 * c.r)) - 2.0 * np.cos(2.0 * c.r)).max())
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert order.min() > 3.5, (errs, order)


def _couette(Nr, zeta=0.5, Re_o=-30.0):
    c = Case(Nr, 8, 8, zeta, 100.0, Re_o, 1e-3)
    s = OracleSolver(c)
    Ri, Ro, Wo = c.Ri, c.Ro, c.W_outer
    A = (Wo * Ro - Ri) / (Ro * Ro - Ri * Ri)
    B = Ri - A * Ri * Ri
    exact = 2.0 * c.nu * B * B * (1.0 / Ri ** 2 - 1.0 / Ro ** 2) / (0.5 * (Ro * Ro - Ri * Ri))
    return c, s, exact


def test_laminar_dissipation_equals_wall_power():
    errs = []
    for Nr in (33, 65):
        c, s, exact = _couette(Nr)
        u, v, w = s.velocity()
        eps = dg.dissipation(c, s.S, u, v, w)
        P = dg.wall_power(c, s.S, s.W)
        assert abs(eps / exact - 1.0) < 1e-5 and abs(P / exact - 1.0) < 2e-5
        errs.append(max(abs(eps / exact - 1.0), abs(P / exact - 1.0)))
    assert errs[0] / errs[1] > 10.0          # fourth order: 16x per halving of h


def test_strain_form_matches_vorticity_form():
    gaps = []
    for Nr in (17, 33, 65):
        c = Case(Nr, 16, 16, 0.7, 200.0, 0.0, 1e-3)
        s = OracleSolver(c)
        v0, e0 = inputs(Nr, 16, 16, 0.7, 11, "box", 5e-2, jmax=3, nmax=3)
        s.set_fields(v=v0, eta=e0)
        u, v, w = s.velocity()
        strain = dg._volume_mean(c, dg.strain_density(c, s.S, u, v, w))
        vort = dg._volume_mean(c, dg.enstrophy_density(c, s.S, u, v, w))
        wall = 2.0 * (s.W[0] ** 2 - s.W[-1] ** 2) / (0.5 * (c.Ro ** 2 - c.Ri ** 2))
        gaps.append(abs(strain - (vort + wall)) / strain)
    assert gaps[-1] < 2e-5
    assert gaps[0] / gaps[1] > 8.0 and gaps[1] / gaps[2] > 8.0, gaps


def _budget(Nr, dt=1e-3, nsteps=50):
    c = Case(Nr, 16, 16, 0.7, 200.0, 0.0, dt)
    s = OracleSolver(c)
    v0, e0 = inputs(Nr, 16, 16, 0.7, 11, "box", 5e-2, jmax=3, nmax=3)
    s.set_fields(v=v0, eta=e0)
    E, F = [], []
    for n in range(nsteps + 1):
        u, v, w = s.velocity()
        E.append(dg.kinetic_energy(c, u, v, w))
        F.append(dg.wall_power(c, s.S, s.W) - dg.dissipation(c, s.S, u, v, w))
        if n < nsteps:
            s.step(1)
    F = np.array(F)
    integral = dt * (0.5 * F[0] + F[1:-1].sum() + 0.5 * F[-1])
    return (E[-1] - E[0] - integral) / (np.abs(F).sum() * dt)


def test_energy_budget_along_a_run():
    g33, g65 = abs(_budget(33)), abs(_budget(65))
    assert g65 < 1e-3
    assert g33 / g65 > 4.0, (g33, g65)
