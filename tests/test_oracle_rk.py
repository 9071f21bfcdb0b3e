"""Pins of the 3-substep IMEX Runge-Kutta scheme (Sec. 2.1, Sec. 3.1):
order conditions in exact arithmetic and the measured temporal order of the
oracle's own stepper."""
from fractions import Fraction
import math

import numpy as np

from oracle.rk import SMR91, OracleSolver
from oracle.grid import Case
from paper_0711_1429_gb300.synthetic import initial_perturbation


def _polymul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _polyadd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def test_explicit_part_is_third_order():
    """y' = lambda y through the explicit recurrence
    y_k = y_(k-1) + z (gamma_k y_(k-1) + zeta_k y_(k-2)) gives exactly
    1 + z + z^2/2 + z^3/6 (the amplification of any 3-stage third-order RK)."""
    g, zt = SMR91.gamma, SMR91.zeta
    y = [[Fraction(1)], [Fraction(1)]]            # y_(-1) (unused), y_0
    for k in range(3):
        prev, prev2 = y[-1], y[-2]
        new = _polyadd(prev, _polyadd(_polymul([0, g[k]], prev), _polymul([0, zt[k]], prev2)))
        y.append(new)
    amp = y[-1] + [Fraction(0)] * 4
    assert amp[:4] == [Fraction(1), Fraction(1), Fraction(1, 2), Fraction(1, 6)]


def test_coefficient_sums_and_crank_nicolson():
    a, b, g, z = SMR91.alpha, SMR91.beta, SMR91.gamma, SMR91.zeta
    assert sum(a) + sum(b) == 1 and sum(g) + sum(z) == 1
    for k in range(3):
        assert a[k] == b[k] == (g[k] + z[k]) / 2


def test_imex_scheme_second_order_in_time():
    """The oracle's full step on a small nonlinear case converges at second
    order in dt (Crank-Nicolson limits the IMEX scheme to order 2).  The
    initial state is first taken through one short step so that it satisfies
    the discrete boundary rows (otherwise the first solve projects it, a
    dt-independent jump)."""
    cs0 = Case(17, 8, 8, 0.7, 300.0, 0.0, 1e-4)
    s0 = OracleSolver(cs0)
    v, e = initial_perturbation(17, 8, 8, 7, "box", 0.05, jmax=3, nmax=3)
    s0.set_fields(v=v, eta=e)
    s0.step(1)
    x0 = (s0.v.copy(), s0.eta.copy(), s0.W.copy())

    def run(dt, T=0.08):
        cs = Case(17, 8, 8, 0.7, 300.0, 0.0, dt)
        s = OracleSolver(cs, stencils=s0.S)
        s.set_fields(v=x0[0], eta=x0[1], W=x0[2])
        s.step(int(round(T / dt)))
        return np.concatenate([s.v.ravel(), s.eta.ravel(), s.W, s.U])
    ref = run(0.08 / 256)
    errs = [np.linalg.norm(run(0.08 / n) - ref) for n in (4, 8, 16)]
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.8, (errs, orders)
