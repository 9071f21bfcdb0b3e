"""Pins of the oracle's radial stencils (Sec. 2.1: 5 points, order >= 4,
coefficients by polynomial matching)."""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle.grid import radial_grid
from oracle.stencils import build_stencils, op_D, op_DDs, op_DDsDDs


def test_chain_operator_expansions_match_sympy():
    """The expanded forms of D, D D_* and D D_* D D_* agree with symbolic
    differentiation of (r - rc)^q (catches a dropped term or sign)."""
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    rc = sp.Rational(31, 2)
    D = lambda f: sp.diff(f, r)
    Ds = lambda f: sp.diff(f, r) + f / r
    ops = [(op_D, D), (op_DDs, lambda f: D(Ds(f))), (op_DDsDDs, lambda f: D(Ds(D(Ds(f)))))]
    for q in range(9):
        p = (r - rc) ** q
        for x in (sp.Rational(29, 2), sp.Rational(33, 2), sp.Rational(16, 1)):
            for mine, ref in ops:
                val = mine(q, Fraction(int(x.p), int(x.q)), Fraction(31, 2))
                exact = sp.simplify(ref(p).subs(r, x))
                assert sp.simplify(sp.Rational(val.numerator, val.denominator) - exact) == 0


def _smooth(x):
    """f = sin(3x) exp(x/5) and its derivatives up to 4 (hand-written)."""
    s, c, e = np.sin(3 * x), np.cos(3 * x), np.exp(x / 5)
    a, b = 0.2, 3.0
    # derivatives of e^{a x} (sin bx): use complex form Im(e^{(a + i b) x})
    z = complex(a, b)
    d = [np.imag(z ** k * np.exp(z * x)) for k in range(5)]
    assert np.allclose(d[0], s * e)
    return d


def _ops(x, d):
    f, f1, f2, f3, f4 = d
    return {
        "l1": f1,
        "l2": f2 + f1 / x - f / x ** 2,
        "l4": f4 + 2 * f3 / x - 3 * f2 / x ** 2 + 3 * f1 / x ** 3 - 3 * f / x ** 4,
    }


@pytest.mark.parametrize("zeta", [0.5, 0.883])
def test_interior_truncation_order(zeta):
    """Residual of  l_X . f - d0 . (X f)  on interior rows decreases at least
    as h^4 for a smooth non-polynomial f (formal order >= 4)."""
    # l4 weights grow like h^-4, so its residual meets round-off sooner:
    # it is measured on coarser grids than l1, l2.
    errs = {k: [] for k in ("l1", "l2", "l4")}
    Ns = {"l1": (33, 65, 129), "l2": (33, 65, 129), "l4": (17, 33, 65)}
    for N in sorted(set(Ns["l1"]) | set(Ns["l4"])):
        r = radial_grid(zeta, N)
        S = build_stencils(r)
        d = _smooth(r)
        X = _ops(r, d)
        for k in errs:
            if N not in Ns[k]:
                continue
            w = getattr(S, k)
            res = S.apply(w, d[0]) - S.apply(S.d0, X[k])
            errs[k].append(np.max(np.abs(res[2:N - 2])))
    for k, e in errs.items():
        orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
        assert min(orders) > 3.7, (k, orders)


def test_wall_rows_and_normalisation():
    r = radial_grid(0.883, 33)
    S = build_stencils(r)
    N = len(r)
    assert np.allclose(S.d0[2:N - 2].sum(axis=1), 1.0, atol=1e-14)
    # explicit near-wall rows: d0 is the identity row
    assert S.d0[1, 1] == 1.0 and S.d0[N - 2, 3] == 1.0
    # one-sided wall derivative is exact on quartics, and 4th-order on f
    for k in range(5):
        p = (r - r[0]) ** k
        assert abs(S.dwall[0] @ p[:5] - (k == 1)) < 1e-9
    # interior d0 diagonally dominant (LU without pivoting is safe)
    ratio = min(abs(S.d0[j, 2]) / (np.abs(S.d0[j]).sum() - abs(S.d0[j, 2])) for j in range(2, N - 2))
    assert ratio > 1.5


def test_compact_derivative_order():
    """The compact first derivative used to rebuild u, w converges at order 4."""
    from oracle.operators import radial_derivative
    errs = []
    for N in (33, 65, 129):
        r = radial_grid(0.5, N)
        S = build_stencils(r)
        x = (r - r[0]) / (r[-1] - r[0])
        f = (x * (1 - x)) ** 2 * np.exp(x)        # f = f' = 0 at both walls
        fp = (2 * x * (1 - x) ** 2 - 2 * x ** 2 * (1 - x) + x ** 2 * (1 - x) ** 2) * np.exp(x) / (r[-1] - r[0])
        Df = radial_derivative(S, f.astype(np.complex128)).real
        errs.append(np.max(np.abs(Df - fp)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 3.5, orders
