"""Five-point compact explicit radial stencils (Sec. 2.1 and Appendix).

The paper fixes: 5 arbitrarily spaced points, formal order at least 4,
coefficients found by matching the discrete derivative of a polynomial to its
analytical derivative; compact yet explicit because the equations contain no
third derivative (Thomas' procedure).  Written as one row of the discretised
equations, every term becomes

    sum_s  l_X[j, s] * g(r_{start_j + s})  ~=  sum_s d0[j, s] * (X g)(r_{start_j + s})

for the chain operators X in {I, D, D D_*, D D_* D D_*} (D g = g',
D_* g = g' + g/r), with one common averaging stencil d0 per row.

Reading used here (the paper gives only the principle):
  * interior rows 2..Nr-3, points j-2..j+2: d0 and l4 (for D D_* D D_*)
    together make DD*DD* exact on every polynomial of degree <= 8, with the
    normalisation sum(d0) = 1 (10 conditions, 10 unknowns); l2 (D D_*) and
    l1 (D) are then exact on degree <= 4 against the same d0;
  * near-wall rows 1 and Nr-2: explicit rows (d0 = delta) with one-sided
    l1, l2 on points 0..4 (resp. Nr-5..Nr-1), exact on degree <= 4;
  * wall rows 0 and Nr-1: explicit one-sided first derivative at the wall on
    the same 5 points (Neumann condition Dv = 0, wall shear for the torque).

All coefficients are found in exact rational arithmetic from the float64
grid values (each float is an exact rational), then rounded once to float64.
"""
from dataclasses import dataclass
from fractions import Fraction
from math import factorial
import numpy as np


# ---- chain operators applied to the monomial (r - rc)^q, evaluated at x -----

def _dk(q, k, x, rc):
    """k-th derivative of (r - rc)^q at r = x (exact)."""
    if k > q:
        return Fraction(0)
    return Fraction(factorial(q), factorial(q - k)) * (x - rc) ** (q - k)


def op_D(q, x, rc):
    """D f = f'."""
    return _dk(q, 1, x, rc)


def op_DDs(q, x, rc):
    """D D_* f = f'' + f'/r - f/r^2   (D_* f = f' + f/r)."""
    return _dk(q, 2, x, rc) + _dk(q, 1, x, rc) / x - _dk(q, 0, x, rc) / (x * x)


def op_DDsDDs(q, x, rc):
    """D D_* D D_* f = f'''' + 2 f'''/r - 3 f''/r^2 + 3 f'/r^3 - 3 f/r^4."""
    return (_dk(q, 4, x, rc) + 2 * _dk(q, 3, x, rc) / x - 3 * _dk(q, 2, x, rc) / x ** 2
            + 3 * _dk(q, 1, x, rc) / x ** 3 - 3 * _dk(q, 0, x, rc) / x ** 4)


def op_I(q, x, rc):
    return _dk(q, 0, x, rc)


def _solve_exact(A, b):
    """Gaussian elimination with row exchanges on Fractions (exact)."""
    n = len(b)
    A = [row[:] for row in A]
    b = b[:]
    for col in range(n):
        piv = next(i for i in range(col, n) if A[i][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for i in range(col + 1, n):
            f = A[i][col] / A[col][col]
            if f != 0:
                for k in range(col, n):
                    A[i][k] -= f * A[col][k]
                b[i] -= f * b[col]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        s = b[i] - sum(A[i][k] * x[k] for k in range(i + 1, n))
        x[i] = s / A[i][i]
    return x


def compact_row(pts, rc):
    """Interior row: d0 and l4 with D D_* D D_* exact to degree 8, sum(d0)=1;
    then l2 and l1 exact to degree 4 against that d0."""
    A, b = [], []
    for q in range(9):
        # sum_s l4_s p_q(x_s) - sum_s d0_s (L4 p_q)(x_s) = 0
        A.append([-op_DDsDDs(q, x, rc) for x in pts] + [op_I(q, x, rc) for x in pts])
        b.append(Fraction(0))
    A.append([Fraction(1)] * 5 + [Fraction(0)] * 5)
    b.append(Fraction(1))
    sol = _solve_exact(A, b)
    d0, l4 = sol[:5], sol[5:]

    def follow(op):
        M = [[op_I(q, x, rc) for x in pts] for q in range(5)]
        rhs = [sum(d0[s] * op(q, pts[s], rc) for s in range(5)) for q in range(5)]
        return _solve_exact(M, rhs)

    return d0, follow(op_D), follow(op_DDs), l4


def explicit_row(pts, xe, op):
    """One-sided explicit stencil: sum_s w_s p(x_s) = (op p)(xe), degree <= 4."""
    M = [[op_I(q, x, xe) for x in pts] for q in range(5)]
    rhs = [op(q, xe, xe) for q in range(5)]
    return _solve_exact(M, rhs)


@dataclass
class Stencils:
    """Per-row stencils.  Row j reads points start[j] .. start[j]+4.
    d0/l1/l2/l4 rows 0 and Nr-1 are zero (boundary rows are built apart);
    l4 is zero on rows 1 and Nr-2.  dwall[0] is D at r_0 on points 0..4,
    dwall[1] is D at r_{Nr-1} on points Nr-5..Nr-1."""
    start: np.ndarray
    d0: np.ndarray
    l1: np.ndarray
    l2: np.ndarray
    l4: np.ndarray
    dwall: np.ndarray

    @property
    def Nr(self):
        return len(self.start)

    def apply(self, w, g):
        """out[j] = sum_s w[j, s] g[start[j] + s] along axis 0 of g."""
        idx = self.start[:, None] + np.arange(5)[None, :]
        ww = w.reshape(w.shape + (1,) * (g.ndim - 1))
        return np.sum(ww * g[idx], axis=1)


def build_stencils(r):
    """Stencil tables for the float64 grid r (length Nr >= 9)."""
    Nr = len(r)
    R = [Fraction(float(x)) for x in r]
    start = np.zeros(Nr, dtype=np.int64)
    d0 = np.zeros((Nr, 5)); l1 = np.zeros((Nr, 5)); l2 = np.zeros((Nr, 5)); l4 = np.zeros((Nr, 5))
    for j in range(2, Nr - 2):
        st = j - 2
        start[j] = st
        a, b1, b2, b4 = compact_row(R[st:st + 5], R[j])
        d0[j] = [float(x) for x in a]
        l1[j] = [float(x) for x in b1]
        l2[j] = [float(x) for x in b2]
        l4[j] = [float(x) for x in b4]
    for j, st in ((1, 0), (Nr - 2, Nr - 5)):
        start[j] = st
        d0[j] = 0.0
        d0[j, j - st] = 1.0
        l1[j] = [float(x) for x in explicit_row(R[st:st + 5], R[j], op_D)]
        l2[j] = [float(x) for x in explicit_row(R[st:st + 5], R[j], op_DDs)]
    start[Nr - 1] = Nr - 5
    dwall = np.array([[float(x) for x in explicit_row(R[0:5], R[0], op_D)],
                      [float(x) for x in explicit_row(R[Nr - 5:Nr], R[Nr - 1], op_D)]])
    return Stencils(start, d0, l1, l2, l4, dwall)
