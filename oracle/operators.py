"""Radial rows of the discretised v and eta equations (Eqs. 6-7), the mean
flow, the boundary conditions and the velocity reconstruction.

Notation (Appendix): D f = df/dr, D_* f = df/dr + f/r, k^2 = alpha^2 + m^2/r^2,
c = 1/k^2 with analytic r-derivatives c1 = Dc, c2 = DDc, c3 = DDDc.  The
viscous coefficient is nu = 2/Re (lengths in h, Re built on the gap 2h).

A chain operator X applied to (coefficient * field) becomes, on row j, the
stencil l_X applied to the pointwise product on the 5 stencil points, with
d0 for the identity chain (see stencils.py).  The chain D D (twice D), which
Eq. 6 also uses, is rewritten D D g = D D_* g - D(g/r).

Readings of Eq. 6 where the printed text is garbled (each checked by
re-deriving Eq. 6 from Eq. 4, and Eq. 4 from the primitive cylindrical
equations, see tests/test_oracle_rows.py):
  * "D_1(1/k^2)" is D(1/k^2);
  * "D[(1/r) D D(1/k^2) v]" is D[(c2/r) v];
  * hat-u^2, hat-v^2, hat-w^2 are the products uu, vv, ww.

Implicit / explicit split (Appendix and Sec. 2.1): the terms in v of Eq. 6
and in eta of Eq. 7 multiplied by 1/Re are implicit; the curvature terms in
u and w, the continuity term -3 D D_*[c1 (i alpha u + i m/r w)], the
coupling 2 m alpha/r^2 v of Eq. 7 and all non-linear terms are explicit.

Row ranges: v rows 2..Nr-3 (rows 0, 1, Nr-2, Nr-1 hold v = 0 and Dv = 0 at
the walls); eta rows 1..Nr-2 (rows 0, Nr-1 hold eta = 0); mean flow rows
1..Nr-2 with Dirichlet rows 0, Nr-1.
"""
import numpy as np
from scipy.linalg import solve_banded


# ---- wavenumber-dependent coefficients ------------------------------------

def coefficients(r, m, alpha):
    """k^2, c = 1/k^2 and its first three r-derivatives.

    With g = alpha^2 r^2 + m^2:  c = r^2/g,  c1 = 2 r m^2 / g^2,
    c2 = 2 m^2 (m^2 - 3 alpha^2 r^2) / g^3,
    c3 = -24 m^2 alpha^2 r (m^2 - alpha^2 r^2) / g^4.
    Broadcasts r (Nr,1,1) against m, alpha.
    """
    k2 = alpha ** 2 + m ** 2 / r ** 2
    c = 1.0 / k2
    g = alpha ** 2 * r ** 2 + m ** 2
    c1 = 2.0 * r * m ** 2 / g ** 2
    c2 = 2.0 * m ** 2 * (m ** 2 - 3.0 * alpha ** 2 * r ** 2) / g ** 3
    c3 = -24.0 * m ** 2 * alpha ** 2 * r * (m ** 2 - alpha ** 2 * r ** 2) / g ** 4
    return k2, c, c1, c2, c3


# ---- band operators ---------------------------------------------------------

def band(S, terms, shape):
    """Band matrix of sum_t l_t . (coef_t * x): entry [j, s] multiplies
    x[start[j] + s].  terms = [(stencil weights (Nr,5), coef or scalar)]."""
    Nr = S.Nr
    out = np.zeros((Nr, 5) + shape, dtype=np.complex128 if any(
        np.iscomplexobj(c) for _, c in terms) else np.float64)
    idx = S.start[:, None] + np.arange(5)[None, :]
    for w, coef in terms:
        ww = w.reshape((Nr, 5) + (1,) * len(shape))
        if np.isscalar(coef):
            out = out + ww * coef
        else:
            cf = np.broadcast_to(coef, (Nr,) + shape)
            out = out + ww * cf[idx]
    return out


def band_apply(S, B, x):
    """y[j] = sum_s B[j, s] x[start[j] + s]."""
    idx = S.start[:, None] + np.arange(5)[None, :]
    return np.sum(B * x[idx], axis=1)


def v_operators(S, r, m, alpha, nu, coef):
    """Mass and implicit operators of Eq. 6 as bands (rows 2..Nr-3 meaningful).

    Mass:  v - D D_*(c v) + D(c1 v).
    Implicit (times nu): 2 D D_* v - D D_* D D_*(c v) + D[(c2/r) v]
        - 2 D D_*[(c1/r) v] + D[c3 v] - D[(c1/r^2) v] - 2 m^2 D[(c/r^3) v] - k^2 v.
    """
    k2, c, c1, c2, c3 = coef
    shape = np.broadcast_shapes(np.shape(m), np.shape(alpha))[1:]
    M = band(S, [(S.d0, 1.0), (S.l2, -c), (S.l1, c1)], shape)
    L = band(S, [(S.l2, 2.0), (S.l4, -c), (S.l1, c2 / r), (S.l2, -2.0 * c1 / r),
                 (S.l1, c3), (S.l1, -c1 / r ** 2), (S.l1, -2.0 * m ** 2 * c / r ** 3),
                 (S.d0, -k2)], shape)
    return M, nu * L


def eta_operators(S, r, m, alpha, nu, coef):
    """Mass d0 and implicit nu (D D_* eta - k^2 eta) of Eq. 7 (rows 1..Nr-2)."""
    k2 = coef[0]
    shape = np.broadcast_shapes(np.shape(m), np.shape(alpha))[1:]
    M = band(S, [(S.d0, 1.0)], shape)
    L = band(S, [(S.l2, 1.0), (S.d0, -k2)], shape)
    return M, nu * L


def v_explicit(S, r, m, alpha, nu, coef, u, v, w, P):
    """Explicit part of Eq. 6 on rows 2..Nr-3: curvature-viscous terms and the
    non-linear terms, in the order the paper prints them."""
    k2, c, c1, c2, c3 = coef
    A = lambda wts, g: S.apply(wts, g)
    I = 1j
    phi = I * alpha * u + I * m / r * w
    visc = (-3.0 * A(S.l2, c1 * phi)
            + 2 * I * m * A(S.l1, c / r ** 3 * w)
            + 2 * I * m * (A(S.l2, c / r ** 2 * w) - A(S.l1, c / r ** 3 * w)
                           - A(S.l1, c1 / r ** 2 * w))
            - 2 * I * m * A(S.d0, w / r ** 2))
    uu, uv, uw, vv, vw, ww = (P[k] for k in ("uu", "uv", "uw", "vv", "vw", "ww"))
    nl = (-I * alpha * (A(S.l2, c * uv) - A(S.l1, c1 * uv))
          - I * m * (A(S.l2, c * vw / r) - A(S.l1, c * vw / r ** 2)
                     + 3.0 * A(S.l1, c * vw / r ** 2) - A(S.l1, c1 / r * vw))
          + A(S.l1, c * (alpha ** 2 * uu + 2.0 * alpha * m / r * uw + m ** 2 / r ** 2 * ww))
          - I * alpha * A(S.d0, uv) - A(S.l1, vv) - I * m * A(S.d0, vw / r)
          - A(S.d0, vv / r) + A(S.d0, ww / r))
    return nu * visc + nl


def eta_explicit(S, r, m, alpha, nu, u, v, w, P):
    """Explicit part of Eq. 7 on rows 1..Nr-2."""
    A = lambda wts, g: S.apply(wts, g)
    I = 1j
    visc = 2 * I * m * (A(S.l1, u / r ** 2) + 2.0 * A(S.d0, u / r ** 3)
                        - I * alpha * A(S.d0, v / r ** 2))
    uu, uv, uw, vv, vw, ww = (P[k] for k in ("uu", "uv", "uw", "vv", "vw", "ww"))
    nl = (-I * m * (I * alpha * A(S.d0, uu / r) + A(S.l1, uv / r)
                    + 2.0 * A(S.d0, uv / r ** 2) + I * m * A(S.d0, uw / r ** 2))
          + I * alpha * (I * alpha * A(S.d0, uw) + A(S.l1, vw)
                         + I * m * A(S.d0, ww / r) + 2.0 * A(S.d0, vw / r)))
    return nu * visc + nl


def mean_operators(S, r, nu):
    """Mean flow (m = alpha = 0), rows 1..Nr-2, zero mean pressure gradient
    in theta and z (Sec. 4).  Azimuthal W: dW/dt = nu D D_* W + [HW]_00,
    axial U: dU/dt = nu (D D_* U + U/r^2) + [HU]_00, with
    [HW]_00 = -(D(vw) + 2 vw/r), [HU]_00 = -(D(uv) + uv/r)."""
    rr = r.reshape(-1)
    MW = band(S, [(S.d0, 1.0)], ())
    LW = nu * band(S, [(S.l2, 1.0)], ())
    MU = MW
    LU = nu * band(S, [(S.l2, 1.0), (S.d0, 1.0 / rr ** 2)], ())
    return MW, LW, MU, LU


def mean_explicit(S, r, uv00, vw00):
    rr = r.reshape(-1)
    EW = -S.apply(S.l1, vw00) - 2.0 * S.apply(S.d0, vw00 / rr)
    EU = -S.apply(S.l1, uv00) - S.apply(S.d0, uv00 / rr)
    return EU, EW


# ---- banded solves ----------------------------------------------------------

def _ab_from_rows(S, B, bc_rows, bc_vals_rows, Nr):
    """LAPACK (3,3) band storage of the Nr x Nr matrix whose rows are B[j]
    (5 entries from start[j]) except the boundary rows given explicitly as
    (row, start, weights)."""
    ab = np.zeros((7,) + (Nr,) + B.shape[2:], dtype=B.dtype)
    rows = [j for j in range(Nr) if j not in bc_rows]
    for j in rows:
        for s in range(5):
            col = S.start[j] + s
            ab[3 + j - col, col] = B[j, s]
    for (j, st, wts) in bc_vals_rows:
        for s, wv in enumerate(wts):
            col = st + s
            ab[3 + j - col, col] = wv
    return ab


def solve_rows(ab, rhs):
    """Solve each pair's banded system (partial pivoting, LAPACK gbsv).
    ab (7, Nr, npairs) real, rhs (Nr, npairs) complex."""
    out = np.empty_like(rhs)
    for p in range(rhs.shape[1]):
        out[:, p] = solve_banded((3, 3), ab[:, :, p], rhs[:, p])
    return out


def v_system(S, A_band):
    """Rows of the v system: interior rows from A_band, then v_0 = 0,
    Dv(r_0) = 0 on row 1, Dv(r_{Nr-1}) = 0 on row Nr-2, v_{Nr-1} = 0."""
    Nr = S.Nr
    npairs = A_band.shape[2]
    one = np.ones(npairs)
    bc = [(0, 0, [one]), (1, 0, [w * one for w in S.dwall[0]]),
          (Nr - 2, Nr - 5, [w * one for w in S.dwall[1]]), (Nr - 1, Nr - 1, [one])]
    return _ab_from_rows(S, A_band, {0, 1, Nr - 2, Nr - 1}, bc, Nr)


def eta_system(S, A_band):
    """Rows of the eta (or mean-flow) system: rows 1..Nr-2 from A_band,
    identity rows 0 and Nr-1 (Dirichlet)."""
    Nr = S.Nr
    shape = A_band.shape[2:]
    one = np.ones(shape)
    bc = [(0, 0, [one]), (Nr - 1, Nr - 1, [one])]
    return _ab_from_rows(S, A_band, {0, Nr - 1}, bc, Nr)


# ---- velocity reconstruction ------------------------------------------------

def radial_derivative(S, v):
    """Dv on every row: 0 at the walls (Dv = 0 is a boundary condition),
    explicit one-sided rows 1 and Nr-2, and the compact rows
    d0 . Dv = l1 . v on rows 2..Nr-3.  v is (Nr, ...) complex."""
    Nr = S.Nr
    flat = v.reshape(Nr, -1)
    rhs = S.apply(S.l1, flat)
    rhs[0] = 0.0
    rhs[Nr - 1] = 0.0
    ab = np.zeros((7, Nr))
    for j in range(1, Nr - 1):
        for s in range(5):
            col = S.start[j] + s
            ab[3 + j - col, col] = S.d0[j, s]
    ab[3, 0] = 1.0
    ab[3, Nr - 1] = 1.0
    Dv = solve_banded((3, 3), ab, rhs)
    return Dv.reshape(v.shape)


def reconstruct_uw(S, r, m, alpha, k2, v, eta):
    """u and w from continuity i alpha u + (i m/r) w + D_* v = 0 and the
    definition of the radial vorticity eta = (i m/r) u - i alpha w:
        u = (i alpha D_*v - (i m/r) eta)/k^2,  w = ((i m/r) D_*v + i alpha eta)/k^2."""
    Dsv = radial_derivative(S, v) + v / r
    u = (1j * alpha * Dsv - 1j * m / r * eta) / k2
    w = (1j * m / r * Dsv + 1j * alpha * eta) / k2
    return u, w
