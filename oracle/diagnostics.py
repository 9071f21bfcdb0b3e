"""Torque, friction Reynolds number and kinetic energy.

Torque (Eq. 2): the printed bracket is garbled; the reading used is the
wall shear of the azimuthal mean flow, |dW/dr - W/r| at the wall, which makes
the laminar value G = 4 pi/(1 - zeta^2) and reproduces Table 2's laminar rows
(16.7551 at zeta = 0.5).  Non-dimensional torque per unit axial length,
G = T / (mu W_i L R_i):
    G_i = 2 pi R_i |W' - W/r|_{R_i},   G_o = 2 pi (R_o^2 / R_i) |W' - W/r|_{R_o},
with W' from the explicit one-sided 5-point derivative at the wall.

Friction Reynolds number (Sec. 5): u_tau = sqrt(tau_w/rho) per wall,
Re_tau = u_tau delta / nu with delta = h = 1:  Re_tau = sqrt(nu |W' - W/r|)/nu.

Kinetic energy per unit volume: E = (1/2) <|u|^2>, Parseval in theta and z
(half spectrum: j = 0 counted once, j > 0 twice) and a fourth-order radial
quadrature with weight r.

Energy budget (Sec. 2 diagnostics; the paper prints none of these values):
for incompressible flow between walls that move tangentially,
dE/dt = P_in - eps per unit volume, with
  eps  = nu < 2 S:S >, the viscous dissipation, S the strain rate in
         cylindrical components (u axial, v radial, w azimuthal):
           S_rr = Dv, S_tt = (i m/r) w + v/r, S_zz = i alpha u,
           S_rt = (Dw - w/r + (i m/r) v)/2, S_rz = (i alpha v + Du)/2,
           S_tz = ((i m/r) u + i alpha w)/2,
         2 S:S = 2 (S_rr^2 + S_tt^2 + S_zz^2) + 4 (S_rt^2 + S_rz^2 + S_tz^2);
  P_in = nu [R_o W_o (W' - W/r)_(R_o) - R_i W_i (W' - W/r)_(R_i)] / V,
         the work of the wall shear stress on the moving walls, V the volume
         per unit box area (R_o^2 - R_i^2)/2; only the mean W enters since
         the fluctuations vanish on the walls.
Radial derivatives in eps use the compact first derivative `radial_D`: the
explicit one-sided 5-point D on the walls and on rows 1, Nr-2, and the
compact rows d0 . Df = l1 . f inside (the operator of continuity).
"""
import math
import numpy as np
from scipy.linalg import solve_banded


def wall_shear(S, r, W):
    dWi = float(np.dot(S.dwall[0], W[0:5]))
    dWo = float(np.dot(S.dwall[1], W[-5:]))
    return abs(dWi - W[0] / r[0]), abs(dWo - W[-1] / r[-1])


def torque(case, S, W):
    si, so = wall_shear(S, case.r, W)
    Ri, Ro = case.r[0], case.r[-1]
    Gi = 2.0 * math.pi * Ri * si
    Go = 2.0 * math.pi * Ro ** 2 / Ri * so
    return Gi, Go


def re_tau(case, S, W):
    si, so = wall_shear(S, case.r, W)
    nu = case.nu
    return math.sqrt(nu * si) / nu, math.sqrt(nu * so) / nu


def radial_weights(r, stretch=0.0):
    """Fourth-order quadrature in the grid coordinate s (uniform), trapezoid
    with end corrections 3/8, 7/6, 23/24, times the Jacobian dr/ds of the
    radial map (1 on the uniform grid)."""
    from .grid import radial_jacobian
    N = len(r)
    h = 2.0 / (N - 1) if stretch != 0.0 else (r[-1] - r[0]) / (N - 1)
    w = np.ones(N)
    w[[0, -1]] = 3.0 / 8.0
    w[[1, -2]] = 7.0 / 6.0
    w[[2, -3]] = 23.0 / 24.0
    return h * w * radial_jacobian(N, stretch)


def kinetic_energy(case, u, v, w):
    """E = (1/2) int |u|^2 r dr / int r dr, Parseval over theta and z."""
    wt = np.ones(case.Nh) * 2.0
    wt[0] = 1.0
    spec = (np.abs(u) ** 2 + np.abs(v) ** 2 + np.abs(w) ** 2) * wt[None, None, :]
    prof = spec.sum(axis=(1, 2))
    q = radial_weights(case.r, case.stretch) * case.r
    return 0.5 * float(np.dot(q, prof) / np.sum(q))


def radial_D(S, f):
    """Compact first derivative along axis 0 of f (any trailing shape):
    rows 0 and Nr-1 from the explicit one-sided wall stencils, rows 1 and
    Nr-2 explicit one-sided, rows 2..Nr-3 compact d0 . Df = l1 . f."""
    Nr = S.Nr
    flat = f.reshape(Nr, -1)
    rhs = S.apply(S.l1, flat)
    rhs[0] = S.dwall[0] @ flat[0:5]
    rhs[Nr - 1] = S.dwall[1] @ flat[Nr - 5:Nr]
    ab = np.zeros((7, Nr))
    for j in range(1, Nr - 1):
        for s in range(5):
            col = S.start[j] + s
            ab[3 + j - col, col] = S.d0[j, s]
    ab[3, 0] = 1.0
    ab[3, Nr - 1] = 1.0
    return solve_banded((3, 3), ab, rhs).reshape(f.shape)


def _volume_mean(case, prof):
    """<prof> = int prof r dr / int r dr with the fourth-order weights."""
    q = radial_weights(case.r, case.stretch) * case.r
    return float(np.dot(q, prof) / np.sum(q))


def _parseval_weights(case):
    wt = np.ones(case.Nh) * 2.0
    wt[0] = 1.0
    return wt[None, None, :]


def strain_density(case, S, u, v, w):
    """sum over modes of 2 S:S (Parseval weights) at every radial point."""
    r = case.r.reshape(-1, 1, 1)
    m = case.m_of()
    al = case.alpha_of()
    Du, Dv, Dw = radial_D(S, u), radial_D(S, v), radial_D(S, w)
    Srr = Dv
    Stt = 1j * m / r * w + v / r
    Szz = 1j * al * u
    Srt = 0.5 * (Dw - w / r + 1j * m / r * v)
    Srz = 0.5 * (1j * al * v + Du)
    Stz = 0.5 * (1j * m / r * u + 1j * al * w)
    sq = lambda a: np.abs(a) ** 2
    dens = 2.0 * (sq(Srr) + sq(Stt) + sq(Szz)) + 4.0 * (sq(Srt) + sq(Srz) + sq(Stz))
    return (dens * _parseval_weights(case)).sum(axis=(1, 2))


def dissipation(case, S, u, v, w):
    """eps = nu < 2 S:S > per unit volume (u, v, w spectral with the mean
    flow in the (0, 0) slot)."""
    return case.nu * _volume_mean(case, strain_density(case, S, u, v, w))


def enstrophy_density(case, S, u, v, w):
    """sum over modes of |omega|^2: omega_r = (i m/r) u - i alpha w (= eta),
    omega_t = i alpha v - Du, omega_z = Dw + w/r - (i m/r) v."""
    r = case.r.reshape(-1, 1, 1)
    m = case.m_of()
    al = case.alpha_of()
    Du, Dw = radial_D(S, u), radial_D(S, w)
    om_r = 1j * m / r * u - 1j * al * w
    om_t = 1j * al * v - Du
    om_z = Dw + w / r - 1j * m / r * v
    dens = np.abs(om_r) ** 2 + np.abs(om_t) ** 2 + np.abs(om_z) ** 2
    return (dens * _parseval_weights(case)).sum(axis=(1, 2))


def wall_power(case, S, W):
    """P_in per unit volume from the mean azimuthal velocity W(r)."""
    r = case.r
    dWi = float(np.dot(S.dwall[0], W[0:5]))
    dWo = float(np.dot(S.dwall[1], W[-5:]))
    Ri, Ro = r[0], r[-1]
    ti = dWi - W[0] / Ri
    to = dWo - W[-1] / Ro
    vol = 0.5 * (Ro * Ro - Ri * Ri)
    return case.nu * (Ro * W[-1] * to - Ri * W[0] * ti) / vol
