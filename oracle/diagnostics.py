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
"""
import math
import numpy as np


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
