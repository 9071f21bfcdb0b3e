"""Fourier expansion in theta and z, and the pseudo-spectral products.

Paper: the homogeneous directions are expanded in Fourier series (Sec. 2.1,
Appendix) and the non-linear terms are those of the primitive-variable
equations (Appendix, below Eq. 3).  The paper does not say how the products
are formed; the reading used here is the usual pseudo-spectral one with the
3/2 rule: transform the three velocity components to a grid of
Mt = 3 Ntheta/2 by Mz = 3 Nz/2 points, multiply, transform back and keep the
retained modes.  With both Nyquist modes dropped this is free of aliasing for
quadratic products.

Transform convention:
    u(theta_p, z_q) = sum_{j, n} u_hat[j, n] exp(i (m_j theta_p + alpha_n z_q))
over the full (Hermitian) spectrum, theta_p = p Theta/Mt, z_q = q Lz/Mz; the
forward transform carries the factor 1/(Mt Mz).  numpy's FFT is used as the
library primitive for both sums; direct_* below are the same sums written
out, used only to pin the FFT route on tiny grids.
"""
import numpy as np


def _slot_positions(case):
    """Retained axial FFT slots (Nyquist excluded) and their rows in the
    padded Mz-point grid."""
    n = np.fft.fftfreq(case.Nz, d=1.0 / case.Nz).astype(np.int64)
    slots = np.array([s for s in range(case.Nz) if s != case.Nz // 2], dtype=np.int64)
    return slots, np.mod(n[slots], case.Mz)


def to_physical(case, F):
    """Spectral (Nr, Nz, Nh) -> physical (Nr, Mz, Mt) on the 3/2 grid."""
    slots, pos = _slot_positions(case)
    pad = np.zeros((F.shape[0], case.Mz, case.Mt // 2 + 1), dtype=np.complex128)
    pad[:, pos, :case.Nh] = F[:, slots, :]
    return np.fft.irfft2(pad, s=(case.Mz, case.Mt), axes=(1, 2)) * (case.Mz * case.Mt)


def to_spectral(case, P):
    """Physical (Nr, Mz, Mt) -> spectral (Nr, Nz, Nh), truncated; Nyquist slot 0."""
    slots, pos = _slot_positions(case)
    S = np.fft.rfft2(P, axes=(1, 2)) / (case.Mz * case.Mt)
    F = np.zeros((P.shape[0], case.Nz, case.Nh), dtype=np.complex128)
    F[:, slots, :] = S[:, pos, :case.Nh]
    return F


PRODUCTS = ("uu", "uv", "uw", "vv", "vw", "ww")


def products(case, u, v, w):
    """The six quadratic products of the velocity, returned in spectral space
    as a dict name -> (Nr, Nz, Nh)."""
    pu, pv, pw = to_physical(case, u), to_physical(case, v), to_physical(case, w)
    phys = {"uu": pu * pu, "uv": pu * pv, "uw": pu * pw,
            "vv": pv * pv, "vw": pv * pw, "ww": pw * pw}
    return {k: to_spectral(case, phys[k]) for k in PRODUCTS}


# ---- the same sums written out (pins only; O(N^4)) -------------------------

def full_spectrum(case, F):
    """Dict (j, n) -> coefficient over the full Hermitian spectrum of one
    radial plane F (Nz, Nh)."""
    n_of = np.fft.fftfreq(case.Nz, d=1.0 / case.Nz).astype(int)
    out = {}
    for s in range(case.Nz):
        if s == case.Nz // 2:
            continue
        for j in range(case.Nh):
            c = complex(F[s, j])
            out[(j, int(n_of[s]))] = c
            if j > 0:
                out[(-j, -int(n_of[s]))] = c.conjugate()
    return out


def direct_to_physical(case, F):
    """Direct double sum for one plane F (Nz, Nh) -> (Mz, Mt)."""
    spec = full_spectrum(case, F)
    out = np.zeros((case.Mz, case.Mt))
    for q in range(case.Mz):
        for p in range(case.Mt):
            s = 0j
            for (j, n), c in spec.items():
                s += c * np.exp(2j * np.pi * (j * p / case.Mt + n * q / case.Mz))
            out[q, p] = s.real
    return out


def direct_to_spectral(case, P):
    """Direct double sum for one plane P (Mz, Mt) -> (Nz, Nh)."""
    n_of = np.fft.fftfreq(case.Nz, d=1.0 / case.Nz).astype(int)
    out = np.zeros((case.Nz, case.Nh), dtype=np.complex128)
    qq, pp = np.meshgrid(np.arange(case.Mz), np.arange(case.Mt), indexing="ij")
    for s in range(case.Nz):
        if s == case.Nz // 2:
            continue
        for j in range(case.Nh):
            ph = np.exp(-2j * np.pi * (j * pp / case.Mt + n_of[s] * qq / case.Mz))
            out[s, j] = np.sum(P * ph) / (case.Mt * case.Mz)
    return out
