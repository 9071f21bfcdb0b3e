"""Geometry, radial grid and Fourier mode sets of one Taylor-Couette case.

Paper references (Pirro & Quadrio):
  * Sec. 2: zeta = R_i/R_o, gap R_o - R_i = 2h, Re built on W_i = Omega_i R_i,
    the gap 2h and nu; lengths are made non-dimensional with h, velocities
    with W_i.  With lengths in h the viscous coefficient is therefore
    nu = 2/Re (the equations of the Appendix write it 1/Re).
  * Sec. 4: box of the turbulent run, L_z = 5h and L_theta = 10 pi h at the
    centreline of the gap; this is the default box here.
  * Appendix: Fourier expansion in theta and z with wavenumbers m (azimuthal)
    and alpha (axial); k^2 = alpha^2 + m^2/r^2.

Mode layout (the convention of the library's C header as well): azimuthal index
j = 0..Ntheta/2-1 with m_j = j*m0 (the half spectrum; the theta Nyquist is
dropped), axial slots in FFT order n = 0..Nz/2-1, [Nz/2 = Nyquist, always 0],
-Nz/2+1..-1 with alpha_n = n*alpha0.  Spectral arrays are shaped
(Nr, Nz, Ntheta/2), complex128.
"""
from dataclasses import dataclass, field
import math
import numpy as np


def radial_grid(zeta, Nr, stretch=0.0):
    """Radial grid from R_i to R_i + 2 (units of h).

    R_i = 2 zeta / (1 - zeta) follows from zeta = R_i/R_o and R_o - R_i = 2.
    Uniform (stretch = 0): r_j = R_i + (2 j)/(Nr - 1).  The paper uses a
    smoothly stretched grid (Sec. 2.1; Table 4 gives a finer spacing at the
    walls than at the centre) without giving the map; the reading used here
    is the tanh map r_j = (R_i + 1) + tanh(a s_j)/tanh(a) with
    s_j = -1 + (2 j)/(Nr - 1), a = stretch > 0 (denser at both walls).
    """
    Ri = 2.0 * zeta / (1.0 - zeta)
    j = np.arange(Nr, dtype=np.float64)
    if stretch == 0.0:
        return Ri + (2.0 * j) / float(Nr - 1)
    s = -1.0 + (2.0 * j) / float(Nr - 1)
    return (Ri + 1.0) + np.tanh(stretch * s) / np.tanh(stretch)


def radial_jacobian(Nr, stretch=0.0):
    """dr/ds at the grid points of the map above (1 for the uniform grid)."""
    if stretch == 0.0:
        return np.ones(Nr)
    s = -1.0 + (2.0 * np.arange(Nr)) / float(Nr - 1)
    return stretch * (1.0 - np.tanh(stretch * s) ** 2) / np.tanh(stretch)


@dataclass
class Case:
    """Parameters of one case: the arguments of tc_create plus the box."""
    Nr: int
    Ntheta: int
    Nz: int
    zeta: float
    Re_i: float
    Re_o: float
    dt: float
    Theta: float = None      # azimuthal extent of the box (radians)
    Lz: float = 5.0          # axial extent of the box (units of h)
    stretch: float = 0.0     # tanh stretching of the radial grid (0: uniform)
    r: np.ndarray = field(init=False, repr=False)

    def __post_init__(self):
        if self.Nr < 9:
            raise ValueError("Nr must be >= 9")
        for nm in ("Ntheta", "Nz"):
            N = getattr(self, nm)
            if N < 4 or N % 2:
                raise ValueError(f"{nm} must be even and >= 4")
        if not (0.0 < self.zeta < 1.0):
            raise ValueError("radius ratio must lie in (0, 1)")
        if self.dt <= 0:
            raise ValueError("dt must be positive")
        self.Ri = 2.0 * self.zeta / (1.0 - self.zeta)
        self.Ro = self.Ri + 2.0
        self.rc = self.Ri + 1.0
        if self.Theta is None:
            # L_theta = 10 pi h measured at the centreline (Sec. 4)
            self.Theta = 10.0 * math.pi / self.rc
        self.m0 = 2.0 * math.pi / self.Theta
        self.alpha0 = 2.0 * math.pi / self.Lz
        self.nu = 2.0 / self.Re_i
        self.W_outer = self.Re_o / self.Re_i
        self.r = radial_grid(self.zeta, self.Nr, self.stretch)
        self.Nh = self.Ntheta // 2
        self.Mt = 3 * self.Ntheta // 2
        self.Mz = 3 * self.Nz // 2

    # ---- Fourier mode sets -------------------------------------------------
    def n_index(self):
        """Signed axial index n of each FFT slot; the Nyquist slot gets 0."""
        n = np.fft.fftfreq(self.Nz, d=1.0 / self.Nz).astype(np.int64)
        n[self.Nz // 2] = 0
        return n

    def m_of(self):
        """m_j = j*m0, shaped (1, 1, Nh) for broadcasting against (Nr, Nz, Nh)."""
        return (np.arange(self.Nh) * self.m0).reshape(1, 1, self.Nh)

    def alpha_of(self):
        """alpha_n = n*alpha0, shaped (1, Nz, 1)."""
        return (self.n_index() * self.alpha0).astype(np.float64).reshape(1, self.Nz, 1)

    def active_mask(self):
        """Pairs whose v and eta are evolved: every (j, n) except (0, 0), the
        axial Nyquist slot, and the m = 0 pairs with n < 0 (those hold the
        complex conjugates of n > 0, so that the field is real)."""
        mask = np.ones((self.Nz, self.Nh), dtype=bool)
        mask[self.Nz // 2, :] = False
        mask[0, 0] = False
        n = np.fft.fftfreq(self.Nz, d=1.0 / self.Nz)
        mask[(n < 0), 0] = False
        return mask

    @property
    def gridpoints(self):
        """Grid points of one field, Nr * Ntheta * Nz (the unit of the
        grid-point RK-steps/s metric)."""
        return self.Nr * self.Ntheta * self.Nz
