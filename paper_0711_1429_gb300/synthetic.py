"""Seeded synthetic initial conditions (input recipe only, no method arithmetic).

Both the CUDA path (through tc_set_field) and the CPU oracle receive the same
arrays from here.  The recipe follows the paper's procedure (Sec. 4.1): the
laminar profile plus random-phase disturbances on a set of Fourier modes; the
shapes vanish with their radial derivative at the walls so that the
boundary conditions v = Dv = eta = 0 hold.

Per Fourier pair (j, n), with x = -1 + 2 i/(Nr - 1) in [-1, 1]:
    v_hat(x)   = a_jn  [xi_1 (1 - x^2)^2 + xi_2 x (1 - x^2)^2]
    eta_hat(x) = b_jn  [xi_3 (1 - x^2)   + xi_4 x (1 - x^2)]
with xi complex standard normals.  Random numbers: splitmix64 (Steele, Lea &
Flood 2014) on the counter seed + (i + 1) * 0x9E3779B97F4A7C15, uniform
u = ((z >> 11) + 1) * 2^-53 in (0, 1], two uniforms per complex normal by
Box-Muller (re = s cos(2 pi u2), im = s sin(2 pi u2), s = sqrt(-2 ln u1)).
Draw order: field (v then eta), azimuthal index j ascending, axial index n
ascending from -Nz/2+1 to Nz/2-1, then the shape index.

Spectra:
  * "box": a = b = amp on j <= jmax and |n| <= nmax, zero elsewhere;
  * "k2":  a = amp * k_h^(-3/2), b = a * k_h with k_h = sqrt((m/r_c)^2 +
    alpha^2), on every retained pair; then one common factor scales v so its
    r.m.s. over the gap is `amp` (shell energy ~ k^-2).
The m = 0 column is made Hermitian (slot -n = conj(slot n)); (0, 0) and the
axial Nyquist slot are zero.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count):
    """Outputs 0..count-1 of splitmix64 started at `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniforms(seed, count):
    z = splitmix64(seed, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def complex_normals(seed, count):
    u = uniforms(seed, 2 * count).reshape(count, 2)
    s = np.sqrt(-2.0 * np.log(u[:, 0]))
    return s * np.cos(2.0 * np.pi * u[:, 1]) + 1j * s * np.sin(2.0 * np.pi * u[:, 1])


def initial_perturbation(Nr, Ntheta, Nz, seed, spectrum="box", amp=1e-3,
                         jmax=4, nmax=4, m0=1.0, alpha0=1.0, rc=1.0):
    """Returns (v_hat, eta_hat), complex128 arrays (Nr, Nz, Ntheta/2) in the
    library's spectral layout (axial slots in FFT order)."""
    Nh = Ntheta // 2
    nvals = np.arange(-Nz // 2 + 1, Nz // 2)           # ascending signed n
    nmodes = Nh * len(nvals)
    xi = complex_normals(seed, 2 * nmodes * 2).reshape(2, Nh, len(nvals), 2)
    x = -1.0 + 2.0 * np.arange(Nr) / (Nr - 1)
    bump = 1.0 - x * x
    shapes_v = np.stack([bump ** 2, x * bump ** 2])     # (2, Nr)
    shapes_e = np.stack([bump, x * bump])
    jj = np.arange(Nh).reshape(Nh, 1)
    nn = nvals.reshape(1, -1)
    if spectrum == "box":
        a = np.where((jj <= jmax) & (np.abs(nn) <= nmax), amp, 0.0)
        b = a
    elif spectrum == "k2":
        kh = np.sqrt((jj * m0 / rc) ** 2 + (nn * alpha0) ** 2)
        zero = kh == 0
        kh[zero] = 1.0
        a = np.where(zero, 0.0, kh ** -1.5)
        b = a * kh
    else:
        raise ValueError(spectrum)
    a = np.broadcast_to(a, (Nh, len(nvals))).copy()
    b = np.broadcast_to(b, (Nh, len(nvals))).copy()
    a[0, nvals <= 0] = 0.0
    b[0, nvals <= 0] = 0.0
    # (Nr, Nh, nmodes_n)
    v = np.einsum("jn,jnp,pr->rjn", a, xi[0], shapes_v)
    e = np.einsum("jn,jnp,pr->rjn", b, xi[1], shapes_e)
    slot = np.mod(nvals, Nz)
    V = np.zeros((Nr, Nz, Nh), dtype=np.complex128)
    Eta = np.zeros_like(V)
    V[:, slot, :] = np.transpose(v, (0, 2, 1))
    Eta[:, slot, :] = np.transpose(e, (0, 2, 1))
    for F in (V, Eta):
        for n in range(1, Nz // 2):
            F[:, Nz - n, 0] = np.conj(F[:, n, 0])
    if spectrum == "k2":
        wt = np.full(Nh, 2.0)
        wt[0] = 1.0
        rms = np.sqrt(np.mean(np.sum(np.abs(V) ** 2 * wt, axis=(1, 2))))
        s = amp / rms
        V *= s
        Eta *= s
    return V, Eta


# Named workloads: grid, physics and initial-condition recipe.
WORKLOADS = {
    "tc-small-33x16x16": dict(Nr=33, Ntheta=16, Nz=16, zeta=0.883, Re_i=200.0, Re_o=0.0,
                              dt=1e-3, seed=1, spectrum="box", amp=1e-3, steps=20),
    "tc-129x128x128": dict(Nr=129, Ntheta=128, Nz=128, zeta=0.883, Re_i=3000.0, Re_o=0.0,
                           dt=1e-3, seed=2, spectrum="k2", amp=0.05, steps=100),
    "tc-257x512x512": dict(Nr=257, Ntheta=512, Nz=512, zeta=0.883, Re_i=3000.0, Re_o=0.0,
                           dt=1e-3, seed=3, spectrum="k2", amp=0.05, steps=500),
    # the paper's turbulent run (Sec. 4, Table 4): zeta 0.882, Re 10500,
    # Nr 129, 512 x 170 modes, dt 0.012, disturbances O(1e-4) on all modes
    "paper-129x512x170": dict(Nr=129, Ntheta=512, Nz=170, zeta=0.882, Re_i=10500.0, Re_o=0.0,
                              dt=0.012, seed=4, spectrum="k2", amp=1e-4, steps=100),
}


def box_defaults(zeta, Lz=5.0):
    """Default box of the library: L_z = 5 h and L_theta = 10 pi h at the
    centreline; returns (m0, alpha0, rc)."""
    Ri = 2.0 * zeta / (1.0 - zeta)
    rc = Ri + 1.0
    return rc / 5.0, 2.0 * np.pi / Lz, rc
