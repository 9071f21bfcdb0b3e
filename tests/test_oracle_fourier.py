"""Pins of the oracle's Fourier transforms and dealiased products against the
directly written sums and a brute-force convolution (3/2 rule exactness)."""
import numpy as np

from oracle.grid import Case
from oracle import fourier as fo


def _rand_spec(case, seed):
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((case.Nr, case.Nz, case.Nh)) + 1j * rng.standard_normal((case.Nr, case.Nz, case.Nh))
    F[:, case.Nz // 2, :] = 0
    F[:, 0, 0] = F[:, 0, 0].real
    for n in range(1, case.Nz // 2):
        F[:, case.Nz - n, 0] = np.conj(F[:, n, 0])
    return F


def test_fft_route_equals_direct_sums():
    cs = Case(9, 8, 6, 0.5, 100.0, 0.0, 1e-3)
    F = _rand_spec(cs, 1)
    P = fo.to_physical(cs, F)
    for i in (0, 4):
        Pd = fo.direct_to_physical(cs, F[i])
        assert np.max(np.abs(P[i] - Pd)) < 1e-12
        Fd = fo.direct_to_spectral(cs, P[i])
        assert np.max(np.abs(fo.to_spectral(cs, P)[i] - Fd)) < 1e-13
    # round trip on the retained modes
    assert np.max(np.abs(fo.to_spectral(cs, P) - F)) < 1e-13


def test_products_are_alias_free_truncated_convolutions():
    """Padded-FFT product == sum over all pairs of retained modes whose
    wavenumbers add up to the target, for every retained target mode."""
    cs = Case(9, 8, 8, 0.5, 100.0, 0.0, 1e-3)
    a, b = _rand_spec(cs, 2), _rand_spec(cs, 3)
    zero = np.zeros_like(a)
    P = fo.products(cs, a, b, zero)["uv"]
    n_of = np.fft.fftfreq(cs.Nz, d=1.0 / cs.Nz).astype(int)
    i = 3
    sa, sb = fo.full_spectrum(cs, a[i]), fo.full_spectrum(cs, b[i])
    for s in range(cs.Nz):
        if s == cs.Nz // 2:
            continue
        for j in range(cs.Nh):
            target = (j, int(n_of[s]))
            acc = 0j
            for (j1, n1), c1 in sa.items():
                c2 = sb.get((target[0] - j1, target[1] - n1))
                if c2 is not None:
                    acc += c1 * c2
            assert abs(P[i, s, j] - acc) < 1e-12, (target, P[i, s, j], acc)


def test_mean_of_product_is_parseval_sum():
    cs = Case(9, 8, 8, 0.5, 100.0, 0.0, 1e-3)
    a = _rand_spec(cs, 5)
    P = fo.products(cs, a, a, a)["uu"]
    wt = np.full(cs.Nh, 2.0)
    wt[0] = 1.0
    ref = np.sum(np.abs(a) ** 2 * wt, axis=(1, 2))
    assert np.max(np.abs(P[:, 0, 0] - ref)) < 1e-12
