"""The allocation-free entry point tc_to_physical_noalloc.

It exists for callers that may not allocate device memory (fixed memory
budgets, host applications that own every buffer, loops that forbid
cudaMalloc).  Here the test plays such a caller: it owns the input and output
device buffers (allocated through torch, outside the entry point) and checks
two calls in a row against the physical field that tc_get_field returns for
the same state, within the tolerance of the other GPU tests.  The shapes
cover the z plans (radix 3/16/8/4/2, and the paired odd-prime stages of
axial lengths with factors 5 and 17), every z tile width, several radial
planes per pass, and a plane that nearly fills the fixed scratch array.  The
file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import paper_0711_1429_gb300 as tc

from helpers import ensure_lib, gpu_case, inputs, relerr

pytestmark = pytest.mark.gpu


def _check_twice(h, Nr, Nt, Nz):
    torch = pytest.importorskip("torch")
    Mt, Mz = 3 * Nt // 2, 3 * Nz // 2
    stream = torch.cuda.current_stream()
    out = torch.empty(Nr * Mz * Mt, dtype=torch.float64, device="cuda")
    for which in (tc.TC_FIELD_V, tc.TC_FIELD_ETA):       # two calls in a row
        spec = tc.tc_get_field(h, which, tc.TC_SPECTRAL)
        ref = tc.tc_get_field(h, which, tc.TC_PHYSICAL)
        d_spec = torch.from_numpy(spec.view(np.float64).copy()).cuda()
        out.fill_(float("nan"))                           # stale values would show
        torch.cuda.synchronize()
        tc.tc_to_physical_noalloc(Nr, Nt, Nz, d_spec.data_ptr(), out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert relerr(got, ref) < 1e-10, (which, relerr(got, ref))


@pytest.mark.parametrize("Nr, Nt, Nz", [
    (17, 48, 24),     # padded 72 x 36: radix-3 and radix-2 stages, z tile 8
    (11, 12, 20),     # Nz = 20: padded 30 = 2 3 5 (prime stage); Ntheta/2 = 6: z tile 2
    (9, 16, 34),      # Nz = 34: padded 51 = 3 17; z tile 8
    (13, 24, 16),     # Ntheta/2 = 12: z tile 4
    (10, 36, 16),     # Ntheta/2 = 18: z tile 2, theta length 54
])
def test_noalloc_transform_matches_tc_get_field_twice(Nr, Nt, Nz):
    pytest.importorskip("torch")
    ensure_lib()
    v, e = inputs(Nr, Nt, Nz, 0.7, 21, "box", 3e-2, jmax=Nt // 4, nmax=Nz // 4)
    h = gpu_case(Nr, Nt, Nz, 0.7, 400.0, 0.0, 1e-3, v=v, eta=e)
    try:
        tc.tc_step(h, 1)
        _check_twice(h, Nr, Nt, Nz)
    finally:
        tc.tc_destroy(h)


def test_noalloc_plane_just_under_the_scratch_limit():
    """Ntheta = 1024, Nz = 1350: one padded plane is 2025 x 512 complex
    values, 16.59 MB of the 16.78 MB array, so each pass takes one radial
    plane; the z tile is 2 (4 or 8 columns of 2025 points exceed the shared
    memory of a block)."""
    pytest.importorskip("torch")
    ensure_lib()
    Nr, Nt, Nz = 9, 1024, 1350
    assert 2025 * 512 * 16 < tc.TC_NOALLOC_SCRATCH_BYTES < 2 * 2025 * 512 * 16
    v, e = inputs(Nr, Nt, Nz, 0.883, 5, "k2", 0.05)
    h = gpu_case(Nr, Nt, Nz, 0.883, 3000.0, 0.0, 1e-3, v=v, eta=e)
    try:
        _check_twice(h, Nr, Nt, Nz)
    finally:
        tc.tc_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    pytest.importorskip("torch")
    ensure_lib()
    # (3*4096/2) x (4096/2) complex plane = 201 MB > the 16 MiB scratch
    with pytest.raises(tc.TcError) as ex:
        tc.tc_to_physical_noalloc(1, 4096, 4096, 1, 1, None)
    assert ex.value.code == tc.TC_ERR_SIZE
    assert "scratch" in str(ex.value)
