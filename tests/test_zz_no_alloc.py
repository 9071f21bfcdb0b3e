"""The allocation-free entry point tc_to_physical_noalloc.

It exists for callers that may not allocate device memory (fixed memory
budgets, host applications that own every buffer, loops that forbid
cudaMalloc).  Here the test plays such a caller: it owns the input and output
device buffers (allocated through torch, outside the entry point) and checks
two calls in a row against the physical field that tc_get_field returns for
the same state, within the tolerance of the other GPU tests.  The file is
named so that pytest collects it last.
"""
import numpy as np
import pytest

import paper_0711_1429_gb300 as tc

from helpers import ensure_lib, gpu_case, inputs, relerr

pytestmark = pytest.mark.gpu


def test_noalloc_transform_matches_tc_get_field_twice():
    torch = pytest.importorskip("torch")
    ensure_lib()
    Nr, Nt, Nz = 17, 48, 24                  # padded 72 x 36: radix-3 and radix-2 stages
    Mt, Mz = 3 * Nt // 2, 3 * Nz // 2
    v, e = inputs(Nr, Nt, Nz, 0.7, 21, "box", 3e-2, jmax=10, nmax=6)
    h = gpu_case(Nr, Nt, Nz, 0.7, 400.0, 0.0, 1e-3, v=v, eta=e)
    try:
        tc.tc_step(h, 1)
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
            assert relerr(got, ref) < 1e-10
    finally:
        tc.tc_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    ensure_lib()
    # (3*4096/2) x (4096/2) complex plane = 50 MB > the 16 MiB scratch
    with pytest.raises(tc.TcError) as ex:
        tc.tc_to_physical_noalloc(1, 4096, 4096, 1, 1, None)
    assert ex.value.code == tc.TC_ERR_SIZE
    assert "scratch" in str(ex.value)
