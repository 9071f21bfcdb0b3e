"""tc_set_field_async / tc_get_field_async give the bits of their waiting
counterparts: the state set without waiting (from page-locked memory) and
stepped, then read back on a second stream while another call runs on the
handle's stream."""
import numpy as np
import pytest

import paper_0711_1429_gb300 as tc

from helpers import ensure_lib, gpu_case, inputs

pytestmark = pytest.mark.gpu


def test_async_copies_equal_the_waiting_ones():
    torch = pytest.importorskip("torch")
    ensure_lib()
    Nr, Nt, Nz = 33, 32, 32
    v, e = inputs(Nr, Nt, Nz, 0.883, 8, "k2", 0.05)
    ref = gpu_case(Nr, Nt, Nz, 0.883, 1000.0, 0.0, 1e-3, v=v, eta=e)
    h = gpu_case(Nr, Nt, Nz, 0.883, 1000.0, 0.0, 1e-3)
    try:
        tc.tc_step(ref, 2)
        nb = tc.tc_field_bytes(h, tc.TC_FIELD_V)
        pin = {k: torch.empty(nb // 8, dtype=torch.float64, pin_memory=True) for k in ("vi", "ei", "vo", "eo")}
        pin["vi"].numpy().view(np.complex128)[:] = v.ravel()
        pin["ei"].numpy().view(np.complex128)[:] = e.ravel()
        tc.tc_set_field_async(h, tc.TC_FIELD_V, pin["vi"].data_ptr(), nb)
        tc.tc_set_field_async(h, tc.TC_FIELD_ETA, pin["ei"].data_ptr(), nb)
        tc.tc_step(h, 2)
        side = torch.cuda.Stream()
        tc.tc_get_field_async(h, tc.TC_FIELD_V, pin["vo"].data_ptr(), nb, side.cuda_stream)
        tc.tc_get_field_async(h, tc.TC_FIELD_ETA, pin["eo"].data_ptr(), nb, side.cuda_stream)
        st = tc.tc_torque_stats(h)
        side.synchronize()
        assert np.array_equal(pin["vo"].numpy().view(np.complex128), tc.tc_get_field(ref, tc.TC_FIELD_V))
        assert np.array_equal(pin["eo"].numpy().view(np.complex128), tc.tc_get_field(ref, tc.TC_FIELD_ETA))
        assert st["G_inner"] == tc.tc_torque_stats(ref)["G_inner"]
        with pytest.raises(tc.TcError):
            tc.tc_get_field_async(h, tc.TC_FIELD_V, pin["vo"].data_ptr(), nb - 16)
    finally:
        tc.tc_destroy(ref)
        tc.tc_destroy(h)


def test_async_copies_through_device_staging_buffers():
    """The same with device buffers on both sides: the input staged on the
    device (as a pipelined caller does) and the result read into device
    memory, then checked on the host."""
    torch = pytest.importorskip("torch")
    ensure_lib()
    Nr, Nt, Nz = 33, 32, 32
    v, e = inputs(Nr, Nt, Nz, 0.883, 8, "k2", 0.05)
    ref = gpu_case(Nr, Nt, Nz, 0.883, 1000.0, 0.0, 1e-3, v=v, eta=e)
    h = gpu_case(Nr, Nt, Nz, 0.883, 1000.0, 0.0, 1e-3)
    try:
        tc.tc_step(ref, 2)
        nb = tc.tc_field_bytes(h, tc.TC_FIELD_V)
        dev = {k: torch.empty(nb // 8, dtype=torch.float64, device="cuda") for k in ("vi", "ei", "vo", "eo")}
        dev["vi"].copy_(torch.from_numpy(v.ravel().view(np.float64)))
        dev["ei"].copy_(torch.from_numpy(e.ravel().view(np.float64)))
        torch.cuda.synchronize()
        tc.tc_set_stream(h, torch.cuda.current_stream().cuda_stream)
        tc.tc_set_field_async(h, tc.TC_FIELD_V, dev["vi"].data_ptr(), nb)
        tc.tc_set_field_async(h, tc.TC_FIELD_ETA, dev["ei"].data_ptr(), nb)
        tc.tc_step(h, 2)
        tc.tc_get_field_async(h, tc.TC_FIELD_V, dev["vo"].data_ptr(), nb)
        tc.tc_get_field_async(h, tc.TC_FIELD_ETA, dev["eo"].data_ptr(), nb)
        torch.cuda.synchronize()
        assert np.array_equal(dev["vo"].cpu().numpy().view(np.complex128), tc.tc_get_field(ref, tc.TC_FIELD_V))
        assert np.array_equal(dev["eo"].cpu().numpy().view(np.complex128), tc.tc_get_field(ref, tc.TC_FIELD_ETA))
    finally:
        tc.tc_destroy(ref)
        tc.tc_destroy(h)
