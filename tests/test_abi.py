"""Host-side checks of the C ABI (no GPU needed): the in-tree library builds
and loads, exports every function include/tc.h declares, and rejects invalid
arguments before touching the device."""
import os

import pytest

import paper_0711_1429_gb300 as tc
from paper_0711_1429_gb300 import build as tcbuild


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(tc.LIB_PATH):
        tcbuild.build()
    return tc.lib()


def test_exports_every_declared_function(lib):
    names = tc.declared_functions()
    assert "tc_create" in names and "tc_step" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("args,msg", [
    ((5, 16, 16, 0.883, 200.0, 0.0, 1e-3), "Nr"),
    ((33, 10, 16, 0.883, 200.0, 0.0, 1e-3), "Ntheta"),
    ((33, 18, 16, 0.883, 200.0, 0.0, 1e-3), "Ntheta"),
    ((33, 16, 38, 0.883, 200.0, 0.0, 1e-3), "Nz"),
    ((33, 16, 16, 1.0, 200.0, 0.0, 1e-3), "radius ratio"),
    ((33, 16, 16, 0.5, -1.0, 0.0, 1e-3), "Re_inner"),
    ((33, 16, 16, 0.5, 100.0, 0.0, 0.0), "dt"),
    ((9, 16, 4374, 0.883, 200.0, 0.0, 1e-3), "shared memory"),     # z columns of 6561 points
    ((9, 3072, 16, 0.883, 200.0, 0.0, 1e-3), "shared memory"),     # float64 theta rows of 4608 points
])
def test_invalid_arguments_are_rejected(lib, args, msg):
    with pytest.raises(tc.TcError) as e:
        tc.tc_create(*args)
    assert msg in str(e.value)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.tc_step(None, 1) == tc.TC_ERR_ARG
    assert lib.tc_get_field(None, 0, 0, None, 0) == tc.TC_ERR_ARG
    assert lib.tc_field_bytes(None, 0, 0) == 0
    assert lib.tc_set_tiles(None, 4, 128, 1) == tc.TC_ERR_ARG
    assert lib.tc_get_tiles(None, None, None, None) == tc.TC_ERR_ARG
    assert lib.tc_state_bytes(None) == 0
    assert lib.tc_save_state(None, None, 0) == tc.TC_ERR_ARG
    assert lib.tc_load_state(None, None, 0) == tc.TC_ERR_ARG
    assert lib.tc_set_rk_deferral(None, 1) == tc.TC_ERR_ARG
    assert lib.tc_get_rk_deferral(None, None) == tc.TC_ERR_ARG
    assert lib.tc_set_field_async(None, 0, None, 0) == tc.TC_ERR_ARG
    assert lib.tc_get_field_async(None, 0, None, 0, None) == tc.TC_ERR_ARG
    lib.tc_destroy(None)


def test_device_byte_estimate_on_host(lib):
    small = tc.make_params(33, 16, 16, 0.883, 200.0, 0.0, 1e-3)
    big = tc.make_params(257, 512, 512, 0.883, 3000.0, 0.0, 1e-3)
    bad = tc.make_params(5, 16, 16, 0.883, 200.0, 0.0, 1e-3)
    assert tc.tc_estimate_device_bytes(bad) == 0
    b_small, b_big = tc.tc_estimate_device_bytes(small), tc.tc_estimate_device_bytes(big)
    assert 0 < b_small < b_big
    # the 257 x 512 x 512 case: 11 spectral fields, 8 plane buffers, 8.5 tables per point
    P = 257 * 512 * 256
    assert b_big > P * (11 * 16 + 8 * 16 * 1.5 + 37 * 8)


@pytest.mark.parametrize("Ntheta, Nz", [(4, 4374), (6144, 4)])
def test_noalloc_rejects_transform_lengths_beyond_shared_memory(lib, Ntheta, Nz):
    """3 Nz/2 = 6561 (one z column of 2 x 6561 complex values is 210 KB) and
    3 Ntheta/2 = 9216 (295 KB) exceed the 200 KB a transform block may use;
    both planes fit the fixed array, so only the shared-memory check can
    refuse them, and it does so before any device call."""
    with pytest.raises(tc.TcError) as e:
        tc.tc_to_physical_noalloc(1, Ntheta, Nz, 1, 1, None)
    assert e.value.code == tc.TC_ERR_SIZE
    assert "shared memory" in str(e.value)


def test_noalloc_argument_checks_on_host(lib):
    with pytest.raises(tc.TcError) as e:
        tc.tc_to_physical_noalloc(4, 20, 16, 1, 1, None)      # Ntheta = 20 is not 2^a 3^b
    assert e.value.code == tc.TC_ERR_ARG
    with pytest.raises(tc.TcError) as e:
        tc.tc_to_physical_noalloc(4, 16, 38, 1, 1, None)      # Nz = 38 has the factor 19
    assert e.value.code == tc.TC_ERR_ARG
    with pytest.raises(tc.TcError) as e:
        tc.tc_to_physical_noalloc(4, 16, 16, None, 1, None)
    assert e.value.code == tc.TC_ERR_ARG
