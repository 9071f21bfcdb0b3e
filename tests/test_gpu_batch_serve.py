"""Many cases on one GPU: the batch (one graph per step; one launch per
plane kernel and shape class, one line kernel and one mean-flow launch per
precision form) and the
server (continuous batching by device budget).  Each case's result must be
the one the same case gives alone (bit for bit: the arithmetic per case is
the single-case path and has no order-dependent reductions)."""
import time

import numpy as np
import pytest

import paper_0711_1429_gb300 as tc

from helpers import ensure_lib, inputs

pytestmark = pytest.mark.gpu

CASES = [  # Nr, Ntheta, Nz, zeta, Re_i, dt, precision, seed
    (33, 32, 32, 0.70, 500.0, 1e-3, tc.TC_PREC_FP64, 1000),
    (65, 64, 32, 0.90, 2000.0, 1e-3, tc.TC_PREC_FP64, 1001),
    (17, 16, 64, 0.80, 1200.0, 2e-3, tc.TC_PREC_MIXED, 1002),
    (49, 48, 24, 0.95, 3000.0, 5e-4, tc.TC_PREC_FP64, 1003),
]


# shape classes of the batch (form, Ntheta, Nz) with several cases each:
# different Nr, radius ratio, Re and dt share one launch per kernel
BATCH_CASES = CASES + [
    (21, 32, 32, 0.85, 900.0, 1e-3, tc.TC_PREC_FP64, 1004),
    (40, 64, 32, 0.75, 1500.0, 2e-3, tc.TC_PREC_FP64, 1005),
    (25, 16, 64, 0.90, 700.0, 1e-3, tc.TC_PREC_MIXED, 1006),
    (30, 32, 32, 0.80, 1000.0, 1e-3, tc.TC_PREC_DF64, 1007),
    (19, 32, 32, 0.60, 800.0, 1e-3, tc.TC_PREC_DF64, 1008),
    (45, 32, 32, 0.92, 2500.0, 5e-4, tc.TC_PREC_FP64, 1009),
]
N_CLASSES = 5


def _params(c, autotune=0):
    Nr, Nt, Nz, z, Re, dt, prec, _ = c
    return tc.make_params(Nr, Nt, Nz, z, Re, 0.0, dt, precision=prec, autotune=autotune)


def _ic(c):
    Nr, Nt, Nz, z, Re, dt, prec, seed = c
    return inputs(Nr, Nt, Nz, z, seed, "k2", 0.05)


def _alone(c, nsteps, autotune=0):
    v, e = _ic(c)
    p = _params(c, autotune)
    h = tc.lib().tc_create_ex(tc.ctypes.byref(p))
    assert h, tc.tc_last_error()
    try:
        tc.tc_set_field(h, tc.TC_FIELD_V, v)
        tc.tc_set_field(h, tc.TC_FIELD_ETA, e)
        tc.tc_step(h, nsteps)
        return tc.tc_get_field(h, tc.TC_FIELD_V), tc.tc_get_field(h, tc.TC_FIELD_ETA)
    finally:
        tc.tc_destroy(h)


def test_batch_equals_alone_and_autotune_changes_nothing():
    ensure_lib()
    ref = [_alone(c, 4) for c in BATCH_CASES]
    tuned = _alone(CASES[1], 4, autotune=1)
    assert np.array_equal(tuned[0], ref[1][0]) and np.array_equal(tuned[1], ref[1][1])
    b = tc.tc_batch_create([_params(c, autotune=1) for c in BATCH_CASES])
    try:
        assert tc.tc_batch_launches_per_step(b) == 3 * (3 * N_CLASSES + 2 * 3)   # 3 precision forms
        for i, c in enumerate(BATCH_CASES):
            v, e = _ic(c)
            h = tc.tc_batch_case(b, i)
            tc.tc_set_field(h, tc.TC_FIELD_V, v)
            tc.tc_set_field(h, tc.TC_FIELD_ETA, e)
        tc.tc_batch_step(b, 3)
        tc.tc_batch_step(b, 1)
        for i in range(len(BATCH_CASES)):
            h = tc.tc_batch_case(b, i)
            assert np.array_equal(tc.tc_get_field(h, tc.TC_FIELD_V), ref[i][0]), i
            assert np.array_equal(tc.tc_get_field(h, tc.TC_FIELD_ETA), ref[i][1]), i
            assert tc.tc_torque_stats(h)["step"] == 4
        assert tc.tc_batch_device_bytes(b) > 0
    finally:
        tc.tc_batch_destroy(b)


@pytest.mark.parametrize("mode", [tc.TC_SERVE_GROUPED, tc.TC_SERVE_PER_CASE])
def test_server_results_equal_alone_within_budget(mode):
    ensure_lib()
    steps = [6, 11, 4, 9, 7, 5]
    cases = [CASES[i % len(CASES)] for i in range(len(steps))]
    ref = [_alone(c, n) for c, n in zip(cases, steps)]
    need = sorted(tc.tc_estimate_device_bytes(_params(c)) for c in cases)
    budget = need[-1] + need[-2] + 1          # at most two large cases at a time
    s = tc.tc_server_create(budget, max_active=8, mode=mode)
    outs = []
    try:
        ids = []
        for k, (c, n) in enumerate(zip(cases, steps)):
            v, e = _ic(c)
            ov, oe = np.empty_like(v.ravel()), np.empty_like(e.ravel())
            outs.append((ov, oe))
            ids.append(tc.tc_server_submit(s, _params(c), v, e, n, ov, oe))
            time.sleep(0.01 * (k % 3))        # staggered arrivals
        with pytest.raises(tc.TcError) as ex:  # alone larger than the budget
            tc.tc_server_submit(s, tc.make_params(129, 256, 256, 0.9, 1000.0, 0.0, 1e-3), None, None, 1)
        assert ex.value.code == tc.TC_ERR_SIZE
        tc.tc_server_drain(s, 300.0)
        res = {r["id"]: r for r in tc.tc_server_poll(s)}
        st = tc.tc_server_stats(s)
    finally:
        tc.tc_server_destroy(s)
    assert st["finished"] == len(steps) and st["peak_used_bytes"] <= budget
    assert st["peak_active"] >= 2                 # requests overlapped on the device
    assert st["steps"] == sum(steps) and st["step_ms_p99"] >= st["step_ms_p50"] > 0
    for k, rid in enumerate(ids):
        r = res[rid]
        assert r["status"] == tc.TC_OK and r["steps"] == steps[k], r
        assert np.array_equal(outs[k][0], ref[k][0]), k
        assert np.array_equal(outs[k][1], ref[k][1]), k
