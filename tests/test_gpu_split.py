"""One case split across ranks, on one GPU: the libtc split calls with the
exchanges of paper_0711_1429_gb300/split.py done in one process.

Two and three shares of the same case, each a handle of its own with its
radial planes and azimuthal columns (tc_split_set), are stepped with the
exchanges as device copies between the handles' arrays (no share's kernels
wait on another's).  Each share's columns of v and eta, and the mean flow of
the share owning column 0, must equal the unsplit tc_step bit for bit, in
all three precision forms.
"""
import numpy as np
import pytest

import paper_0711_1429_gb300 as tc

from helpers import ensure_lib, inputs

pytestmark = pytest.mark.gpu

CASE = (33, 32, 24, 0.85, 800.0, -60.0, 1e-3)     # Nr, Ntheta, Nz, zeta, Re_i, Re_o, dt
STEPS = 4


def _handle(v, e, prec, stream):
    Nr, Nt, Nz, z, Re, Ro, dt = CASE
    h = tc.tc_create_ex(Nr, Nt, Nz, z, Re, Ro, dt, precision=prec)
    tc.tc_set_stream(h, stream)
    tc.tc_set_field(h, tc.TC_FIELD_V, v)
    tc.tc_set_field(h, tc.TC_FIELD_ETA, e)
    return h


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("prec", [tc.TC_PREC_FP64, tc.TC_PREC_MIXED, tc.TC_PREC_DF64])
def test_split_on_one_gpu_equals_tc_step(world, prec):
    torch = pytest.importorskip("torch")
    from paper_0711_1429_gb300 import split as sp
    ensure_lib()
    Nr, Nt, Nz = CASE[:3]
    v, e = inputs(Nr, Nt, Nz, CASE[3], 23, "k2", 5e-2)
    stream = torch.cuda.current_stream().cuda_stream
    ref = _handle(v, e, prec, stream)
    hs = [_handle(v, e, prec, stream) for _ in range(world)]
    try:
        tc.tc_step(ref, STEPS)
        plan = sp.SplitPlan(Nr, Nt, Nz, world)
        shares = [sp.libtc_share(h, plan, r, prec) for r, h in enumerate(hs)]
        for _ in range(STEPS):
            sp.step_in_process(shares)
        for h in hs:
            tc.tc_split_finish(h)
        rv = tc.tc_get_field(ref, tc.TC_FIELD_V).reshape(Nr, Nz, Nt // 2)
        re = tc.tc_get_field(ref, tc.TC_FIELD_ETA).reshape(Nr, Nz, Nt // 2)
        for r, h in enumerate(hs):
            j0, j1 = plan.cols[r]
            gv = tc.tc_get_field(h, tc.TC_FIELD_V).reshape(Nr, Nz, Nt // 2)
            ge = tc.tc_get_field(h, tc.TC_FIELD_ETA).reshape(Nr, Nz, Nt // 2)
            assert np.array_equal(gv[:, :, j0:j1], rv[:, :, j0:j1]), r
            assert np.array_equal(ge[:, :, j0:j1], re[:, :, j0:j1]), r
        for which in (tc.TC_FIELD_MEAN_U, tc.TC_FIELD_MEAN_W):
            assert np.array_equal(tc.tc_get_field(hs[0], which), tc.tc_get_field(ref, which))
        assert tc.tc_torque_stats(hs[0])["step"] == STEPS
    finally:
        for h in [ref] + hs:
            tc.tc_destroy(h)
