"""GPU parity of the mean-flow rows with a non-zero axial mean flow U(r).

The other parity tests start from U = 0, where U stays O(amplitude^2) and
its rows barely enter.  Here U starts from a profile comparable to the
perturbation, set through tc_set_field(TC_FIELD_MEAN_U), and the
perturbation is large enough (r.m.s. ~ 5e-2) that the forcing -(1/r) d(r
<uv>)/dr of the axial row and -(1/r^2) d(r^2 <vw>)/dr of the azimuthal row
change U and W well above the tolerances within 50 steps.  The GPU path must
match the oracle to 1e-10 after one step and 1e-8 after 50 (float64 and
double-float forms), U and W included.  The oracle's mean rows are pinned
against the averaged momentum equations in tests/test_oracle_mean.py.
"""
import numpy as np
import pytest

import paper_0711_1429_gb300 as tc
from oracle.grid import Case
from oracle.rk import OracleSolver

from helpers import compare, gpu_case, gpu_state, inputs, oracle_state

pytestmark = pytest.mark.gpu

CFG = dict(Nr=33, Ntheta=16, Nz=16, zeta=0.883, Re_i=200.0, Re_o=0.0, dt=2e-3)


def _U0(Nr):
    x = -1.0 + 2.0 * np.arange(Nr) / (Nr - 1)
    return 0.05 * (1.0 - x * x) * (1.0 + 0.5 * x)


@pytest.mark.parametrize("precision", [tc.TC_PREC_FP64, tc.TC_PREC_DF64])
def test_nonzero_axial_mean_flow_matches_oracle(precision):
    c = CFG
    v, e = inputs(c["Nr"], c["Ntheta"], c["Nz"], c["zeta"], 31, "box", 5e-2)
    U0 = _U0(c["Nr"])
    cs = Case(c["Nr"], c["Ntheta"], c["Nz"], c["zeta"], c["Re_i"], c["Re_o"], c["dt"])
    s = OracleSolver(cs)
    s.set_fields(v=v, eta=e, U=U0)
    h = gpu_case(c["Nr"], c["Ntheta"], c["Nz"], c["zeta"], c["Re_i"], c["Re_o"], c["dt"],
                 v=v, eta=e, precision=precision)
    try:
        tc.tc_set_field(h, tc.TC_FIELD_MEAN_U, U0)
        assert np.array_equal(tc.tc_get_field(h, tc.TC_FIELD_MEAN_U), U0)
        for nsteps, tol in ((1, 1e-10), (49, 1e-8)):
            tc.tc_step(h, nsteps)
            s.step(nsteps)
            err = compare(gpu_state(h, cs.Nr, cs.Nz, cs.Nh), oracle_state(s))
            assert all(x < tol for x in err.values()), (nsteps, err)
        # the mean rows did work: U moved well beyond the tolerance, and the
        # non-linear forcing contributed (the same run without perturbation
        # ends elsewhere)
        assert np.linalg.norm(s.U - U0) > 1e-4 * np.linalg.norm(U0)
        s2 = OracleSolver(cs)
        s2.set_fields(U=U0)
        s2.step(50)
        assert np.linalg.norm(s2.U - s.U) > 1e-5 * np.linalg.norm(U0)
    finally:
        tc.tc_destroy(h)
