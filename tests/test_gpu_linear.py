"""The GPU hot path reproduces the critical Reynolds numbers of Sec. 3.

A Taylor-vortex mode (m = 0, alpha = 2 pi/4, the straight-vortex box of
Table 1) of amplitude 1e-6 is time-marched through tc_step just below and
just above the paper's brackets: 68.2 < Re_c < 68.4 at zeta = 0.5 and
184 < Re_c < 186 at zeta = 0.95.  After the transients decay, the growth
rate of |v_hat| must change sign across the bracket and agree with the
leading eigenvalue of the oracle's linearised rows (same discretisation, no
time-stepping error worth the name at this dt).
"""
import math

import numpy as np
import pytest

import paper_0711_1429_gb300 as tc
from oracle.grid import Case
from oracle.stencils import build_stencils
from oracle.linear import growth_rate

from helpers import ensure_lib

pytestmark = pytest.mark.gpu


def _gpu_rate(Re, Nr=33, dt=0.05, t1=40.0, t2=80.0, zeta=0.5):
    ensure_lib()
    h = tc.tc_create_ex(Nr, 4, 4, zeta, Re, 0.0, dt, Lz=4.0)
    try:
        Nz, Nh = 4, 2
        x = -1.0 + 2.0 * np.arange(Nr) / (Nr - 1)
        v = np.zeros((Nr, Nz, Nh), dtype=np.complex128)
        v[:, 1, 0] = 1e-6 * (1 - x * x) ** 2
        tc.tc_set_field(h, tc.TC_FIELD_V, v)
        amp = []
        n1, n2 = int(round(t1 / dt)), int(round((t2 - t1) / dt))
        tc.tc_step(h, n1)
        amp.append(np.linalg.norm(tc.tc_get_field(h, tc.TC_FIELD_V).reshape(Nr, Nz, Nh)[:, 1, 0]))
        tc.tc_step(h, n2)
        amp.append(np.linalg.norm(tc.tc_get_field(h, tc.TC_FIELD_V).reshape(Nr, Nz, Nh)[:, 1, 0]))
        return math.log(amp[1] / amp[0]) / (t2 - t1)
    finally:
        tc.tc_destroy(h)


def test_critical_reynolds_bracket_on_gpu():
    S = build_stencils(Case(33, 4, 4, 0.5, 68.0, 0.0, 0.05).r)
    rates = {}
    for Re in (68.0, 68.6):
        g = _gpu_rate(Re)
        e = growth_rate(Case(33, 4, 4, 0.5, Re, 0.0, 0.05, Lz=4.0), S, 0.0, 2 * math.pi / 4.0)
        rates[Re] = (g, e)
        assert abs(g - e) < 2e-4, (Re, g, e)
    assert rates[68.0][0] < 0 < rates[68.6][0], rates


def test_critical_reynolds_bracket_on_gpu_zeta_095():
    """zeta = 0.95 (R_i = 38 h): the growth rates at 184 and 186 are only
    -/+ 3.8e-4, and the next eigenvalue lies 0.12 below; the rate is taken
    between t = 100 and 200, where the second mode has decayed by e^-12."""
    S = build_stencils(Case(33, 4, 4, 0.95, 185.0, 0.0, 0.05).r)
    rates = {}
    for Re in (184.0, 186.0):
        g = _gpu_rate(Re, t1=100.0, t2=200.0, zeta=0.95)
        e = growth_rate(Case(33, 4, 4, 0.95, Re, 0.0, 0.05, Lz=4.0), S, 0.0, 2 * math.pi / 4.0)
        rates[Re] = (g, e)
        assert abs(g - e) < 5e-5, (Re, g, e)
    assert rates[184.0][0] < 0 < rates[186.0][0], rates
