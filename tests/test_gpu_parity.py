"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: relative L2 1e-10 after one step and 1e-8 after 50 steps for the
plain float64 path; the mixed form (float32 FFTs and products) is held to a
stated error bound instead.
"""
import numpy as np
import pytest

import paper_0711_1429_gb300 as tc
from oracle.grid import Case
from oracle.rk import OracleSolver
from oracle import fourier as fo
from oracle import diagnostics as dg

from helpers import (compare, gpu_case, gpu_state, inputs, oracle_state, relerr,
                     workload_inputs, ensure_lib)

pytestmark = pytest.mark.gpu

SMALL = dict(Nr=33, Ntheta=16, Nz=16, zeta=0.883, Re_i=200.0, Re_o=0.0, dt=1e-3)


def _pair(cfg, v, e, precision=tc.TC_PREC_FP64):
    c = Case(cfg["Nr"], cfg["Ntheta"], cfg["Nz"], cfg["zeta"], cfg["Re_i"], cfg["Re_o"], cfg["dt"])
    s = OracleSolver(c)
    s.set_fields(v=v, eta=e)
    h = gpu_case(cfg["Nr"], cfg["Ntheta"], cfg["Nz"], cfg["zeta"], cfg["Re_i"], cfg["Re_o"], cfg["dt"],
                 v=v, eta=e, precision=precision)
    return c, s, h


def _check(c, s, h, tol):
    gs = gpu_state(h, c.Nr, c.Nz, c.Nh)
    os_ = oracle_state(s)
    err = compare(gs, os_)
    bad = {k: e for k, e in err.items() if not e < tol}
    assert not bad, (err, tol)
    return err


def test_one_step_small():
    v, e = workload_inputs("tc-small-33x16x16")
    c, s, h = _pair(SMALL, v, e)
    try:
        tc.tc_step(h, 1)
        s.step(1)
        _check(c, s, h, 1e-10)
    finally:
        tc.tc_destroy(h)


def test_fifty_steps_small():
    v, e = workload_inputs("tc-small-33x16x16")
    c, s, h = _pair(SMALL, v, e)
    try:
        tc.tc_step(h, 50)
        s.step(50)
        _check(c, s, h, 1e-8)
    finally:
        tc.tc_destroy(h)


def test_radix3_sizes_counter_rotation_ragged_tiles():
    """Ntheta = 24, Nz = 12 (padded 36 x 18: radix 3 and 2 stages, 12
    azimuthal columns: z tiles of 4), Nr = 17, outer wall counter-rotating."""
    cfg = dict(Nr=17, Ntheta=24, Nz=12, zeta=0.6, Re_i=150.0, Re_o=-40.0, dt=2e-3)
    v, e = inputs(17, 24, 12, 0.6, 11, "box", 2e-2, jmax=8, nmax=5)
    c, s, h = _pair(cfg, v, e)
    try:
        tc.tc_step(h, 1)
        s.step(1)
        _check(c, s, h, 1e-10)
        tc.tc_step(h, 9)
        s.step(9)
        _check(c, s, h, 1e-9)
    finally:
        tc.tc_destroy(h)


def test_one_step_129():
    """Nr = 129, 128 x 128 modes, k^-2 spectrum at 0.05 rms (several warps
    and CTAs per plane, every FFT stage radix)."""
    cfg = dict(Nr=129, Ntheta=128, Nz=128, zeta=0.883, Re_i=3000.0, Re_o=0.0, dt=1e-3)
    v, e = workload_inputs("tc-129x128x128")
    c, s, h = _pair(cfg, v, e)
    try:
        tc.tc_step(h, 1)
        s.step(1)
        _check(c, s, h, 1e-10)
    finally:
        tc.tc_destroy(h)


@pytest.mark.parametrize("precision", [tc.TC_PREC_FP64, tc.TC_PREC_MIXED, tc.TC_PREC_DF64])
def test_graph_step_equals_substeps_and_is_deterministic(precision):
    """The captured step (in the double-float and mixed forms with the RK
    memory's implicit part deferred to its own kernel beside the theta rows)
    equals the substeps launched one by one, bit for bit."""
    v, e = workload_inputs("tc-small-33x16x16")
    cfg = SMALL
    hs = [gpu_case(cfg["Nr"], cfg["Ntheta"], cfg["Nz"], cfg["zeta"], cfg["Re_i"], cfg["Re_o"], cfg["dt"],
                   v=v, eta=e, precision=precision) for _ in range(5)]
    try:
        tc.tc_step(hs[0], 3)
        tc.tc_advance_substeps(hs[1], 9)
        tc.tc_step(hs[2], 3)
        # the deferred RK memory: three steps in one call (first and next
        # step graphs), and three calls of one step each
        tc.tc_set_rk_deferral(hs[3], 1)
        tc.tc_step(hs[3], 3)
        tc.tc_set_rk_deferral(hs[4], 1)
        for _ in range(3):
            tc.tc_step(hs[4], 1)
        assert tc.tc_get_rk_deferral(hs[3]) == (precision != tc.TC_PREC_FP64)
        ref = gpu_state(hs[1], 33, 16, 8)
        for h in hs[:1] + hs[2:]:
            g = gpu_state(h, 33, 16, 8)
            for k in ref:
                assert np.array_equal(g[k], ref[k]), k
        st = tc.tc_torque_stats(hs[1])
        assert st["step"] == 3 and abs(st["t"] - 3e-3) < 1e-15
    finally:
        for h in hs:
            tc.tc_destroy(h)


def test_boundary_conditions_and_hermitian_symmetry():
    cfg = dict(Nr=33, Ntheta=32, Nz=32, zeta=0.883, Re_i=800.0, Re_o=0.0, dt=2e-3)
    v, e = inputs(33, 32, 32, 0.883, 5, "k2", 0.05)
    c, s, h = _pair(cfg, v, e)
    try:
        tc.tc_step(h, 5)
        g = gpu_state(h, 33, 32, 16)
        for k in ("v", "eta", "u", "w"):
            assert np.max(np.abs(g[k][0, :, 1:])) == 0 and np.max(np.abs(g[k][-1, :, 1:])) == 0, k
        # Dv = 0 at both walls (explicit one-sided derivative), to round-off
        dv_in = np.tensordot(s.S.dwall[0], g["v"][0:5], axes=(0, 0))
        dv_out = np.tensordot(s.S.dwall[1], g["v"][-5:], axes=(0, 0))
        scale = np.max(np.abs(g["v"])) * np.max(np.abs(s.S.dwall))
        assert np.max(np.abs(dv_in)) < 1e-12 * scale and np.max(np.abs(dv_out)) < 1e-12 * scale
        # m = 0 column Hermitian, Nyquist slot zero
        for k in ("v", "eta", "u", "w"):
            col = g[k][:, :, 0]
            for n in range(1, 16):
                assert np.array_equal(col[:, 32 - n], np.conj(col[:, n])), k
            assert np.max(np.abs(g[k][:, 16, :])) == 0
        assert np.max(np.abs(g["U"][[0, -1]])) == 0
        assert g["W"][0] == 1.0 and g["W"][-1] == 0.0
    finally:
        tc.tc_destroy(h)


def test_physical_field_and_stats_match_oracle():
    v, e = workload_inputs("tc-small-33x16x16")
    c, s, h = _pair(SMALL, v, e)
    try:
        tc.tc_step(h, 3)
        s.step(3)
        u, vv, w = s.velocity()
        for which, F in ((tc.TC_FIELD_U, u), (tc.TC_FIELD_V, vv), (tc.TC_FIELD_W, w), (tc.TC_FIELD_ETA, s.eta)):
            P = tc.tc_get_field(h, which, tc.TC_PHYSICAL).reshape(c.Nr, c.Mz, c.Mt)
            assert relerr(P, fo.to_physical(c, F)) < 1e-10, which
        st = tc.tc_torque_stats(h)
        Gi, Go = dg.torque(c, s.S, s.W)
        ti, to = dg.re_tau(c, s.S, s.W)
        E = dg.kinetic_energy(c, u, vv, w)
        assert abs(st["G_inner"] - Gi) < 1e-10 * Gi and abs(st["G_outer"] - Go) < 1e-10 * Go
        assert abs(st["Re_tau_inner"] - ti) < 1e-10 * ti and abs(st["Re_tau_outer"] - to) < 1e-10 * to
        assert abs(st["energy"] - E) < 1e-10 * E
        eps = dg.dissipation(c, s.S, u, vv, w)
        Pin = dg.wall_power(c, s.S, s.W)
        assert abs(st["dissipation"] - eps) < 1e-10 * eps
        assert abs(st["power_in"] - Pin) < 1e-10 * abs(Pin)
        assert st["step"] == 3
    finally:
        tc.tc_destroy(h)


@pytest.mark.parametrize("stretch", [0.0, 1.5])
def test_dissipation_and_wall_power_match_oracle(stretch):
    """eps and P_in of a perturbed state with a moving outer wall, on the
    uniform and the stretched radial grid, several tiles of slots."""
    cfg = dict(Nr=41, Ntheta=24, Nz=18, zeta=0.7, Re_i=300.0, Re_o=-60.0, dt=2e-3)
    c = Case(41, 24, 18, 0.7, 300.0, -60.0, 2e-3, stretch=stretch)
    s = OracleSolver(c)
    v, e = inputs(41, 24, 18, 0.7, 21, "k2", 0.05)
    s.set_fields(v=v, eta=e)
    h = gpu_case(41, 24, 18, 0.7, 300.0, -60.0, 2e-3, v=v, eta=e, stretch=stretch)
    try:
        tc.tc_step(h, 2)
        s.step(2)
        u, vv, w = s.velocity()
        st = tc.tc_torque_stats(h)
        eps = dg.dissipation(c, s.S, u, vv, w)
        Pin = dg.wall_power(c, s.S, s.W)
        assert abs(st["dissipation"] - eps) < 1e-10 * eps, (st["dissipation"], eps)
        assert abs(st["power_in"] - Pin) < 1e-10 * abs(Pin), (st["power_in"], Pin)
    finally:
        tc.tc_destroy(h)


def test_laminar_dissipation_balances_wall_power():
    """Circular Couette flow: eps = P_in = 2 nu B^2 (1/R_i^2 - 1/R_o^2)/V."""
    h = gpu_case(65, 8, 8, 0.5, 100.0, -30.0, 1e-3)
    try:
        st = tc.tc_torque_stats(h)
        c = Case(65, 8, 8, 0.5, 100.0, -30.0, 1e-3)
        Ri, Ro, Wo = c.Ri, c.Ro, c.W_outer
        A = (Wo * Ro - Ri) / (Ro * Ro - Ri * Ri)
        B = Ri - A * Ri * Ri
        exact = 2.0 * c.nu * B * B * (1.0 / Ri ** 2 - 1.0 / Ro ** 2) / (0.5 * (Ro * Ro - Ri * Ri))
        assert abs(st["dissipation"] / exact - 1.0) < 1e-6
        assert abs(st["power_in"] / exact - 1.0) < 2e-6
    finally:
        tc.tc_destroy(h)


def test_laminar_state_stays_laminar():
    cfg = SMALL
    h = gpu_case(cfg["Nr"], cfg["Ntheta"], cfg["Nz"], cfg["zeta"], cfg["Re_i"], cfg["Re_o"], cfg["dt"])
    try:
        tc.tc_step(h, 10)
        g = gpu_state(h, 33, 16, 8)
        assert np.max(np.abs(g["v"])) == 0 and np.max(np.abs(g["eta"])) == 0
        c = Case(33, 16, 16, 0.883, 200.0, 0.0, 1e-3)
        z = c.zeta
        exact = 1.0 / (1.0 - z * z) * (c.Ri / c.r - z * z * c.r / c.Ri)
        assert np.max(np.abs(g["W"] - exact)) < 1e-6
        st = tc.tc_torque_stats(h)
        assert abs(st["G_inner"] - 4 * np.pi / (1 - z * z)) < 1e-4 * st["G_inner"]
    finally:
        tc.tc_destroy(h)


@pytest.mark.parametrize("precision", [tc.TC_PREC_FP64, tc.TC_PREC_MIXED, tc.TC_PREC_DF64])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_state_is_reported(precision, bad):
    """A NaN or an infinity planted in the host input makes tc_step return
    TC_ERR_NONFINITE in every form, through the float32 and double-float
    conversions of the state (no device fault: the kernels only test values)."""
    v, e = workload_inputs("tc-small-33x16x16")
    v = v.copy()
    v[10, 2, 3] = bad
    cfg = SMALL
    h = gpu_case(cfg["Nr"], cfg["Ntheta"], cfg["Nz"], cfg["zeta"], cfg["Re_i"], cfg["Re_o"], cfg["dt"], v=v, eta=e,
                 precision=precision)
    try:
        with pytest.raises(tc.TcError) as ex:
            tc.tc_step(h, 1)
        assert ex.value.code == tc.TC_ERR_NONFINITE
    finally:
        tc.tc_destroy(h)


def test_mixed_precision_error_is_bounded():
    """FP32 FFTs/products, FP64 radial rows and solves: error against the FP64
    oracle after 10 steps of a 33 x 64 x 64 case with a 0.05 rms k^-2 field
    stays below 1e-5 relative per field (it is set by float32 rounding of the
    products, which enter only through dt * E)."""
    cfg = dict(Nr=33, Ntheta=64, Nz=64, zeta=0.883, Re_i=3000.0, Re_o=0.0, dt=1e-3)
    v, e = inputs(33, 64, 64, 0.883, 2, "k2", 0.05)
    c, s, h = _pair(cfg, v, e, precision=tc.TC_PREC_MIXED)
    try:
        tc.tc_step(h, 10)
        s.step(10)
        err = _check(c, s, h, 1e-5)
        assert max(err.values()) > 1e-12      # it really ran in float32
    finally:
        tc.tc_destroy(h)


def test_full_size_first_substep_sampled_pairs():
    """The 257 x 512 x 512 bench workload, in the launch configuration the
    benchmark times: one RK substep on the GPU against the oracle on 53
    sampled Fourier pairs (edges included) and the mean profiles.  The oracle
    forms the products of every radial plane (in chunks of planes) and runs
    its line phase only for the sampled pairs."""
    from oracle.fourier import products
    from oracle import operators as op
    from paper_0711_1429_gb300.synthetic import WORKLOADS
    w = WORKLOADS["tc-257x512x512"]
    Nr, Nt, Nz = w["Nr"], w["Ntheta"], w["Nz"]
    Nh = Nt // 2
    v, e = workload_inputs("tc-257x512x512")
    c = Case(Nr, Nt, Nz, w["zeta"], w["Re_i"], w["Re_o"], w["dt"])
    h = gpu_case(Nr, Nt, Nz, w["zeta"], w["Re_i"], w["Re_o"], w["dt"], v=v, eta=e)
    try:
        tc.tc_advance_substeps(h, 1)
        g = {"v": tc.tc_get_field(h, tc.TC_FIELD_V).reshape(Nr, Nz, Nh),
             "eta": tc.tc_get_field(h, tc.TC_FIELD_ETA).reshape(Nr, Nz, Nh),
             "U": tc.tc_get_field(h, tc.TC_FIELD_MEAN_U), "W": tc.tc_get_field(h, tc.TC_FIELD_MEAN_W)}
    finally:
        tc.tc_destroy(h)
    # oracle: full velocity and products, then the sampled pairs' line phase
    full = OracleSolver(c, pairs=np.zeros((Nz, Nh), dtype=bool))   # no bands; used for helpers
    full.set_fields(v=v, eta=e)
    mask_all = c.active_mask()
    act = np.nonzero(mask_all)
    m = (np.arange(Nh) * c.m0)[act[1]].reshape(1, -1)
    al = (c.n_index() * c.alpha0).astype(float)[act[0]].reshape(1, -1)
    k2 = op.coefficients(c.r.reshape(-1, 1), m, al)[0]
    ua, wa = op.reconstruct_uw(full.S, c.r.reshape(-1, 1), m, al, k2, full.v[:, act[0], act[1]],
                               full.eta[:, act[0], act[1]])
    u = np.zeros((Nr, Nz, Nh), dtype=np.complex128)
    ww = np.zeros_like(u)
    u[:, act[0], act[1]] = ua
    ww[:, act[0], act[1]] = wa
    full._hermitian(u)
    full._hermitian(ww)
    del ua, wa, k2
    u[:, 0, 0] = full.U
    ww[:, 0, 0] = full.W
    vv = full.v.copy()
    P = {k: np.empty_like(vv) for k in ("uu", "uv", "uw", "vv", "vw", "ww")}
    for r0 in range(0, Nr, 16):
        sl = slice(r0, min(Nr, r0 + 16))
        chunk = products(c, u[sl], vv[sl], ww[sl])
        for k in P:
            P[k][sl] = chunk[k]
    del u, ww, vv
    rng = np.random.default_rng(5)
    sample = np.zeros((Nz, Nh), dtype=bool)
    sample.flat[rng.choice(Nz * Nh, 48, replace=False)] = True
    for s_, j_ in ((1, 0), (Nz // 2 - 1, 0), (Nz // 2 - 1, Nh - 1), (Nz // 2 + 1, Nh - 1), (0, 1)):
        sample[s_, j_] = True
    sub = OracleSolver(c, stencils=full.S, pairs=sample)
    sub.set_fields(v=v, eta=e)
    sub.advance(0, sub.explicit_terms(P))
    sel = np.nonzero(sample & mask_all)
    for key, G, O in (("v", g["v"], sub.v), ("eta", g["eta"], sub.eta)):
        err = relerr(G[:, sel[0], sel[1]], O[:, sel[0], sel[1]])
        assert err < 1e-10, (key, err)
    assert relerr(g["U"], sub.U) < 1e-10 and relerr(g["W"], sub.W) < 1e-10


@pytest.mark.parametrize("steps,tol", [(1, 1e-10), (50, 1e-8)])
def test_df64_form_meets_fp64_tolerances_small(steps, tol):
    """Double-float FFTs and products (float32 pairs) hold the FP64 parity bar."""
    v, e = workload_inputs("tc-small-33x16x16")
    c, s, h = _pair(SMALL, v, e, precision=tc.TC_PREC_DF64)
    try:
        tc.tc_step(h, steps)
        s.step(steps)
        err = _check(c, s, h, tol)
        assert max(err.values()) > 0.0
    finally:
        tc.tc_destroy(h)


def test_df64_form_one_step_129():
    cfg = dict(Nr=129, Ntheta=128, Nz=128, zeta=0.883, Re_i=3000.0, Re_o=0.0, dt=1e-3)
    v, e = workload_inputs("tc-129x128x128")
    c, s, h = _pair(cfg, v, e, precision=tc.TC_PREC_DF64)
    try:
        tc.tc_step(h, 1)
        s.step(1)
        _check(c, s, h, 1e-10)
    finally:
        tc.tc_destroy(h)


def test_stretched_grid_parity_and_stats():
    """tanh-stretched radial grid (denser at the walls): one and ten steps,
    and the torque/energy statistics, against the oracle."""
    cfg = dict(Nr=41, Ntheta=32, Nz=24, zeta=0.8, Re_i=600.0, Re_o=0.0, dt=1e-3)
    v, e = inputs(41, 32, 24, 0.8, 17, "k2", 0.05)
    c = Case(41, 32, 24, 0.8, 600.0, 0.0, 1e-3, stretch=1.4)
    s = OracleSolver(c)
    s.set_fields(v=v, eta=e)
    h = gpu_case(41, 32, 24, 0.8, 600.0, 0.0, 1e-3, v=v, eta=e, stretch=1.4)
    try:
        tc.tc_step(h, 1)
        s.step(1)
        _check(c, s, h, 1e-10)
        tc.tc_step(h, 9)
        s.step(9)
        _check(c, s, h, 1e-9)
        st = tc.tc_torque_stats(h)
        u, vv, w = s.velocity()
        Gi, Go = dg.torque(c, s.S, s.W)
        assert abs(st["G_inner"] - Gi) < 1e-10 * Gi and abs(st["G_outer"] - Go) < 1e-10 * Go
        E = dg.kinetic_energy(c, u, vv, w)
        assert abs(st["energy"] - E) < 1e-10 * E
    finally:
        tc.tc_destroy(h)


@pytest.mark.parametrize("Nz", [10, 14, 34])
def test_prime_radix_axial_sizes(Nz):
    """Axial sizes with prime factors 5, 7, 17 (padded 15, 21, 51): the
    transforms take direct-sum prime stages.  The paper's production grid
    has Nz = 170 = 2 5 17."""
    cfg = dict(Nr=21, Ntheta=16, Nz=Nz, zeta=0.85, Re_i=500.0, Re_o=0.0, dt=1e-3)
    v, e = inputs(21, 16, Nz, 0.85, 31, "k2", 0.05)
    c, s, h = _pair(cfg, v, e)
    try:
        tc.tc_step(h, 2)
        s.step(2)
        _check(c, s, h, 1e-10)
    finally:
        tc.tc_destroy(h)


def test_minimum_sizes():
    """The smallest accepted case: Nr = 9 (one interior compact row of each
    kind), Ntheta = Nz = 4 (two azimuthal columns, padded 6 x 6)."""
    cfg = dict(Nr=9, Ntheta=4, Nz=4, zeta=0.6, Re_i=100.0, Re_o=10.0, dt=2e-3)
    v, e = inputs(9, 4, 4, 0.6, 3, "box", 5e-2, jmax=1, nmax=1)
    c, s, h = _pair(cfg, v, e)
    try:
        tc.tc_step(h, 3)
        s.step(3)
        _check(c, s, h, 1e-10)
    finally:
        tc.tc_destroy(h)


@pytest.mark.parametrize("precision", [tc.TC_PREC_FP64, tc.TC_PREC_MIXED, tc.TC_PREC_DF64])
def test_launch_shapes_change_no_bits(precision):
    """Every z tile, line-kernel launch shape and column grouping of the
    overlapped step gives the same bits: the autotuner's choice and the
    overlap change no arithmetic (the overlapped step's dependencies are
    complete, or a group would read stale data)."""
    cfg = dict(Nr=33, Ntheta=32, Nz=24, zeta=0.883, Re_i=800.0, Re_o=0.0, dt=2e-3)
    v, e = inputs(33, 32, 24, 0.883, 9, "k2", 0.05)

    def run(ztile, variant, chunks, rk=0):
        h = gpu_case(cfg["Nr"], cfg["Ntheta"], cfg["Nz"], cfg["zeta"], cfg["Re_i"], cfg["Re_o"], cfg["dt"],
                     v=v, eta=e, precision=precision)
        try:
            tc.tc_set_tiles(h, ztile, variant, chunks)
            tc.tc_set_rk_deferral(h, rk)
            tc.tc_step(h, 2)
            return gpu_state(h, 33, 24, 16)
        finally:
            tc.tc_destroy(h)

    ref = run(8, 128, 1)
    for zt, lv, ch, rk in [(1, 0, 0, 0), (2, 0, 0, 0), (4, 0, 0, 0)] + [(0, x, 0, 0) for x in tc.LINE_VARIANTS] + \
            [(1, 0, 2, 0), (1, 0, 4, 0), (1, 0, 8, 0), (2, 0, 8, 0)] + \
            [(0, 0, 1, 1), (0, 0, 2, 1), (1, 0, 4, 1), (0, 3001, 1, 1), (0, 1004, 2, 1), (0, 0, 0, -1)]:
        g = run(zt, lv, ch, rk)
        for k in ref:
            assert np.array_equal(g[k], ref[k]), (zt, lv, ch, rk, k)
    h = gpu_case(33, 32, 24, 0.883, 800.0, 0.0, 2e-3, precision=precision)
    try:
        for bad in ((3, 0, 0), (0, 100, 0), (16, 0, 0), (0, 0, 3)):
            with pytest.raises(tc.TcError):
                tc.tc_set_tiles(h, *bad)
        for bad in (-2, 2):
            with pytest.raises(tc.TcError):
                tc.tc_set_rk_deferral(h, bad)
    finally:
        tc.tc_destroy(h)


def test_checkpoint_resume_is_bit_identical():
    """A run saved after 5 steps (and after a further substep) and resumed in
    a fresh handle ends bit for bit where the uninterrupted run ends; images
    of another shape or size are refused."""
    cfg = dict(Nr=33, Ntheta=32, Nz=24, zeta=0.8, Re_i=600.0, Re_o=-50.0, dt=2e-3)
    v, e = inputs(33, 32, 24, 0.8, 13, "k2", 0.05)
    mk = lambda prec=tc.TC_PREC_FP64: gpu_case(cfg["Nr"], cfg["Ntheta"], cfg["Nz"], cfg["zeta"], cfg["Re_i"],
                                               cfg["Re_o"], cfg["dt"], v=v, eta=e, precision=prec)
    a, b, c = mk(), mk(), mk()
    try:
        tc.tc_step(a, 5)
        img = tc.tc_save_state(a)
        tc.tc_advance_substeps(a, 1)
        img_mid = tc.tc_save_state(a)
        tc.tc_advance_substeps(a, 2)
        tc.tc_step(a, 4)
        tc.tc_load_state(b, img)
        tc.tc_step(b, 5)
        tc.tc_load_state(c, img_mid)
        tc.tc_advance_substeps(c, 2)
        tc.tc_step(c, 4)
        ga = gpu_state(a, 33, 24, 16)
        for h in (b, c):
            g = gpu_state(h, 33, 24, 16)
            for k in ga:
                assert np.array_equal(g[k], ga[k]), k
        sa, sb = tc.tc_torque_stats(a), tc.tc_torque_stats(b)
        assert abs(sa.pop("t") - sb.pop("t")) < 1e-15     # summed in another order
        assert sa == sb and sa["step"] == 10
        with pytest.raises(tc.TcError) as ex:
            tc.tc_load_state(b, img[:-8])
        assert ex.value.code == tc.TC_ERR_SIZE
        bad = bytearray(img)
        bad[0:8] = b"XXXXXXXX"
        with pytest.raises(tc.TcError) as ex:
            tc.tc_load_state(b, bytes(bad))
        assert ex.value.code == tc.TC_ERR_ARG
    finally:
        for h in (a, b, c):
            tc.tc_destroy(h)
    # another shape: refused
    h = gpu_case(33, 32, 32, 0.8, 600.0, -50.0, 2e-3)
    try:
        with pytest.raises(tc.TcError):
            tc.tc_load_state(h, img)
    finally:
        tc.tc_destroy(h)


@pytest.mark.parametrize("name", ["tc-129x128x128", "tc-257x512x512"])
def test_physical_transform_matches_cufft(name):
    """The z and theta transforms against cuFFT (torch.fft on the device):
    the physical field u(theta_p, z_q) = sum u^ exp(i(m theta_p + alpha z_q))
    of tc_get_field(PHYSICAL) equals irfft2 of the zero-padded spectrum."""
    torch = pytest.importorskip("torch")
    from paper_0711_1429_gb300.synthetic import WORKLOADS
    w = WORKLOADS[name]
    Nr, Nt, Nz = w["Nr"], w["Ntheta"], w["Nz"]
    Nh, Mt, Mz = Nt // 2, 3 * Nt // 2, 3 * Nz // 2
    v, e = workload_inputs(name)
    h = gpu_case(Nr, Nt, Nz, w["zeta"], w["Re_i"], w["Re_o"], w["dt"], v=v, eta=e)
    try:
        tc.tc_step(h, 1)
        spec = torch.from_numpy(tc.tc_get_field(h, tc.TC_FIELD_U).reshape(Nr, Nz, Nh)).cuda()
        phys = tc.tc_get_field(h, tc.TC_FIELD_U, tc.TC_PHYSICAL).reshape(Nr, Mz, Mt)
    finally:
        tc.tc_destroy(h)
    X = torch.zeros((Nr, Mz, Mt // 2 + 1), dtype=torch.complex128, device="cuda")
    X[:, :Nz // 2, :Nh] = spec[:, :Nz // 2, :]
    X[:, Mz - Nz // 2 + 1:, :Nh] = spec[:, Nz // 2 + 1:, :]
    ref = (torch.fft.irfft2(X, s=(Mz, Mt)) * (Mz * Mt)).cpu().numpy()
    assert relerr(phys, ref) < 1e-12
