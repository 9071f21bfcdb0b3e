"""One case split across ranks (transpose form), host side, on the CPU.

The partition and the two exchanges of paper_0711_1429_gb300/split.py are
driven with the oracle as each rank's compute: the plane phase of a rank is
the oracle's products on its radial planes, its line phase the oracle's rows
and solves on its azimuthal columns (OracleSolver restricted to those
pairs), the mean flow on the rank that owns column 0.  The split step must
reproduce the unsplit oracle step bit for bit: in one process (the shares
exchanging by copies) for 2 and 3 ranks, and as two gloo ranks (the
exchanges through torch.distributed.all_to_all_single).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

from paper_0711_1429_gb300 import split as sp

CASE = dict(Nr=17, Ntheta=16, Nz=12, zeta=0.8, Re_i=400.0, Re_o=-50.0, dt=2e-3)
STEPS = 3


def _inputs():
    from paper_0711_1429_gb300.synthetic import initial_perturbation, box_defaults
    m0, a0, rc = box_defaults(CASE["zeta"])
    return initial_perturbation(CASE["Nr"], CASE["Ntheta"], CASE["Nz"], 17, "k2", 5e-2, m0=m0, alpha0=a0, rc=rc)


def _case():
    from oracle.grid import Case
    return Case(CASE["Nr"], CASE["Ntheta"], CASE["Nz"], CASE["zeta"], CASE["Re_i"], CASE["Re_o"], CASE["dt"])


def _f32(a):
    """float32-word view of a complex128 array, trailing axis of 4 words."""
    return torch.from_numpy(a.view(np.float32).reshape(a.shape + (4,)))


PRODUCTS = ("uu", "uv", "uw", "vv", "vw", "ww")


def oracle_share(plan, rank):
    """A rank's share with the oracle as its compute (arrays are numpy,
    viewed by the tensors the exchanges move)."""
    from oracle.rk import OracleSolver
    from oracle.fourier import products
    cs = _case()
    (r0, r1), (j0, j1) = plan.slabs[rank], plan.cols[rank]
    mask = np.zeros((cs.Nz, cs.Nh), dtype=bool)
    mask[:, j0:j1] = True
    s = OracleSolver(cs, pairs=mask)
    v0, e0 = _inputs()
    s.set_fields(v=v0 * mask, eta=e0 * mask)
    u, v, w = (np.ascontiguousarray(x) for x in s.velocity())
    prod = np.zeros((6, cs.Nr, cs.Nz, cs.Nh), dtype=np.complex128)
    slab = np.zeros((6, r1 - r0, cs.Nz, cs.Nh), dtype=np.complex128)
    arrays = {"u": _f32(u), "v": _f32(v), "w": _f32(w), "prod": _f32(prod), "prod_slab": _f32(slab)}

    def planes():
        P = products(cs, u[r0:r1], v[r0:r1], w[r0:r1])
        for i, k in enumerate(PRODUCTS):
            slab[i] = P[k]

    def pairs(k):
        P = {name: prod[i] for i, name in enumerate(PRODUCTS)}
        s.advance(k, s.explicit_terms(P))
        if k == 2:
            s.E_prev = None
            s.t += cs.dt
            s.steps += 1
        uu, vv, ww = s.velocity()
        for arr, new in ((u, uu), (v, vv), (w, ww)):
            arr[:, :, j0:j1] = new[:, :, j0:j1]

    sh = sp.Share(plan, rank, arrays, planes, pairs)
    sh.solver = s
    return sh


def reference():
    from oracle.rk import OracleSolver
    s = OracleSolver(_case())
    v0, e0 = _inputs()
    s.set_fields(v=v0, eta=e0)
    s.step(STEPS)
    return s


def _collect(plan, results):
    """Assemble v, eta from the ranks' own columns; U, W from the owner of
    column 0."""
    v = np.zeros_like(results[0]["v"])
    eta = np.zeros_like(v)
    for rank, r in enumerate(results):
        j0, j1 = plan.cols[rank]
        v[:, :, j0:j1] = r["v"][:, :, j0:j1]
        eta[:, :, j0:j1] = r["eta"][:, :, j0:j1]
    return v, eta, results[0]["U"], results[0]["W"]


def test_partition_covers_everything_once():
    for n, parts in ((17, 2), (17, 3), (257, 8), (8, 8)):
        rs = sp.balanced(n, parts)
        assert rs[0][0] == 0 and rs[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [b - a for a, b in rs]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        sp.balanced(3, 4)


@pytest.mark.parametrize("world", [2, 3])
def test_split_in_process_equals_unsplit_bit_for_bit(world):
    ref = reference()
    plan = sp.SplitPlan(CASE["Nr"], CASE["Ntheta"], CASE["Nz"], world)
    shares = [oracle_share(plan, r) for r in range(world)]
    for _ in range(STEPS):
        sp.step_in_process(shares)
    res = [{"v": s.solver.v, "eta": s.solver.eta, "U": s.solver.U, "W": s.solver.W} for s in shares]
    v, eta, U, W = _collect(plan, res)
    assert np.array_equal(v, ref.v) and np.array_equal(eta, ref.eta)
    assert np.array_equal(U, ref.U) and np.array_equal(W, ref.W)
    assert np.max(np.abs(ref.U)) > 0            # the mean flow moved


def test_split_with_a_dropped_exchange_differs():
    """The pin has teeth: skipping exchange A of the first substep (each rank
    keeps stale columns of the others) changes the result."""
    ref = reference()
    plan = sp.SplitPlan(CASE["Nr"], CASE["Ntheta"], CASE["Nz"], 2)
    shares = [oracle_share(plan, r) for r in range(2)]
    for s in shares:                            # first substep without exchange A
        s.planes()
    recvs = sp.exchange_in_process([sp.pack_to_pairs(plan, s.rank, s.a["prod_slab"]) for s in shares])
    for s in shares:
        sp.unpack_to_pairs(plan, s.rank, s.a["prod"], recvs[s.rank])
        s.pairs(0)
    for k in (1, 2):
        recvs = sp.exchange_in_process([sp.pack_to_planes(plan, s.rank, s.fields()) for s in shares])
        for s in shares:
            sp.unpack_to_planes(plan, s.rank, s.fields(), recvs[s.rank])
            s.planes()
        recvs = sp.exchange_in_process([sp.pack_to_pairs(plan, s.rank, s.a["prod_slab"]) for s in shares])
        for s in shares:
            sp.unpack_to_pairs(plan, s.rank, s.a["prod"], recvs[s.rank])
            s.pairs(k)
    for _ in range(STEPS - 1):
        sp.step_in_process(shares)
    res = [{"v": s.solver.v, "eta": s.solver.eta, "U": s.solver.U, "W": s.solver.W} for s in shares]
    v, eta, U, W = _collect(plan, res)
    assert not np.array_equal(v, ref.v)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = sp.SplitPlan(CASE["Nr"], CASE["Ntheta"], CASE["Nz"], world)
    sh = oracle_share(plan, rank)
    for _ in range(STEPS):
        sp.step_distributed(sh)
    q.put((rank, {"v": sh.solver.v, "eta": sh.solver.eta, "U": sh.solver.U, "W": sh.solver.W}))
    dist.barrier()
    dist.destroy_process_group()


def test_split_over_two_gloo_ranks_equals_unsplit_bit_for_bit():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = reference()
    plan = sp.SplitPlan(CASE["Nr"], CASE["Ntheta"], CASE["Nz"], 2)
    v, eta, U, W = _collect(plan, [got[0], got[1]])
    assert np.array_equal(v, ref.v) and np.array_equal(eta, ref.eta)
    assert np.array_equal(U, ref.U) and np.array_equal(W, ref.W)
