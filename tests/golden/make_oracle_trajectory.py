"""Writes the stored oracle trajectory of the 129 x 128 x 128 workload.

The oracle needs minutes per 129 x 128 x 128 step on one CPU core, so a
50-step comparison cannot recompute it inside the GPU test.  This script runs
the oracle (and only the oracle, from the seeded synthetic inputs) for the
workload "tc-129x128x128" -- radius ratio 0.883, Re_i = 3000, Nr = 129,
128 x 128 modes, dt = 1e-3, k^-2 perturbation of r.m.s. 0.05 -- and stores,
after 50 steps:

  * the radial lines of v, eta, u and w at a seeded sample of Fourier pairs
    (every radial point), plus fixed pairs at both ends of the spectrum;
  * the mean profiles U and W;
  * the torques G_i, G_o and the kinetic energy.

Run from the repository root:  python tests/golden/make_oracle_trajectory.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.grid import Case                                   # noqa: E402
from oracle.rk import OracleSolver                             # noqa: E402
from oracle import diagnostics as dg                           # noqa: E402
from paper_0711_1429_gb300.synthetic import WORKLOADS, initial_perturbation, box_defaults  # noqa: E402

NAME = "tc-129x128x128"
STEPS = 50
NSAMPLE = 44
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tc-129x128x128_50steps.npz")


def sample_pairs(cs, seed=12345):
    """(n-slot, j) of the stored lines: four fixed pairs (lowest and highest
    azimuthal and axial indices) and a seeded draw among the active pairs."""
    mask = cs.active_mask()
    fixed = [(1, 0), (0, 1), (cs.Nz // 2 - 1, cs.Nh - 1), (cs.Nz // 2 + 1, cs.Nh - 1)]
    act = np.argwhere(mask)
    rng = np.random.default_rng(seed)
    pick = act[rng.choice(len(act), size=NSAMPLE - len(fixed), replace=False)]
    pairs = fixed + [tuple(int(x) for x in p) for p in pick if tuple(p) not in fixed]
    return np.array(pairs[:NSAMPLE], dtype=np.int64)


def main():
    w = WORKLOADS[NAME]
    cs = Case(w["Nr"], w["Ntheta"], w["Nz"], w["zeta"], w["Re_i"], w["Re_o"], w["dt"])
    m0, a0, rc = box_defaults(w["zeta"])
    v0, e0 = initial_perturbation(w["Nr"], w["Ntheta"], w["Nz"], w["seed"], w["spectrum"], w["amp"],
                                  m0=m0, alpha0=a0, rc=rc)
    s = OracleSolver(cs)
    s.set_fields(v=v0, eta=e0)
    t0 = time.time()
    for k in range(STEPS):
        s.step(1)
        print(f"step {k + 1}/{STEPS}  {time.time() - t0:.0f} s", flush=True)
    u, v, w_ = s.velocity()
    pairs = sample_pairs(cs)
    lines = {name: F[:, pairs[:, 0], pairs[:, 1]] for name, F in
             (("v", s.v), ("eta", s.eta), ("u", u), ("w", w_))}
    Gi, Go = dg.torque(cs, s.S, s.W)
    E = dg.kinetic_energy(cs, u, v, w_)
    np.savez_compressed(OUT, workload=NAME, steps=STEPS, pairs=pairs, U=s.U, W=s.W,
                        G_inner=Gi, G_outer=Go, energy=E, **lines)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
