"""Shared helpers of the GPU tests: build the same case on the GPU (through
the C ABI) and in the oracle, from the same seeded inputs."""
import os

import numpy as np

import paper_0711_1429_gb300 as tc
from paper_0711_1429_gb300 import build as tcbuild
from paper_0711_1429_gb300.synthetic import WORKLOADS, initial_perturbation, box_defaults


def ensure_lib():
    if not os.path.exists(tc.LIB_PATH):
        tcbuild.build()
    return tc.lib()


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def inputs(Nr, Ntheta, Nz, zeta, seed, spectrum="box", amp=1e-3, **kw):
    m0, a0, rc = box_defaults(zeta)
    return initial_perturbation(Nr, Ntheta, Nz, seed, spectrum, amp, m0=m0, alpha0=a0, rc=rc, **kw)


def workload_inputs(name):
    w = WORKLOADS[name]
    return inputs(w["Nr"], w["Ntheta"], w["Nz"], w["zeta"], w["seed"], w["spectrum"], w["amp"])


def gpu_case(Nr, Ntheta, Nz, zeta, Re_i, Re_o, dt, v=None, eta=None, precision=tc.TC_PREC_FP64, **kw):
    ensure_lib()
    h = tc.tc_create_ex(Nr, Ntheta, Nz, zeta, Re_i, Re_o, dt, precision=precision, **kw)
    if v is not None:
        tc.tc_set_field(h, tc.TC_FIELD_V, v)
    if eta is not None:
        tc.tc_set_field(h, tc.TC_FIELD_ETA, eta)
    return h


def gpu_state(h, Nr, Nz, Nh):
    g = lambda which: tc.tc_get_field(h, which).reshape(Nr, Nz, Nh)
    return {"v": g(tc.TC_FIELD_V), "eta": g(tc.TC_FIELD_ETA), "u": g(tc.TC_FIELD_U),
            "w": g(tc.TC_FIELD_W), "U": tc.tc_get_field(h, tc.TC_FIELD_MEAN_U),
            "W": tc.tc_get_field(h, tc.TC_FIELD_MEAN_W)}


def oracle_state(s):
    u, v, w = s.velocity()
    return {"v": s.v, "eta": s.eta, "u": u, "w": w, "U": s.U, "W": s.W}


def compare(gs, os_, keys=("v", "eta", "u", "w", "U", "W")):
    return {k: relerr(gs[k], os_[k]) for k in keys}
