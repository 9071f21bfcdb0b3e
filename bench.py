#!/usr/bin/env python
"""Benchmark: grid-point Runge-Kutta steps per second of the Taylor-Couette
DNS step on GB300, through the libtc C ABI.

Default workload: tc-257x512x512 (radius ratio 0.883, Re_i = 3000, Nr = 257,
Ntheta = Nz = 512 Fourier modes, 768 x 768 dealiased planes), float64,
seeded k^-2 perturbation on circular Couette flow.  One step = 3 RK substeps
over the whole state (about 24 GB on the device, far larger than L2, so no L2
flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference      # the CPU oracle on a bounded sample

Under torchrun each rank runs an independent replica (the method does not
shard across GPUs here: "replicas only"); value = all ranks' grid-point
steps / max over ranks of the timed region.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point RK-steps/s"
UNIT = "gridpoint-steps/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--workload", default="tc-257x512x512")
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "df64"])
    p.add_argument("--e2e-steps", type=int, default=10)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the other precision forms")
    p.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    p.add_argument("--sample-planes", type=int, default=4)
    p.add_argument("--sample-pairs", type=int, default=1024)
    p.add_argument("--sample-repeat", type=int, default=1)
    p.add_argument("--ncases", type=int, default=64, help="batch64: number of cases")
    p.add_argument("--serve-seconds", type=float, default=2.0, help="served: arrival window (s)")
    p.add_argument("--serve-rate", type=float, default=20.0, help="served: Poisson rate (1/s)")
    p.add_argument("--budget-gb", type=float, default=150.0, help="served: device budget")
    p.add_argument("--torque-steps", type=int, default=500,
                   help="steps of the torque run of the fp64 and mixed forms (0: none)")
    p.add_argument("--no-many-cases", action="store_true", help="skip the batch64 and served results")
    p.add_argument("--nr", type=int, default=0,
                   help="radial points instead of the workload's (profiling captures of the per-pair "
                        "kernels at the full pair count with a smaller device footprint)")
    p.add_argument("--column-groups", type=int, default=0,
                   help="pin the column groups of the step graph (0: chosen by timing)")
    p.add_argument("--line-variant", type=int, default=0,
                   help="pin the line-kernel variant (0: chosen by timing; the launch shape changes no bits)")
    p.add_argument("--ztile", type=int, default=0,
                   help="pin the z tile of the z kernels (0: chosen by timing)")
    p.add_argument("--rk-deferral", type=int, default=-1, choices=[-1, 0, 1],
                   help="pin the deferred RK memory of the df64 and mixed forms (-1: chosen by timing)")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    def __init__(self, world, rank, backend):
        self.world, self.rank = world, rank
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per launch (the roofline numerators)
def algorithmic(w, prec):
    """FLOPs and bytes per launch of each kernel of the step, counted for the
    work the method needs in this formulation: a complex FFT of length M is
    5 M log2 M flops, a real one half of that; per substep the theta rows
    transform 3 real fields back (u, v, w) and 5 real products forward
    (uu - vv, uv, uw, vw, ww - vv), and the z direction 3 + 5 complex
    columns per retained azimuthal index."""
    import math
    Nr, Nt, Nz = w["Nr"], w["Ntheta"], w["Nz"]
    Nh, Mt, Mz = Nt // 2, 3 * Nt // 2, 3 * Nz // 2
    f = lambda M: 5.0 * M * math.log2(M)
    cb = 8 if prec == "mixed" else 16           # bytes of one complex intermediate
    P = Nr * Nz * Nh
    npr = 5
    return {
        "z_inverse": {"flops": 3 * Nr * Nh * f(Mz), "bytes": 3 * P * 16 + 3 * Nr * Mz * Nh * cb},
        "theta_rows_products": {"flops": Nr * Mz * (8 * 0.5 * f(Mt) + 9 * Mt),
                                "bytes": 3 * Nr * Mz * Nh * cb + npr * Nr * Mz * Nh * cb},
        "z_forward": {"flops": npr * Nr * Nh * f(Mz), "bytes": npr * Nr * Mz * Nh * cb + npr * P * cb},
        # line: products, u, v, w, H (read+write), new v, eta, u, w, LU, L and c tables
        "line": {"flops": None, "bytes": P * (npr * cb + 48 + 64 + 64 + 120 + 16)},
        "mean": {"flops": None, "bytes": Nr * 8 * 12},
    }


# ---------------------------------------------------------------------------
def cpu_sample(args):
    """Time the oracle (as it stands) on a bounded sample of the workload and
    extrapolate to grid-point steps per second.  The sample builds only what
    it times, so that one process per core fits in host memory:
      * plane phase: the products with the 3/2 rule (inverse transforms of u,
        v, w, the six products, forward transforms and truncation) on
        `sample_planes` radial planes of the workload's Ntheta x Nz grid;
      * line phase: reconstruction, explicit rows, right sides and banded
        solves of one substep for every pair of a case with the workload's
        radial grid (Nr, radius ratio, Re) and a small Fourier box of about
        `sample_pairs` pairs; the oracle's per-pair work does not depend on
        the pair's wavenumbers.
    Both are repeated `sample_repeat` times; one step of the workload costs
    3 (Nr t_plane + npairs t_pair)."""
    import math
    import numpy as np
    from oracle.grid import Case
    from oracle.rk import OracleSolver
    from oracle.fourier import products
    from paper_0711_1429_gb300.synthetic import WORKLOADS, initial_perturbation, box_defaults
    w = WORKLOADS[args.workload]
    cs = Case(w["Nr"], w["Ntheta"], w["Nz"], w["zeta"], w["Re_i"], w["Re_o"], w["dt"])
    m0, a0, rc = box_defaults(w["zeta"])
    K = min(args.sample_planes, cs.Nr)
    vp, ep = initial_perturbation(K + 2, w["Ntheta"], w["Nz"], w["seed"], w["spectrum"], w["amp"],
                                  m0=m0, alpha0=a0, rc=rc)
    vp, ep = vp[1:-1], ep[1:-1]
    side = 1 << max(2, int(round(math.log2(max(4, args.sample_pairs)) / 2)))
    cl = Case(w["Nr"], 2 * side, side, w["zeta"], w["Re_i"], w["Re_o"], w["dt"])
    vl, el = initial_perturbation(cl.Nr, cl.Ntheta, cl.Nz, w["seed"], w["spectrum"], w["amp"],
                                  m0=m0, alpha0=a0, rc=rc)
    s = OracleSolver(cl)
    s.set_fields(v=vl, eta=el)
    npairs = len(s.act[0])
    P = {k: np.zeros_like(vl) for k in ("uu", "uv", "uw", "vv", "vw", "ww")}
    t_plane = t_pair = 0.0
    reps = max(1, args.sample_repeat)
    for _ in range(reps):
        t0 = time.perf_counter()
        products(cs, vp, vp, ep)
        t_plane += (time.perf_counter() - t0) / K / reps
        t0 = time.perf_counter()
        s.advance(0, s.explicit_terms(P))
        t_pair += (time.perf_counter() - t0) / npairs / reps
    total_pairs = int(cs.active_mask().sum())
    t_step = 3.0 * (cs.Nr * t_plane + total_pairs * t_pair)
    return {"value": cs.gridpoints / t_step, "t_step_s": t_step, "t_plane_s": t_plane,
            "t_pair_s": t_pair, "planes": K, "pairs": npairs, "repeat": reps,
            "sample": f"oracle plane phase on {K} radial planes of {w['Ntheta']} x {w['Nz']} modes and line "
                      f"phase on the {npairs} pairs of a {cl.Ntheta} x {cl.Nz}-mode case with the same "
                      f"{cs.Nr}-point radial grid, one substep each, repeated {reps} times, extrapolated to a "
                      f"full 3-substep step of {args.workload} ({cs.Nr} planes, {total_pairs} pairs)"}


def _sample_cmd(args):
    return [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--workload", args.workload,
            "--sample-planes", str(args.sample_planes), "--sample-pairs", str(args.sample_pairs),
            "--sample-repeat", str(args.sample_repeat)]


def _sample_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        env.pop(k, None)
    return env


def run_cpu_sample_subprocess(args):
    """One oracle process, one thread."""
    p = subprocess.run(_sample_cmd(args), capture_output=True, text=True, env=_sample_env())
    if p.returncode != 0:
        raise RuntimeError(p.stderr[-2000:])
    res = json.loads(p.stdout.strip().splitlines()[-1])
    res["cores"] = 1
    return res


def run_cpu_sample_all_cores(args, ncores=None):
    """One single-threaded oracle process per host core, all at once, each on
    the sample above.  The oracle's planes and pairs are independent, so the
    cores would share a step's work; the rate of all cores together is
    ncores x gridpoints / (the slowest process's extrapolated step time)."""
    ncores = ncores or os.cpu_count() or 1
    procs = [subprocess.Popen(_sample_cmd(args), stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=_sample_env()) for _ in range(ncores)]
    res = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    t_max = max(r["t_step_s"] for r in res)
    gp = res[0]["value"] * res[0]["t_step_s"]
    return {"value": ncores * gp / t_max, "t_step_s": t_max / ncores, "cores": ncores,
            "per_process_t_step_s": [round(r["t_step_s"], 3) for r in res],
            "sample": res[0]["sample"] + f"; {ncores} such processes at once, one per core"}


def state_bytes_floor(w):
    """Bytes of the six spectral fields every form keeps resident (v, eta, u,
    w and the two RK memories), a lower bound of the step's working set."""
    P = w["Nr"] * w["Nz"] * (w["Ntheta"] // 2)
    return 6 * P * 16


def config_of(args, w, world):
    """The config dict of the bench line, shared by both arms."""
    sb = state_bytes_floor(w)
    name = args.workload if not getattr(args, "nr", 0) else f"{args.workload} with Nr = {args.nr}"
    return {"workload": name, "Nr": w["Nr"], "Ntheta": w["Ntheta"], "Nz": w["Nz"],
            "radius_ratio": w["zeta"], "Re_inner": w["Re_i"], "dt": w["dt"],
            "precision": args.precision, "parallelism": f"replicas{world}",
            "l2": (f"inputs larger than L2 (resident spectral state >= {sb / 1e9:.1f} GB), not flushed"
                   if sb > 129e6 else "state may fit in L2 (not flushed)")}


# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle on the machine's host cores: every step is one all-core sample
    (one process per core, as above), extrapolated to a full step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_0711_1429_gb300.synthetic import WORKLOADS
    w = WORKLOADS[args.workload]
    vals = []
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        r = run_cpu_sample_all_cores(args)
        if i >= args.warmup:
            vals.append(r)
    wall = time.perf_counter() - t_all
    t_step = statistics.mean(x["t_step_s"] for x in vals)
    value = (w["Nr"] * w["Ntheta"] * w["Nz"]) / t_step
    cores = vals[0]["cores"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_of(args, w, world),
            "extrapolated": True,
            "extrapolation": (f"each of the {args.steps} timed steps is one sample of the oracle on all "
                              f"{cores} host cores (per process: one substep of the plane phase on "
                              f"{args.sample_planes} planes and of the line phase on ~{args.sample_pairs} "
                              f"pairs), scaled to the full 3-substep step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
def warmup_steps(args):
    return max(args.warmup, 5)


def e2e_pipelined(args, tc, torch, h, v, e, gp, world, dist, local):
    """The metric end to end through the public API with host buffers.  Every
    step: the state v, eta in from page-locked host memory, one step, v, eta
    out to page-locked host memory, and the torque statistics.  The copies are
    pipelined as a data loader does: while step i runs, the input of step
    i + 1 crosses the host link into a device staging buffer (its own
    stream) and the result of step i - 1 crosses back from another; before
    the step, tc_set_field_async loads the staged input into the state
    (device to device), and after it tc_get_field_async copies the state
    into the outgoing staging buffer.  Setting the state restarts the RK
    memory, so each step also runs k_init."""
    import numpy as np
    nb = tc.tc_field_bytes(h, tc.TC_FIELD_V)
    n8 = nb // 8
    stream = torch.cuda.current_stream()            # the handle's launch stream
    pin = {k: torch.empty(n8, dtype=torch.float64, pin_memory=True) for k in ("vi", "ei", "vo", "eo")}
    pin["vi"].numpy().view(np.complex128)[:] = v.ravel()
    pin["ei"].numpy().view(np.complex128)[:] = e.ravel()
    pin["vo"].zero_()
    pin["eo"].zero_()
    stage = {k: torch.empty(n8, dtype=torch.float64, device=f"cuda:{local}") for k in ("vi", "ei", "vo", "eo")}
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: torch.cuda.Event() for k in ("in_ready", "in_free", "out_ready", "out_free")}
    torch.cuda.synchronize()

    def upload():                                   # host -> staging, once the last input was loaded
        s_in.wait_event(ev["in_free"])
        with torch.cuda.stream(s_in):
            stage["vi"].copy_(pin["vi"], non_blocking=True)
            stage["ei"].copy_(pin["ei"], non_blocking=True)
        ev["in_ready"].record(s_in)

    def download():                                 # staging -> host, during the next step
        s_out.wait_event(ev["out_ready"])
        with torch.cuda.stream(s_out):
            pin["vo"].copy_(stage["vo"], non_blocking=True)
            pin["eo"].copy_(stage["eo"], non_blocking=True)
        ev["out_free"].record(s_out)

    def run(k):
        ev["in_free"].record(stream)
        ev["out_free"].record(stream)
        upload()
        stats = None
        for i in range(k):
            stream.wait_event(ev["in_ready"])
            tc.tc_set_field_async(h, tc.TC_FIELD_V, stage["vi"].data_ptr(), nb)
            tc.tc_set_field_async(h, tc.TC_FIELD_ETA, stage["ei"].data_ptr(), nb)
            ev["in_free"].record(stream)
            if i + 1 < k:
                upload()                            # the next step's input, during this step
            tc.tc_step(h, 1)
            stream.wait_event(ev["out_free"])
            tc.tc_get_field_async(h, tc.TC_FIELD_V, stage["vo"].data_ptr(), nb)
            tc.tc_get_field_async(h, tc.TC_FIELD_ETA, stage["eo"].data_ptr(), nb)
            ev["out_ready"].record(stream)
            download()                              # this step's result, during the next step
            stats = tc.tc_torque_stats(h)
        s_out.synchronize()
        return stats

    run(1)                                          # untimed warm-up of the pipeline
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stats = run(args.e2e_steps)
    wall = dist.max(time.perf_counter() - t0)
    ok = bool(np.isfinite(pin["vo"].numpy()).all()) and float(np.abs(pin["vo"].numpy()).max()) > 0
    return {"value": gp * args.e2e_steps * world / wall, "unit": UNIT,
            "h2d_bytes_per_step": 2 * nb, "d2h_bytes_per_step": 2 * nb + ctypes.sizeof(tc.tc_stats),
            "steps": args.e2e_steps, "torque_inner": stats["G_inner"], "ms_per_step": 1e3 * wall / args.e2e_steps,
            "pipelined": "host copies of step i+1's input and step i-1's result overlap step i (device staging buffers)",
            "result_read_back": ok}


def time_form(tc, torch, w, prec, v, e, args, local, dist, measure_clocks=False, torque_steps=0):
    """Create the case in one precision form, warm up, time K steps with CUDA
    events on the launch stream, then time each kernel (tc_phase_times).
    With torque_steps > 0, the state is then reset to the initial condition
    and run for torque_steps steps, recording the torques after every step
    (outside the timed region)."""
    Nr, Nt, Nz = w["Nr"], w["Ntheta"], w["Nz"]
    h = tc.tc_create_ex(Nr, Nt, Nz, w["zeta"], w["Re_i"], w["Re_o"], w["dt"], precision=prec, device=local,
                        autotune=1)
    stream = torch.cuda.current_stream()
    tc.tc_set_stream(h, stream.cuda_stream)
    tc.tc_set_field(h, tc.TC_FIELD_V, v)
    tc.tc_set_field(h, tc.TC_FIELD_ETA, e)
    W0 = tc.tc_get_field(h, tc.TC_FIELD_MEAN_W)
    if args.column_groups or args.line_variant or args.ztile:
        tc.tc_set_tiles(h, args.ztile, args.line_variant, args.column_groups)
    if args.rk_deferral >= 0:
        tc.tc_set_rk_deferral(h, args.rk_deferral)
    # warm-up steps (the first call of five or more steps also runs the
    # autotuner's timed choice of column groups and RK-memory deferral)
    tc.tc_step(h, warmup_steps(args))
    torch.cuda.synchronize()
    clocks = ClockSampler(local) if measure_clocks else None
    dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    # the timed region: K steps in one call, CUDA events on the launch stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    tc.tc_step(h, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop() if clocks else None
    total_ms = dist.max(ev0.elapsed_time(ev1))
    # per-step latency: K more steps, one call each (outside the timed region)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for i in range(args.steps):
        tc.tc_step(h, 1)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps))
    state = {"v": tc.tc_get_field(h, tc.TC_FIELD_V), "eta": tc.tc_get_field(h, tc.TC_FIELD_ETA),
             "W": tc.tc_get_field(h, tc.TC_FIELD_MEAN_W), "U": tc.tc_get_field(h, tc.TC_FIELD_MEAN_U)}
    torque = tc.tc_torque_stats(h)
    ph = tc.tc_phase_times(h, 1)
    series = None
    if torque_steps > 0:
        import numpy as np
        tc.tc_set_field(h, tc.TC_FIELD_V, v)
        tc.tc_set_field(h, tc.TC_FIELD_ETA, e)
        tc.tc_set_field(h, tc.TC_FIELD_MEAN_W, W0)
        tc.tc_set_field(h, tc.TC_FIELD_MEAN_U, np.zeros_like(W0))
        series = {"G_inner": [], "G_outer": [], "energy": []}
        for _ in range(torque_steps):
            tc.tc_step(h, 1)
            st = tc.tc_torque_stats(h)
            for k in series:
                series[k].append(st[k])
    zt, lv, ch = tc.tc_get_tiles(h)
    shapes = {"ztile": zt, "line_variant": lv, "column_groups": ch, "rk_memory_deferred": tc.tc_get_rk_deferral(h)}
    return h, {"total_ms": total_ms, "per": per, "clk": clk, "state": state, "phase_ms": ph,
               "torque": torque, "series": series, "launch_shapes": shapes}


def torque_summary(series):
    import numpy as np
    g, go = np.array(series["G_inner"]), np.array(series["G_outer"])
    return {"steps": len(g), "G_inner_mean": float(g.mean()), "G_outer_mean": float(go.mean()),
            "G_inner_first": float(g[0]), "G_inner_last": float(g[-1]),
            "energy_last": float(series["energy"][-1])}


# DRAM bytes per z row of k_rows<double> (Ntheta = 512, Mt = 768): one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the current
# kernel on the paper workload 129 x 512 x 170, 32895 rows per launch; the
# per-row traffic does not depend on Nr or Nz.
ROWS_FP64_BYTES_PER_ROW = {512: (404781824 + 630402816) / 32895}
ROWS_FP64_CAPTURE_CURRENT = True


def roofline_of(w, prec_name, ph, peaks):
    alg = algorithmic(w, prec_name)
    dom = max(ph, key=ph.get)
    meas_peaks = {}
    try:
        meas_peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = meas_peaks.get("hbm_gbs")
    a = alg[dom]
    t = ph[dom] * 1e-3
    if a["flops"] is not None:
        pk = peaks["fp64_tflops"] if prec_name == "fp64" else peaks["fp32_tflops"]
        roof = {"bound": "alu", "achieved": a["flops"] / t / 1e12, "peak": pk, "unit": "TFLOP/s",
                "frac": a["flops"] / t / 1e12 / pk, "traffic": None, "kernel": dom,
                "peak_source": ("measured FP64 FMA probe (tc_fma_peak) in this run" if prec_name == "fp64"
                                else "measured FP32 FMA probe (tc_fma_peak) in this run"),
                "hbm_gbs_of_kernel": a["bytes"] / t / 1e9}
    else:
        roof = {"bound": "hbm", "achieved": a["bytes"] / t / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": (a["bytes"] / t / 1e9 / hbm) if hbm else None, "traffic": None,
                "kernel": dom, "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst)",
                "note": "the line kernel is float64-issue-bound (ncu); bytes/time is reported against HBM"}
    if dom == "theta_rows_products" and prec_name == "fp64" and w["Ntheta"] in ROWS_FP64_BYTES_PER_ROW:
        rows = w["Nr"] * 3 * w["Nz"] // 2
        scaled = ROWS_FP64_BYTES_PER_ROW[w["Ntheta"]] * rows
        src = "ncu dram bytes per row of k_rows<double> on paper-129x512x170, scaled by rows"
        if ROWS_FP64_CAPTURE_CURRENT:
            roof["traffic"] = scaled
            roof["traffic_source"] = src
        else:
            roof["traffic_last_capture"] = {"bytes": scaled, "source": src + ", taken before the kernel's "
                                            "last change (forward plan order, products' scale factor)"}
    roof["phase_ms"] = ph
    return roof


def workload_of(args):
    from paper_0711_1429_gb300.synthetic import WORKLOADS
    w = dict(WORKLOADS[args.workload])
    if args.nr:
        w["Nr"] = args.nr
    return w


def run_gpu(args):
    import numpy as np
    import torch
    import paper_0711_1429_gb300 as tc
    from paper_0711_1429_gb300.synthetic import WORKLOADS, initial_perturbation, box_defaults

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist(world, rank, "nccl")
    if not os.path.exists(tc.LIB_PATH):
        from paper_0711_1429_gb300 import build as b
        b.build()
    w = workload_of(args)
    PREC = {"fp64": tc.TC_PREC_FP64, "mixed": tc.TC_PREC_MIXED, "df64": tc.TC_PREC_DF64}
    DTYPE = {"fp64": "f64", "mixed": "f32+f64", "df64": "f32x2+f64"}
    Nr, Nt, Nz = w["Nr"], w["Ntheta"], w["Nz"]
    gp = Nr * Nt * Nz
    m0, a0, rc = box_defaults(w["zeta"])
    v, e = initial_perturbation(Nr, Nt, Nz, w["seed"] + rank, w["spectrum"], w["amp"], m0=m0, alpha0=a0, rc=rc)
    peaks = tc.tc_fma_peak(local)

    # the torque run is a one-GPU diagnostic of the headline workload
    tq = args.torque_steps if args.precision in ("fp64", "mixed") and world == 1 else 0
    h, main = time_form(tc, torch, w, PREC[args.precision], v, e, args, local, dist, measure_clocks=True,
                        torque_steps=tq)
    value = gp * args.steps * world / (main["total_ms"] / 1e3)
    per = main["per"]
    p50 = statistics.median(per)
    p99 = per[min(len(per) - 1, int(round(0.99 * (len(per) - 1))))]
    roof = roofline_of(w, args.precision, main["phase_ms"], peaks)

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if args.e2e_steps > 0:
        e2e = e2e_pipelined(args, tc, torch, h, v, e, gp, world, dist, local)
    device_bytes = tc.tc_device_bytes(h)
    shapes = main["launch_shapes"]
    tc.tc_destroy(h)

    # ---- the other precision forms, same input and step count; error against this run
    forms = {}
    series = {args.precision: main["series"]} if main["series"] else {}
    if not args.no_forms:
        ref = main["state"]
        for name in [p for p in ("df64", "mixed", "fp64") if p != args.precision]:
            hf, res = time_form(tc, torch, w, PREC[name], v, e, args, local, dist,
                                torque_steps=args.torque_steps if name in ("fp64", "mixed") and world == 1 else 0)
            tc.tc_destroy(hf)
            if res["series"]:
                series[name] = res["series"]
            err = {k: float(np.linalg.norm(res["state"][k] - ref[k]) / np.linalg.norm(ref[k]))
                   for k in ("v", "eta", "W")}
            err["U"] = float(np.linalg.norm(res["state"]["U"] - ref["U"]) / max(np.linalg.norm(ref["U"]), 1e-300))
            err["torque_inner"] = abs(res["torque"]["G_inner"] - main["torque"]["G_inner"]) / main["torque"]["G_inner"]
            rper = res["per"]
            forms[name] = {"value": gp * args.steps * world / (res["total_ms"] / 1e3), "unit": UNIT,
                           "ms_per_step": res["total_ms"] / args.steps, "dtype": DTYPE[name],
                           "latency_ms": {"p50": statistics.median(rper),
                                          "p99": rper[min(len(rper) - 1, int(round(0.99 * (len(rper) - 1))))]},
                           "rel_l2_error_vs_" + args.precision: err,
                           "launch_shapes": res["launch_shapes"],
                           "roofline": roofline_of(w, name, res["phase_ms"], peaks)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import argparse as _ap
        sargs = _ap.Namespace(**vars(args))
        sargs.sample_repeat = max(args.sample_repeat, 3)
        try:
            allc = run_cpu_sample_all_cores(sargs)
            one = run_cpu_sample_subprocess(sargs)
            cpu = {"value": allc["value"], "unit": UNIT, "cores": allc["cores"], "kind": "oracle",
                   "sample": allc["sample"],
                   "single_core": {"value": one["value"], "unit": UNIT, "cores": 1, "sample": one["sample"]}}
        except Exception as ex:        # reported, not fatal
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "error": str(ex)[-300:]}

    # ---- the paper's own timed workload (Sec. 3.1: 182 s per step on one
    # 2.66 GHz Xeon, i.e. 129 x 512 x 170 / 182 = 6.17e4 grid-point steps/s)
    paper = None
    if not args.no_forms and args.workload == "tc-257x512x512":
        wp = WORKLOADS["paper-129x512x170"]
        vp, ep = initial_perturbation(wp["Nr"], wp["Ntheta"], wp["Nz"], wp["seed"], wp["spectrum"], wp["amp"],
                                      m0=box_defaults(wp["zeta"])[0], alpha0=box_defaults(wp["zeta"])[1],
                                      rc=box_defaults(wp["zeta"])[2])
        gpp = wp["Nr"] * wp["Ntheta"] * wp["Nz"]
        paper = {"workload": "paper-129x512x170", "paper_value": 6.17e4,
                 "paper_hardware": "1 x Intel Xeon 2.66 GHz (182 s per step, Sec. 3.1)", "forms": {}}
        for name in ("fp64", "df64", "mixed"):
            hp, res = time_form(tc, torch, wp, PREC[name], vp, ep, args, local, dist)
            tc.tc_destroy(hp)
            val = gpp * args.steps * world / (res["total_ms"] / 1e3)
            paper["forms"][name] = {"value": val, "ms_per_step": res["total_ms"] / args.steps,
                                    "vs_paper": val / 6.17e4, "dtype": DTYPE[name],
                                    "launch_shapes": res["launch_shapes"]}

    torque_run = None
    if "fp64" in series and "mixed" in series:
        import numpy as np
        gf, gm = np.array(series["fp64"]["G_inner"]), np.array(series["mixed"]["G_inner"])
        torque_run = {"what": f"inner/outer torque G (Eq. 2, Table 2 reading) after each of "
                              f"{len(gf)} steps from the initial condition, mean over the run",
                      "fp64": torque_summary(series["fp64"]), "mixed": torque_summary(series["mixed"]),
                      "rel_diff_G_inner_mean": float(abs(gm.mean() - gf.mean()) / gf.mean()),
                      "max_rel_diff_G_inner_per_step": float(np.max(np.abs(gm - gf) / gf))}

    many = None
    if not args.no_many_cases and args.workload == "tc-257x512x512" and world == 1:
        many = {"batch64": {}, "served": {}}
        for name in ("fp64", "mixed"):
            many["batch64"][name] = batch_measure(args, tc, torch, name, local, dist)
            many["served"][name] = served_measure(args, tc, torch, name, local)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": warmup_steps(args), "ms_per_step": main["total_ms"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": config_of(args, w, world), "device_bytes": device_bytes,
            "latency_ms": {"p50": p50, "p99": p99},
            "gpu_launches": tc.step_kernels(shapes["column_groups"], shapes["rk_memory_deferred"]) * args.steps,
            "launch_shapes": shapes,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": main["clk"],
            "alu_peaks_tflops": peaks, "forms": forms, "paper_workload": paper,
            "torque_run": torque_run, "many_cases": many}
    if rank == 0:
        print(json.dumps(line))
    dist.close()


# ---------------------------------------------------------------------------
# many cases on one GPU: the batched ensemble and the served stream
def ensemble_case(rng, i, prec, big_prob=0.0):
    """One case of the ensemble recipe: Nr ~ U{33..129}, Ntheta, Nz ~ U{32, 64,
    128} independently, zeta ~ U[0.7, 0.95], Re_i ~ U[500, 3000], k^-2
    perturbation of 0.05 rms with seed 1000 + i; with probability big_prob a
    257 x 256 x 256 case instead."""
    import paper_0711_1429_gb300 as tc
    if rng.random() < big_prob:
        Nr, Nt, Nz = 257, 256, 256
    else:
        Nr = int(rng.integers(33, 130))
        Nt, Nz = (int(x) for x in rng.choice([32, 64, 128], size=2))
    z = float(rng.uniform(0.7, 0.95))
    Re = float(rng.uniform(500.0, 3000.0))
    p = tc.make_params(Nr, Nt, Nz, z, Re, 0.0, 1e-3, precision=prec, autotune=1)
    return p, (Nr, Nt, Nz, z, 1000 + i)


def ensemble_ic(spec):
    from paper_0711_1429_gb300.synthetic import initial_perturbation, box_defaults
    Nr, Nt, Nz, z, seed = spec
    m0, a0, rc = box_defaults(z)
    return initial_perturbation(Nr, Nt, Nz, seed, "k2", 0.05, m0=m0, alpha0=a0, rc=rc)


def batch_measure(args, tc, torch, prec_name, local, dist):
    """The batched ensemble: args.ncases independent cases stepped together,
    K timed steps after W warm-up steps; returns the result dict."""
    import numpy as np
    world, rank, _ = dist_env()
    prec = {"fp64": tc.TC_PREC_FP64, "mixed": tc.TC_PREC_MIXED, "df64": tc.TC_PREC_DF64}[prec_name]
    rng = np.random.default_rng(1000 + rank)
    cases = [ensemble_case(rng, i, prec) for i in range(args.ncases)]
    for p, _ in cases:
        p.device = local
    b = tc.tc_batch_create([p for p, _ in cases])
    stream = torch.cuda.current_stream()
    tc.tc_batch_set_stream(b, stream.cuda_stream)
    gp = 0
    for i, (p, spec) in enumerate(cases):
        v, e = ensemble_ic(spec)
        h = tc.tc_batch_case(b, i)
        tc.tc_set_field(h, tc.TC_FIELD_V, v)
        tc.tc_set_field(h, tc.TC_FIELD_ETA, e)
        gp += p.Nr * p.Ntheta * p.Nz
    tc.tc_batch_step(b, max(args.warmup, 3))
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    dist.barrier()
    clocks.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for i in range(args.steps):
        tc.tc_batch_step(b, 1)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    per = sorted(ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps))
    total = dist.max(ev[0].elapsed_time(ev[args.steps]))
    launches = tc.tc_batch_launches_per_step(b)
    res = {"value": gp * args.steps * world / (total / 1e3), "unit": UNIT,
           "ms_per_step": total / args.steps, "steps": args.steps, "warmup": max(args.warmup, 3),
           "dtype": {"fp64": "f64", "mixed": "f32+f64", "df64": "f32x2+f64"}[prec_name],
           "cases": args.ncases, "gridpoints": gp, "device_bytes": tc.tc_batch_device_bytes(b),
           "latency_ms": {"p50": statistics.median(per),
                          "p99": per[min(len(per) - 1, int(round(0.99 * (len(per) - 1))))]},
           "gpu_launches": launches * args.steps, "clocks": clk}
    tc.tc_batch_destroy(b)
    return res


def run_batch(args):
    import torch
    import paper_0711_1429_gb300 as tc
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = Dist(world, rank, "nccl")
    r = batch_measure(args, tc, torch, args.precision, local, dist)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": r["warmup"], "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"], "data": "synthetic",
            "config": {"workload": f"batch{args.ncases}", "cases": args.ncases, "gridpoints": r["gridpoints"],
                       "precision": args.precision, "autotune": True},
            "device_bytes": r["device_bytes"], "latency_ms": r["latency_ms"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    if rank == 0:
        print(json.dumps(line))
    dist.close()


def served_measure(args, tc, torch, prec_name, local):
    """The served stream: Poisson arrivals over the window, each request
    submitted at its arrival time; returns the result dict."""
    import numpy as np
    world, rank, _ = dist_env()
    prec = {"fp64": tc.TC_PREC_FP64, "mixed": tc.TC_PREC_MIXED, "df64": tc.TC_PREC_DF64}[prec_name]
    rng = np.random.default_rng(7 + rank)
    # Poisson arrivals over the window, cases as the ensemble plus 5% 257 x 256 x 256
    t, arrivals = 0.0, []
    while True:
        t += rng.exponential(1.0 / args.serve_rate)
        if t > args.serve_seconds:
            break
        p, spec = ensemble_case(rng, len(arrivals), prec, big_prob=0.05)
        p.device = local
        arrivals.append((t, p, spec, int(rng.integers(50, 501))))
    ics = [ensemble_ic(spec) for _, _, spec, _ in arrivals]
    s = tc.tc_server_create(int(args.budget_gb * 1e9), max_active=256, device=local)
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    h2d = d2h = 0
    outs = []
    for (ta, p, spec, n), (v, e) in zip(arrivals, ics):
        dt_wait = ta - (time.perf_counter() - t0)
        if dt_wait > 0:
            time.sleep(dt_wait)
        ov, oe = np.empty_like(v.ravel()), np.empty_like(e.ravel())
        outs.append((ov, oe))
        tc.tc_server_submit(s, p, v, e, n, ov, oe)
        h2d += v.nbytes + e.nbytes
        d2h += ov.nbytes + oe.nbytes
    tc.tc_server_drain(s, 3600.0)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = tc.tc_server_stats(s)
    res = tc.tc_server_poll(s, 4096)
    tc.tc_server_destroy(s)
    bad = [r for r in res if r["status"] != tc.TC_OK]
    nsteps = sum(n for _, _, _, n in arrivals)
    return {"value": st["gridpoint_steps"] / (st["busy_ms"] / 1e3), "unit": UNIT,
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "df64": "f32x2+f64"}[prec_name],
            "requests": len(arrivals), "steps": int(st["steps"]), "rate_per_s": args.serve_rate,
            "mode": "per case: every admitted case on its own stream, one step in flight each",
            "window_s": args.serve_seconds, "budget_gb": args.budget_gb,
            "peak_active": st["peak_active"], "peak_used_gb": st["peak_used_bytes"] / 1e9,
            "within_budget": st["peak_used_bytes"] <= st["budget_bytes"], "failed": len(bad),
            "latency_ms": {"p50": st["step_ms_p50"], "p99": st["step_ms_p99"]},
            "busy_s": st["busy_ms"] / 1e3, "wall_s": wall,
            "e2e": {"value": st["gridpoint_steps"] / wall, "unit": UNIT,
                    "h2d_bytes_per_step": h2d / max(1, nsteps), "d2h_bytes_per_step": d2h / max(1, nsteps)},
            "clocks": clk}


def run_served(args):
    import torch
    import paper_0711_1429_gb300 as tc
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    r = served_measure(args, tc, torch, args.precision, local)
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": r["steps"],
            "warmup": 0, "ms_per_step": r["busy_s"] * 1e3 / max(1, r["steps"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": r["dtype"],
            "data": "synthetic",
            "config": {"workload": "served", "requests": r["requests"], "rate_per_s": args.serve_rate,
                       "window_s": args.serve_seconds, "budget_gb": args.budget_gb, "precision": args.precision},
            "peak_active": r["peak_active"], "peak_used_gb": r["peak_used_gb"], "failed": r["failed"],
            "latency_ms": r["latency_ms"], "e2e": r["e2e"], "clocks": r["clocks"], "wall_s": r["wall_s"]}
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    if args.cpu_sample:
        print(json.dumps(cpu_sample(args)))
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("batch"):
        run_batch(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
