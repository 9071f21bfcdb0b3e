"""The reference arm of bench.py (the CPU oracle timed on a bounded sample) on
CPU: the JSON line it prints, and its multi-rank behaviour (rank 0 alone runs
and prints; the other ranks exit 0 without work)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "tc-small-33x16x16", "--steps", "2", "--warmup", "1",
        "--sample-planes", "1", "--sample-pairs", "8"]


def _run(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + ARGS, cwd=ROOT,
                          capture_output=True, text=True, env=env, timeout=300)


def test_reference_arm_prints_one_contract_line():
    p = _run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == "grid-point RK-steps/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0
    # ms_per_step and value describe the same sampled step time
    gp = 33 * 16 * 16
    assert abs(line["value"] * line["ms_per_step"] / 1e3 - gp) < 1e-6 * gp
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] == (os.cpu_count() or 1) and cpu["value"] == line["value"]
    assert "1 radial planes of 16 x 16 modes" in cpu["sample"] and "one per core" in cpu["sample"]
    assert line["extrapolated"] is True
    # the same config keys and values as the GPU arm's line (bench.config_of)
    cfg = line["config"]
    assert cfg["workload"] == "tc-small-33x16x16" and cfg["Nr"] == 33 and cfg["Ntheta"] == 16 and cfg["Nz"] == 16
    assert cfg["precision"] == "fp64" and cfg["parallelism"] == "replicas1"
    assert set(cfg) == {"workload", "Nr", "Ntheta", "Nz", "radius_ratio", "Re_inner", "dt", "precision",
                        "parallelism", "l2"}
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""
