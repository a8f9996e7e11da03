"""The reference arm of bench.py (`--impl reference`): the FP64 oracle timed on
the host cores on a bounded sample of the benchmark workload, printed as the
same JSON line as the CUDA arm (no GPU)."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_json_line():
    from paper_1602_02306_gb300 import workloads
    # the 64^3 Hamiltonian keeps this CPU test short; the default workload
    # (2M-row power-law CSR) runs the same code
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--ref-probes", "4",
                        "--workload", "fd64"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    W = workloads.WORKLOADS["fd64"]()
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cfg = d["config"]
    assert cfg["workload"] == W.name and cfg["n"] == W.n
    assert cfg["shifts"] == len(W.shifts) and cfg["probes_per_shift"] == W.nprobe
    assert cfg["lanczos_steps_max"] == W.maxsteps
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert 1 <= cb["cores"] <= (os.cpu_count() or 1) and "4 probes" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # probe-steps over the sample: 2 shifts x 4 probes x 30 steps in ms_per_step
    assert d["value"] == pytest.approx(2 * 4 * 30 / (d["ms_per_step"] / 1e3), rel=0.02)


def test_default_workload_is_the_largest_single_gpu_config():
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'ap.add_argument("--workload", default="powerlaw2m")' in src
    from paper_1602_02306_gb300 import workloads
    W = workloads.WORKLOADS["powerlaw2m"]()
    assert W.n == 2_000_000 and W.nprobe == 128 and W.maxsteps == 50 and len(W.shifts) == 2


def test_reference_arm_on_other_ranks_prints_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""
