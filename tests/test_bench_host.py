"""Host logic of bench.py (no GPU): the roofline of the dominant kernel class
from the launch list (span records of concurrent chunk groups included), the
latency-bound label for small problems, the ncu traffic record attached only
while the kernel source is the one captured, and the clock summary that
decides whether a run is kept."""
import json
import os
import shutil

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _Evc:
    KERNEL_NAMES = ["init", "jacobi", "stencil", "csr", "dots", "reduce", "update", "finish"]


def test_roofline_uses_span_records_and_counts_launches():
    # one step: a span (2 ms, 10 GB) over four untimed stencil launches, one dots launch
    recs = [(2, 1, 2.0, 10e9, 1)] + [(2, 1, -1.0, 2.5e9, 0)] * 4 + [(4, 1, 1.0, 6e9, 0)]
    roof, kinds = bench._roofline(_Evc, recs, 6800.0, "measured", "stencil_patch_kernel")
    assert roof["bound"] == "hbm" and roof["kernel"] == "stencil_patch_kernel"
    assert roof["achieved"] == pytest.approx(5000.0)          # 10 GB / 2 ms
    assert roof["frac"] == pytest.approx(5000.0 / 6800.0, abs=1e-4)
    assert roof["launches"] == 4 and kinds["stencil"]["launches"] == 4
    assert kinds["dots"]["GB/s"] == pytest.approx(6000.0)
    assert roof["share_of_step"] == pytest.approx(2.0 / 3.0, abs=1e-3)


def test_roofline_picks_the_class_with_the_most_time():
    recs = [(2, 1, 1.0, 5e9, 0), (6, 1, 1.5, 9e9, 0), (4, 1, 1.2, 7e9, 0)]
    roof, _ = bench._roofline(_Evc, recs, 6800.0, "measured")
    assert roof["kernel"] == "reorth_update_kernel"
    assert roof["achieved"] == pytest.approx(6000.0)


def test_latency_bound_class_has_no_bandwidth_roofline():
    recs = [(7, 40, 2.3, 0.0, 0), (4, 1, 0.5, 1e6, 0), (3, 1, 0.3, 1e6, 0)]
    roof, _ = bench._roofline(_Evc, recs, 6800.0, "measured")
    assert roof["bound"] == "latency"
    assert roof["achieved"] is None and roof["frac"] is None and roof["peak"] is None


def test_traffic_attached_only_while_the_source_matches(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "stencil_patch_fd64_traffic.json")))
    roof = {"kernel": "stencil_patch_kernel", "traffic": None}
    bench._attach_traffic(roof)
    assert roof["traffic"] == rec["dram_bytes"]
    assert roof["traffic_launch_algorithmic_bytes"] == rec["algorithmic_bytes"]
    assert rec["dram_bytes"] < 1.05 * rec["algorithmic_bytes"]     # no wasted re-reads
    # the same record against a changed source: no traffic
    fake = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "profiles"), fake / "profiles")
    src = fake / rec["source"]
    src.parent.mkdir(parents=True)
    src.write_text(open(os.path.join(ROOT, rec["source"])).read() + "\n// edited\n")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    roof2 = {"kernel": "stencil_patch_kernel", "traffic": None}
    bench._attach_traffic(roof2)
    assert roof2["traffic"] is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _row(sm, mx, hw="Not Active", thermal="Not Active", swth="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, thermal, swth, cap]


def test_clock_summary_flags_throttle_reasons(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    c = bench.ClockSampler(0)
    c.proc = _Proc()
    c.rows = [_row(2070, 2070), _row(2055, 2070, cap="Active"), _row(2070, 2070)]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    c.rows = [_row(1500, 2070, thermal="Active"), ["garbage"]]
    out = c.stop()
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["samples"] == 1
    c2 = bench.ClockSampler(0)
    assert c2.stop()["reasons"] == ["nvidia-smi unavailable"]
