"""Host logic of bench.py (no GPU): the roofline of the dominant kernel class
from the launch list (span records of concurrent chunk groups included), the
latency-bound label for small problems, the ncu traffic record attached only
while the kernel source is the one captured, and the clock summary that
decides whether a run is kept."""
import json
import os
import shutil

import numpy as np
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


class _W:
    name = "toy_workload"


def _fake_repo(tmp_path, body):
    fake = tmp_path / "repo"
    (fake / "profiles").mkdir(parents=True)
    (fake / "k").mkdir()
    (fake / "k" / "toy.cu").write_text(body)
    return fake


_SRC = """// toy kernels
struct Args { int n; };

__device__ float helper(float x) { return 2.0f * x; }

template <typename T>
__global__ void __launch_bounds__(128)
toy_kernel(Args a)
{
    if (a.n) { float y = helper(1.0f); (void)y; }
}

void host_launch(Args a) { toy_kernel<float><<<1, 1>>>(a); helper(3.0f); }
"""


def test_function_text_finds_definitions_not_calls():
    t = bench._function_text(_SRC, "toy_kernel")
    assert t.startswith("template <typename T> __global__ void __launch_bounds__(128) toy_kernel(Args a)")
    assert t.endswith("}")
    assert bench._function_text(_SRC, "helper").startswith("__device__ float helper(float x)")
    assert bench._function_text(_SRC, "struct Args") == "struct Args { int n; }"
    with pytest.raises(KeyError):
        bench._function_text(_SRC, "missing_kernel")


def test_traffic_attached_only_while_the_device_code_matches(tmp_path, monkeypatch):
    fake = _fake_repo(tmp_path, _SRC)
    monkeypatch.setattr(bench, "ROOT", str(fake))
    spec = [["k/toy.cu", ["struct Args", "helper", "toy_kernel"]]]
    rec = {"kernel": "toy_kernel", "device_code": spec,
           "device_code_sha256": bench._device_code_sha(spec),
           "launch": "toy", "dram_bytes": 90.0, "algorithmic_bytes": 100.0, "profile": "p.md"}
    (fake / "profiles" / "toy_kernel_toy_workload_traffic.json").write_text(json.dumps(rec))
    roof = {"kernel": "toy_kernel", "traffic": None, "bytes_per_launch_avg": 1000.0}
    bench._attach_traffic(roof, _W)
    assert roof["traffic"] == pytest.approx(900.0)        # scaled to the bench's launch
    assert roof["traffic_per_algorithmic_byte"] == pytest.approx(0.9)
    # host code and comments around the kernel may change
    (fake / "k" / "toy.cu").write_text(_SRC.replace("host_launch(Args a) {", "host_launch(Args a) { /* x */")
                                       .replace("// toy kernels", "// toy kernels, edited"))
    roof = {"kernel": "toy_kernel", "traffic": None, "bytes_per_launch_avg": 1000.0}
    bench._attach_traffic(roof, _W)
    assert roof["traffic"] == pytest.approx(900.0)
    # a change in a device function the kernel calls, or in its arguments: no traffic
    for old, new in (("2.0f * x", "3.0f * x"), ("int n;", "long n;"), ("(128)", "(256)")):
        (fake / "k" / "toy.cu").write_text(_SRC.replace(old, new))
        roof = {"kernel": "toy_kernel", "traffic": None, "bytes_per_launch_avg": 1000.0}
        bench._attach_traffic(roof, _W)
        assert roof["traffic"] is None and "changed" in roof["traffic_note"]


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


def test_early_stop_rates_split_at_the_first_stop():
    # steps 1-2 with every shift running, step 3 after one stopped; the
    # records carry the compulsory bytes of the chunks still active
    recs = [(2, 1, 1.0, 5e9, 0), (2, 2, 1.0, 5e9, 0), (2, 3, 0.5, 2e9, 0),
            (4, 1, 1.0, 6e9, 0), (4, 3, 1.0, 3e9, 0), (6, 2, -1.0, 1e9, 0)]
    r = {"steps_used": np.array([2, 3]), "recs": recs}
    out = bench._early_stop_rates(None, r)
    assert out["first_stop_step"] == 2
    assert out["stencil_all_running_GBps"] == pytest.approx(5000.0)
    assert out["stencil_some_stopped_GBps"] == pytest.approx(4000.0)
    assert out["dots_all_running_GBps"] == pytest.approx(6000.0)
    assert out["dots_some_stopped_GBps"] == pytest.approx(3000.0)
    assert out["update_all_running_GBps"] is None       # untimed record only


def test_quad_bound_summary_per_shift():
    # per shift, the median and the largest of the per-probe Eq. qbound factors
    class _E:
        @staticmethod
        def evc_get_quad_bound(h, ncol):
            assert ncol == 6
            return np.array([1.0, -3.0, 2.0, 10.0, 12.0, 11.0])

    class _C:
        h = None

    class _W2:
        shifts = [-0.5, 0.5]
        nprobe = 3

    out = bench._quad_bound_summary(_E, _C, _W2)
    assert out["log10_median"] == [1.0, 11.0]
    assert out["log10_max"] == [2.0, 12.0]


def test_every_tracked_traffic_record_matches_its_device_code():
    # a committed DRAM-traffic record is attached to a bench line only while
    # the device code it was captured from is unchanged; every record in
    # profiles/ must still match the sources (else it is stale)
    import glob
    for rec in glob.glob(os.path.join(ROOT, "profiles", "*_traffic.json")):
        d = json.load(open(rec))
        assert bench._device_code_sha(d["device_code"]) == d["device_code_sha256"], rec
