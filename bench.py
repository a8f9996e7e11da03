"""Benchmark: Lanczos probe-steps/s of the preconditioned eigenvalue-count
estimator on one GB300, FP32-mixed (headline) and FP64, with the HBM
roofline of the dominant kernel and the FP64 CPU oracle timed beside it.

Workload (default, the largest single-GPU configuration): a generic sparse
symmetric indefinite matrix, n = 2,000,000, power-law row lengths (mean ~30,
at most ~2000), N(0,1) values, diagonal U(-5, 5); interval [-0.5, 0.5];
Jacobi preconditioner 1/(|a_ii - sigma| + 1e-3); 128 Rademacher probes per
shift; 50 Lanczos steps.  One benchmark step = one full count (2 shifts x 128
probes x 50 Lanczos steps, every kernel of the path) with the matrix resident
in HBM.  The same line carries the other workloads of the path under
`extra_workloads` (the 64^3 FD Hamiltonian with the Chebyshev kinetic
preconditioner, and 32-shift spectrum slicing of the 13-point 96^3
Hamiltonian with early stop), each with its own time and roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--extras a,b]

Multi-GPU (torchrun): the path shards by probe columns with no data
exchange; N ranks run one count of N x m probes per shift, rank r holding
probe ids r*m .. (r+1)*m - 1 of the same seed, and the per-probe quadratures
are combined on the host after the timed region.  The job reports the sum
of all ranks' probe-steps over the slowest rank's time ("weak" scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "probe Lanczos steps/s + HBM GB/s, FP32-mixed vs FP64 at count error <=0.5"
UNIT = "probe-steps/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


_CHEB_FORM = [0]     # EVC_CHEB_FACTORED; --cheb-form clenshaw sets 1
_METHOD = [0]        # EVC_METHOD_LANCZOS; --method arnoldi sets 1
_SHAPES = {"patch": 0, "zb": 0, "groups": 0, "csr_threads": 0}   # 0: library default
_MAXSTEPS = [0]      # --maxsteps (profiling aid); 0 keeps the workload's own
_PROBE_OFFSET = [0]  # under torchrun: rank * m, the rank's block of one sharded count


def _make_ctx(evc, W, precision, stream_ptr, V=None, nshift=None):
    if W.kind == "stencil":
        ctx = evc.Context.stencil(W.N, W.h, W.order, W.potential() if V is None else V,
                                  precision=precision, stream=stream_ptr)
    else:
        ctx = evc.Context.csr(W.csr(), precision=precision, stream=stream_ptr)
    kind = {"identity": evc.EVC_PREC_IDENTITY, "jacobi": evc.EVC_PREC_JACOBI,
            "cheb": evc.EVC_PREC_CHEB_KINETIC}[W.precond]
    ctx.set_precond(kind, *W.prec_params)
    evc.evc_set_option(ctx.h, evc.EVC_OPT_MIN_STEPS, W.min_steps)
    if W.precond == "cheb":
        evc.evc_set_option(ctx.h, evc.EVC_OPT_CHEB_FORM, _CHEB_FORM[0])
    evc.evc_set_option(ctx.h, evc.EVC_OPT_METHOD, _METHOD[0])
    if _PROBE_OFFSET[0]:
        evc.evc_set_option(ctx.h, evc.EVC_OPT_PROBE_OFFSET, _PROBE_OFFSET[0])
    if W.kind == "csr" and _SHAPES["csr_threads"]:
        evc.evc_set_option(ctx.h, evc.EVC_OPT_CSR_THREADS, _SHAPES["csr_threads"])
    if W.kind == "stencil":
        # fixed tile shapes (the autotuner, when it runs, starts from these)
        if _SHAPES["patch"]:
            evc.evc_set_option(ctx.h, evc.EVC_OPT_STENCIL_PATCH, _SHAPES["patch"])
        if _SHAPES["zb"]:
            evc.evc_set_option(ctx.h, evc.EVC_OPT_STENCIL_ZB, _SHAPES["zb"])
        if _SHAPES["groups"]:
            evc.evc_set_option(ctx.h, evc.EVC_OPT_STENCIL_GROUPS, _SHAPES["groups"])
    ctx.reserve(len(W.shifts) if nshift is None else nshift, W.nprobe, W.maxsteps)
    return ctx


def _roofline(evc, recs, peak, peak_kind, stencil_name="stencil_pass_kernel", W=None):
    """Roofline of the kernel class with the largest device time in the launch
    list: achieved = sum of its launches' algorithmic bytes / sum of their
    CUDA-event durations.  Launches that ran as concurrent chunk groups are
    timed by the span record of their segment (its wall time and the bytes of
    all its launches) and carry no time of their own."""
    per_kind = {}
    best = None
    for k, name in enumerate(evc.KERNEL_NAMES):
        rr = [r for r in recs if r[0] == k and r[2] > 0]
        if not rr:
            continue
        t = sum(r[2] for r in rr)
        b = sum(r[3] for r in rr)
        nl = sum(1 for r in recs if r[0] == k and not r[4])
        per_kind[name] = {"launches": nl, "ms": round(t, 4),
                          "GB/s": round(b / (t * 1e-3) / 1e9, 1) if t > 0 else None}
        if best is None or t > best[1]:
            best = (name, t, b, nl)
    if best is None:
        return None, per_kind
    name, t, b, cnt = best
    if name in ("finish", "reduce", "init"):
        # per-column FP64 scalar work (eigensolves, reductions): chains of
        # dependent operations, bound by their latency, not by a bandwidth
        kernel = {"finish": "quad_kernel", "reduce": "reorth_reduce_kernel"}.get(name, name)
        roof = {"bound": "latency", "kernel": kernel, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None, "launches": cnt, "ms_per_launch_avg": t / cnt,
                "share_of_step": None,
                "note": "small problem: the dominant class is FP64 per-column work bound by its "
                        "dependency chains; no bandwidth roofline applies"}
        tot = sum(v["ms"] for v in per_kind.values())
        roof["share_of_step"] = round(t / tot, 3) if tot > 0 else None
        return roof, per_kind
    kernel = {"stencil": stencil_name, "csr": "csr_pass_kernel",
              "dots": "reorth_dots_kernel", "update": "reorth_update_kernel"}.get(name, name)
    ach = b / (t * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": kernel, "achieved": round(ach, 1), "peak": peak,
            "unit": "GB/s", "frac": round(ach / peak, 4), "peak_source": peak_kind,
            "traffic": None, "bytes_per_launch_avg": b / cnt, "ms_per_launch_avg": t / cnt,
            "launches": cnt, "share_of_step": None}
    tot = sum(v["ms"] for v in per_kind.values())
    roof["share_of_step"] = round(t / tot, 3) if tot > 0 else None
    _attach_traffic(roof, W)
    return roof, per_kind


def _function_text(src, name):
    """Text of the definition of function (or `struct X`) `name` in src, with
    whitespace collapsed: from the name to the end of its brace-delimited body."""
    import re
    if name.startswith("struct "):
        pats = [r"\bstruct\s+" + re.escape(name.split()[1]) + r"\s*\{"]
    else:
        pats = [r"\b" + re.escape(name) + r"\s*\("]
    for mt in re.finditer(pats[0], src):
        j = mt.end() - 1
        if src[j] == "(":
            depth = 0
            while j < len(src):
                depth += {"(": 1, ")": -1}.get(src[j], 0)
                if depth == 0:
                    break
                j += 1
            j += 1
            while j < len(src) and src[j] in " \t\n":
                j += 1
            if j >= len(src) or src[j] != "{":
                continue            # a call or a declaration, not the definition
        depth, e = 0, j
        while e < len(src):
            depth += {"{": 1, "}": -1}.get(src[e], 0)
            if depth == 0:
                break
            e += 1
        # the declaration lines just above the name (template parameters,
        # __global__ / __launch_bounds__ qualifiers), up to a blank line, a
        # comment or the end of the previous statement
        st = src.rfind("\n", 0, mt.start()) + 1
        for _ in range(3):
            prev = src.rfind("\n", 0, st - 1) + 1 if st > 0 else 0
            line = src[prev:st].strip()
            if st == 0 or not line or line.startswith("//") or line.endswith((";", "}", "*/")):
                break
            st = prev
        return " ".join(src[st:e + 1].split())
    raise KeyError(f"no definition of {name}")


def _device_code_sha(spec):
    """sha256 over the device code a kernel runs: spec = [[file, [function or
    'struct X' names]], ...], each definition's text in the listed order."""
    import hashlib
    h = hashlib.sha256()
    for rel, names in spec:
        src = open(os.path.join(ROOT, rel)).read()
        for nm in names:
            h.update(_function_text(src, nm).encode())
    return h.hexdigest()


def _attach_traffic(roof, W=None):
    """DRAM traffic of one launch of the dominant kernel from the committed ncu
    capture (profiles/<kernel>_<workload>_traffic.json), attached only while the
    device code of that kernel -- its definition and every device function and
    argument struct it uses, hashed as text -- is unchanged since the capture."""
    if W is None:
        return
    rec = os.path.join(ROOT, "profiles", f"{roof['kernel']}_{W.name}_traffic.json")
    if not os.path.exists(rec):
        roof["traffic_note"] = "no ncu capture of this kernel on this workload"
        return
    d = json.load(open(rec))
    try:
        sha = _device_code_sha(d["device_code"])
    except (KeyError, OSError) as e:
        roof["traffic_note"] = f"device code of the capture not found: {e}"
        return
    if sha != d["device_code_sha256"]:
        roof["traffic_note"] = "device code changed since the ncu capture"
        return
    per_unit = d["dram_bytes"] / d["algorithmic_bytes"]
    # the capture's launch may be smaller than the bench's; DRAM bytes scale with
    # the algorithmic bytes of the launch (same kernel, same shape per chunk)
    roof["traffic"] = per_unit * roof["bytes_per_launch_avg"]
    roof["traffic_per_algorithmic_byte"] = round(per_unit, 4)
    roof["traffic_launch"] = d["launch"]
    roof["traffic_source"] = d["profile"]
    if "note" in d:
        roof["traffic_note"] = d["note"]


def _measure(evc, W, args, stream, peak, peak_kind, steps, warmup, seed, tune=True):
    """Time `steps` counts of W on a mixed context with the matrix resident
    (after `warmup` untimed counts), then one profiled count for the per-kernel
    device times.  Returns the open context and the measurements."""
    import torch
    S, m, k = len(W.shifts), W.nprobe, W.maxsteps
    ctx = _make_ctx(evc, W, evc.EVC_MIXED, stream.cuda_stream)
    ws = evc.evc_workspace_bytes(ctx.h, S, m, k)
    # the library's autotuner picks the tile shapes for this launch shape
    # (short counts, before and outside the timed region)
    tuning = ctx.autotune(S, m, k) if tune and not args.no_autotune else None
    dq = torch.empty(S * m, dtype=torch.float64, device="cuda")
    dL = torch.empty(S, dtype=torch.float64, device="cuda")
    ds = torch.empty(S, dtype=torch.int32, device="cuda")

    def timed(nsteps, nwarm, profile):
        evc.evc_set_option(ctx.h, evc.EVC_OPT_PROFILE, 1 if profile else 0)
        for _ in range(nwarm):
            evc.evc_count_slices_async(ctx.h, W.shifts, m, k, W.tol, seed, dL.data_ptr(),
                                       dq.data_ptr(), ds.data_ptr())
        evc.evc_sync(ctx.h)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        _barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(nsteps):
            evc.evc_count_slices_async(ctx.h, W.shifts, m, k, W.tol, seed, dL.data_ptr(),
                                       dq.data_ptr(), ds.data_ptr())
        e1.record(stream)
        evc.evc_sync(ctx.h)
        torch.cuda.synchronize()
        _barrier()
        return e0.elapsed_time(e1), dL.cpu().numpy(), ds.cpu().numpy(), dq.cpu().numpy()

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ms, L, st, q = timed(steps, warmup, profile=False)
    clk = clocks.stop()
    # per-kernel device times: one more count of the same workload, replayed
    # with a pair of timing events around every kernel, or around each step's
    # stencil segment when its chunk groups run concurrently (kept out of the
    # timed region above, whose events see only the whole counts)
    timed(1, 0, profile=True)
    recs = evc.evc_get_profile(ctx.h)
    qbound = _quad_bound_summary(evc, ctx, W) if not _METHOD[0] else None
    evc.evc_set_option(ctx.h, evc.EVC_OPT_PROFILE, 0)
    launches = sum(1 for r in recs if not r[4])   # span records are not launches
    # the stencil class runs the patch kernel when the tuner chose 2 x 2 patches
    # (passes without Jacobi scaling, N even), the tiled kernel for patch 3
    # (N a multiple of its 8 x 8 tile, else the patch kernel)
    sname = "stencil_pass_kernel"
    patch = tuning.get("stencil_patch") if tuning else _SHAPES["patch"]
    if W.kind == "stencil" and patch in (2, 3) and W.precond != "jacobi" and W.N % 2 == 0:
        sname = "stencil_tma_kernel" if patch == 3 and W.N % 8 == 0 else "stencil_patch_kernel"
    roof, per_kind = _roofline(evc, recs, peak, peak_kind, sname, W)
    psteps = float(m * int(np.sum(st)))
    return ctx, {"ms": ms, "L": L, "steps_used": st, "quad": q, "clocks": clk, "roofline": roof,
                 "quad_bound": qbound,
                 "kernels": per_kind, "launches": launches, "psteps": psteps, "ws": ws,
                 "tuning": tuning, "kmax": k, "recs": recs}


_WORLD = [1]


def _early_stop_rates(evc, r):
    """Rate of compulsory bytes of the streaming classes over the steps where
    every shift runs against the steps after the first shift stopped: the
    launches of later steps still cover the stopped chunks, whose blocks return
    at once, so a drop in rate would be their cost."""
    first = int(np.min(r["steps_used"]))
    out = {"first_stop_step": first}
    for kind, name in ((2, "stencil"), (4, "dots"), (6, "update")):
        for label, sel in (("all_running", lambda st: st <= first),
                           ("some_stopped", lambda st: st > first)):
            rr = [x for x in r["recs"] if x[0] == kind and x[2] > 0 and sel(x[1])]
            t = sum(x[2] for x in rr)
            b = sum(x[3] for x in rr)
            out[f"{name}_{label}_GBps"] = round(b / (t * 1e-3) / 1e9, 1) if t > 0 else None
    return out


def _device_time(r, steps):
    """How much of a count the kernels fill: the per-kernel device times of the
    profiled count against the timed counts' wall time on the device.  With
    early stop, the launches of a step still cover stopped chunks, whose blocks
    return at once; the gap also holds the graph's launch-to-launch gaps."""
    busy = sum(v["ms"] for v in r["kernels"].values())
    t = r["ms"] / steps
    done = int(np.sum(r["steps_used"]))
    return {"count_ms": round(t, 3), "kernels_ms": round(busy, 3),
            "idle_ms": round(t - busy, 3), "idle_frac": round((t - busy) / t, 4),
            "shift_steps_run": done, "shift_steps_max": len(r["steps_used"]) * int(r["kmax"])}


def _quad_bound_summary(evc, ctx, W):
    """Per shift, the median and the largest over probes of the computable
    factor of the Gauss quadrature error bound (Sec. 3, Eq. qbound) of the last
    count: log10(||v||^2 beta_2^2 ... beta_{k+1}^2 / (2k)!)."""
    S, m = len(W.shifts), W.nprobe
    qb = evc.evc_get_quad_bound(ctx.h, S * m).reshape(S, m)
    return {"log10_median": [round(float(np.median(x)), 2) for x in qb],
            "log10_max": [round(float(np.max(x)), 2) for x in qb],
            "note": "log10(||v||^2 beta_2^2...beta_{k+1}^2/(2k)!) per probe (Eq. qbound): times a bound "
                    "on the 2k-th derivative of a smooth stand-in for the step function it bounds "
                    "the quadrature error"}


def _barrier():
    if _WORLD[0] > 1:
        import torch.distributed as dist
        dist.barrier()


def _tinv_leg(evc, ctx, W, stream, seed, steps):
    """The same mixed count by the T^{-1}-inner-product process (Sec. 4,
    Eq. lanT1; Jacobi T = M^2): timed with events like the headline, then one
    profiled count for its per-kernel device times."""
    import torch
    S, m, k = len(W.shifts), W.nprobe, W.maxsteps
    evc.evc_set_option(ctx.h, evc.EVC_OPT_TINV_LANCZOS, 1)
    ctx.reserve(S, m, k)          # one more per-shift array (the T^{-1} weights)
    dq = torch.empty(S * m, dtype=torch.float64, device="cuda")
    dL = torch.empty(S, dtype=torch.float64, device="cuda")
    ds = torch.empty(S, dtype=torch.int32, device="cuda")

    def run():
        evc.evc_count_slices_async(ctx.h, W.shifts, m, k, W.tol, seed, dL.data_ptr(),
                                   dq.data_ptr(), ds.data_ptr())
    run()
    evc.evc_sync(ctx.h)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    evc.evc_sync(ctx.h)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    L, st = dL.cpu().numpy(), ds.cpu().numpy()
    evc.evc_set_option(ctx.h, evc.EVC_OPT_PROFILE, 1)
    run()
    evc.evc_sync(ctx.h)
    recs = evc.evc_get_profile(ctx.h)
    evc.evc_set_option(ctx.h, evc.EVC_OPT_PROFILE, 0)
    evc.evc_set_option(ctx.h, evc.EVC_OPT_TINV_LANCZOS, 0)
    _, per_kind = _roofline(evc, recs, 1.0, "", "stencil_pass_kernel", None)
    psteps = float(m * int(np.sum(st)))
    return {"value": round(psteps / (ms * 1e-3), 1), "ms_per_step": round(ms, 3), "steps": steps,
            "L": L, "kernels": {kk: {"ms": v["ms"], "GB/s": v["GB/s"]} for kk, v in per_kind.items()
                                if kk in ("csr", "stencil", "dots", "update")}}


def _fp64_leg(evc, W, args, stream, seed, ws_mixed, shifts=None):
    """The FP64 path on the same workload (or a subset of its shifts), timed."""
    import torch
    torch.cuda.empty_cache()
    shifts = list(W.shifts) if shifts is None else list(shifts)
    S, m, k = len(shifts), W.nprobe, W.maxsteps
    free, _ = torch.cuda.mem_get_info()
    need = 2 * ws_mixed * S / len(W.shifts)
    if need > 0.9 * free:
        return None, f"FP64 workspace {need / 1e9:.0f} GB does not fit next to the rest"
    ctx = _make_ctx(evc, W, evc.EVC_FP64, stream.cuda_stream, nshift=S)
    if not args.no_autotune:
        ctx.autotune(S, m, k)
    nsteps = max(1, min(3, args.steps // 2))
    for _ in range(1):
        L, q, st = ctx.count_slices(shifts, m, k, tol=W.tol, seed=seed)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nsteps):
        L, q, st = ctx.count_slices(shifts, m, k, tol=W.tol, seed=seed)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / nsteps
    ctx.close()
    torch.cuda.empty_cache()
    return {"ms_per_step": ms, "psteps": float(m * int(np.sum(st))), "L": L, "steps_used": st,
            "quad": q}, None


def _serving_extra(args, nreq=1000, low_nreq=250):
    """A shorter serving run for the default line: nreq requests at the
    offered rate, then low_nreq at the low rate (the full run is
    `--workload serving`)."""
    import torch
    torch.cuda.empty_cache()
    main, low, clk, _, budget = _serving_run(args, nreq, args.rate, low_nreq, args.low_rate)
    return {"workload": f"serving_8x_fd_7pt_32^3-128^3_{args.serving_precond}",
            "requests": nreq, "offered_rps": args.rate, "slots": args.slots,
            "hbm_budget_GB": round(budget / 1e9, 1),
            "value": round(main["probe_steps"] / main["span_s"], 1), "unit": UNIT,
            "serving": main, "serving_low_rate": low, "clocks": clk}


def _extra(evc, name, args, stream, peak, peak_kind, seed):
    """Another workload of the path, measured the same way, for the same line."""
    import torch
    from paper_1602_02306_gb300 import workloads
    W = workloads.WORKLOADS[name]()
    if _MAXSTEPS[0]:
        W.maxsteps = _MAXSTEPS[0]
    torch.cuda.empty_cache()
    ctx, r = _measure(evc, W, args, stream, peak, peak_kind, args.extra_steps, 1, seed)
    ctx.close()
    out = {"workload": W.name, "n": W.n, "shifts": len(W.shifts), "probes_per_shift": W.nprobe,
           "lanczos_steps_max": W.maxsteps, "tol": W.tol,
           "steps_used": [int(x) for x in r["steps_used"]],
           "value": round(r["psteps"] / (r["ms"] / args.extra_steps * 1e-3), 1), "unit": UNIT,
           "ms_per_step": round(r["ms"] / args.extra_steps, 3), "steps": args.extra_steps,
           "roofline": r["roofline"], "kernels": r["kernels"], "clocks": r["clocks"],
           "tiles": r["tuning"], "gpu_launches_per_step": r["launches"],
           "device_time": _device_time(r, args.extra_steps)}
    if W.tol > 0:
        out["early_stop"] = _early_stop_rates(evc, r)
    if name == "slicing96" and not args.skip_fp64:
        # the FP64 basis of all 32 shifts does not fit beside anything; every
        # shift's columns (and its stop rule) are independent of the others, so
        # FP64 runs on three of the shifts and each is compared with the same
        # shift of the mixed run
        sub = [0, 15, 31]
        f64, note = _fp64_leg(evc, W, args, stream, seed, r["ws"], shifts=[W.shifts[s] for s in sub])
        if f64 is None:
            out["fp64_subset"] = {"skipped": note}
        else:
            out["fp64_subset"] = {
                "shifts": sub, "n_below_fp64": [round(float(x), 4) for x in f64["L"]],
                "n_below_mixed": [round(float(r["L"][s]), 4) for s in sub],
                "mixed_minus_fp64": [float(r["L"][s] - f64["L"][j]) for j, s in enumerate(sub)],
                "steps_fp64": [int(x) for x in f64["steps_used"]],
                "steps_mixed": [int(r["steps_used"][s]) for s in sub],
                "value_fp64": round(f64["psteps"] / (f64["ms_per_step"] * 1e-3), 1)}
    elif W.kind == "stencil" and not args.skip_fp64:
        f64, note = _fp64_leg(evc, W, args, stream, seed, r["ws"])
        if f64 is not None:
            out["fp64"] = {"value": round(f64["psteps"] / (f64["ms_per_step"] * 1e-3), 1),
                           "ms_per_step": round(f64["ms_per_step"], 3)}
            est_m = float(r["L"][-1] - r["L"][0])
            est_f = float(f64["L"][-1] - f64["L"][0])
            out["estimate"] = {"mixed": est_m, "fp64": est_f, "mixed_minus_fp64": est_m - est_f}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1602_02306_gb300 import evc, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    _WORLD[0] = world
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    evc.load()
    W = workloads.WORKLOADS[args.workload]()
    if _MAXSTEPS[0]:
        W.maxsteps = _MAXSTEPS[0]
    S, m, k = len(W.shifts), W.nprobe, W.maxsteps
    # N ranks run one count of N*m probes: rank r holds probe ids r*m ..
    # (r+1)*m - 1 (same seed), and the per-probe quadratures are combined on
    # the host after the timed region (the only exchange of the path)
    seed = args.seed
    _PROBE_OFFSET[0] = rank * m
    peak, peak_kind = _peaks()
    stream = torch.cuda.Stream()

    # ---- headline: FP32-mixed, inputs resident
    ctx, r = _measure(evc, W, args, stream, peak, peak_kind, args.steps, args.warmup, seed)
    ms_mixed, L_mixed, steps_mixed = r["ms"], r["L"], r["steps_used"]
    # ---- e2e: the step's inputs from pinned host memory (V of a stencil
    # context, the CSR values otherwise, in the type they were given in),
    # count, per-probe results back to the host
    if W.kind == "stencil":
        hv = W.potential()
    else:
        hv = W.csr()[2]
    Vh = torch.from_numpy(np.ascontiguousarray(hv)).pin_memory()
    t_e2e = None
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    if not args.skip_e2e:
        evc.evc_count_slices(ctx.h, W.shifts, m, k, W.tol, seed)
        torch.cuda.synchronize()
        _barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            evc.evc_set_values(ctx.h, Vh.data_ptr(), False)
            evc.evc_count_slices(ctx.h, W.shifts, m, k, W.tol, seed)
        t_e2e = time.perf_counter() - t0
        _barrier()
    h2d = int(Vh.numel() * Vh.element_size())
    d2h = S * m * 8 + S * 8 + S * 4
    del Vh
    # ---- the T^{-1}-inner-product form of the same count (Jacobi workloads)
    tinv = None
    if W.precond == "jacobi" and not args.skip_tinv and _METHOD[0] == 0:
        tinv = _tinv_leg(evc, ctx, W, stream, seed, max(1, args.extra_steps))
    # ---- accuracy trial: the same count with the basis rounded to BF16 when stored
    L_bf16 = None
    if not args.skip_bf16:
        evc.evc_set_option(ctx.h, evc.EVC_OPT_BASIS_BF16, 1)
        L_bf16, _, _ = ctx.count_slices(W.shifts, m, k, tol=W.tol, seed=seed)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_BASIS_BF16, 0)
    ctx.close()
    torch.cuda.empty_cache()
    # ---- FP64 path on the same GPU
    f64, fp64_note = (None, "--skip-fp64") if args.skip_fp64 else \
        _fp64_leg(evc, W, args, stream, seed, r["ws"])

    psteps = r["psteps"]
    t_step = ms_mixed / args.steps
    t_max = t_step
    e2e_t = (t_e2e / e2e_steps) if t_e2e is not None else float("nan")
    if world > 1:
        t = torch.tensor([t_step, e2e_t], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max, e2e_t = float(t[0]), float(t[1])
    value = world * psteps / (t_max * 1e-3)
    if world > 1:
        # the sharded count's estimate over all N*m probes
        from paper_1602_02306_gb300 import replicas
        g = dist.new_group(backend="gloo")
        q_all, L_all = replicas.combine(r["quad"].reshape(S, m), world * m, group=g)
        L_mixed = L_all
    est_mixed = float(L_mixed[-1] - L_mixed[0])
    est_fp64 = float(f64["L"][-1] - f64["L"][0]) if f64 is not None else None
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_max, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": W.name, "n": W.n, "shifts": S, "probes_per_shift": m,
                   "lanczos_steps_max": k, "tol": W.tol,
                   "steps_used": [int(x) for x in steps_mixed],
                   "precond": {"cheb": f"chebyshev-{int(W.prec_params[0])} kinetic (c={W.prec_params[1]}), "
                                       f"{['factored', 'clenshaw'][_CHEB_FORM[0]]}",
                               "jacobi": "jacobi (eps 1e-3)", "identity": "none"}[W.precond],
                   "precision": "FP32 vectors/operator, FP64 alpha/beta/reorth coefficients/eig"
                                + (", FP64 diagonal and Jacobi set-up" if W.kind == "csr" else ""),
                   "step": "one full count: all shifts x probes x executed Lanczos steps",
                   "l2": f"inputs larger than L2 (Lanczos basis {r['ws'] / 1e9:.1f} GB workspace "
                         f"streamed every step)",
                   "parallelism": f"probe shards x{world}" if world > 1 else "one GPU",
                   "method": ["lanczos (Algorithms 1-2)", "arnoldi (Sec. 4, Algorithm 3)"][_METHOD[0]],
                   "tiles": r["tuning"] if r["tuning"] is not None else "defaults (--no-autotune)"},
        "gpu_launches": r["launches"] * args.steps,
        "clocks": r["clocks"],
        "roofline": r["roofline"],
        "kernels": r["kernels"],
        "device_time": _device_time(r, args.steps),
        "e2e": {"value": round(world * psteps / e2e_t, 1) if t_e2e is not None else None, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": ("evc_set_values(V" if W.kind == "stencil" else "evc_set_values(CSR values")
                        + " float64 from pinned host) + evc_count_slices (host outputs)",
                "steps": e2e_steps},
        "fp64": {"skipped": fp64_note} if f64 is None else {
            "value": round(world * f64["psteps"] / (f64["ms_per_step"] * 1e-3), 1), "unit": UNIT,
            "ms_per_step": round(f64["ms_per_step"], 3)},
        "quad_bound": r.get("quad_bound"),
        "estimate": {"mixed": est_mixed, "fp64": est_fp64,
                     # this rank's probes on both paths (the whole count at N = 1)
                     "mixed_minus_fp64": (float(r["L"][-1] - r["L"][0]) - est_fp64)
                     if est_fp64 is not None else None,
                     "n_below_mixed": [round(float(x), 4) for x in L_mixed],
                     "probes_per_shift": world * m,
                     "n_below_fp64": None if f64 is None else [round(float(x), 4) for x in f64["L"]],
                     "max_abs_per_probe_mixed_minus_fp64": None if f64 is None else
                     float(np.max(np.abs(r["quad"] - f64["quad"].reshape(-1))))},
        "tinv_lanczos": None if tinv is None else {
            "value": tinv["value"], "unit": UNIT, "ms_per_step": tinv["ms_per_step"],
            "steps": tinv["steps"], "kernels": tinv["kernels"],
            "estimate": float(tinv["L"][-1] - tinv["L"][0]),
            "minus_fp64": (float(tinv["L"][-1] - tinv["L"][0]) - est_fp64)
            if est_fp64 is not None else None,
            "n_below": [round(float(x), 4) for x in tinv["L"]],
            "note": "the T^-1-inner-product Lanczos process (Sec. 4, Eq. lanT1) with T = M^2: "
                    "operator rows scaled by T, inner products weighted by T^-1; the same J_k "
                    "in exact arithmetic (FP64: per-probe equal to Algorithm 1 within 1e-6 "
                    "at this size)"},
        "bf16_basis": None if L_bf16 is None else {
            "estimate": float(L_bf16[-1] - L_bf16[0]),
            "minus_fp64": (float(L_bf16[-1] - L_bf16[0]) - est_fp64) if est_fp64 is not None else None,
            "minus_mixed": float(L_bf16[-1] - L_bf16[0]) - est_mixed,
            "n_below": [round(float(x), 4) for x in L_bf16],
            "note": "basis rounded to BF16 when stored (storage kept FP32): count error of BF16 "
                    "storage; its traffic would halve the reorthogonalisation bytes"},
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(W, args.cpu_probes, seed=args.seed)
    # ---- the other workloads of the path, each with its own time and roofline
    if rank == 0 and world == 1 and args.extras:
        line["extra_workloads"] = {}
        for name in [x for x in args.extras.split(",") if x and x != args.workload]:
            if name == "serving":
                line["extra_workloads"][name] = _serving_extra(args)
                continue
            line["extra_workloads"][name] = _extra(evc, name, args, stream, peak, peak_kind, seed)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(W, nprobe_sample, seed=0):
    """The FP64 oracle as it stands, on a bounded sample of the workload."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    if W.kind == "stencil":
        V = W.potential()
        pk = {"identity": O.PREC_NONE, "jacobi": O.PREC_JACOBI, "cheb": O.PREC_CHEB}[W.precond]
        P = O.Problem.stencil(W.N, W.h, W.order, V, pk, cheb_degree=int(W.prec_params[0]),
                              cheb_c=float(W.prec_params[1]), jac_eps=float(W.prec_params[0]))
    else:
        pk = {"identity": O.PREC_NONE, "jacobi": O.PREC_JACOBI}[W.precond]
        P = O.Problem.csr_matrix(W.csr(), pk, jac_eps=float(W.prec_params[0]))
    t0 = time.perf_counter()
    if _METHOD[0] == 1:
        # the Arnoldi oracle is numpy on one core: a quarter of the sample
        from oracle import arnoldi as AR
        nprobe_sample = max(1, nprobe_sample // 4)
        cores = 1
        q, st, L = AR.count(P, W.shifts, nprobe_sample, W.maxsteps, tol=W.tol, seed=seed)
    else:
        q, st, L = O.count(P, W.shifts, nprobe_sample, W.maxsteps, tol=W.tol, seed=seed,
                           nthreads=cores)
    dt = time.perf_counter() - t0
    ps = float(nprobe_sample * int(np.sum(st)))      # the steps each shift actually ran
    return {"value": round(ps / dt, 2), "unit": UNIT, "cores": min(cores, len(W.shifts) * nprobe_sample),
            "kind": "oracle",
            "sample": f"{len(W.shifts)} shifts x {nprobe_sample} probes x at most {W.maxsteps} steps "
                      f"at full n",
            "seconds": round(dt, 2)}


def _serving_run(args, nreq, rate, low_nreq, low_rate, rank=0):
    """Count requests on 8 resident FD Hamiltonians arriving as a Poisson
    stream, served by the library's request server: a phase of nreq requests
    at `rate` per second (clocks sampled), then a lighter one (low_nreq at
    low_rate; none when low_rate <= 0).  Returns (main, low, clocks, stats,
    HBM budget)."""
    import torch
    from paper_1602_02306_gb300 import evc, inputs

    Ns = [32, 40, 48, 64, 80, 96, 112, 128]
    h = 0.3
    ctxs, vmin = [], []
    pk = {"identity": evc.EVC_PREC_IDENTITY, "jacobi": evc.EVC_PREC_JACOBI}[args.serving_precond]
    for N in Ns:
        V = inputs.gaussian_wells(N, h, nwells=32, seed=1)
        c = evc.Context.stencil(N, h, 2, V, precision=evc.EVC_MIXED)
        c.set_precond(pk, 1e-3)
        # no tolerance stop before step 10: the first Ritz values have not yet
        # reached the low end of the spectrum, where L stagnates near zero
        evc.evc_set_option(c.h, evc.EVC_OPT_MIN_STEPS, 10)
        ctxs.append(c)
        vmin.append(float(V.min()))
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.85 * free)
    srv = evc.evc_server_create(budget, slots=args.slots, max_batch=16)
    mids = [evc.evc_server_add_matrix(srv, c.h) for c in ctxs]
    # warm-up: one request per matrix size, not timed
    for mi in mids:
        tk = evc.evc_server_submit(srv, mi, vmin[mi], vmin[mi] + 1.0, 32, 5, 0.0, 3)
        evc.evc_server_wait(srv, tk)

    def phase(nreq, rate, seed):
        """nreq Poisson arrivals at `rate` per second; returns the results."""
        rng = np.random.default_rng(seed)
        arrive = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
        reqs = []
        for q in range(nreq):
            mi = int(rng.integers(0, len(Ns)))
            a, b = np.sort(rng.uniform(0.0, 4.0, size=2))
            if b - a < 0.05:
                b = a + 0.05
            reqs.append(dict(matrix_id=mids[mi], xi=vmin[mi] + float(a), eta=vmin[mi] + float(b),
                             nprobe=int(rng.choice([32, 64, 128])), maxsteps=30,
                             tol=float(rng.choice([0.25, 0.5])), seed=3))
        st0 = evc.evc_server_stats(srv)
        tickets = [None] * nreq
        t0 = time.perf_counter()

        def submitter():
            for q in range(nreq):
                dt = arrive[q] - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                tickets[q] = evc.evc_server_submit(srv, **reqs[q])

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        results = [evc.evc_server_wait(srv, tickets[q]) for q in range(nreq)]
        wall = time.perf_counter() - t0
        st = evc.evc_server_stats(srv)
        ok = [(q, r) for q, (rc, r) in zip(reqs, results) if rc == evc.EVC_OK]
        lat = np.array([r["t_done"] - r["t_submit"] for _, r in ok])
        span = max(r["t_done"] for _, r in ok) - min(r["t_submit"] for _, r in ok)
        psteps = sum(q["nprobe"] * sum(r["steps"]) for q, r in ok)
        return {"offered_rps": rate, "requests": nreq, "completed": len(ok),
                "failed": nreq - len(ok), "throughput_rps": round(len(ok) / span, 2),
                "p50_ms": round(1000 * float(np.percentile(lat, 50)), 2),
                "p99_ms": round(1000 * float(np.percentile(lat, 99)), 2),
                "mean_batch": round(float(np.mean([r["batch_size"] for _, r in ok])), 2),
                "merged": st["merged"] - st0["merged"], "batches": st["batches"] - st0["batches"],
                "wall_s": round(wall, 2), "span_s": round(span, 3),
                "mean_steps": round(float(np.mean([np.mean(r["steps"]) for _, r in ok])), 2),
                "probe_steps": psteps}

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    main = phase(nreq, rate, 3 + rank)
    clk = clocks.stop()
    low = phase(low_nreq, low_rate, 103 + rank) if low_rate > 0 else None
    st = evc.evc_server_stats(srv)
    evc.evc_server_destroy(srv)
    for c in ctxs:
        c.close()
    main = dict(main, peak_hbm_GB=round(st["peak_bytes"] / 1e9, 2))
    return main, low, clk, st, budget


def run_serving(args):
    """Serving workload: count requests on 8 resident FD Hamiltonians arriving
    as a Poisson stream, served by the library's request server."""
    import torch
    from paper_1602_02306_gb300 import evc

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    evc.load()
    main, low, clk, st, budget = _serving_run(args, args.requests, args.rate, args.low_requests,
                                              args.low_rate, rank)
    value = main["probe_steps"] / main["span_s"]
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.requests, "warmup": len(mids),
            "ms_per_step": round(1000 * main["span_s"] / max(1, main["completed"]), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"serving_8x_fd_7pt_32^3-128^3_{args.serving_precond}",
                       "requests": args.requests, "offered_rps": args.rate, "slots": args.slots,
                       "max_batch": 16, "hbm_budget_GB": round(budget / 1e9, 1),
                       "probes": [32, 64, 128], "tol": [0.25, 0.5], "maxsteps": 30,
                       "min_steps": 10, "precond": args.serving_precond,
                       "step": "one request (2 shifts x m probes, early stop)"},
            "serving": main,
            "serving_low_rate": low,
            "clocks": clk,
            "e2e": {"value": round(value, 1), "unit": UNIT,
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * 3,
                    "path": "evc_server_submit/wait (host arguments and results)"}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_laplace_family(args):
    """The paper's Laplace mesh family (Sec. 7; Table 1 "Laplace", Table 2's
    h = 2^-6 .. 2^-10): estimate against k for the unpreconditioned Lanczos
    estimator (scalar Jacobi), m = 50, tau = 3000, mixed precision, next to the
    closed-form count -- the mesh dependence of k that the paper's
    preconditioners remove.  One JSON line."""
    import torch
    from paper_1602_02306_gb300 import evc, workloads
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    evc.load()
    ks = [int(x) for x in args.family_k.split(",")]
    rows = []
    t_all = time.perf_counter()
    tot_ps, tot_ms = 0.0, 0.0
    for e in range(6, 11):
        W = workloads.laplace_paper(e, k=max(ks))
        exact = workloads.laplace_exact_below(e)
        stream = torch.cuda.Stream()
        ctx = _make_ctx(evc, W, evc.EVC_MIXED, stream.cuda_stream)
        row = {"h": f"2^-{e}", "n": W.n, "exact": exact, "k": {}}
        first5 = None
        for k in ks:
            kk = min(k, W.n)
            ctx.count_slices(W.shifts, W.nprobe, kk, seed=args.seed)   # graph capture, untimed
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            L, q, st = ctx.count_slices(W.shifts, W.nprobe, kk, seed=args.seed)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            se = float(q[0].std(ddof=1) / np.sqrt(W.nprobe))
            rel = abs(float(L[0]) - exact) / exact
            row["k"][kk] = {"estimate": round(float(L[0]), 2), "se": round(se, 2),
                            "rel_err": round(rel, 4), "ms": round(ms, 2)}
            if first5 is None and rel <= 0.05:
                first5 = kk
            tot_ps += W.nprobe * int(st[0])
            tot_ms += ms
        row["smallest_k_within_5pct"] = first5
        rows.append(row)
        ctx.close()
        torch.cuda.empty_cache()
    line = {"metric": METRIC, "value": round(tot_ps / (tot_ms * 1e-3), 1), "unit": UNIT,
            "n_gpus": 1, "steps": len(ks) * 5, "warmup": 1,
            "ms_per_step": round(tot_ms / (len(ks) * 5), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "laplace2d_family_h2^-6..2^-10_tau3000_m50",
                       "precond": "jacobi (a scalar here: the paper's unpreconditioned row)",
                       "k_grid": ks, "step": "one count at one (h, k)"},
            "paper": {"table1_laplace_h2^-7": {"exact": 226, "k": 134, "estimate": 232}},
            "family": rows, "wall_s": round(time.perf_counter() - t_all, 1)}
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.steps < 1:
        raise SystemExit("--steps must be >= 1")
    from paper_1602_02306_gb300 import workloads
    W = workloads.WORKLOADS[args.workload]()
    for _ in range(args.warmup):
        cpu_baseline(W, args.ref_probes, seed=args.seed)
    times, vals = [], []
    for _ in range(args.steps):
        cb = cpu_baseline(W, args.ref_probes, seed=args.seed)
        times.append(cb["seconds"])
        vals.append(cb["value"])
    value = float(np.median(vals))
    config = {"workload": W.name, "n": W.n, "shifts": len(W.shifts), "probes_per_shift": W.nprobe,
              "lanczos_steps_max": W.maxsteps, "tol": W.tol, "precond": W.precond,
              "method": ["lanczos (Algorithms 1-2)", "arnoldi (Sec. 4, Algorithm 3)"][_METHOD[0]],
              "step": "a bounded sample of one count, scaled to probe-steps/s", "sample": cb["sample"]}
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT,
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * float(np.median(times)), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "kind": "oracle",
                             "cores": cb["cores"], "sample": cb["sample"] + " per step"},
            "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="powerlaw2m")
    ap.add_argument("--extras", default="fd64,slicing96,serving",
                    help="other workloads measured for the same line (comma list, '' for none)")
    ap.add_argument("--extra-steps", type=int, default=3, help="timed counts per extra workload")
    ap.add_argument("--e2e-steps", type=int, default=5,
                    help="counts of the end-to-end leg (at most --steps)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--family-k", default="25,50,100,134,200,256",
                    help="laplace-family workload: the Lanczos step counts of the study")
    ap.add_argument("--cpu-probes", type=int, default=6,
                    help="probes per shift of the oracle's bounded sample (cpu_baseline)")
    ap.add_argument("--ref-probes", type=int, default=2,
                    help="probes per shift of each step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the FP64 comparison leg")
    ap.add_argument("--skip-e2e", action="store_true", help="omit the end-to-end leg")
    ap.add_argument("--skip-bf16", action="store_true", help="omit the BF16-basis accuracy trial")
    ap.add_argument("--skip-tinv", action="store_true",
                    help="omit the T^-1-inner-product Lanczos leg (Jacobi workloads)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes")
    ap.add_argument("--stencil-patch", type=int, default=0, choices=[0, 1, 2, 3],
                    help="points per thread of the stencil pass: 1, 2 (2x2 patch) or 3 (2x2 patches of tensor-copied tiles) (with --no-autotune)")
    ap.add_argument("--stencil-zb", type=int, default=0,
                    help="z planes per block of the stencil pass (with --no-autotune)")
    ap.add_argument("--stencil-groups", type=int, default=0, choices=[0, 1, 2, 4],
                    help="concurrent chunk groups of the stencil passes (with --no-autotune)")
    ap.add_argument("--csr-threads", type=int, default=0, choices=[0, 128, 256, 512],
                    help="threads per block of the CSR pass (with --no-autotune)")
    ap.add_argument("--maxsteps", type=int, default=0,
                    help="profiling aid: run the workload with this many Lanczos steps instead "
                         "of its own (a smaller device footprint for ncu captures)")
    ap.add_argument("--method", default="lanczos", choices=["lanczos", "arnoldi"],
                    help="estimator: preconditioned Lanczos (default) or the Arnoldi-type variant")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serving workload: arrivals per s")
    ap.add_argument("--slots", type=int, default=2, help="serving workload: server slots")
    ap.add_argument("--serving-precond", default="identity", choices=["identity", "jacobi"],
                    help="serving workload: preconditioner of the resident Hamiltonians")
    ap.add_argument("--low-rate", type=float, default=50.0,
                    help="serving workload: a second, lighter phase at this rate (0: none)")
    ap.add_argument("--low-requests", type=int, default=500,
                    help="serving workload: requests of the lighter phase")
    ap.add_argument("--cheb-form", default="factored", choices=["factored", "clenshaw"],
                    help="how the Chebyshev preconditioner polynomial is applied")
    args = ap.parse_args()
    _CHEB_FORM[0] = 0 if args.cheb_form == "factored" else 1
    _MAXSTEPS[0] = args.maxsteps
    _METHOD[0] = 0 if args.method == "lanczos" else 1
    _SHAPES["patch"], _SHAPES["zb"] = args.stencil_patch, args.stencil_zb
    _SHAPES["groups"] = args.stencil_groups
    _SHAPES["csr_threads"] = args.csr_threads
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "laplace-family":
        run_laplace_family(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
