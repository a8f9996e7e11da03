"""Benchmark: Lanczos probe-steps/s of the preconditioned eigenvalue-count
estimator on one GB300, FP32-mixed (headline) and FP64, with the HBM
roofline of the dominant kernel and the FP64 CPU oracle timed beside it.

Workload (default): FD Hamiltonian H = -1/2 Lap_h + V, 7-point periodic 64^3
(n = 262,144), h = 0.3, 32 Gaussian wells; shifts lambda_min - 1 and eta;
Chebyshev degree-8 kinetic preconditioner; 64 Rademacher probes per shift;
30 Lanczos steps.  One benchmark step = one full count (2 shifts x 64 probes x
30 Lanczos steps, every kernel of the path) with the matrix resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): the path shards by probe columns with no data
exchange; every rank runs its own replica on its own probes (seed + rank)
and the job reports the sum of all ranks' probe-steps over the slowest
rank's time ("weak" scaling).
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


def _make_ctx(evc, W, precision, stream_ptr, V=None):
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
    ctx.reserve(len(W.shifts), W.nprobe, W.maxsteps)
    return ctx


def _roofline(evc, recs, peak, peak_kind, stencil_name="stencil_pass_kernel"):
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
    _attach_traffic(roof)
    return roof, per_kind


def _attach_traffic(roof):
    """DRAM traffic of one launch of the dominant kernel from the committed ncu
    capture, only while the kernel's source is unchanged since the capture."""
    import hashlib
    rec = {"stencil_pass_kernel": "profiles/stencil_pass_fd64_traffic.json",
           "stencil_patch_kernel": "profiles/stencil_patch_fd64_traffic.json"}.get(roof["kernel"])
    if not rec or not os.path.exists(os.path.join(ROOT, rec)):
        return
    d = json.load(open(os.path.join(ROOT, rec)))
    src = os.path.join(ROOT, d["source"])
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != d["source_sha256"]:
        return
    roof["traffic"] = d["dram_bytes"]
    roof["traffic_launch"] = d["launch"]
    roof["traffic_launch_algorithmic_bytes"] = d["algorithmic_bytes"]
    roof["traffic_source"] = d["profile"]
    if "note" in d:
        roof["traffic_note"] = d["note"]


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1602_02306_gb300 import evc, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    evc.load()
    W = workloads.WORKLOADS[args.workload]()
    S, m, k = len(W.shifts), W.nprobe, W.maxsteps
    seed = args.seed + rank
    peak, peak_kind = _peaks()
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(ctx, steps, warmup, profile):
        evc.evc_set_option(ctx.h, evc.EVC_OPT_PROFILE, 1 if profile else 0)
        dq = torch.empty(S * m, dtype=torch.float64, device="cuda")
        dL = torch.empty(S, dtype=torch.float64, device="cuda")
        ds = torch.empty(S, dtype=torch.int32, device="cuda")
        for _ in range(warmup):
            evc.evc_count_slices_async(ctx.h, W.shifts, m, k, W.tol, seed, dL.data_ptr(),
                                       dq.data_ptr(), ds.data_ptr())
        evc.evc_sync(ctx.h)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            evc.evc_count_slices_async(ctx.h, W.shifts, m, k, W.tol, seed, dL.data_ptr(),
                                       dq.data_ptr(), ds.data_ptr())
        e1.record(stream)
        evc.evc_sync(ctx.h)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        return ms, dL.cpu().numpy(), ds.cpu().numpy()

    # ---- headline: FP32-mixed, inputs resident
    ctx = _make_ctx(evc, W, evc.EVC_MIXED, sp)
    ws_mixed = evc.evc_workspace_bytes(ctx.h, S, m, k)
    # the library's autotuner picks the tile shapes for this launch shape
    # (short counts, before and outside the timed region)
    tuning = None if args.no_autotune else ctx.autotune(S, m, k)
    clocks = ClockSampler(local)
    clocks.start()
    ms_mixed, L_mixed, steps_mixed = timed(ctx, args.steps, args.warmup, profile=False)
    clk = clocks.stop()
    # per-kernel device times: one more count of the same workload, replayed
    # with a pair of timing events around every kernel, or around each step's
    # stencil segment when its chunk groups run concurrently (kept out of the
    # timed region above, whose events see only the whole counts)
    timed(ctx, 1, 0, profile=True)
    recs = evc.evc_get_profile(ctx.h)
    launches_per_step = sum(1 for r in recs if not r[4])   # span records are not launches
    # the stencil class runs the patch kernel when the tuner chose 2 x 2 patches
    # (passes without Jacobi scaling, N even)
    sname = "stencil_pass_kernel"
    patch = tuning.get("stencil_patch") if tuning else _SHAPES["patch"]
    if W.kind == "stencil" and patch == 2 and W.precond != "jacobi" and W.N % 2 == 0:
        sname = "stencil_patch_kernel"
    roof, per_kind = _roofline(evc, recs, peak, peak_kind, sname)
    # ---- e2e: host V (pinned) -> device, count, per-probe results -> host
    Vh = torch.from_numpy(W.potential()).pin_memory() if W.kind == "stencil" else None
    evc.evc_set_option(ctx.h, evc.EVC_OPT_PROFILE, 0)
    t_e2e = None
    if not args.skip_e2e:
        evc.evc_count_slices(ctx.h, W.shifts, m, k, W.tol, seed)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            if Vh is not None:
                evc.evc_set_values(ctx.h, Vh.data_ptr(), False)
            evc.evc_count_slices(ctx.h, W.shifts, m, k, W.tol, seed)
        t_e2e = time.perf_counter() - t0
        barrier()
    h2d = W.n * 8 if Vh is not None else 0
    d2h = S * m * 8 + S * 8 + S * 4
    # ---- accuracy trial: the same count with the basis rounded to BF16 when stored
    L_bf16 = None
    if not args.skip_bf16:
        evc.evc_set_option(ctx.h, evc.EVC_OPT_BASIS_BF16, 1)
        _, L_bf16, _ = timed(ctx, 1, 0, profile=False)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_BASIS_BF16, 0)
    ctx.close()
    torch.cuda.empty_cache()
    # ---- FP64 path on the same GPU
    ms_fp64, L_fp64, fp64_note = None, None, None
    if not args.skip_fp64:
        free, _ = torch.cuda.mem_get_info()
        need = 2 * ws_mixed
        if need > 0.9 * free:
            fp64_note = f"FP64 workspace {need / 1e9:.0f} GB does not fit next to the rest"
        else:
            ctx64 = _make_ctx(evc, W, evc.EVC_FP64, sp)
            if not args.no_autotune:
                ctx64.autotune(S, m, k)
            ms_fp64, L_fp64, steps_fp64 = timed(ctx64, max(1, args.steps // 2), 1, profile=False)
            psteps64 = float(m * int(np.sum(steps_fp64)))
            ctx64.close()

    # probe-steps per count: every probe of a shift runs that shift's steps
    psteps = float(m * int(np.sum(steps_mixed)))
    t_step = ms_mixed / args.steps
    t_max = t_step
    e2e_t = (t_e2e / args.steps) if t_e2e is not None else float("nan")
    if world > 1:
        t = torch.tensor([t_step, e2e_t], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max, e2e_t = float(t[0]), float(t[1])
    value = world * psteps / (t_max * 1e-3)
    est_mixed = float(L_mixed[-1] - L_mixed[0])
    est_fp64 = float(L_fp64[-1] - L_fp64[0]) if L_fp64 is not None else None
    fp64_steps = max(1, args.steps // 2)
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
                   "precision": "FP32 vectors/operator, FP64 alpha/beta/reorth coefficients/eig",
                   "step": "one full count: all shifts x probes x executed Lanczos steps",
                   "l2": f"inputs larger than L2 (Lanczos basis {ws_mixed / 1e9:.1f} GB workspace streamed every step)",
                   "parallelism": f"replicas{world}",
                   "method": ["lanczos (Algorithms 1-2)", "arnoldi (Sec. 4, Algorithm 3)"][_METHOD[0]],
                   "tiles": tuning if tuning is not None else "defaults (--no-autotune)"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "roofline": roof,
        "kernels": per_kind,
        "e2e": {"value": round(world * psteps / e2e_t, 1) if t_e2e is not None else None, "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "path": "evc_set_values(V from pinned host) + evc_count_slices (host outputs)"},
        "fp64": {"skipped": fp64_note or "--skip-fp64"} if ms_fp64 is None else {
            "value": round(world * psteps64 / (ms_fp64 / fp64_steps * 1e-3), 1), "unit": UNIT,
            "ms_per_step": round(ms_fp64 / fp64_steps, 3)},
        "estimate": {"mixed": est_mixed, "fp64": est_fp64,
                     "mixed_minus_fp64": (est_mixed - est_fp64) if est_fp64 is not None else None,
                     "n_below_mixed": [round(float(x), 4) for x in L_mixed],
                     "n_below_fp64": None if L_fp64 is None else [round(float(x), 4) for x in L_fp64]},
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


def run_serving(args):
    """Serving workload: count requests on 8 resident FD Hamiltonians arriving
    as a Poisson stream, served by the library's request server."""
    import torch
    from paper_1602_02306_gb300 import evc, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    evc.load()
    Ns = [32, 40, 48, 64, 80, 96, 112, 128]
    h = 0.3
    ctxs, vmin = [], []
    for N in Ns:
        V = inputs.gaussian_wells(N, h, nwells=32, seed=1)
        c = evc.Context.stencil(N, h, 2, V, precision=evc.EVC_MIXED)
        c.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        # no tolerance stop before step 10: the first Ritz values have not yet
        # reached the low end of the spectrum, where L stagnates near zero
        evc.evc_set_option(c.h, evc.EVC_OPT_MIN_STEPS, 10)
        ctxs.append(c)
        vmin.append(float(V.min()))
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.85 * free)
    srv = evc.evc_server_create(budget, slots=args.slots, max_batch=16)
    mids = [evc.evc_server_add_matrix(srv, c.h) for c in ctxs]
    rng = np.random.default_rng(3 + rank)
    nreq, rate = args.requests, args.rate
    gaps = rng.exponential(1.0 / rate, size=nreq)
    arrive = np.cumsum(gaps)
    reqs = []
    for q in range(nreq):
        mi = int(rng.integers(0, len(Ns)))
        a, b = np.sort(rng.uniform(0.0, 4.0, size=2))
        if b - a < 0.05:
            b = a + 0.05
        reqs.append(dict(matrix_id=mids[mi], xi=vmin[mi] + float(a), eta=vmin[mi] + float(b),
                         nprobe=int(rng.choice([32, 64, 128])), maxsteps=30,
                         tol=float(rng.choice([0.25, 0.5])), seed=3))
    # warm-up: one request per matrix size, not timed
    for mi in mids:
        tk = evc.evc_server_submit(srv, mi, vmin[mi], vmin[mi] + 1.0, 32, 5, 0.0, 3)
        evc.evc_server_wait(srv, tk)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
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
    results = []
    for q in range(nreq):
        rc, r = evc.evc_server_wait(srv, tickets[q])
        results.append((rc, r))
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = evc.evc_server_stats(srv)
    evc.evc_server_destroy(srv)
    for c in ctxs:
        c.close()
    ok = [r for rc, r in results if rc == evc.EVC_OK]
    lat = np.array([r["t_done"] - r["t_submit"] for r in ok])
    first = min(r["t_submit"] for r in ok)
    last = max(r["t_done"] for r in ok)
    span = last - first
    psteps = sum(q["nprobe"] * sum(r["steps"]) for q, (rc, r) in zip(reqs, results) if rc == 0)
    value = psteps / span
    line = {"metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": nreq, "warmup": len(mids), "ms_per_step": round(1000 * span / max(1, len(ok)), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "serving_8x_fd_7pt_32^3-128^3_jacobi", "requests": nreq,
                       "offered_rps": rate, "slots": args.slots, "max_batch": 16,
                       "hbm_budget_GB": round(budget / 1e9, 1),
                       "probes": [32, 64, 128], "tol": [0.25, 0.5], "maxsteps": 30,
                       "min_steps": 10,
                       "step": "one request (2 shifts x m probes, early stop)"},
            "serving": {"completed": len(ok), "failed": nreq - len(ok),
                        "throughput_rps": round(len(ok) / span, 2),
                        "p50_ms": round(1000 * float(np.percentile(lat, 50)), 2),
                        "p99_ms": round(1000 * float(np.percentile(lat, 99)), 2),
                        "mean_batch": round(float(np.mean([r["batch_size"] for r in ok])), 2),
                        "merged": st["merged"], "batches": st["batches"],
                        "peak_hbm_GB": round(st["peak_bytes"] / 1e9, 2), "wall_s": round(wall, 2),
                        "mean_steps": round(float(np.mean([np.mean(r["steps"]) for r in ok])), 2)},
            "clocks": clk,
            "e2e": {"value": round(value, 1), "unit": UNIT,
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * 3,
                    "path": "evc_server_submit/wait (host arguments and results)"}}
    if rank == 0:
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
        cpu_baseline(W, args.cpu_probes, seed=args.seed)
    times, vals = [], []
    for _ in range(args.steps):
        cb = cpu_baseline(W, args.cpu_probes, seed=args.seed)
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
    ap.add_argument("--workload", default="fd64")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-probes", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true", help="omit the FP64 comparison leg")
    ap.add_argument("--skip-e2e", action="store_true", help="omit the end-to-end leg")
    ap.add_argument("--skip-bf16", action="store_true", help="omit the BF16-basis accuracy trial")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tile shapes")
    ap.add_argument("--stencil-patch", type=int, default=0, choices=[0, 1, 2],
                    help="points per thread of the stencil pass (with --no-autotune)")
    ap.add_argument("--stencil-zb", type=int, default=0,
                    help="z planes per block of the stencil pass (with --no-autotune)")
    ap.add_argument("--stencil-groups", type=int, default=0, choices=[0, 1, 2, 4],
                    help="concurrent chunk groups of the stencil passes (with --no-autotune)")
    ap.add_argument("--csr-threads", type=int, default=0, choices=[0, 128, 256, 512],
                    help="threads per block of the CSR pass (with --no-autotune)")
    ap.add_argument("--method", default="lanczos", choices=["lanczos", "arnoldi"],
                    help="estimator: preconditioned Lanczos (default) or the Arnoldi-type variant")
    ap.add_argument("--requests", type=int, default=2000, help="serving workload: requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serving workload: arrivals per s")
    ap.add_argument("--slots", type=int, default=4, help="serving workload: server slots")
    ap.add_argument("--cheb-form", default="factored", choices=["factored", "clenshaw"],
                    help="how the Chebyshev preconditioner polynomial is applied")
    args = ap.parse_args()
    _CHEB_FORM[0] = 0 if args.cheb_form == "factored" else 1
    _METHOD[0] = 0 if args.method == "lanczos" else 1
    _SHAPES["patch"], _SHAPES["zb"] = args.stencil_patch, args.stencil_zb
    _SHAPES["groups"] = args.stencil_groups
    _SHAPES["csr_threads"] = args.csr_threads
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
