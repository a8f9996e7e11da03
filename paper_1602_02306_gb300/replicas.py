"""Sharding one count over several processes (one GPU each) by probes.

The estimator's probe columns are independent (Algorithm 2: one Lanczos run
per probe; Sec. 3: one run per shift), so a count with m probes splits into
shards of consecutive probe ids with no exchange during the computation.  The
one exchange step is the final combination: every rank contributes its
per-probe quadratures, all_gather collects them in rank order, and the
estimate is their mean per shift -- the same numbers, in the same order, as
one unsharded run with probe ids 0..m-1 (up to the order of the final sum).

The combination works on host tensors through any torch.distributed backend
(gloo on CPU in the tests, NCCL between GPUs).  With a tolerance-driven stop
the shards would decide their steps on different probe subsets, so sharded
counts use a fixed number of steps (tol <= 0).
"""
from __future__ import annotations

import numpy as np


def shard_range(m: int, rank: int, world: int):
    """Probe ids [lo, hi) of this rank: consecutive blocks, sizes differing by at most one."""
    base, extra = divmod(m, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def combine(local_quad: np.ndarray, m: int, group=None):
    """All-gather per-probe quadratures [S, m_local] from every rank and return
    (quad [S, m] in probe-id order, L [S] = per-shift means)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    S = local_quad.shape[0]
    # pad to the largest shard so every rank sends the same shape
    mmax = max(hi - lo for lo, hi in (shard_range(m, r, world) for r in range(world)))
    buf = torch.zeros((S, mmax), dtype=torch.float64)
    buf[:, :local_quad.shape[1]] = torch.from_numpy(np.ascontiguousarray(local_quad, dtype=np.float64))
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    cols = []
    for r in range(world):
        lo, hi = shard_range(m, r, world)
        cols.append(parts[r][:, :hi - lo].numpy())
    quad = np.concatenate(cols, axis=1)
    return quad, quad.mean(axis=1)


def sharded_count_slices(ctx, shifts, m, maxsteps, seed=0, group=None):
    """One count sharded over the ranks of `group` through the C library: this
    rank runs its probe block (EVC_OPT_PROBE_OFFSET), then the per-probe
    quadratures are combined on the host.  Returns (L [S], quad [S, m])."""
    import torch.distributed as dist
    from . import evc
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, hi = shard_range(m, rank, world)
    evc.evc_set_option(ctx.h, evc.EVC_OPT_PROBE_OFFSET, lo)
    try:
        if hi > lo:
            _, q, _ = ctx.count_slices(shifts, hi - lo, maxsteps, tol=0.0, seed=seed)
        else:
            q = np.zeros((len(shifts), 0))
    finally:
        evc.evc_set_option(ctx.h, evc.EVC_OPT_PROBE_OFFSET, 0)
    quad, L = combine(q, m, group)
    return L, quad
