"""Probe sharding across ranks (gloo, world size 2, CPU): the combination step
reproduces an unsharded count.  The per-rank work is done by the FP64 oracle
on the rank's probe ids, standing in for the GPU library on each rank."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1602_02306_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_1602_02306_gb300 import inputs as I
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = O.Problem.csr_matrix(I.laplace2d_dirichlet(12), O.PREC_JACOBI)
        m = 11
        lo, hi = replicas.shard_range(m, rank, world)
        q, _, _ = O.count(P, [1.0, 2.5], hi - lo, 15, seed=3, probe_ids=list(range(lo, hi)))
        quad, L = replicas.combine(q, m)
        out[rank] = (quad, L)
    finally:
        dist.destroy_process_group()


def test_shard_ranges_cover_all_probes():
    for m in (1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            ids = []
            for r in range(world):
                lo, hi = replicas.shard_range(m, r, world)
                ids += list(range(lo, hi))
            assert ids == list(range(m))


def test_gloo_two_ranks_combine_equals_unsharded():
    from oracle import oracle as O
    from paper_1602_02306_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    P = O.Problem.csr_matrix(I.laplace2d_dirichlet(12), O.PREC_JACOBI)
    qref, _, Lref = O.count(P, [1.0, 2.5], 11, 15, seed=3)
    for r in range(2):
        quad, L = out[r]
        np.testing.assert_array_equal(quad, qref)
        np.testing.assert_allclose(L, Lref, rtol=1e-15)
