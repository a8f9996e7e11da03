"""Probe sharding through the C library on the GPU: ranks of a gloo group run
their probe blocks (EVC_OPT_PROBE_OFFSET) and combine the per-probe
quadratures on the host; the result equals one unsharded count bit for bit.

The ranks are processes on the one GPU of the box; their kernels never wait on
each other (the only exchange is the host-side all_gather after the counts).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    from paper_1602_02306_gb300 import inputs as I
    return I.powerlaw_symmetric(6000, cap=200, seed=2), [-0.5, 0.5], 45, 12


def _worker(rank, world, port, prec, out):
    import torch
    import torch.distributed as dist
    from paper_1602_02306_gb300 import evc, replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        evc.load()
        csr, shifts, m, k = _case()
        with evc.Context.csr(csr, precision=prec) as ctx:
            ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
            L, quad = replicas.sharded_count_slices(ctx, shifts, m, k, seed=4)
        out[rank] = (quad, L)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02306_gb300 import build, evc
    build.build()
    evc.load()


@pytest.mark.parametrize("world", [1, 2])
@pytest.mark.parametrize("prec", [0, 1])   # EVC_FP64, EVC_MIXED
def test_sharded_count_equals_unsharded(world, prec):
    from paper_1602_02306_gb300 import evc
    csr, shifts, m, k = _case()
    with evc.Context.csr(csr, precision=prec) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        Lref, qref, _ = ctx.count_slices(shifts, m, k, seed=4)
    ctx_mp = mp.get_context("spawn")
    mgr = ctx_mp.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx_mp.Process(target=_worker, args=(r, world, port, prec, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(world):
        quad, L = out[r]
        np.testing.assert_array_equal(quad, qref)
        np.testing.assert_allclose(L, Lref, rtol=1e-14)
