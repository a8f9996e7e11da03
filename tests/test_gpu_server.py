"""The request server: continuous admission by HBM footprint, merged
launches, overlapping slots, and results that do not depend on the mix."""
import threading

import numpy as np
import pytest

from paper_1602_02306_gb300 import evc
from paper_1602_02306_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02306_gb300 import build
    build.build()
    evc.load()


def _matrices():
    ctxs = []
    for N in (10, 12, 16):
        V = I.gaussian_wells(N, 0.3, nwells=4, seed=1)
        c = evc.Context.stencil(N, 0.3, 2, V, precision=evc.EVC_MIXED)
        c.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        ctxs.append(c)
    return ctxs


def test_result_same_alone_and_in_the_mix():
    ctxs = _matrices()
    # a larger grid for the long counts that hold the slots
    Vb = I.gaussian_wells(40, 0.3, nwells=4, seed=1)
    big = evc.Context.stencil(40, 0.3, 2, Vb, precision=evc.EVC_MIXED)
    big.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
    ctxs.append(big)
    srv = evc.evc_server_create(24 << 30, slots=3, max_batch=8)
    try:
        mids = [evc.evc_server_add_matrix(srv, c.h) for c in ctxs]
        probe = dict(matrix_id=mids[1], xi=-2.0, eta=0.5, nprobe=32, maxsteps=20, tol=0.25, seed=7)
        alone = np.zeros(64)
        t = evc.evc_server_submit(srv, **probe, quad_buf=alone)
        rc, ra = evc.evc_server_wait(srv, t)
        assert rc == evc.EVC_OK and ra["batch_size"] == 1
        # every slot busy with a long count (distinct seeds: no two share a
        # launch), so that the requests below wait and are merged whatever
        # the timing
        blockers = [evc.evc_server_submit(srv, mids[3], -1.0, 1.0, 64, 80, 0.0, 11 + j)
                    for j in range(3)]
        # now the same request among many others, submitted from two threads
        bufs, tickets = [], []
        lock = threading.Lock()

        def submitter(seed):
            g = np.random.default_rng(seed)
            for k in range(20):
                if k % 5 == 2:
                    b = np.zeros(64)
                    tk = evc.evc_server_submit(srv, **probe, quad_buf=b)
                    with lock:
                        bufs.append(b)
                        tickets.append(("probe", tk))
                else:
                    xi = float(g.uniform(-3, 0))
                    tk = evc.evc_server_submit(srv, int(g.integers(0, 3)), xi, xi + float(g.uniform(0.5, 2)),
                                               32, 20, 0.25, 7)
                    with lock:
                        tickets.append(("other", tk))

        th = [threading.Thread(target=submitter, args=(s,)) for s in (1, 2)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        res = {}
        for kind, tk in tickets:
            rc, r = evc.evc_server_wait(srv, tk)
            assert rc == evc.EVC_OK
            res[tk] = (kind, r)
        for tk in blockers:
            rc, r = evc.evc_server_wait(srv, tk)
            assert rc == evc.EVC_OK and r["batch_size"] == 1
        st = evc.evc_server_stats(srv)
        assert st["completed"] == 1 + len(tickets) + len(blockers)
        assert st["merged"] > 0                      # requests did share launches
        merged_probe = [r for kind, r in res.values() if kind == "probe" and r["batch_size"] > 1]
        assert merged_probe, "the repeated request never ran inside a batch"
        for kind, r in res.values():
            if kind == "probe":
                assert r["estimate"] == ra["estimate"]
                assert r["steps"] == ra["steps"]
        for b in bufs:
            np.testing.assert_array_equal(b, alone)
    finally:
        evc.evc_server_destroy(srv)
        for c in ctxs:
            c.close()


def test_admission_respects_budget_and_overlaps():
    ctxs = _matrices()
    one = evc.evc_workspace_bytes(ctxs[2].h, 2, 64, 20)
    srv = evc.evc_server_create(int(2.5 * one), slots=4, max_batch=1)
    try:
        mid = evc.evc_server_add_matrix(srv, ctxs[2].h)
        tks = [evc.evc_server_submit(srv, mid, -2.0 + 0.1 * k, 0.5, 64, 20, 0.0, k) for k in range(12)]
        rs = []
        for tk in tks:
            rc, r = evc.evc_server_wait(srv, tk)
            assert rc == evc.EVC_OK
            rs.append(r)
        st = evc.evc_server_stats(srv)
        assert st["peak_bytes"] <= st["budget_bytes"]
        assert st["peak_bytes"] >= 2 * one           # two batches ran at the same time
        assert st["used_bytes"] == 0 and st["pending"] == 0
        # first come, first served: admissions in submission order
        starts = [r["t_start"] for r in rs]
        assert starts == sorted(starts)
    finally:
        evc.evc_server_destroy(srv)
        for c in ctxs:
            c.close()


def test_request_larger_than_budget_fails_cleanly():
    ctxs = _matrices()
    srv = evc.evc_server_create(1 << 20, slots=1, max_batch=4)
    try:
        mid = evc.evc_server_add_matrix(srv, ctxs[0].h)
        tk = evc.evc_server_submit(srv, mid, -1.0, 0.0, 32, 10)
        rc, r = evc.evc_server_wait(srv, tk, 30.0)
        assert rc == evc.EVC_ENOMEM
        with pytest.raises(evc.EvcError):
            evc.evc_server_submit(srv, mid, 1.0, 0.0, 32, 10)   # xi > eta
    finally:
        evc.evc_server_destroy(srv)
        for c in ctxs:
            c.close()


def test_served_request_matches_the_oracle_fp64():
    # one request through the server (merged with others) against the FP64
    # oracle per probe, stop rule included
    from oracle import oracle as O
    N, h = 10, 0.3
    V = I.gaussian_wells(N, h, nwells=4, seed=1)
    ctx = evc.Context.stencil(N, h, 2, V, precision=evc.EVC_FP64)
    ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
    srv = evc.evc_server_create(4 << 30, slots=1, max_batch=8)
    try:
        mid = evc.evc_server_add_matrix(srv, ctx.h)
        req = dict(matrix_id=mid, xi=-2.5, eta=0.25, nprobe=24, maxsteps=25, tol=0.25, seed=5)
        bufs = [np.zeros(48) for _ in range(4)]
        tks = [evc.evc_server_submit(srv, **dict(req, xi=req["xi"] + 0.1 * q), quad_buf=bufs[q])
               for q in range(4)]
        res = [evc.evc_server_wait(srv, tk) for tk in tks]
        P = O.Problem.stencil(N, h, 2, V, O.PREC_JACOBI, jac_eps=1e-3)
        for q, (rc, r) in enumerate(res):
            assert rc == evc.EVC_OK
            qr, sr, Lr = O.count(P, [req["xi"] + 0.1 * q, req["eta"]], req["nprobe"],
                                 req["maxsteps"], tol=req["tol"], seed=req["seed"])
            assert list(r["steps"]) == list(sr)
            np.testing.assert_allclose(bufs[q], qr.reshape(-1), rtol=0, atol=1e-8)
            assert abs(r["estimate"] - (Lr[1] - Lr[0])) < 1e-9
    finally:
        evc.evc_server_destroy(srv)
        ctx.close()


def test_numeric_failure_stays_with_its_request():
    # a shift that is finite in FP64 but overflows FP32 makes its own columns
    # non-finite; merged with good requests, only that request fails and the
    # others equal their results alone
    N = 10
    V = I.gaussian_wells(N, 0.3, nwells=4, seed=1)
    ctx = evc.Context.stencil(N, 0.3, 2, V, precision=evc.EVC_MIXED)
    ctx.set_precond(evc.EVC_PREC_IDENTITY)
    # one Lanczos run per shift (with shared runs the shift never reaches the
    # FP32 operator, and the merged requests share their columns)
    ctx.set_option(evc.EVC_OPT_SHARED_KRYLOV, 0)
    Vb = I.gaussian_wells(40, 0.3, nwells=4, seed=1)
    big = evc.Context.stencil(40, 0.3, 2, Vb, precision=evc.EVC_MIXED)
    big.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
    srv = evc.evc_server_create(8 << 30, slots=1, max_batch=8)
    try:
        mid = evc.evc_server_add_matrix(srv, ctx.h)
        mbig = evc.evc_server_add_matrix(srv, big.h)
        good = [dict(matrix_id=mid, xi=-2.0 + 0.2 * q, eta=0.5, nprobe=32, maxsteps=15, tol=0.0,
                     seed=9) for q in range(3)]
        alone = []
        for g in good:
            rc, r = evc.evc_server_wait(srv, evc.evc_server_submit(srv, **g))
            assert rc == evc.EVC_OK
            alone.append(r)
        blocker = evc.evc_server_submit(srv, mbig, -1.0, 1.0, 64, 80, 0.0, 1)
        bad = evc.evc_server_submit(srv, mid, -1e300, 0.5, 32, 15, 0.0, 9)
        tks = [evc.evc_server_submit(srv, **g) for g in good]
        rc, rb = evc.evc_server_wait(srv, bad)
        assert rc == evc.EVC_ENUMERIC
        for tk, ra in zip(tks, alone):
            rc, r = evc.evc_server_wait(srv, tk)
            assert rc == evc.EVC_OK
            assert r["estimate"] == ra["estimate"]
        assert rb["batch_size"] > 1                      # it did share a launch
        assert evc.evc_server_wait(srv, blocker)[0] == evc.EVC_OK
    finally:
        evc.evc_server_destroy(srv)
        ctx.close()
        big.close()
