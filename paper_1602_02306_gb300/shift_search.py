"""Offline search for the interval endpoint of the 64^3 FD-Hamiltonian workload.

Finds a shift eta with exactly `target` eigenvalues of H = -1/2 Lap_h + V below
it (7-point periodic, N = 64, h = 0.3, 32 wells, seed 1) by Sylvester's law
of inertia: H - eta I = P L D L^T P^T from scipy's SuperLU in symmetric mode
(diagonal pivoting, symmetric fill-reducing ordering), n_-(H - eta I) = number
of negative pivots.  Several shifts are factored in parallel processes per
round (k-section).  Takes hours on a few CPU cores; the result is recorded
as constants in workloads.py.

    python -m paper_1602_02306_gb300.shift_search --lo 0.2 --hi 1.6 --target 300
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import time

import numpy as np


def _hamiltonian(N=64, h=0.3):
    import scipy.sparse as sp
    from . import inputs as I
    V = I.gaussian_wells(N, h, nwells=32, seed=1)
    e = np.ones(N)
    T = sp.diags([-e[:-1], 2 * e, -e[:-1]], [-1, 0, 1], shape=(N, N), format="lil")
    T[0, N - 1] = -1
    T[N - 1, 0] = -1
    L1 = T.tocsr() / h ** 2
    Id = sp.identity(N, format="csr")
    K = 0.5 * (sp.kron(sp.kron(Id, Id), L1) + sp.kron(sp.kron(Id, L1), Id) +
               sp.kron(sp.kron(L1, Id), Id))
    return (K + sp.diags(V)).tocsc()


def negative_inertia(eta: float):
    """(n_-(H - eta I), smallest |pivot|) by symmetric-mode sparse LU."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    H = _hamiltonian()
    lu = sla.splu((H - eta * sp.identity(H.shape[0], format="csc")).tocsc(),
                  permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                  options=dict(SymmetricMode=True))
    if not np.array_equal(lu.perm_r, lu.perm_c):
        raise RuntimeError("row pivoting left the symmetric permutation; inertia undefined")
    d = lu.U.diagonal()
    return int((d < 0).sum()), float(np.min(np.abs(d)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lo", type=float, required=True)
    ap.add_argument("--hi", type=float, required=True)
    ap.add_argument("--target", type=int, default=300)
    ap.add_argument("--procs", type=int, default=4)
    ap.add_argument("--rounds", type=int, default=6)
    ap.add_argument("--out", default="shift_search.json")
    a = ap.parse_args()
    lo, hi = a.lo, a.hi
    log = []
    ctx = mp.get_context("spawn")
    for rnd in range(a.rounds):
        etas = list(np.linspace(lo, hi, a.procs + 2)[1:-1])
        t0 = time.time()
        with ctx.Pool(a.procs) as pool:
            res = pool.map(negative_inertia, etas)
        for eta, (cnt, piv) in zip(etas, res):
            log.append({"eta": eta, "count": cnt, "min_abs_pivot": piv})
            print(json.dumps(log[-1]), f"{time.time() - t0:.0f}s", flush=True)
            if cnt == a.target:
                json.dump({"eta": eta, "count": cnt, "log": log}, open(a.out, "w"), indent=1)
                return
        below = [e for e, (c, _) in zip(etas, res) if c < a.target]
        above = [e for e, (c, _) in zip(etas, res) if c > a.target]
        lo = max(below) if below else lo
        hi = min(above) if above else hi
    json.dump({"eta": None, "log": log}, open(a.out, "w"), indent=1)


if __name__ == "__main__":
    main()
