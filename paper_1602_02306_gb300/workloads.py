"""Named synthetic workloads (shapes, sizes, seeds, shifts) used by the
benchmark and the full-size parity tests.

Each workload is the input recipe only: the matrix comes from ``inputs``, the
shifts are fixed numbers recorded here with how they were obtained.  Nothing
here computes any part of the estimator.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import inputs as I


@dataclass
class Workload:
    name: str
    kind: str                     # "stencil" or "csr"
    shifts: list
    nprobe: int
    maxsteps: int
    tol: float = 0.0
    precond: str = "identity"     # identity | jacobi | cheb
    prec_params: tuple = (0.0, 0.0)
    N: int = 0
    h: float = 0.0
    order: int = 2
    csr_builder: object = None
    nwells: int = 32
    seed: int = 0
    min_steps: int = 3            # no tolerance stop before this step
    notes: dict = field(default_factory=dict)
    _csr: object = field(default=None, repr=False, compare=False)

    @property
    def n(self) -> int:
        if self.kind == "stencil":
            return self.N ** 3
        return self.notes["n"]

    def potential(self) -> np.ndarray:
        return I.gaussian_wells(self.N, self.h, nwells=self.nwells, seed=1)

    def csr(self):
        """The CSR arrays (built once per Workload object)."""
        if self._csr is None:
            self._csr = self.csr_builder()
        return self._csr


# Lowest eigenvalue of H = -1/2 Lap_h + V on the periodic 64^3 grid (7-point,
# h = 0.3, 32 wells, well seed 1) by scipy.sparse.linalg.eigsh (ARPACK,
# which='SA', tol 1e-10).
FD64_LAMBDA_MIN = -3.2826731738772574

# Upper endpoint with exactly 300 eigenvalues below it: n_-(H - eta I) = 300 by
# Sylvester's law of inertia, counting the negative pivots of a symmetric-mode
# sparse LU of H - eta I (shift_search.py, k-section of [0.2, 1.6]: 0.48 -> 284,
# 0.4912 -> 289, 0.5024 -> 294, 0.5136 -> 300, 0.536 -> 309 eigenvalues below).
FD64_ETA = 0.5136


def fd64_eta() -> float:
    return FD64_ETA


def fd_hamiltonian_64() -> Workload:
    """3D FD Hamiltonian, 7-point periodic 64^3 (n = 262,144), h = 0.3, 32
    Gaussian wells; [lambda_min - 1, eta] with exactly 300 eigenvalues in it
    (eta between the 300th and 301st); Chebyshev degree-8 kinetic
    preconditioner (c = 1); 64 probes (seed 0); 30 Lanczos steps."""
    return Workload(name="fd_hamiltonian_64^3_7pt_cheb8_m64_k30", kind="stencil",
                    shifts=[FD64_LAMBDA_MIN - 1.0, fd64_eta()], nprobe=64, maxsteps=30,
                    precond="cheb", prec_params=(8, 1.0), N=64, h=0.3, order=2)


def laplace32() -> Workload:
    """2D Dirichlet 5-point Laplacian 32x32 (n = 1024), [1, 2], Jacobi, 16
    probes, 40 steps, FP64."""
    return Workload(name="laplace2d_32x32_jacobi_m16_k40", kind="csr", shifts=[1.0, 2.0],
                    nprobe=16, maxsteps=40, precond="jacobi", prec_params=(1e-3, 0.0),
                    csr_builder=lambda: I.laplace2d_dirichlet(32), notes={"n": 1024})


# Lowest eigenvalue of the 13-point (4th-order) periodic 96^3 Hamiltonian,
# h = 0.3, 32 wells (seed 1), by scipy.sparse.linalg.eigsh (which='SA', tol 1e-10).
FD96_LAMBDA_MIN = -2.767709970053203


def slicing_96_profile() -> Workload:
    """A smaller case of the 13-point passes for profiling: the 96^3
    Hamiltonian of batched_slicing_96 with its first 2 shifts (4 chunks of
    32 columns, each chunk vector 113 MB, still near L2's size), 4 steps --
    about 3 GB on the device."""
    W = batched_slicing_96()
    W.name = "slicing_96^3_13pt_cheb8_S2_m64_k4"
    W.shifts = W.shifts[:2]
    W.maxsteps = 4
    W.tol = 0.0
    return W


def batched_slicing_96() -> Workload:
    """Spectrum slicing of the 4th-order 13-point periodic 96^3 Hamiltonian
    (n = 884,736, h = 0.3, 32 wells): 32 shifts lambda_min + 8 s/32,
    s = 1..32, 64 probes each in one batched launch, per-shift stop at
    tol 0.25, at least 10 and at most 30 steps, shared Chebyshev-8 kinetic
    preconditioner."""
    lmin = FD96_LAMBDA_MIN
    return Workload(name="slicing_96^3_13pt_cheb8_S32_m64_tol0.25", kind="stencil",
                    shifts=[lmin + 8.0 * s / 32 for s in range(1, 33)], nprobe=64, maxsteps=30,
                    tol=0.25, precond="cheb", prec_params=(8, 1.0), N=96, h=0.3, order=4,
                    min_steps=10)


def powerlaw_2m() -> Workload:
    """Generic sparse symmetric n = 2,000,000, power-law rows (mean ~30, at
    most ~2000), N(0,1) values, diagonal U(-5,5), [-0.5, 0.5], Jacobi
    1/(|d - sigma| + 1e-3), 128 probes, 50 steps."""
    return Workload(name="powerlaw_2M_jacobi_m128_k50", kind="csr", shifts=[-0.5, 0.5],
                    nprobe=128, maxsteps=50, precond="jacobi", prec_params=(1e-3, 0.0),
                    csr_builder=lambda: I.powerlaw_symmetric(2_000_000, cap=2000, seed=2),
                    notes={"n": 2_000_000})


def powerlaw_1m_profile() -> Workload:
    """A smaller case of the same CSR pass for profiling: power-law rows as in
    powerlaw_2m with n = 1,200,000 (each chunk's 32-column x vector, 154 MB,
    is still larger than L2, so the gathers reach DRAM), 64 probes, 4 steps --
    about 2.5 GB on the device."""
    return Workload(name="powerlaw_1.2M_jacobi_m64_k4", kind="csr", shifts=[-0.5, 0.5],
                    nprobe=64, maxsteps=4, precond="jacobi", prec_params=(1e-3, 0.0),
                    csr_builder=lambda: I.powerlaw_symmetric(1_200_000, cap=2000, seed=2),
                    notes={"n": 1_200_000})


# The paper's Laplace test problem (Sec. 7, Table 1 "Laplace" row; the mesh
# family h = 2^-6 .. 2^-10 of its mesh-independence study): the 5-point
# Dirichlet Laplacian on the unit square scaled by 1/h^2, tau = 3000.
LAPLACE_TAU = 3000.0


def laplace_exact_below(e: int, tau: float = LAPLACE_TAU) -> int:
    """n_-(A - tau I) of the h = 2^-e Laplacian from its closed-form spectrum
    (4/h^2)(sin^2(i pi h/2) + sin^2(j pi h/2)), i, j = 1 .. 2^e - 1:
    230, 226, 222, 220, 220 for e = 6 .. 10 (Table 1 prints 226 for e = 7)."""
    h = 2.0 ** -e
    i = np.arange(1, 2 ** e)
    s = 4.0 * np.sin(i * np.pi * h / 2.0) ** 2 / h ** 2
    return int(((s[:, None] + s[None, :]) < tau).sum())


def laplace_paper(e: int, k: int = 134, m: int = 50) -> Workload:
    """Laplace h = 2^-e (N = 2^e - 1 interior points per axis, n = N^2),
    tau = 3000, m = 50 probes, k Lanczos steps (134 is Table 1's k for the
    unpreconditioned run at h = 2^-7).  Jacobi: the diagonal is the constant
    4/h^2, so M is a scalar and the run is the paper's unpreconditioned row."""
    N, h = 2 ** e - 1, 2.0 ** -e
    return Workload(name=f"laplace2d_h2^-{e}_tau3000_m{m}_k{k}", kind="csr",
                    shifts=[LAPLACE_TAU], nprobe=m, maxsteps=k, precond="jacobi",
                    prec_params=(1e-3, 0.0),
                    csr_builder=lambda: I.laplace2d_dirichlet(N, scale=1.0 / h ** 2),
                    notes={"n": N * N, "h": h, "e": e})


WORKLOADS = {
    "fd64": fd_hamiltonian_64,
    "laplace32": laplace32,
    "slicing96": batched_slicing_96,
    "powerlaw2m": powerlaw_2m,
    "powerlaw1m": powerlaw_1m_profile,
    "slicing96x2": slicing_96_profile,
    "laplace2^-7": lambda: laplace_paper(7),
    "laplace2^-10": lambda: laplace_paper(10),
}
