"""Workload definitions and seeded synthetic inputs.

This module holds no arithmetic of the method: it names the lattice/contraction sizes of
the benchmark workloads and draws seeded random inputs (parameter vectors, configuration
batches) that both the CUDA path and the CPU oracle consume.

Workloads (the paper's benchmark shapes, Sec. III.A; no dataset is involved):
  heis4   4x4 open Heisenberg (J1=1), D=2, chi=4, FP64; Ns=2000, eps=1e-4, tau=0.02, 50 steps.
  heis8   8x8 open Heisenberg (J1=1), D=4, chi=16; 8192 chains; tau=0.02, 200 steps.
  j1j2_10 10x10 open J1-J2 (J1=1, J2=0.5), D=6, chi=36; Ns=16384; eps=1e-4, <=100 CG its.
  direct6 6x6 open Heisenberg (J1=1), D=2, chi=16, 30000 reweighted direct samples per SR
          step (App. A, Eqs. A2-A7; the sample count and lattice of the paper's direct-sampled
          runs, Sec. III.B, on the spin model), from the perturbed beta=0 state, b_d from 1.
  hubbard6 6x6 open Fermi-Hubbard (Sec. III.B: t=1, U=8, mu=4), fermionic PEPS with sixteen
          local states, D=4, chi=16, 1024 Metropolis chains, from the perturbed |I>.
  hubbard8 8x8 open Fermi-Hubbard at half filling (t=1, U=8, mu=4), D=6, chi=24, 8192
          samples per SR step, tau=0.01 (bench.py --fermion --workload hubbard8).
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    L: int
    D: int
    chi: int
    J1: float = 1.0
    J2: float = 0.0
    n_samples: int = 1024
    tau: float = 0.02
    eps: float = 1e-4
    n_steps: int = 50
    max_cg: int = 100
    cg_tol: float = 1e-10
    init_noise: float = 1e-3
    seed: int = 0
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "heis4": Workload("heis4", L=4, D=2, chi=4, n_samples=2000, tau=0.02, n_steps=50),
    "heis8": Workload("heis8", L=8, D=4, chi=16, n_samples=8192, tau=0.02, n_steps=200),
    "j1j2_10": Workload("j1j2_10", L=10, D=6, chi=36, J2=0.5, n_samples=16384, tau=0.01,
                        n_steps=300),
    "direct6": Workload("direct6", L=6, D=2, chi=16, n_samples=30000, tau=0.02, n_steps=100,
                        extra={"exponent": 0.5, "b_d0": 1.0, "su_t": 0.0}),
    "hubbard6": Workload("hubbard6", L=6, D=4, chi=16, n_samples=1024, tau=0.02, n_steps=100,
                         extra={"t": 1.0, "U": 8.0, "mu": 4.0}),
    "hubbard8": Workload("hubbard8", L=8, D=6, chi=24, n_samples=8192, tau=0.01, n_steps=200,
                         extra={"t": 1.0, "U": 8.0, "mu": 4.0}),
}


def site_dims(L1, L2, D):
    """Open-boundary leg dimensions (dl, dr, du, dd) of every site, row-major."""
    out = []
    for r in range(L1):
        for c in range(L2):
            out.append((1 if c == 0 else D, 1 if c == L2 - 1 else D,
                        1 if r == 0 else D, 1 if r == L1 - 1 else D))
    return out


def n_params(L1, L2, D):
    """Number of PEPS parameters with trimmed open boundaries: 4 * sum of site sizes."""
    return 4 * sum(int(np.prod(d)) for d in site_dims(L1, L2, D))


def random_theta(L1, L2, D, seed, scale=1.0, diag_bias=0.0):
    """Seeded random parameter vector.  diag_bias adds a constant to the [0,0,0,0] entry of
    the S = 0 and S = 3 slices of every site (a state near the beta = 0 product state)."""
    rng = np.random.default_rng(seed)
    dims = site_dims(L1, L2, D)
    th = scale * rng.standard_normal(n_params(L1, L2, D))
    off = 0
    for d in dims:
        sz = int(np.prod(d))
        th[off] += diag_bias
        th[off + 3 * sz] += diag_bias
        off += 4 * sz
    return th


def random_configs(L1, L2, n, seed, diagonal_fraction=0.5):
    """Seeded configuration batch, uint8 [n][L1*L2], entries S = 2 s + s' in 0..3.  A
    fraction of the rows is diagonal (s = s' on every site), the rest uniform."""
    rng = np.random.default_rng(seed)
    N = L1 * L2
    S = rng.integers(0, 4, size=(n, N), dtype=np.uint8)
    nd = int(round(diagonal_fraction * n))
    S[:nd] = 3 * rng.integers(0, 2, size=(nd, N), dtype=np.uint8)
    return S


def fermion_support_configs(n, N, seed):
    """n seeded configurations of N sixteen-valued sites with equal system and ancilla
    occupations on every site (a | a << 2, a uniform in 0..3)."""
    a = np.random.default_rng(seed).integers(0, 4, (n, N))
    return (a | (a << 2)).astype(np.uint8)
