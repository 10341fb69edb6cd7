"""Seeded synthetic workloads (parameters and neutral random inputs).

This module holds no arithmetic of the method: it only names the synthetic
configurations (sizes, disorder width, localisation length, hop cut-off,
temperature, field, seeds) and draws neutral random inputs (occupations for
property tests) from numpy's seeded generator.  Both the CUDA library's tests
and the CPU oracle's tests take their inputs from here.

The paper draws every input at random (uniform site energies, random initial
configuration, section "Results for the lattice model in two dimensions"), so
there is no dataset to stand in for; the configurations below follow the
paper's 2D lattice model at half filling with the sizes and temperatures of
the benchmark plan.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict

import numpy as np


@dataclass(frozen=True)
class Replica:
    """Parameters of one disorder replica (the arguments of ``cg_create``)."""
    L: int
    nu: float
    W: float          # full width of the uniform site-energy interval
    xi: float
    r_max: int
    T: float
    E: float
    seed: int
    replica: int = 0
    dim: int = 2      # 2: L x L square lattice; 3: L x L x L cubic lattice
    sites: int = 0    # 0: lattice sites; 1: random positions in the L x L box

    def as_dict(self):
        return asdict(self)


@dataclass(frozen=True)
class Workload:
    name: str
    replicas: tuple
    M: int
    hops: int
    precision: str = "fp64"
    refresh_every: int = 0
    notes: str = ""
    extra: dict = field(default_factory=dict)


def l16_fp64() -> Workload:
    """L=16 (N=256), nu=1/2, phi ~ U[-0.5, 0.5], xi=1, r_max=4, T=0.05, E=0,
    M=256, one replica, 1e4 hops, seed 0: the bit-exact trajectory case."""
    r = Replica(L=16, nu=0.5, W=1.0, xi=1.0, r_max=4, T=0.05, E=0.0, seed=0)
    return Workload("L16_T0.05_fp64", (r,), M=256, hops=10_000)


def l64_fp64(T: float = 0.05, seed: int = 0, hops: int = 1_000_000) -> Workload:
    """L=64 (N=4096), nu=1/2, phi ~ U[-0.5, 0.5], xi=1, r_max=6, field E=0.01
    along x, M=4096; T in {0.02, 0.05, 0.1}, disorder seeds 0..7."""
    r = Replica(L=64, nu=0.5, W=1.0, xi=1.0, r_max=6, T=T, E=0.01, seed=seed)
    return Workload(f"L64_T{T}_s{seed}_fp64", (r,), M=4096, hops=hops)


L64_TEMPERATURES = (0.02, 0.05, 0.1)
L64_SEEDS = tuple(range(8))


def l128(seed: int = 0, precision: str = "fp32", M: int = 4096,
         hops: int = 10_000_000) -> Workload:
    """L=128 (N=16384), nu=1/2, phi ~ U[-1, 1] (W=2), xi=1, r_max=8, T=0.01,
    E=0.005; M swept 1024..65536; FP32 eps with an FP64 refresh every 1024
    hops against the plain FP64 form."""
    r = Replica(L=128, nu=0.5, W=2.0, xi=1.0, r_max=8, T=0.01, E=0.005, seed=seed)
    return Workload(f"L128_T0.01_{precision}", (r,), M=M, hops=hops,
                    precision=precision, refresh_every=1024 if precision == "fp32" else 0)


L128_M_SWEEP = (1024, 4096, 16384, 65536)


def l128_batch(R: int, precision: str = "fp32", M: int = 4096,
               hops: int = 1024) -> Workload:
    """R disorder replicas of the L=128, T=0.01 system (seeds 0..R-1): the
    batched form of the L=128 workload."""
    reps = tuple(Replica(L=128, nu=0.5, W=2.0, xi=1.0, r_max=8, T=0.01,
                         E=0.005, seed=s, replica=s) for s in range(R))
    return Workload(f"L128_T0.01_{precision}_R{R}", reps, M=M, hops=hops,
                    precision=precision, refresh_every=1024)


def mixed_batch(R: int = 256, sizes=(32, 48, 64, 96), draw_seed: int = 0) -> Workload:
    """R disorder replicas with L drawn uniformly from ``sizes`` (numpy seeded
    draw), phi ~ U[-0.5, 0.5], xi=1, r_max=6, T=0.03, E=0.01, replica s uses
    Philox seed s; FP32 eps with a split-BF16 refresh per same-L group."""
    rng = np.random.default_rng(draw_seed)
    Ls = rng.choice(np.asarray(sizes), size=R)
    reps = tuple(Replica(L=int(L), nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.03,
                         E=0.01, seed=s, replica=s) for s, L in enumerate(Ls))
    return Workload(f"mixed_L{'-'.join(map(str, sizes))}_R{R}", reps, M=4096,
                    hops=4096, precision="fp32", refresh_every=1024)


def l256(R: int = 16, hops: int = 10_000_000) -> Workload:
    """L=256 (N=65536), nu=1/2, phi ~ U[-0.5, 0.5], xi=1.5, r_max=10, T=0.02,
    E=0.005, 16 replicas, FP32 eps with a refresh every 4096 hops."""
    reps = tuple(Replica(L=256, nu=0.5, W=1.0, xi=1.5, r_max=10, T=0.02,
                         E=0.005, seed=s, replica=s) for s in range(R))
    return Workload(f"L256_T0.02_R{R}", reps, M=16384, hops=hops,
                    precision="fp32", refresh_every=4096)


def pairs(R: int = 304, pair_frac: float = 0.2, hops: int = 1_000_000) -> Workload:
    """Two-electron hops (the paper's multi-electron extension): L=64,
    nu=1/2, phi ~ U[-0.5, 0.5], xi=1, r_max=6, T=0.05, E=0.01, a fraction
    pair_frac of the labels proposing a pair with offsets |e| <= 4, FP32 eps
    refreshed every 1024 hops."""
    reps = tuple(Replica(L=64, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01,
                         seed=s, replica=s) for s in range(R))
    return Workload(f"pairs_L64_T0.05_R{R}_p{pair_frac}", reps, M=4096, hops=hops,
                    precision="fp32", refresh_every=1024,
                    extra={"pair_frac": pair_frac, "pair_rmax": 4})


def cubic(R: int = 152, L: int = 32, hops: int = 1_000_000,
          refresh_every: int = 1024) -> Workload:
    """The cubic lattice the paper's conclusions name as the next extension:
    L x L x L sites (N = 32768 for L=32), nu=1/2, phi ~ U[-0.5, 0.5], xi=1,
    hops inside the ball |d| <= 3 (122 vectors), T=0.05, E=0.01, one replica
    per SM, FP32 eps with a refresh from scratch every `refresh_every` hops
    (a refresh costs N^2 pair terms: larger lattices refresh less often)."""
    reps = tuple(Replica(L=L, nu=0.5, W=1.0, xi=1.0, r_max=3, T=0.05, E=0.01,
                         seed=s, replica=s, dim=3) for s in range(R))
    return Workload(f"cubic_L{L}_T0.05_R{R}", reps, M=4096, hops=hops,
                    precision="fp32", refresh_every=refresh_every)


def random_sites(R: int = 152, L: int = 64, hops: int = 1_000_000,
                 lattice: bool = False) -> Workload:
    """The random-site Coulomb glass (the off-lattice model of the paper's
    introduction): N = L^2 sites at uniform random positions in the L x L
    periodic box, nu=1/2, phi ~ U[-0.5, 0.5], xi=1, partners within
    r_max=6, T=0.05, E=0.01, one replica per SM, binary64 (the N x N
    coupling matrix in device memory).  lattice=True: the same replicas on
    the square lattice, for comparison."""
    reps = tuple(Replica(L=L, nu=0.5, W=1.0, xi=1.0, r_max=6, T=0.05, E=0.01,
                         seed=s, replica=s, sites=0 if lattice else 1) for s in range(R))
    kind = "lattice" if lattice else "random"
    return Workload(f"{kind}_L{L}_T0.05_R{R}", reps, M=4096, hops=hops,
                    precision="fp64", refresh_every=0)


# ---------------------------------------------------------------------------
# neutral random inputs for property tests
# ---------------------------------------------------------------------------

def random_occupation(N: int, n_occ: int, seed: int) -> np.ndarray:
    """A uniformly random occupation with exactly ``n_occ`` electrons."""
    rng = np.random.default_rng(seed)
    n = np.zeros(N, np.uint8)
    n[rng.choice(N, size=n_occ, replace=False)] = 1
    return n


def random_phi(N: int, W: float, seed: int) -> np.ndarray:
    """Site energies uniform in [-W/2, W/2] from numpy's generator."""
    rng = np.random.default_rng(seed)
    return (rng.random(N) - 0.5) * W
