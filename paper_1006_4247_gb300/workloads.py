"""Seeded synthetic inputs for the parallel-tempering engine and its tests.

This module holds no arithmetic of the method: it only draws the quenched
couplings, builds inverse-temperature ladders and test configurations.  Both
the CUDA engine's tests and the CPU oracle's tests take their inputs from here.

Couplings follow section I of Hasenbusch & Schaefer (arXiv:1006.4247): one
independent Gaussian J_xy of zero mean and unit variance per nearest-neighbour
bond of the periodic L^3 lattice.  Layout [3, N], J[mu, x] for the bond
(x, x + e_mu), x = i + L (j + L k); values are float32 so that both sides see
the same numbers.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def couplings(L: int, seed: int) -> np.ndarray:
    """Gaussian couplings J ~ N(0, 1), float32 [3, L^3]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((3, L ** 3)).astype(np.float32)


def linear_betas(n: int, beta_min: float, beta_max: float) -> np.ndarray:
    """n inverse temperatures spaced linearly in [beta_min, beta_max]."""
    return np.linspace(beta_min, beta_max, n, dtype=np.float64)


def geometric_betas(n: int, t_min: float = 0.12, t_max: float = 0.19) -> np.ndarray:
    """The temperature ladder of section IV: T_i = T_max (T_min/T_max)^((i-1)/(n-1)),
    returned as increasing inverse temperatures."""
    i = np.arange(n, dtype=np.float64)
    T = t_max * (t_min / t_max) ** (i / (n - 1))
    return 1.0 / T


def random_spins(L: int, seed: int, count: int | None = None) -> np.ndarray:
    """Unit spins drawn uniformly on the sphere (normalised Gaussian vectors),
    float64 [count, N, 3] (or [N, 3] when count is None)."""
    rng = np.random.default_rng(seed)
    shape = (L ** 3, 3) if count is None else (count, L ** 3, 3)
    v = rng.standard_normal(shape)
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


@dataclass
class Workload:
    """A batch of disorder samples run together."""
    name: str
    L: list
    n_replicas: list
    beta_min: float
    beta_max: float
    n_copies: int = 2
    n_hb: int = 1
    n_or: int = 1
    j_seed0: int = 0
    exchange: str = "plain"
    eps: float = 0.0
    extra: dict = field(default_factory=dict)

    @property
    def n_samples(self) -> int:
        return len(self.L)

    def couplings(self):
        return [couplings(L, self.j_seed0 + s) for s, L in enumerate(self.L)]

    def betas(self):
        return [linear_betas(n, self.beta_min, self.beta_max) for n in self.n_replicas]

    def spins_total(self) -> int:
        return sum(self.n_copies * n * L ** 3 for L, n in zip(self.L, self.n_replicas))


def uniform(name, L, n_samples, n_replicas, beta_min, beta_max, **kw) -> Workload:
    return Workload(name, [L] * n_samples, [n_replicas] * n_samples, beta_min, beta_max, **kw)


# The workloads the engine is measured and checked on.  Sizes: L^3 sites,
# n_replicas inverse temperatures per copy, two copies for the overlap.
WORKLOADS = {
    # L=4, 8 replicas, beta linear in [2.5, 8.0], 1 HB + 3 OR, plain swap.
    "L4_R8_S1": lambda: uniform("L4_R8_S1", 4, 1, 8, 2.5, 8.0, n_hb=1, n_or=3,
                                j_seed0=1, exchange="plain"),
    # L=16, 24 replicas x 2 copies x 64 samples, beta in [2.0, 8.0], 1 HB + 5L/4 OR.
    "L16_R24_S64": lambda: uniform("L16_R24_S64", 16, 64, 24, 2.0, 8.0, n_hb=1, n_or=20,
                                   j_seed0=100, exchange="coolheat", eps=0.017),
    # L=32, 48 replicas x 2 copies x 16 samples, 1 HB + 5L/4 OR, modified exchange.
    "L32_R48_S16": lambda: uniform("L32_R48_S16", 32, 16, 48, 2.0, 8.0, n_hb=1, n_or=40,
                                   j_seed0=200, exchange="decimation", eps=0.007),
}


def uneven_batch(seed: int = 300, n_samples: int = 256) -> Workload:
    """Samples with L drawn from {8, 12, 16, 24, 32} and 16..48 replicas each."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice([8, 12, 16, 24, 32], size=n_samples).tolist()
    nts = rng.integers(16, 49, size=n_samples).tolist()
    w = Workload("uneven_S256", Ls, nts, 2.0, 8.0, n_hb=1, n_or=0, j_seed0=seed * 1000)
    w.extra["n_or_per_L"] = {L: 5 * L // 4 for L in (8, 12, 16, 24, 32)}
    return w
