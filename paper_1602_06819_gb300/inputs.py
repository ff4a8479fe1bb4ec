"""Seeded synthetic inputs: isotropic Gaussian mixtures.

The paper's synthetic dataset is a mixture of Gaussians in R^3 searched with
the Euclidean distance (Sec. 8.1).  The workloads here keep that recipe at
larger dimensions: component means uniform in [-a, a]^d, each point picks a
component uniformly at random and adds sigma * N(0, I).

This module holds no arithmetic of the method itself; it feeds both the CUDA
path and the CPU oracle the same numbers.  Every draw comes from numpy's
PCG64 with an explicit seed, so a (mixture, seed, n) triple always yields the
same float32 array.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Mixture:
    """A d-dimensional isotropic Gaussian mixture with fixed, seeded means."""

    d: int
    components: int
    half_width: float
    sigma: float
    seed: int

    @property
    def means(self) -> np.ndarray:
        rng = np.random.Generator(np.random.PCG64(self.seed))
        return rng.uniform(-self.half_width, self.half_width,
                           size=(self.components, self.d))

    def sample(self, n: int, seed: int, with_labels: bool = False):
        """n float32 points; the seed picks components and noise."""
        rng = np.random.Generator(np.random.PCG64(seed))
        labels = rng.integers(0, self.components, size=n)
        noise = rng.standard_normal(size=(n, self.d))
        x = (self.means[labels] + self.sigma * noise).astype(np.float32)
        return (x, labels) if with_labels else x


@dataclass(frozen=True)
class Workload:
    """Sizes and parameters of one synthetic workload."""

    name: str
    mixture: Mixture
    n_init: int
    n_insert: int
    k: int
    batch: int
    speedups: tuple
    expansion: float = 5.0
    depth: int = 2
    seed_init: int = 1
    seed_stream: int = 2
    seed_query: int = 3
    seed_search: int = 4

    def initial(self) -> np.ndarray:
        return self.mixture.sample(self.n_init, self.seed_init)

    def stream(self, n: int | None = None) -> np.ndarray:
        return self.mixture.sample(self.n_insert if n is None else n, self.seed_stream)

    def queries(self, n: int) -> np.ndarray:
        return self.mixture.sample(n, self.seed_query)


# n = 1,000 initial + 1,000 inserted one at a time, d = 16, 10 components,
# means in [-10, 10]^16, sigma 1, k = 10; update DEPTH 2, expansion 5.
SMALL_D16 = Workload(
    name="gmm-d16-n1k+1k-k10-batch1",
    mixture=Mixture(d=16, components=10, half_width=10.0, sigma=1.0, seed=11),
    n_init=1000, n_insert=1000, k=10, batch=1, speedups=(4, 8, 16, 20, 32))

# n = 100,000 initial + 100,000 inserted in batches of 1,024, d = 128,
# 100 components, means in [-20, 20]^128, sigma 1, k = 10.  The stream is one
# sample of 98 whole batches (100,352 points); a shorter run inserts a prefix
# of it, so every run of any length sees the same points in the same order.
PLAIN_D128 = Workload(
    name="gmm-d128-n100k+100k-k10-batch1024",
    mixture=Mixture(d=128, components=100, half_width=20.0, sigma=1.0, seed=21),
    n_init=100_000, n_insert=98 * 1024, k=10, batch=1024, speedups=(4, 8, 16, 32))

# n = 1,000,000 initial + 1,000,000 inserts, d = 96, 1,000 components,
# k = 20, screening storage BF16 / FP8-E4M3 with an FP32 re-score of 4k;
# inserted in batches of 8,192 (the graph is DRAM-resident and a launch lasts
# about as long as its slowest search, so larger batches share that time).
PRECISION_D96 = Workload(
    name="gmm-d96-n1M+1M-k20-batch8192",
    mixture=Mixture(d=96, components=1000, half_width=20.0, sigma=1.0, seed=31),
    n_init=1_000_000, n_insert=1_000_000, k=20, batch=8192, speedups=(4, 8, 16, 32))

WORKLOADS = {w.name: w for w in (SMALL_D16, PLAIN_D128, PRECISION_D96)}
