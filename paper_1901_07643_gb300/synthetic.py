"""Seeded synthetic inputs: samples of random linear-Gaussian structural equation models.

This module holds input generation only (no step of the scoring method) and is
the one piece of code shared by the oracle's tests and the CUDA path's tests
and benchmark.

Recipe (the paper ships no data; the workloads are synthetic):

* a random DAG over a random variable order: for positions a < b in the order,
  an edge order[a] -> order[b] with probability ``edge_p``;
* edge weights sign * U[0.5, 2] with sign +-1 equally likely;
* noise N(0, sigma_v^2) with sigma_v^2 ~ U[0.5, 1.5] per variable;
* ancestral sampling of n rows;
* optional near-collinear columns: ``collinear`` target columns are each
  replaced by another uniformly chosen column plus N(0, 1e-3) noise (1e-3 is
  the variance), applied after sampling;
* optional bootstrap resampling of the rows (with replacement).

Everything is drawn from ``numpy.random.default_rng(seed)`` (PCG64).  Columns
are returned raw (not centred); the scoring path centres them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Tuple

import numpy as np


def sem_sample(m: int, n: int, edge_p: float, seed: int, collinear: int = 0,
               bootstrap: bool = False) -> np.ndarray:
    """n x m float64 sample (row-major) of a seeded random linear-Gaussian SEM."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(m)
    W = np.zeros((m, m))
    for a in range(m):
        for b in range(a + 1, m):
            if rng.random() < edge_p:
                sign = 1.0 if rng.random() < 0.5 else -1.0
                W[order[a], order[b]] = sign * rng.uniform(0.5, 2.0)
    sigma2 = rng.uniform(0.5, 1.5, size=m)
    X = np.zeros((n, m))
    for a in range(m):
        v = order[a]
        X[:, v] = X @ W[:, v] + rng.normal(0.0, math.sqrt(sigma2[v]), size=n)
    if collinear:
        targets = rng.choice(m, size=collinear, replace=False)
        for t in targets:
            src = int(rng.choice([j for j in range(m) if j != t]))
            X[:, t] = X[:, src] + rng.normal(0.0, math.sqrt(1e-3), size=n)
    if bootstrap:
        X = X[rng.integers(0, n, size=n)]
    return np.ascontiguousarray(X)


@dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    edge_p: float
    seed: int
    collinear: int = 0


# The single-instance workloads, named by what they are.
SMALL_M10 = Workload("sem_m10_n200", 10, 200, 0.3, 1000)
MEDIUM_M20 = Workload("sem_m20_n1000", 20, 1000, 0.2, 2000)
PROFILE_M24 = Workload("sem_m24_n2000", 24, 2000, 0.15, 2400)
LARGE_M26 = Workload("sem_m26_n5000_collinear2", 26, 5000, 0.15, 3000,
                     collinear=int(math.ceil(0.05 * 26)))


def workload_sample(w: Workload) -> np.ndarray:
    return sem_sample(w.m, w.n, w.edge_p, w.seed, w.collinear)


def batched_bootstrap(count: int = 256, seed: int = 4, base_seed: int = 4000,
                      m_range: Tuple[int, int] = (12, 20), n_range: Tuple[int, int] = (100, 5000),
                      edge_p: float = 0.25) -> List[np.ndarray]:
    """Many bootstrap-resampled datasets of uneven m and n, each from its own SEM."""
    sizes = np.random.default_rng(seed)
    ms = sizes.integers(m_range[0], m_range[1] + 1, size=count)
    ns = sizes.integers(n_range[0], n_range[1] + 1, size=count)
    return [sem_sample(int(ms[i]), int(ns[i]), edge_p, base_seed + i, bootstrap=True)
            for i in range(count)]


def gradient_workload(count: int = 64, m: int = 16, n: int = 2000, base_seed: int = 5000,
                      w_seed: int = 5999, edge_p: float = 0.2):
    """Datasets plus per-family weights w ~ N(0,1) for the backward pass."""
    Xs = [sem_sample(m, n, edge_p, base_seed + i) for i in range(count)]
    w = np.random.default_rng(w_seed).standard_normal(m << (m - 1))
    return Xs, w


def integer_sample(m: int, n: int, seed: int, lo: int = -4, hi: int = 4) -> np.ndarray:
    """Small integer-valued matrix (exact rational checks)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(n, m)).astype(np.float64)
