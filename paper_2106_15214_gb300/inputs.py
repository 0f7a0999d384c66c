"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the NMF method: it only draws random
matrices. Both the CUDA path's tests/benchmark and the CPU oracle's tests take
their inputs from here. Every generator is deterministic in its seed.

The paper's datasets (Sec. 4.2-4.5) are not available; each generator below is
a synthetic stand-in with the same shape class, value range and structure.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class DenseProblem:
    name: str
    beta: float
    V: np.ndarray          # F x N, float64
    W0: np.ndarray         # F x K initial W
    H0: np.ndarray         # K x N initial H
    iters: int

    @property
    def shape(self):
        return self.V.shape[0], self.V.shape[1], self.W0.shape[1]


@dataclass
class SparseProblem:
    name: str
    beta: float
    F: int
    N: int
    rowptr: np.ndarray     # int32, F + 1 (CSR)
    col: np.ndarray        # int32, nnz
    val: np.ndarray        # float32/64, nnz
    W0: np.ndarray
    H0: np.ndarray
    iters: int

    @property
    def rows(self):
        return np.repeat(np.arange(self.F, dtype=np.int64), np.diff(self.rowptr))


def uniform_init(F, N, K, seed=1, lo=0.1, hi=1.0):
    """Initial factors W ~ U(lo, hi)^{F x K}, H ~ U(lo, hi)^{K x N}."""
    rng = np.random.default_rng(seed)
    W = rng.uniform(lo, hi, size=(F, K))
    H = rng.uniform(lo, hi, size=(K, N))
    return W, H


def half_normal_init(F, N, K, seed=1):
    """Initial factors drawn half-normal, as in the paper's set-up (Sec. 4.1.2)."""
    rng = np.random.default_rng(seed)
    return np.abs(rng.standard_normal((F, K))), np.abs(rng.standard_normal((K, N)))


def random_dense(F, N, K, seed=0, beta=1.0, offset=0.01):
    """Small generic problem: V = W0 H0 + offset with Gamma(1,1) factors; U(0.1,1) init."""
    rng = np.random.default_rng(seed)
    W0 = rng.gamma(1.0, 1.0, size=(F, K))
    H0 = rng.gamma(1.0, 1.0, size=(K, N))
    V = W0 @ H0 + offset
    W, H = uniform_init(F, N, K, seed=seed + 1)
    return DenseProblem(f"random_{F}x{N}x{K}", beta, V, W, H, 1)


def dense_kl_small(seed=20210629, init_seed=1):
    """Dense KL (beta = 1), F=200, N=500, K=10: V = W0 H0 + 0.01 with
    W0, H0 ~ Gamma(1,1); W, H ~ U(0.1, 1); 200 iterations. Small Olivetti-like
    dense KL case (Sec. 4.2 shape class, reduced)."""
    F, N, K = 200, 500, 10
    rng = np.random.default_rng(seed)
    W0 = rng.gamma(1.0, 1.0, size=(F, K))
    H0 = rng.gamma(1.0, 1.0, size=(K, N))
    V = W0 @ H0 + 0.01
    W, H = uniform_init(F, N, K, seed=init_seed)
    return DenseProblem("dense_kl_200x500x10", 1.0, V, W, H, 200)


def dense_quadratic_faces(seed=20210629, init_seed=1):
    """Dense quadratic loss (beta = 2), F=361 (19x19 images), N=2429, K=49.

    W0 = U(0,1) . Bernoulli(0.3) (sparse-ish parts), H0 ~ Gamma(0.5, 1),
    X = W0 H0 / max(W0 H0), V = clip(X + N(0, 0.02^2), 0, 1). Face-image shape
    class (Sec. 4.2 stand-in); 1000 iterations."""
    F, N, K = 361, 2429, 49
    rng = np.random.default_rng(seed)
    W0 = rng.uniform(0.0, 1.0, size=(F, K)) * (rng.uniform(size=(F, K)) < 0.3)
    H0 = rng.gamma(0.5, 1.0, size=(K, N))
    X = W0 @ H0
    X = X / X.max()
    V = np.clip(X + rng.normal(0.0, 0.02, size=(F, N)), 0.0, 1.0)
    W, H = uniform_init(F, N, K, seed=init_seed)
    return DenseProblem("dense_quadratic_361x2429x49", 2.0, V, W, H, 1000)


def dense_is_spectrogram(seed=20210629, init_seed=1, N=20000):
    """Dense Itakura-Saito (beta = 0), F=513 frequency bins, N frames (20000),
    K=20: V = max((W0 H0) . E, 1e-8) with W0, H0 ~ Gamma(1,1), E ~ Exp(1),
    a power-spectrogram-like matrix (Sec. 4.3 stand-in)."""
    F, K = 513, 20
    rng = np.random.default_rng(seed)
    W0 = rng.gamma(1.0, 1.0, size=(F, K))
    H0 = rng.gamma(1.0, 1.0, size=(K, N))
    E = rng.exponential(1.0, size=(F, N))
    V = np.maximum((W0 @ H0) * E, 1e-8)
    W, H = uniform_init(F, N, K, seed=init_seed)
    return DenseProblem(f"dense_is_513x{N}x20", 0.0, V, W, H, 200)


def sparse_counts(F=20000, N=100000, density=0.001, K=50, seed=20210629,
                  init_seed=1, p=0.3, dtype=np.float32):
    """Sparse play-count-like matrix for KL NMF (Sec. 4.4 stand-in).

    nnz = round(density F N) positions uniform without replacement; values
    1 + Geometric(p) on {0, 1, ...} (numpy's geometric counts trials, so the
    value is rng.geometric(p)), i.e. integer counts >= 1 with mean 1/p.
    Returned in CSR form with sorted columns inside each row.
    """
    rng = np.random.default_rng(seed)
    nnz = int(round(density * F * N))
    total = F * N
    picked = np.unique(rng.integers(0, total, size=int(nnz * 1.05) + 64, dtype=np.int64))
    while picked.size < nnz:
        more = rng.integers(0, total, size=nnz, dtype=np.int64)
        picked = np.unique(np.concatenate([picked, more]))
    picked = np.sort(rng.choice(picked, size=nnz, replace=False))
    rows = (picked // N).astype(np.int64)
    cols = (picked % N).astype(np.int32)
    vals = rng.geometric(p, size=nnz).astype(dtype)
    rowptr = np.zeros(F + 1, dtype=np.int32)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    W, H = uniform_init(F, N, K, seed=init_seed)
    return SparseProblem(f"sparse_kl_{F}x{N}_{nnz}nz_K{K}", 1.0, F, N, rowptr, cols,
                         vals, W, H, 100)


def batched_hyperspectral(count=512, seed=5, init_seed=1, F_range=(64, 256),
                          N_range=(256, 8192), K_range=(4, 32)):
    """Many independent beta = 1.5 problems (Sec. 4.5 stand-in): F, N, K drawn
    uniformly from the inclusive ranges; W0 ~ U(0,1), the columns of H0 are
    Dirichlet(1_K) abundances, V = W0 H0."""
    rng = np.random.default_rng(seed)
    Fs = rng.integers(F_range[0], F_range[1] + 1, size=count)
    Ns = rng.integers(N_range[0], N_range[1] + 1, size=count)
    Ks = rng.integers(K_range[0], K_range[1] + 1, size=count)
    problems = []
    for i in range(count):
        F, N, K = int(Fs[i]), int(Ns[i]), int(Ks[i])
        W0 = rng.uniform(0.0, 1.0, size=(F, K))
        H0 = rng.dirichlet(np.ones(K), size=N).T
        V = W0 @ H0
        W, H = uniform_init(F, N, K, seed=init_seed + i)
        problems.append(DenseProblem(f"hyper_{i}_{F}x{N}x{K}", 1.5, V, W, H, 1))
    return problems


def batched_shapes(count=512, seed=5, F_range=(64, 256), N_range=(256, 8192),
                   K_range=(4, 32)):
    """Just the (F, N, K) triples that batched_hyperspectral draws."""
    rng = np.random.default_rng(seed)
    Fs = rng.integers(F_range[0], F_range[1] + 1, size=count)
    Ns = rng.integers(N_range[0], N_range[1] + 1, size=count)
    Ks = rng.integers(K_range[0], K_range[1] + 1, size=count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(Fs, Ns, Ks)]
