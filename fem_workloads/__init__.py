"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and lays out workloads; it holds none of the
method's arithmetic (no assembly, no solver).  Both the oracle and the CUDA
library consume what it returns, so neither ever feeds the other.

Workloads stand in for the paper's experiments (Sec. 4: unit cube, smooth,
discontinuous and non-homogeneous targets) and for the batched and serving
workloads, which have no counterpart in the paper.
"""
from __future__ import annotations

import numpy as np


def grid_n(N: int) -> int:
    """Cells per side of the Kuhn mesh with N = (n-1)^3 interior unknowns."""
    n = round(N ** (1.0 / 3.0)) + 1
    assert (n - 1) ** 3 == N
    return n


def uniform_xyz(n: int) -> np.ndarray:
    """Vertex coordinates h*(i, j, k) of the (n+1)^3 grid, i fastest."""
    h = 1.0 / n
    i = np.arange(n + 1, dtype=np.float64) * h
    K, J, I = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)


def jittered_xyz(n: int, amp: float = 0.2, seed: int = 0) -> np.ndarray:
    """Uniform grid with every interior vertex moved by U(-amp*h, amp*h) per coordinate."""
    xyz = uniform_xyz(n)
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    d = rng.uniform(-amp * h, amp * h, size=xyz.shape)
    i = np.arange(n + 1)
    K, J, I = np.meshgrid(i, i, i, indexing="ij")
    inside = ((I > 0) & (I < n) & (J > 0) & (J < n) & (K > 0) & (K < n)).ravel()
    xyz[inside] += d[inside]
    return xyz


def sine_target() -> dict:
    """ubar = sin(pi x) sin(pi y) sin(pi z) (Sec. 4.1)."""
    return {"kind": "sine"}


def box_target(lo: float = 0.25, hi: float = 0.75) -> dict:
    """ubar = 1 on (lo, hi)^3, 0 elsewhere (Sec. 4.2)."""
    return {"kind": "box", "lo": lo, "hi": hi}


def sine_plus_one_target() -> dict:
    """ubar = 1 + sin sin sin, violating the boundary condition (Sec. 4.3)."""
    return {"kind": "sine_plus_one"}


def bump_target(seed: int, nb: int = 8) -> dict:
    """Sum of nb Gaussian bumps: centres U[0.1, 0.9]^3, widths U[0.05, 0.2], amplitudes N(0, 1)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.1, 0.9, size=(nb, 3))
    w = rng.uniform(0.05, 0.2, size=nb)
    a = rng.normal(0.0, 1.0, size=nb)
    return {"kind": "bumps", "centers": c, "widths": w, "amps": a}


def log_uniform(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))


def batched_workload(n: int = 128, nrhs: int = 64, seed: int = 1000):
    """Targets ubar_k (seed 1000 + k) and per-instance rho_k log-uniform in [1e-6, 1e-2]."""
    targets = [bump_target(seed + k) for k in range(nrhs)]
    rhos = log_uniform(nrhs, 1e-6, 1e-2, seed)
    return targets, rhos


def request_stream(count: int = 2000, rate: float = 100.0, seed: int = 7,
                   sizes=(32, 64, 96, 128, 192), rho_lo: float = 1e-8, rho_hi: float = 1.0):
    """Poisson arrivals (rate per second) of solve requests with random mesh size,
    log-uniform rho and a Gaussian-bump target."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    ns = rng.choice(np.asarray(sizes), size=count)
    rhos = np.exp(rng.uniform(np.log(rho_lo), np.log(rho_hi), size=count))
    seeds = rng.integers(0, 2 ** 31 - 1, size=count)
    return [{"id": i, "t": float(t[i]), "n": int(ns[i]), "rho": float(rhos[i]),
             "target": bump_target(int(seeds[i]))} for i in range(count)]


def random_vector(N: int, seed: int, nrhs: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(size=(N, nrhs) if nrhs > 1 else N)
    return np.ascontiguousarray(v)
