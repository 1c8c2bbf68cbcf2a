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


# ------------------------------------------------------------------ general tetrahedral meshes
#
# A mesh is (xyz [nv, 3], tets [nt, 4] vertex indices, dirichlet [nv] uint8 flags marking the
# vertices on the boundary of the unit cube).  These generators only lay out vertices and
# connectivity; element arithmetic is left to the oracle and the library.

def _cube_vertex(n: int, i, j, k):
    return i + (n + 1) * (j + (n + 1) * k)


def _cube_boundary(xyz: np.ndarray) -> np.ndarray:
    on = (xyz == 0.0) | (xyz == 1.0)
    return on.any(axis=1).astype(np.uint8)


def kuhn_mesh(n: int, xyz: np.ndarray | None = None):
    """The Kuhn mesh as a general mesh: cube (i, j, k) (i fastest) is split into the 6 tets of
    the paths 0 -> e_a -> e_a + e_b -> (1,1,1), permutations (a, b, c) in lexicographic order;
    tet 6 c + p is path p of cube c."""
    if xyz is None:
        xyz = uniform_xyz(n)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    c = np.arange(n ** 3)
    ci, cj, ck = c % n, (c // n) % n, c // (n * n)
    tets = np.empty((n ** 3, 6, 4), dtype=np.int32)
    for p, perm in enumerate(perms):
        off = np.zeros((n ** 3, 3), dtype=np.int64)
        tets[:, p, 0] = _cube_vertex(n, ci, cj, ck)
        for s, ax in enumerate(perm):
            off[:, ax] += 1
            tets[:, p, s + 1] = _cube_vertex(n, ci + off[:, 0], cj + off[:, 1], ck + off[:, 2])
    grid = uniform_xyz(n)
    return np.array(xyz, dtype=np.float64), tets.reshape(-1, 4), _cube_boundary(grid)


def five_tet_mesh(n: int):
    """Each cube split into 5 tets: 4 corner tets around a central one, the split alternating
    with the parity of i + j + k so that neighbouring cubes share their face diagonals."""
    xyz = uniform_xyz(n)
    tets = []
    corner_sets = {0: [(0, 1, 2, 4), (3, 1, 2, 7), (5, 1, 4, 7), (6, 2, 4, 7), (1, 2, 4, 7)],
                   1: [(1, 0, 3, 5), (2, 0, 3, 6), (4, 0, 5, 6), (7, 3, 5, 6), (0, 3, 5, 6)]}
    for k in range(n):
        for j in range(n):
            for i in range(n):
                cv = [_cube_vertex(n, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1))
                      for a in range(8)]
                for tset in corner_sets[(i + j + k) & 1]:
                    tets.append([cv[a] for a in tset])
    return xyz, np.array(tets, dtype=np.int32), _cube_boundary(xyz)


def bey_refine(xyz: np.ndarray, tets: np.ndarray, dirichlet: np.ndarray):
    """One round of Bey's red refinement: every tet into 8 (4 corner tets and 4 tets of the
    inner octahedron cut along the diagonal between the midpoints of edges 02 and 13).  An
    edge midpoint is a Dirichlet vertex when the edge lies on a boundary face (a face of one
    tet only) whose three vertices are Dirichlet vertices."""
    tets = np.asarray(tets, dtype=np.int64)
    nv = len(xyz)
    pairs = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    e = np.stack([np.sort(tets[:, list(p)], axis=1) for p in pairs], axis=1)   # [nt, 6, 2]
    keys = e[:, :, 0] * nv + e[:, :, 1]
    uk, inv = np.unique(keys.ravel(), return_inverse=True)
    mid = nv + inv.reshape(-1, 6)
    a, b = uk // nv, uk % nv
    new_xyz = np.concatenate([xyz, 0.5 * (xyz[a] + xyz[b])])
    # boundary faces
    faces = np.sort(np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]],
                                    tets[:, [0, 1, 2]]]), axis=1)
    fk = (faces[:, 0] * nv + faces[:, 1]) * nv + faces[:, 2]
    fu, fc = np.unique(fk, return_counts=True)
    bf = fu[fc == 1]
    f0, f1, f2 = bf // (nv * nv), (bf // nv) % nv, bf % nv
    bedges = np.unique(np.concatenate([np.minimum(f0, f1) * nv + np.maximum(f0, f1),
                                       np.minimum(f0, f2) * nv + np.maximum(f0, f2),
                                       np.minimum(f1, f2) * nv + np.maximum(f1, f2)]))
    d_f = np.asarray(dirichlet, dtype=bool)
    face_dir = d_f[f0] & d_f[f1] & d_f[f2]
    bedges_dir = np.unique(np.concatenate([
        (np.minimum(f0, f1) * nv + np.maximum(f0, f1))[face_dir],
        (np.minimum(f0, f2) * nv + np.maximum(f0, f2))[face_dir],
        (np.minimum(f1, f2) * nv + np.maximum(f1, f2))[face_dir]]))
    del bedges
    new_dir = np.concatenate([d_f, np.isin(uk, bedges_dir)]).astype(np.uint8)
    # children: vertex ids of the parent corners and edge midpoints
    m = {p: mid[:, q] for q, p in enumerate(pairs)}
    v = [tets[:, q] for q in range(4)]
    def M(x, y):
        return m[(min(x, y), max(x, y))]
    kids = [(v[0], M(0, 1), M(0, 2), M(0, 3)), (M(0, 1), v[1], M(1, 2), M(1, 3)),
            (M(0, 2), M(1, 2), v[2], M(2, 3)), (M(0, 3), M(1, 3), M(2, 3), v[3]),
            (M(0, 1), M(0, 2), M(0, 3), M(1, 3)), (M(0, 1), M(0, 2), M(1, 2), M(1, 3)),
            (M(0, 2), M(0, 3), M(1, 3), M(2, 3)), (M(0, 2), M(1, 2), M(1, 3), M(2, 3))]
    new_tets = np.stack([np.stack(kd, axis=1) for kd in kids], axis=1).reshape(-1, 4)
    return new_xyz, new_tets.astype(np.int32), new_dir


def relabel_mesh(xyz, tets, dirichlet, seed: int = 0):
    """Random renumbering of the vertices and the tets and a random order of each tet's
    vertices (the mesh itself is unchanged)."""
    rng = np.random.default_rng(seed)
    nv = len(xyz)
    perm = rng.permutation(nv)          # new index of old vertex v is inv[v]
    inv = np.empty(nv, dtype=np.int64)
    inv[perm] = np.arange(nv)
    new_xyz = np.asarray(xyz)[perm]
    new_dir = np.asarray(dirichlet)[perm]
    t = inv[np.asarray(tets, dtype=np.int64)]
    t = t[rng.permutation(len(t))]
    order = np.argsort(rng.random(t.shape), axis=1)
    t = np.take_along_axis(t, order, axis=1)
    return new_xyz, t.astype(np.int32), new_dir
