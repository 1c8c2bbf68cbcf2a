"""Local refinement of a conforming tetrahedral mesh by longest-edge bisection (the adaptive
meshes of Sec. 4.2 and 4.3: the paper refines where a residual indicator is large but does not
say how; this is Rivara's longest-edge bisection with conforming closure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The rules, which the library follows exactly:

* Edges are ordered by squared length, computed as ``(dx*dx + dy*dy) + dz*dz`` with
  d = x_b - x_a and no fused multiply-add, ties broken by the smaller vertex pair
  ``(min, max)`` in lexicographic order.  The longest edge of a tet is the largest of its six
  edges in this order; its local positions are i < j.
* Bisecting a tet on its longest edge with midpoint m = 0.5 * (x_a + x_b) gives child 0 = the
  tet with its vertex j replaced by m (it keeps the tet's index) and child 1 = the tet with
  its vertex i replaced by m (it is appended).  Both keep the orientation.
* A refinement call bisects every marked tet on its longest edge and then whatever
  conformity requires: an edge that is to be bisected is bisected in every tet containing it,
  and a tet is bisected only on its longest edge, so a tet that contains such an edge first
  gets its own longest edge bisected (closure).  This runs in passes: close the set of edges
  to bisect (add the longest edge of every tet that contains one, until nothing changes),
  then bisect every tet whose longest edge is in the set, all at once.  It stops when no tet
  contains an edge of the set.
* New vertices are numbered in each pass in the order of the first tet (lowest index) whose
  longest edge they bisect; appended children in the order of their parents.
* A new vertex is a Dirichlet vertex when it lies on the boundary of the mesh (on a face that
  belongs to one tet only): the homogeneous condition holds on all of the boundary (Sec. 2).
"""
from __future__ import annotations

import numpy as np

_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def edge_len2(xyz: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Squared length of the segments (a, b) in the fixed evaluation order above."""
    d = xyz[b] - xyz[a]
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def longest_edge(xyz: np.ndarray, tets: np.ndarray):
    """Local index (0..5 into the edge list (01, 02, 03, 12, 13, 23)) and vertex pair
    (min, max) of the longest edge of every tet."""
    nt = len(tets)
    best = np.zeros(nt, dtype=np.int64)
    lo = np.minimum(tets[:, 0], tets[:, 1])
    hi = np.maximum(tets[:, 0], tets[:, 1])
    bl = edge_len2(xyz, tets[:, 0], tets[:, 1])
    for q, (i, j) in enumerate(_EDGES[1:], start=1):
        a, b = tets[:, i], tets[:, j]
        l2 = edge_len2(xyz, a, b)
        ea, eb = np.minimum(a, b), np.maximum(a, b)
        better = (l2 > bl) | ((l2 == bl) & ((ea < lo) | ((ea == lo) & (eb < hi))))
        best = np.where(better, q, best)
        bl = np.where(better, l2, bl)
        lo = np.where(better, ea, lo)
        hi = np.where(better, eb, hi)
    return best, lo, hi


def _keys(tets: np.ndarray, nv_bound: int):
    """Edge keys min * nv_bound + max of the six edges of every tet, [nt, 6]."""
    out = np.empty((len(tets), 6), dtype=np.int64)
    for q, (i, j) in enumerate(_EDGES):
        a, b = tets[:, i], tets[:, j]
        out[:, q] = np.minimum(a, b) * nv_bound + np.maximum(a, b)
    return out


def boundary_faces(tets: np.ndarray) -> np.ndarray:
    """Sorted vertex triples of the faces that belong to exactly one tet."""
    f = np.sort(np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]],
                                tets[:, [0, 1, 2]]]), axis=1)
    u, c = np.unique(f, axis=0, return_counts=True)
    return u[c == 1]


def refine(xyz: np.ndarray, tets: np.ndarray, dirichlet: np.ndarray, marked: np.ndarray):
    """Longest-edge bisection of the marked tets with conforming closure (rules above).
    Returns (xyz, tets, dirichlet, passes)."""
    xyz = np.array(xyz, dtype=np.float64)
    tets = np.array(tets, dtype=np.int64)
    nv0 = len(xyz)
    big = np.int64(1) << 31                      # vertex ids stay below 2^31
    _, lo, hi = longest_edge(xyz, tets)
    marked = np.asarray(marked, dtype=bool)
    todo = set((lo[marked] * big + hi[marked]).tolist())       # edges to bisect
    mid = {}                                                   # edge -> midpoint vertex
    passes = 0
    while True:
        keys = _keys(tets, big)
        li, lo, hi = longest_edge(xyz, tets)
        lkey = lo * big + hi
        # closure: the longest edge of every tet containing an edge to bisect
        while True:
            arr = np.fromiter(todo, dtype=np.int64, count=len(todo))
            has = np.isin(keys, arr).any(axis=1)
            add = set(lkey[has].tolist()) - todo
            if not add:
                break
            todo |= add
        arr = np.fromiter(todo, dtype=np.int64, count=len(todo))
        bis = np.flatnonzero(np.isin(lkey, arr))
        if len(bis) == 0:
            break
        passes += 1
        # new midpoints in the order of the first tet that bisects them
        new = [k for k in dict.fromkeys(lkey[bis].tolist()) if k not in mid]
        for r, k in enumerate(new):
            mid[k] = len(xyz) + r
        if new:
            ka = np.array(new, dtype=np.int64)
            a, b = ka // big, ka % big
            xyz = np.concatenate([xyz, 0.5 * (xyz[a] + xyz[b])])
        m = np.array([mid[k] for k in lkey[bis].tolist()], dtype=np.int64)
        ij = np.array(_EDGES, dtype=np.int64)[li[bis]]
        c0 = tets[bis].copy()
        c1 = tets[bis].copy()
        c0[np.arange(len(bis)), ij[:, 1]] = m
        c1[np.arange(len(bis)), ij[:, 0]] = m
        tets[bis] = c0
        tets = np.concatenate([tets, c1])
    d = np.zeros(len(xyz), dtype=np.uint8)
    d[:nv0] = np.asarray(dirichlet, dtype=np.uint8)
    bf = boundary_faces(tets)
    onb = np.zeros(len(xyz), dtype=bool)
    onb[bf.ravel()] = True
    d[nv0:] = onb[nv0:]
    return xyz, tets.astype(np.int32), d, passes
