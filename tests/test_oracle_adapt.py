"""The adaptive loop's pieces in the oracle (Sec. 4.2-4.3: residual indicator after Verfurth,
bulk marking, local refinement), pinned to what the mathematics fixes:

* refinement: a plain recursive restatement of Rivara's longest-edge bisection (one tet at a
  time) reaches the same set of tets; the result is conforming, nested in the input, keeps
  every tet's orientation and the volume, refines every marked tet, and flags exactly the new
  vertices on the cube's surface;
* indicator: the volume term for u_h = 0 sums to the closed-form integral of the target, with
  the weight (h_T / sqrt(rho))^2 when that is below 1; the face term equals a separate
  computation of the normal-derivative jumps (gradients by least squares, areas by Heron's
  formula, normals by SVD); jumps vanish for a linear u_h; the indicator tracks the energy
  error under refinement;
* marking: brute force over all thresholds.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import fem_workloads as W
from oracle import core
from oracle import refine as R


# ------------------------------------------------------------------ refinement


def _recursive_leb(xyz, tets, marked):
    """Rivara's algorithm one tet at a time: to bisect an edge, first bisect (recursively)
    every tet around it whose longest edge is another one, then split all tets around it."""
    xyz = [tuple(p) for p in np.asarray(xyz, dtype=np.float64)]
    mesh = {}                              # id -> tuple of 4 vertex ids
    for t, v in enumerate(np.asarray(tets).tolist()):
        mesh[t] = tuple(v)
    nxt = [len(mesh)]
    mids = {}

    def l2(a, b):
        dx, dy, dz = (xyz[b][0] - xyz[a][0], xyz[b][1] - xyz[a][1], xyz[b][2] - xyz[a][2])
        return (dx * dx + dy * dy) + dz * dz

    def longest(v):
        best = None
        for i, j in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)):
            e = (min(v[i], v[j]), max(v[i], v[j]))
            k = (l2(v[i], v[j]), -e[0], -e[1])
            if best is None or k > best[0]:
                best = (k, e)
        return best[1]

    def bisect_edge(e):
        while True:
            star = [t for t, v in mesh.items() if e[0] in v and e[1] in v]
            bad = [t for t in star if longest(mesh[t]) != e]
            if not bad:
                break
            bisect_edge(longest(mesh[bad[0]]))
        if e not in mids:
            mids[e] = len(xyz)
            a, b = xyz[e[0]], xyz[e[1]]
            xyz.append(tuple(0.5 * (a[d] + b[d]) for d in range(3)))
        m = mids[e]
        for t in star:
            v = mesh.pop(t)
            for drop in e:
                w = tuple(m if x == drop else x for x in v)
                mesh[nxt[0]] = w
                nxt[0] += 1

    for t in np.flatnonzero(marked):
        if t in mesh:
            bisect_edge(longest(mesh[t]))
    return np.array(xyz), np.array(list(mesh.values()))


def _geometric_set(xyz, tets):
    return sorted(tuple(sorted(tuple(xyz[v]) for v in t)) for t in np.asarray(tets).tolist())


def _mesh_cases():
    yield "kuhn3", W.kuhn_mesh(3)
    yield "kuhn3_jittered", W.kuhn_mesh(3, W.jittered_xyz(3, 0.25, 5))
    yield "five3", W.five_tet_mesh(3)


@pytest.mark.parametrize("name,mesh", list(_mesh_cases()))
def test_refinement_equals_recursive_rivara(name, mesh):
    xyz, tets, d = mesh
    rng = np.random.default_rng(11)
    for _ in range(3):
        marked = rng.random(len(tets)) < 0.15
        x2, t2, d2, _ = R.refine(xyz, tets, d, marked)
        xr, tr = _recursive_leb(xyz, tets, marked)
        assert len(t2) == len(tr) and len(x2) == len(xr)
        assert _geometric_set(x2, t2) == _geometric_set(xr, tr)
        xyz, tets, d = x2, t2, d2


def _locate(xyz0, tets0, p):
    """Index of the input tet containing point p strictly inside (barycentric > 0)."""
    X = xyz0[tets0]
    E = X[:, 1:, :] - X[:, :1, :]
    lam = np.linalg.solve(E.transpose(0, 2, 1), (p[None, :] - X[:, 0, :])[:, :, None])[:, :, 0]
    bary = np.concatenate([1 - lam.sum(axis=1, keepdims=True), lam], axis=1)
    inside = np.flatnonzero(np.all(bary > 1e-12, axis=1))
    assert len(inside) == 1
    return inside[0]


@pytest.mark.parametrize("name,mesh", list(_mesh_cases()))
def test_refined_mesh_is_conforming_nested_and_oriented(name, mesh):
    xyz, tets, d = mesh
    rng = np.random.default_rng(3)
    x0, t0 = xyz, tets
    sign0 = np.sign(core.tet_dets(t0, x0))
    for _ in range(3):
        marked = rng.random(len(tets)) < 0.2
        x2, t2, d2, passes = R.refine(xyz, tets, d, marked)
        assert passes >= 1
        # every marked tet was split: none of them survives as a vertex set
        old = set(tuple(sorted(v)) for v in np.asarray(tets)[marked].tolist())
        assert not old & set(tuple(sorted(v)) for v in t2.tolist())
        # conforming, boundary on the cube's surface, Dirichlet flags = surface vertices
        faces = np.sort(np.concatenate([t2[:, [1, 2, 3]], t2[:, [0, 2, 3]], t2[:, [0, 1, 3]],
                                        t2[:, [0, 1, 2]]]), axis=1)
        _, cnt = np.unique(faces, axis=0, return_counts=True)
        assert cnt.max() == 2
        for f in R.boundary_faces(t2):
            assert np.any(np.all((x2[f] == 0.0) | (x2[f] == 1.0), axis=0))
        assert np.array_equal(d2, W._cube_boundary(x2))
        det = core.tet_dets(t2, x2)
        assert abs(np.abs(det).sum() / 6.0 - 1.0) <= 1e-14
        # nested in the input mesh and oriented as the tet it came from
        cen = x2[t2].mean(axis=1)
        for t in range(0, len(t2), 7):
            assert np.sign(det[t]) == sign0[_locate(x0, t0, cen[t])]
        xyz, tets, d = x2, t2, d2


def test_no_marks_leave_the_mesh_unchanged():
    xyz, tets, d = W.five_tet_mesh(2)
    x2, t2, d2, passes = R.refine(xyz, tets, d, np.zeros(len(tets), bool))
    assert passes == 0 and np.array_equal(t2, tets) and np.array_equal(x2, xyz)


def test_single_kuhn_cube_bisects_its_diagonal():
    # the 6 tets of a Kuhn cube share the main diagonal, the longest edge of each
    xyz, tets, d = W.kuhn_mesh(1)
    x2, t2, d2, passes = R.refine(xyz, tets, d, np.eye(6, dtype=bool)[0])
    assert passes == 1 and len(t2) == 12 and len(x2) == 9
    assert np.array_equal(x2[8], [0.5, 0.5, 0.5]) and d2[8] == 0


# ------------------------------------------------------------------ indicator


def test_volume_term_integrates_the_target():
    # u_h = 0: no jumps, eta^2 = a_T^2 ||ubar||^2_T; with a_T = 1 the sum is int sin^2 = 1/8
    n, rho = 6, 1e-4
    xyz, tets, d = W.kuhn_mesh(n)
    s = core.assemble_mesh(xyz, tets, d, W.sine_target())
    u0 = np.zeros(s.K.shape[0])
    tot = core.error_indicator(s, rho, u0, W.sine_target(), qlevel=2).sum()
    assert abs(tot / 0.125 - 1.0) <= 2e-4
    # a_T = h_T / sqrt(rho) < 1, h_T = sqrt(3) / n on every Kuhn tet
    rho2 = 4.0
    tot2 = core.error_indicator(s, rho2, u0, W.sine_target(), qlevel=2).sum()
    assert abs(tot2 / (tot * 3.0 / (n * n * rho2)) - 1.0) <= 1e-13


def _torn(xyz, tets):
    """The same tets with their own copies of the vertices: no shared faces."""
    t = np.asarray(tets)
    return xyz[t.ravel()], np.arange(4 * len(t), dtype=np.int32).reshape(-1, 4)


def _plane_gradient(P, vals):
    """Gradient of the affine function through 4 points by least squares."""
    A = np.concatenate([np.ones((4, 1)), P], axis=1)
    return np.linalg.lstsq(A, vals, rcond=None)[0][1:]


@pytest.mark.parametrize("mesh", ["kuhn2_jittered", "five2"])
def test_face_term_equals_separate_jump_computation(mesh):
    xyz, tets, _ = (W.kuhn_mesh(2, W.jittered_xyz(2, 0.2, 9)) if mesh == "kuhn2_jittered"
                    else W.five_tet_mesh(2))
    rho = 0.05
    nv = len(xyz)
    nod = np.zeros(nv, np.uint8)                     # every vertex an unknown
    s = core.assemble_mesh(xyz, tets, nod, W.sine_target())
    u = W.random_vector(s.K.shape[0], 4)
    U = s.full_vector(u)
    eta = core.error_indicator(s, rho, u, W.sine_target())
    xt, tt = _torn(xyz, tets)
    st = core.assemble_mesh(xt, tt, np.zeros(len(xt), np.uint8), W.sine_target())
    ut = np.empty(st.K.shape[0])
    ut[st.dof] = U[np.asarray(tets).ravel()]
    eta_t = core.error_indicator(st, rho, ut, W.sine_target())
    face = eta - eta_t
    # separate computation, face by face
    ref = np.zeros(len(tets))
    where = {}
    for t, v in enumerate(np.asarray(tets).tolist()):
        for a in range(4):
            where.setdefault(tuple(sorted(v[:a] + v[a + 1:])), []).append(t)
    for f, ts in where.items():
        if len(ts) != 2:
            continue
        P = xyz[list(f)]
        g = [_plane_gradient(xyz[tets[t]], U[tets[t]]) for t in ts]
        n = np.linalg.svd(np.stack([P[1] - P[0], P[2] - P[0]]))[2][2]
        la, lb, lc = (np.linalg.norm(P[1] - P[0]), np.linalg.norm(P[2] - P[1]),
                      np.linalg.norm(P[0] - P[2]))
        sp_ = 0.5 * (la + lb + lc)
        area = math.sqrt(sp_ * (sp_ - la) * (sp_ - lb) * (sp_ - lc))
        aF = min(max(la, lb, lc) / math.sqrt(rho), 1.0)
        c = aF * area * rho ** 1.5 * float(np.dot(g[0] - g[1], n)) ** 2
        for t in ts:
            ref[t] += 0.5 * c
    assert np.max(np.abs(face - ref)) <= 1e-10 * np.max(ref)
    # an affine u_h has no jumps
    ul = 0.3 + xyz @ np.array([1.0, -2.0, 0.5])
    eta_l = core.error_indicator(s, rho, ul[s.dof >= 0][np.argsort(s.dof[s.dof >= 0])],
                                 W.sine_target())
    ul_t = np.empty(st.K.shape[0])
    ul_t[st.dof] = ul[np.asarray(tets).ravel()]
    eta_lt = core.error_indicator(st, rho, ul_t, W.sine_target())
    assert np.max(np.abs(eta_l - eta_lt)) <= 1e-14 * np.max(eta_l)


def test_indicator_tracks_the_energy_error_under_refinement():
    # rho = 1 keeps a_T = h_T < 1 from the first mesh on (asymptotic regime); the efficiency
    # index eta / ||u - u_h||_rho stays put (about 6.6) while both halve at each refinement
    rho = 1.0
    exact = {"kind": "sine_scaled", "scale": 1.0 / (3.0 * rho * math.pi ** 2 + 1.0)}
    mesh = W.five_tet_mesh(2)
    ratios = []
    for _ in range(3):
        mesh = W.bey_refine(*mesh)
        s = core.assemble_mesh(*mesh, W.sine_target())
        u = spl.spsolve(s.A(rho).tocsc(), s.f)
        l2, h1 = core.errors(s, u, exact, qlevel=1)
        eta = math.sqrt(core.error_indicator(s, rho, u, W.sine_target()).sum())
        ratios.append(eta / math.sqrt(rho * h1 + l2))
    assert all(1.0 <= r <= 20.0 for r in ratios), ratios
    assert max(ratios) / min(ratios) <= 1.05, ratios


# ------------------------------------------------------------------ marking


@pytest.mark.parametrize("seed,theta", [(0, 0.5), (1, 0.3), (2, 0.9), (3, 1.0)])
def test_bulk_marking_brute_force(seed, theta):
    rng = np.random.default_rng(seed)
    eta = rng.random(60) ** 3
    eta[10:20] = eta[5]                             # ties
    got = core.dorfler_mark(eta, theta)
    goal = theta * eta.sum()
    best = None
    for t in np.unique(eta):
        if eta[eta >= t].sum() >= goal * (1 - 1e-15):
            best = t
    assert np.array_equal(got, eta >= best)
    assert eta[got].sum() >= goal * (1 - 1e-15)


def test_tet_gradients_reproduce_the_barycentric_coordinates():
    # lambda_a is the affine function with lambda_a(x_b) = delta_ab: its gradient dotted with
    # x_b - x_0 is delta_ab - delta_a0, the four gradients sum to zero, and the volume is the
    # tet's (a unit reference tet, scaled and sheared copies, and a jittered Kuhn mesh)
    ref = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    A = np.array([[2.0, 0.3, 0.0], [0.0, 0.5, 0.1], [0.2, 0.0, 1.5]])
    xyz = np.concatenate([ref, ref @ A.T + 3.0])
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    vol, g = core.tet_gradients(xyz, tets)
    assert np.allclose(vol, [1.0 / 6.0, abs(np.linalg.det(A)) / 6.0], rtol=1e-14)
    assert np.allclose(g[0], np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]]),
                       atol=1e-15)
    x2, t2, _ = W.kuhn_mesh(4, W.jittered_xyz(4, 0.2, seed=2))
    for X, T in ((xyz, tets), (x2, t2)):
        vol, g = core.tet_gradients(X, T)
        P = X[T]
        lam = np.einsum("tad,tbd->tab", g, P - P[:, :1, :])   # grad lambda_a . (x_b - x_0)
        want = np.eye(4)[None] - np.eye(4)[None, :, :1]
        assert np.allclose(lam, want, atol=1e-12)
        assert np.allclose(g.sum(axis=1), 0.0, atol=1e-12)
        assert np.allclose(vol, np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6.0, rtol=1e-13)
