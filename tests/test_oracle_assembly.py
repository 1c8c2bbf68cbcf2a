"""Pins of the oracle's mesh, assembly, quadrature and direct/iterative solvers.

Each check ties the oracle to something other than itself: closed forms,
invariants of the P1 space, symmetries of the Kuhn mesh, brute force, and the
values the paper prints (Tables 1 and 3, Sec. 4.1).
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import fem_workloads as W
from oracle import core
from tests.conftest import golden


def test_reference_element_closed_form():
    # unit reference tet: K_e = (1/6) [[3,-1,-1,-1],[-1,1,0,0],[-1,0,1,0],[-1,0,0,1]],
    # M_e = (1/120) (1 + delta_ab)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    det, Ke, Me = core.element(X)
    assert det == pytest.approx(1.0)
    Kref = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    Mref = (np.ones((4, 4)) + np.eye(4)) / 120.0
    np.testing.assert_allclose(Ke, Kref, atol=1e-15)
    np.testing.assert_allclose(Me, Mref, atol=1e-15)


def test_element_affine_invariance():
    # K_e scales like h, M_e like h^3 under x -> h Q x + t (Q orthogonal)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((4, 3))
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    h = 0.37
    det0, K0, M0 = core.element(X)
    det1, K1, M1 = core.element(h * X @ Q.T + np.array([0.3, -1.0, 2.0]))
    np.testing.assert_allclose(K1, h * K0, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(M1, h ** 3 * M0, rtol=1e-12, atol=1e-16)
    # rows of K_e sum to zero (constants are in the kernel of the Laplacian)
    np.testing.assert_allclose(K0.sum(axis=1), 0.0, atol=1e-12 * np.abs(K0).max())


@pytest.mark.parametrize("level", [0, 1])
def test_quadrature_exact_to_degree_two(level):
    # int over the unit tet of x^a y^b z^c = a! b! c! / (a+b+c+3)!
    bary, wt = core.qrule(level)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    pts = bary @ X
    vol = 1.0 / 6.0
    assert wt.sum() == pytest.approx(1.0, abs=1e-15)
    for a in range(3):
        for b in range(3 - a):
            for c in range(3 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(
                    a + b + c + 3)
                got = vol * np.sum(wt * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert got == pytest.approx(exact, rel=1e-13)
    # degree 4 is not exact: the rule is the degree-2 one, not something stronger by accident
    got = vol * np.sum(wt * pts[:, 0] ** 4)
    assert abs(got - 24.0 / math.factorial(7)) > 1e-8


@pytest.mark.parametrize("jitter", [False, True])
def test_full_mesh_invariants(jitter):
    n = 4
    xyz = W.jittered_xyz(n, 0.2, seed=5) if jitter else None
    s = core.assemble(n, W.sine_target(), xyz=xyz, full=True)
    K, M = s.K, s.M
    one = np.ones(K.shape[0])
    # constants are in the kernel of K; total mass is |Omega| = 1
    assert np.abs(K @ one).max() < 1e-13
    assert M.sum() == pytest.approx(1.0, abs=1e-14)
    # linear functions are harmonic: (K L)_i = 0 at interior vertices
    coords = s.xyz
    interior = core.interior_dof_map(n) >= 0
    for d in range(3):
        assert np.abs((K @ coords[:, d])[interior]).max() < 1e-13
    # symmetry and positive diagonals
    assert abs(K - K.T).max() < 1e-15 and abs(M - M.T).max() < 1e-18
    assert (K.diagonal() > 0).all() and (M.diagonal() > 0).all()
    # M applied to the coordinates integrates them: sum_ij M_ij x_j = int x = 1/2
    for d in range(3):
        assert (M @ coords[:, d]).sum() == pytest.approx(0.5, abs=1e-14)


def test_kuhn_stencil_values():
    # uniform Kuhn mesh: K = h * (7-point Laplacian, 0 on face/body diagonals);
    # M = h^3 * (2/5 centre, 1/20 on axis and body diagonals, 1/30 on face diagonals)
    n = 8
    h = 1.0 / n
    s = core.assemble(n, W.sine_target())
    m = n - 1
    expect_K = {0: 6.0, 1: -1.0, 2: 0.0, 3: 0.0}
    expect_M = {0: 0.4, 1: 1 / 20, 2: 1 / 30, 3: 1 / 20}
    for (i, j, k) in [(3, 3, 3), (2, 4, 5)]:
        r = i + m * (j + m * k)
        cols = s.K.indices[s.K.indptr[r]:s.K.indptr[r + 1]]
        kv = s.K.data[s.K.indptr[r]:s.K.indptr[r + 1]]
        mv = s.M.data[s.M.indptr[r]:s.M.indptr[r + 1]]
        assert len(cols) == 15
        for c, a, b in zip(cols, kv, mv):
            di, dj, dk = c % m - i, (c // m) % m - j, c // (m * m) - k
            off = (di, dj, dk)
            if off != (0, 0, 0):
                # Kuhn neighbours: +-e_i, +-(e_i + e_j), +-(1,1,1)
                assert len({x for x in off if x != 0}) == 1
            typ = sum(abs(x) for x in off)
            assert a / h == pytest.approx(expect_K[typ], abs=1e-12)
            assert b / h ** 3 == pytest.approx(expect_M[typ], rel=1e-12)
    # interior M row sums are int phi_i = h^3
    r = 3 + m * (3 + m * 3)
    assert s.M[r].sum() == pytest.approx(h ** 3, rel=1e-13)


def test_jittered_mesh_stays_admissible():
    n = 16
    tets = core.kuhn_tets(n)
    d0 = core.tet_dets(tets, core.uniform_xyz(n))
    d1 = core.tet_dets(tets, W.jittered_xyz(n, 0.2, seed=0))
    assert (d1 / d0 > 0).all()
    # the cube is filled: sum of volumes is 1
    assert np.abs(d1).sum() / 6.0 == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("n,rho", [(6, 1.0), (8, 1.0 / 64), (10, 1e-6)])
def test_direct_and_iterative_solvers_agree(n, rho):
    s = core.assemble(n, W.sine_target())
    A = s.A(rho)
    x_chol = core.cholesky_solve(A.toarray(), s.f)
    x_np = np.linalg.solve(A.toarray(), s.f)
    x_cg, it, rr = core.jacobi_pcg(s, rho, s.f, tol=1e-14)
    assert rr < 1e-13
    nrm = np.linalg.norm(x_np)
    assert np.linalg.norm(x_chol - x_np) <= 1e-12 * nrm
    assert np.linalg.norm(x_cg - x_np) <= 1e-11 * nrm
    # the oracle's operator matches the matrix
    x = W.random_vector(A.shape[0], 1)
    np.testing.assert_allclose(core.apply(s, rho, x), A @ x, rtol=1e-13, atol=1e-18)


def test_solution_symmetries():
    # the Kuhn mesh is invariant under axis permutations and under x -> 1 - x;
    # so is the sine target: the discrete solution inherits these symmetries.
    n, rho = 8, 1.0 / 64
    s = core.assemble(n, W.sine_target())
    u = spl.spsolve(s.A(rho).tocsc(), s.f).reshape(n - 1, n - 1, n - 1)  # [k, j, i]
    scale = np.abs(u).max()
    for perm in [(0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)]:
        assert np.abs(u - u.transpose(perm)).max() < 1e-12 * scale
    assert np.abs(u - u[::-1, ::-1, ::-1]).max() < 1e-12 * scale


def test_table1_l2_errors_and_orders():
    rows = golden("table1_l2_error.txt")
    ns = [4, 8, 16, 32]
    for row in rows:
        rho, paper, paper_eoc = row[0], np.array(row[1:5]), np.array(row[5:8])
        exact = {"kind": "sine_scaled", "scale": 1.0 / (3.0 * rho * math.pi ** 2 + 1.0)}
        errs = []
        for n in ns:
            s = core.assemble(n, W.sine_target())
            u = spl.spsolve(s.A(rho).tocsc(), s.f)
            errs.append(math.sqrt(core.errors(s, u, exact, qlevel=2)[0]))
        errs = np.array(errs)
        eoc = np.log2(errs[:-1] / errs[1:])
        assert np.all(np.abs(errs / paper - 1.0) < 0.15), (rho, errs / paper)
        assert np.all(np.abs(eoc - paper_eoc) < 0.1), (rho, eoc, paper_eoc)


def test_theorem1_rate_at_rho_equal_h2():
    # Theorem 1: ||u_rho,h - ubar||_L2 <= c h^2 for rho = h^2
    ratios = []
    for n in [4, 8, 16, 32]:
        rho = 1.0 / n ** 2
        s = core.assemble(n, W.sine_target())
        u = spl.spsolve(s.A(rho).tocsc(), s.f)
        ratios.append(math.sqrt(core.errors(s, u, W.sine_target(), qlevel=2)[0]) * n ** 2)
    ratios = np.array(ratios)
    # error / h^2 settles to a constant: increments shrink geometrically, and the
    # order between h = 1/16 and 1/32 is close to 2
    inc = np.diff(ratios)
    assert np.all(inc[1:] < 0.6 * inc[:-1]), ratios
    assert np.log2(ratios[2] / 16 ** 2 / (ratios[3] / 32 ** 2)) > 1.85, ratios


def test_table3_closed_form_and_error_routine():
    # Table 3's L2 column is, to 5e-4 (the FE error of the printed run), ||ubar - u_rho||^2 = (1/8) (3 rho pi^2 / (3 rho pi^2 + 1))^2:
    # it pins the manufactured solution u_rho = ubar / (3 rho pi^2 + 1) (Sec. 4.1).
    for rho, printed in golden("table3_target_error.txt"):
        c = 3 * rho * math.pi ** 2
        assert (c / (c + 1)) ** 2 / 8 == pytest.approx(printed, rel=5e-4)
    # the oracle's error routine integrates (s sin sin sin)^2 = s^2 / 8
    s = core.assemble(16, W.sine_target())
    l2, h1 = core.errors(s, np.zeros(s.K.shape[0]), {"kind": "sine_scaled", "scale": 0.5},
                         qlevel=2)
    assert l2 == pytest.approx(0.25 / 8, rel=1e-4)
    assert h1 == pytest.approx(0.25 * 3 * math.pi ** 2 / 8, rel=1e-3)


def test_small_rho_gives_l2_projection():
    # rho -> 0: A -> M and u_h -> M^{-1} f, the L2 projection of ubar (Sec. 3.1 remark)
    n = 8
    s = core.assemble(n, W.box_target())
    u0 = spl.spsolve(s.M.tocsc(), s.f)
    u = spl.spsolve(s.A(1e-14).tocsc(), s.f)
    assert np.linalg.norm(u - u0) <= 1e-9 * np.linalg.norm(u0)
    # the box target gives f > 0 only near the box, and positive mass
    assert s.f.sum() == pytest.approx(0.125, rel=0.2)


def test_load_vector_of_constant_target_is_lumped_mass():
    # ubar = 1 is integrated exactly: f = M 1 restricted to the unknowns
    n = 6
    s = core.assemble(n, {"kind": "box", "lo": -1.0, "hi": 2.0})
    full = core.assemble(n, {"kind": "box", "lo": -1.0, "hi": 2.0}, full=True)
    rowsum = np.asarray(full.M.sum(axis=1)).ravel()
    dof = core.interior_dof_map(n)
    np.testing.assert_allclose(s.f, rowsum[dof >= 0], rtol=1e-13)


@pytest.mark.parametrize("jitter", [False, True])
def test_single_rows_match_full_assembly(jitter):
    # the row routine (used for sampled checks on meshes too large to assemble on the CPU)
    # restates the same integrals: it must reproduce the assembled rows exactly
    n = 9
    xyz = W.jittered_xyz(n, 0.2, seed=4) if jitter else None
    t = W.bump_target(12)
    s = core.assemble(n, t, xyz=xyz)
    rows = np.arange(s.K.shape[0])
    cols, K, M, f = core.kuhn_rows(n, t, rows, xyz=xyz)
    for r in rows:
        sl = slice(s.K.indptr[r], s.K.indptr[r + 1])
        ln = s.K.indptr[r + 1] - s.K.indptr[r]
        assert np.array_equal(cols[r, :ln], s.K.indices[sl]) and np.all(cols[r, ln:] == -1)
        np.testing.assert_allclose(K[r, :ln], s.K.data[sl], rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(M[r, :ln], s.M.data[sl], rtol=1e-13, atol=1e-19)
    np.testing.assert_allclose(f, s.f, rtol=1e-13, atol=1e-18)
