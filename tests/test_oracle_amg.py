"""Pins of the oracle's smoothed-aggregation hierarchy, smoother, V-cycle and PCG.

The hierarchy's rules are checked against brute force (greedy MIS-2, dense
products), the defining formulas in dense arithmetic, the closed form of the
Chebyshev error polynomial, and the exact discrete solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import fem_workloads as W
from oracle import amg, core


def _greedy_mis2(adj, prio, isolated):
    """Scan nodes by decreasing priority; take a node if no taken node is within distance 2."""
    n = len(adj)
    taken = np.zeros(n, dtype=bool)
    for i in sorted(range(n), key=lambda t: -int(prio[t])):
        if isolated[i]:
            continue
        ball = set(adj[i])
        for j in adj[i]:
            ball |= set(adj[j])
        ball.discard(i)
        if not any(taken[j] for j in ball):
            taken[i] = True
    return taken


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    M = rng.random((n, n)) < p
    M = np.triu(M, 1)
    M = M | M.T
    return sp.csr_matrix(M.astype(float))


@pytest.mark.parametrize("seed", range(6))
def test_mis2_equals_greedy_by_priority(seed):
    S = _random_graph(60, 0.06, seed)
    S.sort_indices()
    adj = [list(S.indices[S.indptr[i]:S.indptr[i + 1]]) for i in range(60)]
    isolated = np.diff(S.indptr) == 0
    prio = amg.priority(60, seed)
    state = amg.mis2(S, prio, isolated)
    assert np.array_equal(state == amg.IN, _greedy_mis2(adj, prio, isolated))


def test_priorities_are_unique_and_hash_is_murmur_finaliser():
    # fmix32 reference values computed by hand from its definition
    h = amg.fmix32(np.array([0, 1, 0xFFFFFFFF], dtype=np.uint32))
    assert int(h[0]) == 0
    assert int(h[1]) == 0x514E28B7
    assert int(h[2]) == 0x81F16F39
    p = amg.priority(1000, 3)
    assert len(np.unique(p)) == 1000
    assert np.array_equal(p & np.uint64(0x7FFFFFFF), np.arange(1000, dtype=np.uint64))


def _hier_problem(n=12, rho=1.0 / 144):
    s = core.assemble(n, W.sine_target())
    return s, s.A(rho)


def test_aggregates_are_valid():
    s, A = _hier_problem()
    agg, nagg, smask = amg.aggregate(A, 0.05, 0)
    r = amg.rows_of(A)
    strong = sp.csr_matrix((np.ones(int(smask.sum())), (r[smask], A.indices[smask])),
                           shape=A.shape)
    deg = np.diff(strong.indptr)
    assert np.all((agg >= 0) == (deg > 0))
    assert set(np.unique(agg[agg >= 0])) == set(range(nagg))
    # each aggregate is connected in the strong graph
    for a in range(nagg):
        nodes = np.flatnonzero(agg == a)
        sub = strong[nodes][:, nodes]
        ncomp, _ = sp.csgraph.connected_components(sub, directed=False)
        assert ncomp == 1
    # roots (one per aggregate) are pairwise at strong-graph distance >= 3
    S2 = (strong + strong @ strong).tocsr()
    state = amg.mis2(strong, amg.priority(A.shape[0], 0), deg == 0)
    roots = np.flatnonzero(state == amg.IN)
    assert len(roots) == nagg
    sub = S2[roots][:, roots].tolil()
    sub.setdiag(0)
    assert sp.csr_matrix(sub).count_nonzero() == 0


def test_spgemm_matches_dense_and_keeps_structural_zeros():
    rng = np.random.default_rng(0)
    A = sp.random(40, 30, density=0.15, random_state=1, format="csr")
    B = sp.random(30, 20, density=0.2, random_state=2, format="csr")
    C = amg.spgemm(A, B)
    np.testing.assert_allclose(C.toarray(), A.toarray() @ B.toarray(), rtol=1e-14, atol=1e-15)
    # cancellation: [1 1] @ [[1],[-1]] = 0 is kept as a stored entry
    Z = amg.spgemm(sp.csr_matrix([[1.0, 1.0]]), sp.csr_matrix([[1.0], [-1.0]]))
    assert Z.nnz == 1 and Z.data[0] == 0.0
    del rng


def test_prolongator_and_galerkin_operator_formulas():
    s, A = _hier_problem()
    agg, nagg, smask = amg.aggregate(A, 0.05, 0)
    P, omega = amg.smoothed_prolongator(A, smask, agg, nagg)
    Ad = A.toarray()
    n = Ad.shape[0]
    Pt = np.zeros((n, nagg))
    Pt[np.arange(n)[agg >= 0], agg[agg >= 0]] = 1.0
    strongD = np.zeros_like(Ad)
    r = amg.rows_of(A)
    strongD[r[smask], A.indices[smask]] = 1.0
    F = np.where(strongD > 0, Ad, 0.0) + np.diag(np.diag(Ad))
    lam = np.max(np.abs(F).sum(axis=1) / np.diag(Ad))
    assert omega == pytest.approx(4.0 / (3.0 * lam), rel=1e-15)
    Pd = Pt - omega * (F / np.diag(Ad)[:, None]) @ Pt
    np.testing.assert_allclose(P.toarray(), Pd, rtol=1e-13, atol=1e-15)
    # coarse operator
    H = amg.build_hierarchy(A, dict(coarse_max=50))
    Ac = H[1].A.toarray()
    Pd = H[0].P.toarray()
    np.testing.assert_allclose(Ac, Pd.T @ Ad @ Pd, rtol=1e-12, atol=1e-12 * np.abs(Ac).max())
    assert np.abs(Ac - Ac.T).max() <= 1e-14 * np.abs(Ac).max()
    assert np.linalg.eigvalsh(Ac).min() > 0


@pytest.mark.parametrize("n,rho", [(12, 1.0 / 144), (11, 1.0), (10, 1e-6)])
def test_smoothed_prolongator_is_a_stencil_on_the_aggregates(n, rho):
    """On the uniform Kuhn grid every row of A holds the interior row's values at the same
    offsets and every diagonal is the same, so P x_c = [agg >= 0] ((1 - omega) t +
    sum_strong (-omega a_d / a_ii) t(. + d)) with t = P_t x_c: the smoothed prolongator
    written as a stencil on the aggregates' values (the form the uniform finest level
    prolongs with).  Checked against the oracle's sparse P for three strong sets."""
    s, A = _hier_problem(n, rho)
    m = n - 1
    agg, nagg, smask = amg.aggregate(A, 0.05, 0)
    P, omega = amg.smoothed_prolongator(A, smask, agg, nagg)
    # the interior row at the grid's centre: value and strength per offset
    c = (m // 2) * (1 + m + m * m)
    lo, hi = A.indptr[c], A.indptr[c + 1]
    aii = A[c, c]
    coef = {}
    for e in range(lo, hi):
        j = int(A.indices[e])
        dz, rem = divmod(j - c + (1 + m + m * m), m * m)
        dy, dx = divmod(rem, m)
        off = (dx - 1, dy - 1, dz - 1)
        assert j == c + off[0] + m * off[1] + m * m * off[2]
        if smask[e]:
            coef[off] = -omega * (A.data[e] / aii)
    assert 0 < len(coef) <= 14
    # what the stencil form needs: one diagonal value (the assembly sums each row's element
    # contributions in its own order, so equal to rounding), and every row's strong entries
    # are exactly the interior row's strong offsets that stay on the grid, with its values
    np.testing.assert_allclose(A.diagonal(), aii, rtol=1e-14)
    r = amg.rows_of(A)
    on = {}
    for e in range(A.nnz):
        i, j = int(r[e]), int(A.indices[e])
        if i == j:
            continue
        di, dj = np.unravel_index(i, (m, m, m)), np.unravel_index(j, (m, m, m))
        off = (int(dj[2] - di[2]), int(dj[1] - di[1]), int(dj[0] - di[0]))
        assert bool(smask[e]) == (off in coef), (i, j)
        if smask[e]:
            assert -omega * (A.data[e] / aii) == pytest.approx(coef[off], rel=1e-14)
        on[(i, off)] = True
    for i in range(m ** 3):   # every strong offset that stays on the grid is an entry
        k, j, ii = np.unravel_index(i, (m, m, m))
        for (dx, dy, dz) in coef:
            if 0 <= ii + dx < m and 0 <= j + dy < m and 0 <= k + dz < m:
                assert (i, (dx, dy, dz)) in on
    rng = np.random.default_rng(n)
    xc = rng.standard_normal(nagg)
    t = np.where(agg >= 0, xc[np.maximum(agg, 0)], 0.0).reshape(m, m, m)   # [k][j][i]
    tp = np.pad(t, 1)
    y = (1.0 - omega) * t
    for (dx, dy, dz), cd in coef.items():
        y = y + cd * tp[1 + dz:1 + dz + m, 1 + dy:1 + dy + m, 1 + dx:1 + dx + m]
    y = np.where(agg.reshape(m, m, m) >= 0, y, 0.0).ravel()
    ref = P @ xc
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_chebyshev_error_polynomial_closed_form():
    # D = I, A = diag(lam): after k steps from x0 = 0 for A x = A 1, the error is
    # -T_k((theta - lam)/delta) / T_k(theta/delta) (Chebyshev acceleration)
    lam = np.linspace(0.05, 2.0, 25)
    A = sp.diags(lam).tocsr()
    b = lam.copy()
    lmax, ratio = 2.0, 6.0
    a_, b_ = lmax / ratio, lmax
    theta, delta = (a_ + b_) / 2, (b_ - a_) / 2
    for k in [1, 2, 3, 4]:
        x = amg.chebyshev(A, np.ones(25), b, None, lmax, ratio, k)
        Tk = np.polynomial.chebyshev.Chebyshev.basis(k)
        expect = 1.0 - Tk((theta - lam) / delta) / Tk(theta / delta)
        np.testing.assert_allclose(x, expect, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("smoother", ["chebyshev", "l1"])
def test_vcycle_is_symmetric_positive_definite(smoother):
    s, A = _hier_problem(10, 1.0)
    opts = dict(smoother=smoother, coarse_max=40)
    H = amg.build_hierarchy(A, opts)
    assert len(H) >= 3
    N = A.shape[0]
    x, y = W.random_vector(N, 1), W.random_vector(N, 2)
    Vx, Vy = amg.vcycle(H, x, opts), amg.vcycle(H, y, opts)
    assert abs(Vx @ y - x @ Vy) <= 1e-12 * np.linalg.norm(Vx) * np.linalg.norm(y)
    assert x @ Vx > 0 and y @ Vy > 0
    # linear in its argument
    np.testing.assert_allclose(amg.vcycle(H, 2 * x - y, opts), 2 * Vx - Vy, rtol=1e-11,
                               atol=1e-13 * np.abs(Vx).max())


@pytest.mark.parametrize("rho", [1.0, 1.0 / 256, 1e-6])
def test_amg_pcg_reaches_exact_discrete_solution(rho):
    n = 16
    s = core.assemble(n, W.sine_target())
    A = s.A(rho)
    H = amg.build_hierarchy(A)
    x, it, rr, hist = amg.pcg(A, s.f, lambda r: amg.vcycle(H, r), tol=1e-13, maxit=200)
    x_ref = spl_solve(A, s.f)
    assert rr <= 1e-12
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    assert it <= 30
    # flexible CG with the same (fixed) preconditioner converges as well
    xf, itf, rrf, _ = amg.pcg(A, s.f, lambda r: amg.vcycle(H, r), tol=1e-13, maxit=200,
                              flexible=True)
    assert np.linalg.norm(xf - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def spl_solve(A, b):
    import scipy.sparse.linalg as spl
    return spl.spsolve(A.tocsc(), b)


def test_pencil_hierarchy_matches_direct_galerkin():
    # with P fixed, P^T (rho K + M) P = rho P^T K P + P^T M P
    n, rho = 10, 1.0 / 100
    s = core.assemble(n, W.sine_target())
    A = s.A(rho)
    H = amg.build_hierarchy(A, dict(coarse_max=30), K=s.K, M=s.M)
    for L in H[1:]:
        np.testing.assert_allclose(L.A.toarray(), (rho * L.K + L.M).toarray(), rtol=1e-12,
                                   atol=1e-13 * abs(L.A).max())


def test_row_limit_stops_coarsening():
    # a level whose restriction or Galerkin products would have a row longer than max_row is
    # the coarsest: at or above every level's longest product row the hierarchy is the
    # default one; below level 0's, it is level 0 alone, and the V-cycle is then one
    # Chebyshev smoothing from zero
    s = core.assemble(20, W.sine_target())
    A = s.A(1e-2).tocsr()
    H = amg.build_hierarchy(A)
    assert len(H) >= 3

    def longest(L):
        AP = amg.spgemm(L.A, L.P)
        return max(int(np.diff(B.indptr).max()) for B in (L.R, AP, amg.spgemm(L.R, AP)))

    top = max(longest(L) for L in H if not L.coarsest)
    Hs = amg.build_hierarchy(A, {"max_row": top})
    assert len(Hs) == len(H)
    for L, Ls in zip(H, Hs):
        assert (L.A != Ls.A).nnz == 0
    H1 = amg.build_hierarchy(A, {"max_row": longest(H[0]) - 1})
    assert len(H1) == 1 and H1[0].coarsest and H1[0].Ainv is None
    b = W.random_vector(A.shape[0], 3)
    L0 = H1[0]
    ref = amg.chebyshev(A, L0.dinv, b, None, L0.lmax, amg.DEFAULTS["cheb_ratio"],
                        amg.DEFAULTS["degree"])
    assert np.array_equal(amg.vcycle(H1, b), ref)


def test_strength_gershgorin_and_l1_jacobi_against_independent_facts():
    # strength: a brute-force loop over the stored entries of a random symmetric matrix with a
    # positive diagonal (stored zeros are never strong); Gershgorin: the bound lies above the
    # largest eigenvalue of D^-1 A and is 1 for a diagonal matrix; l1-Jacobi: exact in one
    # step for a positive diagonal matrix, and for SPD A its error propagator I - D_l1^-1 A
    # has spectral radius below 1 (the l1 row sums dominate the diagonal part of A)
    rng = np.random.default_rng(8)
    n = 30
    R = sp.random(n, n, density=0.2, random_state=3, format="csr")
    S = (R + R.T).tocsr()
    S.setdiag(np.abs(S).sum(axis=1).A1 * 0.5 + rng.uniform(0.5, 1.5, n))
    S = S.tocsr()
    off = np.flatnonzero(np.repeat(np.arange(n), np.diff(S.indptr)) != S.indices)
    S.data[off[::7]] = 0.0                  # a few stored zeros off the diagonal
    theta = 0.1
    mask = amg.strength(S, theta)
    d = S.diagonal()
    rows = np.repeat(np.arange(n), np.diff(S.indptr))
    for e, (i, j, v) in enumerate(zip(rows, S.indices, S.data)):
        want = i != j and v != 0.0 and abs(v) >= theta * np.sqrt(d[i] * d[j])
        assert bool(mask[e]) == want
    A = core.assemble(6, W.sine_target()).A(1e-2).tocsr()
    Dinv = np.diag(1.0 / A.diagonal())
    lam = np.max(np.linalg.eigvals(Dinv @ A.toarray()).real)
    assert amg.gershgorin(A) >= lam * (1 - 1e-12)
    Dg = sp.diags(rng.uniform(1.0, 2.0, 10)).tocsr()
    assert amg.gershgorin(Dg) == 1.0
    b = rng.standard_normal(10)
    assert np.allclose(amg.l1_jacobi(Dg, Dg.diagonal(), b, None), b / Dg.diagonal(), rtol=0,
                       atol=0)
    l1 = np.abs(A).sum(axis=1).A1
    Ad = A.toarray()
    E = np.eye(len(l1)) - Ad / l1[:, None]
    assert np.max(np.abs(np.linalg.eigvals(E))) < 1.0
    x = rng.standard_normal(len(l1))
    bb = Ad @ rng.standard_normal(len(l1))
    xs = np.linalg.solve(Ad, bb)
    e0, e1 = x - xs, amg.l1_jacobi(A, l1, bb, x) - xs
    assert e1 @ Ad @ e1 < e0 @ Ad @ e0
