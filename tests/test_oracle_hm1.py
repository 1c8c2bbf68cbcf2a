"""Pins of the oracle's discrete H^-1 error (the first column of Tables 3, 6 and 8 measures
||ubar - u_h||^2 in H^-1): ||w - u_h||_{-1,h}^2 = r^T K^-1 r with r = scale * f - M u, the dual
norm of w - u_h on the P1 space with zero boundary values.  Each pin reaches the value by a
route that does not go through the oracle's sparse solve:

* spectral sum: r^T K^-1 r = sum_i (q_i^T r)^2 / lambda_i over the eigenpairs of K, and no
  v gives a larger (r^T v)^2 / (v^T K v) (the dual norm is a supremum);
* a generalized eigenvector K v = lambda M v with scale = 0 has ||v_h||_{-1,h}^2 = v^T M v / lambda;
* the optimal state (rho K + M) u = f has r = rho K u, so the error equals rho^2 u^T K u;
* the L2 projection u = M^-1 f has r = 0; doubling the scale then gives f^T K^-1 f;
* for ubar = sin sin sin and u_h = 0 the value converges at second order to the continuous
  ||ubar||_{H^-1}^2 = ||ubar||^2 / (3 pi^2) = 1 / (24 pi^2) (ubar is the first Dirichlet
  eigenfunction, eigenvalue 3 pi^2).

A plausible slip (M instead of K in the solve, f + M u instead of f - M u, a dropped scale)
fails at least one of them.
"""
import math

import numpy as np
import scipy.linalg as sla

import fem_workloads as W
from oracle import core


def _dense(s):
    return s.K.toarray(), s.M.toarray()


def test_hm1_equals_the_spectral_sum_and_bounds_every_quotient():
    rng = np.random.default_rng(5)
    for n, target, scale in ((4, W.box_target(), 1.0), (5, W.sine_target(), 0.7),
                             (5, W.bump_target(3), -1.3)):
        s = core.assemble(n, target)
        K, M = _dense(s)
        u = rng.standard_normal(len(s.f)) * 0.1
        r = scale * s.f - M @ u
        lam, Q = np.linalg.eigh(K)
        ref = float(np.sum((Q.T @ r) ** 2 / lam))
        got = core.error_hm1(s, u, scale)
        assert abs(got - ref) <= 1e-12 * ref
        V = rng.standard_normal((len(r), 200))
        quot = (r @ V) ** 2 / np.einsum("ij,ij->j", V, K @ V)
        assert np.all(quot <= got * (1 + 1e-12))
        vstar = Q @ ((Q.T @ r) / lam)
        assert abs((r @ vstar) ** 2 / (vstar @ K @ vstar) - got) <= 1e-12 * got


def test_hm1_of_a_generalized_eigenvector():
    s = core.assemble(5, W.sine_target())
    K, M = _dense(s)
    lam, V = sla.eigh(K, M)          # V^T M V = I
    for k in (0, 3, len(lam) - 1):
        got = core.error_hm1(s, V[:, k], scale=0.0)
        assert abs(got - 1.0 / lam[k]) <= 1e-11 / lam[k]


def test_hm1_of_the_optimal_state_is_rho_squared_times_its_energy():
    for rho in (1.0, 1e-2, 1e-5):
        s = core.assemble(6, W.box_target())
        K, M = _dense(s)
        u = core.cholesky_solve(rho * K + M, s.f)
        got = core.error_hm1(s, u)
        ref = rho * rho * float(u @ K @ u)
        assert abs(got - ref) <= 1e-10 * ref


def test_hm1_vanishes_for_the_l2_projection():
    s = core.assemble(6, W.bump_target(2))
    K, M = _dense(s)
    u = core.cholesky_solve(M, s.f)
    full = float(s.f @ np.linalg.solve(K, s.f))
    assert core.error_hm1(s, u) <= 1e-20 * full
    assert abs(core.error_hm1(s, u, scale=2.0) - full) <= 1e-12 * full


def test_hm1_of_the_sine_target_converges_to_the_closed_form():
    exact = 1.0 / (24.0 * math.pi ** 2)
    err = []
    for n in (8, 16, 32):
        s = core.assemble(n, W.sine_target())
        err.append(abs(core.error_hm1(s, np.zeros(len(s.f))) / exact - 1.0))
    eoc = [math.log2(err[i] / err[i + 1]) for i in range(2)]
    assert all(1.85 <= e <= 2.15 for e in eoc), eoc
    assert err[-1] <= 5e-3


def test_table3_hm1_column_is_a_fixed_multiple_of_the_dual_norm():
    # For ubar = sin sin sin the error ubar - u_rho is a multiple of the first Dirichlet
    # eigenfunction, so its squared H^-1 and L2 norms differ by the factor 1 / (3 pi^2); the
    # oracle's discrete dual norm shows that factor on a discrete solution.  Table 3's printed
    # H^-1 column is its printed L2 column times one constant at every rho, 0.898 of that
    # factor: the paper's unstated discrete H^-1 norm differs from the dual norm by a fixed
    # normalisation (context only, not a parity target).
    from tests.conftest import golden
    rows = golden("table3_hm1_error.txt")
    printed = [hm / l2 for _, hm, l2 in rows]
    assert max(printed) / min(printed) - 1.0 <= 2e-4
    rho, n = 1e-2, 24
    s = core.assemble(n, W.sine_target())
    u = core.jacobi_pcg(s, rho, s.f, tol=1e-13)[0]
    ours = core.error_hm1(s, u) / core.errors(s, u, W.sine_target())[0]
    assert abs(ours * 3.0 * math.pi ** 2 - 1.0) <= 0.02
    assert abs(printed[0] * 3.0 * math.pi ** 2 - 0.8984) <= 2e-3
