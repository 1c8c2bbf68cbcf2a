"""Serving loop: continuous batching of mixed (n, rho) requests on the GPU.

Each served solution is checked against the oracle's exact solution (a solve stopped at
||r|| / ||f|| <= 1e-8 is within kappa * 1e-8 of it; the meshes here keep kappa small), and
two requests are re-served alone by a fresh service: the bits must be the same.
"""
import numpy as np
import pytest

import fem_workloads as W
from oracle import core
from tests import gpu_util as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def serving():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_03515_gb300 import build as b
    b.build()
    from paper_2102_03515_gb300 import serving as s
    return s


def _requests(S, count, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.choice([8, 10, 12]))
        rho = float(np.exp(rng.uniform(np.log(1e-8), np.log(1.0))))
        reqs.append(S.Request(id=i, n=n, rho=rho, target=W.bump_target(int(rng.integers(1 << 30))),
                              t_arrival=0.002 * i))
    return reqs


def test_served_results_match_oracle_and_alone(serving):
    S = serving
    cfg = S.ServeConfig(slots=4, steps_per_tick=2, keep_solutions=True, coarse_max=64)
    svc = S.SolveService(cfg)
    reqs = _requests(S, 24, seed=7)
    try:
        stats = svc.run(reqs, realtime=True, time_limit=120)
    finally:
        pass
    assert stats["solved"] == len(reqs) and stats["converged"] == len(reqs), stats
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["hierarchy_builds"] <= 3 * 2
    for r in reqs:
        s = core.assemble(r.n, r.target)
        x = core.cholesky_solve(s.A(r.rho).toarray(), s.f)
        assert r.relres <= 1e-8
        assert G.rel(r.u.cpu().numpy(), x) <= 1e-6, (r.id, r.n, r.rho)
    # the same requests served alone by a fresh service: identical bits
    picks = [reqs[3], reqs[17]]
    mixed = {r.id: r.u.cpu().numpy() for r in picks}
    svc.close()
    for r in picks:
        alone = S.SolveService(S.ServeConfig(slots=4, steps_per_tick=2, keep_solutions=True,
                                             coarse_max=64))
        r2 = S.Request(id=r.id, n=r.n, rho=r.rho, target=r.target)
        alone.run([r2], realtime=False)
        assert np.array_equal(r2.u.cpu().numpy(), mixed[r.id])
        alone.close()


def test_budget_forces_eviction_of_idle_sessions(serving):
    S = serving
    cfg = S.ServeConfig(slots=2, steps_per_tick=4, keep_solutions=False, coarse_max=64)
    svc = S.SolveService(cfg)
    try:
        # n = 8 (h^2 = 1/64): rho = 0.1 is stiffness-dominated, 1e-6 mass-dominated, so the
        # requests alternate between two sessions of the same size
        rhos = [0.1, 1e-6, 0.1, 1e-6]
        reqs = [S.Request(id=i, n=8, rho=r, target=W.bump_target(i)) for i, r in enumerate(rhos)]
        svc.run(reqs[:1], realtime=False)
        hier = max(svc._hier_bytes(h) for h in svc.hier.values())
        # room for both hierarchies but for one session only
        svc.cfg.hbm_budget = svc.bytes_in_use + hier + 1024
        for r in reqs[1:]:
            svc.run([r], realtime=False)
        stats = svc.run_stats()
        assert stats["converged"] == 4, stats
        assert svc.stats["evictions"] >= 2
        assert len(svc.sessions) == 1
    finally:
        svc.close()
