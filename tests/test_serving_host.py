"""Host-side logic of the serving loop (no GPU): bucketing and latency statistics."""
import math

import pytest

pytest.importorskip("torch")


def test_rho_buckets_cover_the_workload_range():
    from paper_2102_03515_gb300.serving import rho_bucket
    assert rho_bucket(1.0) == 0
    assert rho_bucket(0.99) == -1
    assert rho_bucket(1e-8) == -8
    assert rho_bucket(3.2e-5) == -5
    # every rho of [1e-8, 1] falls in one of 9 buckets
    assert {rho_bucket(10 ** (-k / 7.0)) for k in range(0, 57)} <= set(range(-8, 1))


def test_regimes_split_at_h_squared():
    from paper_2102_03515_gb300.serving import regime, regime_rho_setup, rho_bucket
    n = 100  # h^2 = 1e-4
    assert regime(n, rho_bucket(1e-4)) == 1
    assert regime(n, rho_bucket(9.9e-5)) == 0   # its decade [1e-5, 1e-4) lies below h^2
    assert regime(n, rho_bucket(9e-6)) == 0
    assert regime(n, rho_bucket(1.0)) == 1
    assert regime_rho_setup(n, 0) == pytest.approx(1e-4)
    assert regime_rho_setup(n, 1) == 1.0


def test_latency_percentiles():
    from paper_2102_03515_gb300 import serving as S
    svc = S.SolveService.__new__(S.SolveService)  # statistics only, no device state
    svc.done = []
    svc.stats = __import__("collections").Counter(hierarchy_hits=3, hierarchy_builds=1)
    for i in range(100):
        r = S.Request(id=i, n=8, rho=1.0, target={"kind": "sine"}, t_arrival=0.0)
        r.t_done = (i + 1) / 1000.0
        r.status = 1
        svc.done.append(r)
    st = S.SolveService.run_stats(svc)
    assert st["p50_ms"] == pytest.approx(50.0)
    assert st["p99_ms"] == pytest.approx(99.0)
    assert st["cache_hit_rate"] == pytest.approx(0.75)
    assert math.isclose(st["solves_per_s"], 1000.0, rel_tol=1e-9)
