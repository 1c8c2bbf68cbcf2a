"""The seeded input generators follow the recipe the measurements state: the same seed gives
the same input, interior vertices move by at most 0.2 h per coordinate and boundary vertices
not at all, bump parameters lie in their stated ranges, rho values in theirs, and the request
stream's arrivals have the stated mean rate."""
import numpy as np

import fem_workloads as W


def test_generators_are_deterministic_per_seed():
    assert np.array_equal(W.jittered_xyz(9, 0.2, seed=3), W.jittered_xyz(9, 0.2, seed=3))
    assert not np.array_equal(W.jittered_xyz(9, 0.2, seed=3), W.jittered_xyz(9, 0.2, seed=4))
    a, b = W.bump_target(11), W.bump_target(11)
    for k in ("centers", "widths", "amps"):
        assert np.array_equal(a[k], b[k])
    r1, r2 = W.request_stream(50, seed=7), W.request_stream(50, seed=7)
    assert [(r["t"], r["n"], r["rho"]) for r in r1] == [(r["t"], r["n"], r["rho"]) for r in r2]
    assert all(np.array_equal(x["target"]["amps"], y["target"]["amps"]) for x, y in zip(r1, r2))
    assert np.array_equal(W.random_vector(100, 5), W.random_vector(100, 5))


def test_jitter_moves_interior_vertices_within_bounds_and_fixes_the_boundary():
    n = 12
    u, j = W.uniform_xyz(n), W.jittered_xyz(n, 0.2, seed=0)
    d = np.abs(j - u)
    onb = np.any((u < 1e-12) | (u > 1 - 1e-12), axis=1)
    assert np.all(d[onb] == 0.0)
    assert np.all(d[~onb] <= 0.2 / n) and np.all(d[~onb].max(axis=0) > 0.15 / n)


def test_bumps_batched_and_stream_ranges():
    t = W.bump_target(1000, nb=8)
    assert t["centers"].shape == (8, 3) and np.all((t["centers"] >= 0.1) & (t["centers"] <= 0.9))
    assert np.all((t["widths"] >= 0.05) & (t["widths"] <= 0.2))
    targets, rhos = W.batched_workload(n=16, nrhs=64, seed=1000)
    assert len(targets) == 64 and np.all((rhos >= 1e-6) & (rhos <= 1e-2))
    assert np.array_equal(targets[5]["centers"], W.bump_target(1005)["centers"])
    reqs = W.request_stream(4000, rate=100.0, seed=7)
    ts = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(ts) > 0)
    assert abs(len(ts) / ts[-1] / 100.0 - 1.0) < 0.05
    assert {r["n"] for r in reqs} == {32, 64, 96, 128, 192}
    assert all(1e-8 <= r["rho"] <= 1.0 for r in reqs)
