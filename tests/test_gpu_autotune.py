"""Launch-shape autotuner: every variant computes the same operator as the oracle, the
set-up tunes and caches choices, and the environment switches work.

Stencil variants differ only in tiling (each point's arithmetic is the same expression),
CSR variants in the order of a row's partial sums: FP64 results match the oracle's
A x to 1e-14 of sum |a_ij x_j|; FP32 V-cycles of different variants agree to 1e-5.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import fem_workloads as W
from oracle import core

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STENCIL_VARIANTS = 8
CSR_VARIANTS = 6


@pytest.fixture(scope="module")
def fa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_03515_gb300 import build as b
    b.build()
    import paper_2102_03515_gb300 as m
    yield m
    m.fem_autotune_clear()


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,jit", [(41, False), (23, True)])
def test_every_fp64_variant_matches_oracle(fa, n, jit):
    # m = n - 1 = 40: ragged against every tile height (4, 8, 16) and plane count (16..64)
    rho = 1.0 / n ** 2
    xyz = W.jittered_xyz(n, 0.2, seed=5) if jit else None
    s = core.assemble(n, W.sine_target(), xyz=xyz)
    N = (n - 1) ** 3
    x = W.random_vector(N, 11)
    yo = core.apply(s, rho, x)
    scale = np.abs(s.A(rho)).dot(np.abs(x))
    family, count = ("csr_f64", CSR_VARIANTS) if jit else ("stencil_f64", STENCIL_VARIANTS)
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz)
    try:
        for v in range(count):
            fa.fem_autotune_pin(family, v)
            y = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
            fa.fem_spmv(sys_, _dev(x), y)
            err = np.max(np.abs(y.cpu().numpy() - yo) / scale)
            assert err <= 1e-14, (family, v, err)
    finally:
        fa.fem_autotune_pin(family, -1)
        fa.fem_system_destroy(sys_)


@pytest.mark.parametrize("n,jit,prec", [(41, False, 1), (23, True, 1), (23, True, 2)])
def test_every_low_precision_variant_gives_the_same_vcycle(fa, n, jit, prec):
    rho = 1.0 / n ** 2
    xyz = W.jittered_xyz(n, 0.2, seed=6) if jit else None
    N = (n - 1) ** 3
    r = _dev(W.random_vector(N, 12))
    sys_ = fa.fem_assemble(n, rho, W.sine_target(), xyz=xyz)
    if jit:
        family, count = ("csr_bf16" if prec == 2 else "csr_f32"), CSR_VARIANTS
    else:
        family, count = "stencil_f32", STENCIL_VARIANTS
    try:
        h = fa.amg_setup(sys_, precision=prec)
        outs = []
        for v in range(count):
            fa.fem_autotune_pin(family, v)
            z = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
            fa.amg_vcycle(h, r, z)
            outs.append(z.cpu().numpy())
        fa.amg_hier_destroy(h)
        ref = outs[0]
        assert np.all(np.isfinite(ref))
        for v, z in enumerate(outs):
            d = np.max(np.abs(z - ref)) / np.max(np.abs(ref))
            assert d <= 1e-5, (family, v, d)
    finally:
        fa.fem_autotune_pin(family, -1)
        fa.fem_system_destroy(sys_)


def test_setup_tunes_and_caches(fa):
    fa.fem_autotune_clear()
    n = 96
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target())
    try:
        h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
        rep = fa.fem_autotune_report()
        assert rep["enabled"] is True
        kinds = {e["kernel"] for e in rep["entries"]}
        assert {"stencil_f32", "stencil_f64", "csr_f32"} <= kinds, kinds
        for e in rep["entries"]:
            assert e["source"] == "timed"
            assert 0 <= e["pick"] < len(e["variants"])
            assert all(v["us"] > 0 for v in e["variants"])
            if e["kernel"].startswith("stencil"):
                assert e["a"] == n - 1
        count = len(rep["entries"])
        h2 = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
        assert len(fa.fem_autotune_report()["entries"]) == count   # cache hits only
        # a solve with the tuned shapes still converges to the requested residual
        u = torch.zeros((n - 1) ** 3, dtype=torch.float64, device="cuda")
        res = fa.pcg_solve(sys_, h2, None, u, tol=1e-8)[0]
        assert res["status"] == "FEM_OK" and res["relres"] <= 1e-8
        fa.amg_hier_destroy(h)
        fa.amg_hier_destroy(h2)
    finally:
        fa.fem_system_destroy(sys_)


_CHILD = r"""
import json, sys, torch
import paper_2102_03515_gb300 as fa
import fem_workloads as W
n = 72
s = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target())
h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32)
fa.amg_hier_destroy(h)
fa.fem_system_destroy(s)
print(json.dumps(fa.fem_autotune_report()))
"""


def _child(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    out = subprocess.run([sys.executable, "-c", _CHILD], env=env, cwd=ROOT, capture_output=True,
                         text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_environment_switches(fa, tmp_path):
    off = _child({"FEM_AUTOTUNE": "0"})
    assert off["enabled"] is False and off["entries"] == []
    cache = str(tmp_path / "tune.txt")
    first = _child({"FEM_AUTOTUNE_CACHE": cache})
    timed = [e for e in first["entries"] if e["source"] == "timed"]
    assert timed
    lines = open(cache).read().split("\n")
    assert len([ln for ln in lines if ln.strip()]) == len(timed)
    second = _child({"FEM_AUTOTUNE_CACHE": cache})
    assert all(e["source"] == "file" for e in second["entries"])
    picks1 = {(e["kernel"], e["a"], e["b"], e["c"]): e["pick"] for e in timed}
    picks2 = {(e["kernel"], e["a"], e["b"], e["c"]): e["pick"] for e in second["entries"]}
    assert picks1 == picks2


@pytest.mark.parametrize("n,jit", [(17, False), (11, True)])
def test_every_multivector_variant_solves_to_the_oracle(fa, n, jit):
    # m = 16: several column blocks per plane range; B = 8 slots: 1, 2 and 4 slots per thread
    xyz = W.jittered_xyz(n, 0.2, seed=9) if jit else None
    nrhs = 8
    N = (n - 1) ** 3
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target(), xyz=xyz, keep_pencil=True)
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32, coarse_max=64)
    rhos = W.log_uniform(nrhs, 1e-6, 1e-2, seed=7)
    F = torch.empty((N, nrhs), dtype=torch.float64, device="cuda")
    refs = []
    try:
        for k in range(nrhs):
            t = W.bump_target(2000 + k)
            f = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.fem_assemble_rhs(sys_, t, f)
            F[:, k] = f
            s = core.assemble(n, t, xyz=xyz)
            refs.append(core.cholesky_solve(s.A(rhos[k]).toarray(), s.f))
        cases = [("mv_csr_f32", v) for v in range(3)]
        cases += [("mv_csr_f64", v) for v in range(3)] if jit else \
            [("mv_stencil_f32", v) for v in range(6)]
        for family, v in cases:
            fa.fem_autotune_pin(family, v)
            U = torch.zeros((N, nrhs), dtype=torch.float64, device="cuda")
            res = fa.pcg_solve(sys_, h, F, U, nrhs=nrhs, rho_k=rhos, tol=1e-11)
            fa.fem_autotune_pin(family, -1)
            Uh = U.cpu().numpy()
            for k in range(nrhs):
                assert res[k]["status"] == "FEM_OK", (family, v, res[k])
                err = np.linalg.norm(Uh[:, k] - refs[k]) / np.linalg.norm(refs[k])
                assert err <= 1e-9, (family, v, k, err)
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_batched_session_tunes_its_shapes(fa):
    fa.fem_autotune_clear()
    n, nrhs = 48, 16
    N = (n - 1) ** 3
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target(), keep_pencil=True)
    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
    try:
        F = torch.empty((N, nrhs), dtype=torch.float64, device="cuda")
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        for k in range(nrhs):
            fa.fem_assemble_rhs(sys_, W.bump_target(3000 + k), f)
            F[:, k] = f
        U = torch.zeros((N, nrhs), dtype=torch.float64, device="cuda")
        rhos = W.log_uniform(nrhs, 1e-6, 1e-2, seed=8)
        res = fa.pcg_solve(sys_, h, F, U, nrhs=nrhs, rho_k=rhos, tol=1e-8)
        assert all(r["status"] == "FEM_OK" for r in res)
        rep = fa.fem_autotune_report()
        mv = [e for e in rep["entries"] if e["kernel"].startswith("mv_")]
        assert any(e["kernel"] == "mv_stencil_f32" and e["c"] == nrhs for e in mv), mv
        assert any(e["kernel"] == "mv_csr_f32" for e in mv), mv
    finally:
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)


def test_graph_replayed_vcycle_equals_the_plain_one(fa):
    n = 33
    N = (n - 1) ** 3
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target())
    try:
        for prec in (0, 1):
            h = fa.amg_setup(sys_, precision=prec)
            r = _dev(W.random_vector(N, 4))
            z1 = torch.empty_like(r)
            z2 = torch.full_like(r, float("nan"))
            fa.amg_vcycle(h, r, z1)
            ms = fa.amg_vcycle_graph(h, r, z2, reps=5)
            fa.amg_hier_destroy(h)
            assert ms > 0
            assert torch.equal(z1, z2)
    finally:
        fa.fem_system_destroy(sys_)


def test_measured_fp64_rate_is_plausible(fa):
    # FMA throughput of the FP64 pipe: positive and of the order of the nominal 1.25 TFLOP/s
    rate = fa.fem_measure_fp64_rate(3)
    assert 0.05 < rate < 5.0, rate
