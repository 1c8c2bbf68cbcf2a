"""fem_assemble_rhs_noalloc: the load vector for callers that cannot allocate device memory.

The allocation-free entry point must give what fem_assemble_rhs gives, on two calls in a
row (the shared scratch array keeps the previous call's contents), and refuse meshes
beyond its fixed scratch size.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

import fem_workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2102_03515_gb300 import build as b
    b.build()
    import paper_2102_03515_gb300 as m
    return m


@pytest.mark.parametrize("n,jitter", [(16, False), (11, True), (64, False)])
def test_noalloc_rhs_matches_allocating_entry_point(fa, n, jitter):
    xyz = W.jittered_xyz(n, 0.2, seed=3) if jitter else None
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target(), xyz=xyz)
    try:
        N = (n - 1) ** 3
        targets = [W.bump_target(21), W.box_target(), W.sine_plus_one_target(), W.bump_target(22)]
        for t in targets:
            ref = torch.empty(N, dtype=torch.float64, device="cuda")
            fa.fem_assemble_rhs(sys_, t, ref)
            for _ in range(2):  # two calls in a row share the scratch array
                got = torch.full((N,), float("nan"), dtype=torch.float64, device="cuda")
                fa.fem_assemble_rhs_noalloc(sys_, t, got)
                r, g = ref.cpu().numpy(), got.cpu().numpy()
                assert np.all(np.isfinite(g))
                # same kernels and order of operations: equal up to the last bit
                assert np.max(np.abs(g - r)) <= 1e-15 * np.max(np.abs(r))
    finally:
        fa.fem_system_destroy(sys_)


def test_noalloc_rhs_rejects_meshes_beyond_its_scratch(fa):
    sys_ = fa.fem_assemble(65, 1.0 / 65 ** 2, W.sine_target())
    try:
        f = torch.empty(64 ** 3, dtype=torch.float64, device="cuda")
        with pytest.raises(fa.FemError) as ei:
            fa.fem_assemble_rhs_noalloc(sys_, W.sine_target(), f)
        assert ei.value.status == 1  # FEM_EINVAL
        assert "64" in str(ei.value)
    finally:
        fa.fem_system_destroy(sys_)


def test_noalloc_rhs_rejects_point_value_targets(fa):
    n = 8
    sys_ = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target())
    try:
        N = (n - 1) ** 3
        vals = torch.ones(6 * n ** 3 * 4, dtype=torch.float64, device="cuda")
        f = torch.empty(N, dtype=torch.float64, device="cuda")
        with pytest.raises(fa.FemError) as ei:
            fa.fem_assemble_rhs_noalloc(sys_, {"kind": "quadvals", "values": vals}, f)
        assert ei.value.status == 1  # FEM_EINVAL
        assert "quadrature points" in str(ei.value)
    finally:
        fa.fem_system_destroy(sys_)
