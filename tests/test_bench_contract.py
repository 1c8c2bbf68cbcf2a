"""The benchmark's host-side contract without a GPU: the reference arm's JSON line (the oracle
timed on the host's cores) has the keys and types the contract names, and the algorithmic-byte
model of one V-cycle adds up the terms its docstring lists."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, cwd=ROOT,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference"
    for k in ("metric", "unit", "config", "dtype", "data", "scaling"):
        assert isinstance(j[k], (str, dict)) and j[k], k
    assert j["value"] > 0 and j["higher_is_better"] is True
    assert j["n_gpus"] == 1 and j["steps"] == 1 and j["warmup"] == 0
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == j["value"] and cb["cores"] > 0
    assert cb["host_cores"] >= 1 and isinstance(cb["sample"], str)
    e2e = j["e2e"]
    assert e2e["value"] == j["value"] and e2e["unit"] == j["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_vcycle_byte_model_sums_its_terms():
    sys.path.insert(0, ROOT)
    import bench
    info = {"levels": 3, "rows": [1000, 100, 10], "nnz": [16000, 2000, 100],
            "pnnz": [4000, 400, 0], "rnnz": [3000, 300, 0], "finest_stencil": True}
    b = bench.vcycle_bytes(info)
    # the matrix-free finest level prolongs by the smoothed prolongator's stencil: 24 bytes
    # per fine row and the coarse vector
    fine = 84.0 * 1000 + (8 * 3000 + 4 * 100 + 4 * 1000 + 4 * 100) + (24 * 1000 + 4 * 100)
    mid = 64.0 * 100 + 4 * (8 * 2000 + 4 * 100) + (8 * 300 + 4 * 10 + 4 * 100 + 4 * 10) \
        + (8 * 400 + 4 * 100 + 8 * 100 + 4 * 10)
    coarsest = 8.0 * 10 * 10 + 12.0 * 10
    assert b == fine + mid + coarsest
    assert bench.vcycle_bytes(info, flexible_r2=True) == b + 8.0 * 1000
