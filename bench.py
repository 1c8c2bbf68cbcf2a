"""Benchmark: AMG-preconditioned CG for (rho K + M) u = f on the 256^3 Kuhn mesh.

One step = fem_assemble + amg_setup + pcg_solve to ||f - A u|| / ||f|| <= 1e-8 on the
unit cube with n = 256 cells per side (255^3 = 16,581,375 unknowns), rho = h^2, smooth
sine target (the smooth-target experiment of arXiv 2102.03515, Sec. 4.1, at h = 1/256),
with the FP32 V-cycle inside FP64 flexible CG.  The metric is dof-iterations per second
of the whole step (unknowns x CG iterations / step time; setup included, as the paper's
timings include coarsening).  FP64 and BF16 V-cycles of the same workload are reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs independent replicas (one per GPU, launched by torchrun); nothing is sharded.
--impl reference times the FP64 CPU oracle (assembly, smoothed-aggregation hierarchy and
AMG-PCG in numpy/scipy) on a smaller mesh of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 256
TOL = 1e-8
ORACLE_N = 48          # reference-arm step: the same workload on a 48^3 mesh
CPU_SAMPLE_N = 64        # cpu_baseline sample: the same workload on a 64^3 mesh
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from ncu captures of
# the current kernels, by kernel: None until a capture of the current code exists
# (the product's launches as captured; its small row-pointer scans changed since: 0.94 GB of
# these bytes came from them and all sixteen small launches)
TRAFFIC = {"galerkin_l0_n256": (11.852 + 5.813) * 1e9,
           "cg_operator_n256": (265.38 + 104.65) * 1e6,
           "vcycle_fp32_n256": (4161.8 + 437.6) * 1e6}


def reduce_over_ranks(x: float, op: str, world: int, device) -> float:
    """Max or sum of a per-rank scalar over the process group (the value itself at world 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units_local: float, ms_local: float, world: int, device):
    """(whole-job units per second, the slowest rank's ms per step).  Replicas run their own
    steps with nothing shared, so the job processes the units of all ranks in the time of
    the slowest."""
    ms = reduce_over_ranks(ms_local, "max", world, device)
    units = reduce_over_ranks(units_local, "sum", world, device)
    return units / (ms / 1e3), ms


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _measured_hbm_gbs() -> float:
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except Exception:
        return 6800.0   # the profiling recipe's fallback copy rate


def vcycle_bytes(info: dict, flexible_r2: bool = False) -> float:
    """Algorithmic bytes of one FP32 V-cycle (Chebyshev degree 2, matrix-free finest level,
    FP32 CSR4 values on coarser levels, every vector access counted once): finest level
    16 (start from the FP64 residual: read it, write b and d) + 12 (the step after the start:
    d, b -> x) + 12 (residual) + 16 (post start: b, x -> r, d) + 28 (last step: d, r, x,
    FP64 z and <z, r>; + 8 with <z, r_prev>) bytes per row; a CSR level 64 bytes of vectors
    per row (8 + 12 + 12 + 16 + 16) and four passes over its matrix (8 bytes per stored
    entry + 4 per row); R_l and P_l one pass each plus their vectors, except the matrix-free
    finest level's prolongation: the stencil of the smoothed prolongator on the aggregates'
    values (aggregate ids read twice, t written and read, x read and written: 24 bytes per
    row, the coarse vector once); the coarsest dense inverse N^2 x 8 bytes."""
    L = info["levels"]
    rows, nnz, pnnz, rnnz = info["rows"], info["nnz"], info["pnnz"], info["rnnz"]
    total = 0.0
    for lev in range(L):
        N = rows[lev]
        coarsest = lev == L - 1
        if coarsest:
            total += 8.0 * N * N + 12.0 * N
            continue
        if lev == 0 and info["finest_stencil"]:
            total += (84.0 + (8.0 if flexible_r2 else 0.0)) * N
        else:
            total += 64.0 * N + 4 * (8.0 * nnz[lev] + 4.0 * N)
        Nc = rows[lev + 1]
        total += 8.0 * rnnz[lev] + 4.0 * Nc + 4.0 * N + 4.0 * Nc      # restriction
        if lev == 0 and info["finest_stencil"]:
            total += 24.0 * N + 4.0 * Nc                              # stencil prolongation
        else:
            total += 8.0 * pnnz[lev] + 4.0 * N + 8.0 * N + 4.0 * Nc   # prolongation
    return total


def oracle_sample(n: int) -> dict:
    """Run the oracle's full path (assemble, SA hierarchy, AMG-PCG to 1e-8) at n^3."""
    import numpy as np  # noqa: F401
    import fem_workloads as W
    from oracle import amg, core
    t0 = time.perf_counter()
    c0 = time.process_time()
    s = core.assemble(n, W.sine_target())
    rho = 1.0 / n ** 2
    A = s.A(rho)
    H = amg.build_hierarchy(A)
    x, it, rr, _ = amg.pcg(A, s.f, lambda r: amg.vcycle(H, r), tol=TOL)
    dt = time.perf_counter() - t0
    cpu = time.process_time() - c0
    N = A.shape[0]
    return {"n": n, "N": N, "iterations": it, "seconds": dt, "relres": rr,
            "value": N * it / dt, "cores_used": cpu / dt if dt > 0 else 1.0}


def host_cpu() -> dict:
    """Cores this process may run on and the CPU model (from /proc/cpuinfo when present)."""
    try:
        ncores = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        ncores = os.cpu_count() or 0
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "processor name") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "cpu part":   # Arm: the part number (0xd4f: Neoverse V2)
                        model = "CPU part " + model
                    if key == "model name":
                        break
    except OSError:
        pass
    return {"host_cores": ncores, "cpu_model": model}


def oracle_subprocess(n: int, timeout: float = 600.0) -> dict:
    """The oracle in a single-threaded child process (started before any GPU work)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(%d)))" % (ROOT, n))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         env=env, timeout=timeout, cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_reference_start(n: int, path: str):
    """Start (before any GPU work) a child process that assembles and solves the full system
    with the oracle (Jacobi-PCG to a relative residual of 1e-13, the independent row loops on
    all but two host cores) and saves the solution to `path`."""
    threads = max(1, host_cpu()["host_cores"] - 2)
    code = ("import json, sys, time; sys.path.insert(0, %r); import numpy as np; "
            "import fem_workloads as W; from oracle import core; "
            "core.set_threads(%d); t0 = time.perf_counter(); s = core.assemble(%d, W.sine_target()); "
            "t1 = time.perf_counter(); x, it, rr = core.jacobi_pcg(s, 1.0 / %d ** 2, s.f, tol=1e-13); "
            "t2 = time.perf_counter(); np.save(%r, x); "
            "print(json.dumps({'assemble_s': t1 - t0, 'solve_s': t2 - t1, 'iterations': it, "
            "'relres': rr, 'threads': %d, 'N': len(x)}))" % (ROOT, threads, n, n, path, threads))
    env = dict(os.environ)
    env["OMP_NUM_THREADS"] = str(threads)
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                            stderr=subprocess.PIPE, text=True, env=env, cwd=ROOT,
                            preexec_fn=lambda: os.nice(10))


def oracle_reference_finish(proc, path: str, timeout: float = 900.0):
    try:
        out, err = proc.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        proc.kill()
        return None, {"error": "oracle reference timed out"}
    if proc.returncode != 0:
        return None, {"error": err[-500:]}
    import numpy as np
    info = json.loads(out.strip().splitlines()[-1])
    x = np.load(path)
    try:
        os.remove(path)
    except OSError:
        pass
    return x, info


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def batched_sample(fa, torch, dev, n: int = 128, nrhs: int = 64):
    """64 targets and rho_k on the 128^3 mesh: one batched solve (FP32 V-cycle, FP64 flexible
    CG) against 64 sequential FP64 AMG-PCG solves, each with its own hierarchy."""
    import numpy as np
    import fem_workloads as W
    targets, rhos = W.batched_workload(n, nrhs)
    N = (n - 1) ** 3

    def batched():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target(), keep_pencil=True)
        h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32, rho_setup=float(np.max(rhos)))
        F = torch.empty((N, nrhs), dtype=torch.float64, device=dev)
        f = torch.empty(N, dtype=torch.float64, device=dev)
        for k, t in enumerate(targets):
            fa.fem_assemble_rhs(s, t, f)
            F[:, k] = f
        U = torch.zeros((N, nrhs), dtype=torch.float64, device=dev)
        res = fa.pcg_solve(s, h, F, U, nrhs=nrhs, rho_k=rhos, tol=TOL)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(s)
        return U, res, dt

    def sequential():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U = torch.zeros((N, nrhs), dtype=torch.float64, device=dev)
        u = torch.zeros(N, dtype=torch.float64, device=dev)
        its = []
        for k in range(nrhs):
            s = fa.fem_assemble(n, float(rhos[k]), targets[k])
            h = fa.amg_setup(s, precision=fa.AMG_PREC_FP64)
            r = fa.pcg_solve(s, h, None, u, tol=TOL)[0]
            its.append(r["iterations"])
            U[:, k] = u
            fa.amg_hier_destroy(h)
            fa.fem_system_destroy(s)
        torch.cuda.synchronize()
        return U, its, time.perf_counter() - t0

    def solve_only():
        # the same pencil and hierarchy: 64 one-column solves against one 64-column solve
        s = fa.fem_assemble(n, 1.0 / n ** 2, W.sine_target(), keep_pencil=True)
        h = fa.amg_setup(s, precision=fa.AMG_PREC_FP32, rho_setup=float(np.max(rhos)))
        F = torch.empty((N, nrhs), dtype=torch.float64, device=dev)
        f = torch.empty(N, dtype=torch.float64, device=dev)
        for k, t in enumerate(targets):
            fa.fem_assemble_rhs(s, t, f)
            F[:, k] = f
        U = torch.zeros((N, nrhs), dtype=torch.float64, device=dev)
        fa.pcg_solve(s, h, F, U, nrhs=nrhs, rho_k=rhos, tol=TOL)    # warm-up (tuning)
        U.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rb = fa.pcg_solve(s, h, F, U, nrhs=nrhs, rho_k=rhos, tol=TOL)
        torch.cuda.synchronize()
        tb1 = time.perf_counter() - t0
        u1 = torch.zeros((N, 1), dtype=torch.float64, device=dev)
        f1 = torch.empty((N, 1), dtype=torch.float64, device=dev)
        fa.pcg_solve(s, h, F[:, :1].contiguous(), u1, nrhs=1, rho_k=rhos[:1], tol=TOL)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its1 = []
        dmax = 0.0
        for k in range(nrhs):
            f1.copy_(F[:, k:k + 1])
            u1.zero_()
            r1 = fa.pcg_solve(s, h, f1, u1, nrhs=1, rho_k=rhos[k:k + 1], tol=TOL)
            its1.append(r1[0]["iterations"])
            dmax = max(dmax, (torch.linalg.norm(u1[:, 0] - U[:, k]) /
                              torch.linalg.norm(U[:, k])).item())
        torch.cuda.synchronize()
        ts1 = time.perf_counter() - t0
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(s)
        return {"batched_ms": tb1 * 1e3, "sequential_ms": ts1 * 1e3, "speedup": ts1 / tb1,
                "iterations_min_max": [min(r["iterations"] for r in rb),
                                       max(r["iterations"] for r in rb)],
                "sequential_iterations_min_max": [min(its1), max(its1)],
                "max_rel_diff_batched_vs_one_column": dmax}

    batched()  # warm-up
    Ub, res, tb = batched()
    Us, its_s, ts = sequential()
    so = solve_only()
    its_b = [r["iterations"] for r in res]
    err = max((torch.linalg.norm(Ub[:, k] - Us[:, k]) / torch.linalg.norm(Us[:, k])).item()
              for k in range(nrhs))
    return {"workload": "128^3 Kuhn mesh (2,048,383 dofs), 64 Gaussian-bump targets, rho_k "
                        "log-uniform in [1e-6, 1e-2], tol 1e-8",
            "value": N * sum(its_b) / tb, "unit": "dof-iters/s", "ms": tb * 1e3,
            "iterations_min_max": [min(its_b), max(its_b)],
            "sequential_fp64_ms": ts * 1e3, "sequential_iterations_min_max": [min(its_s), max(its_s)],
            "speedup_vs_sequential_fp64": ts / tb, "max_rel_diff_vs_sequential_fp64": err,
            "solve_only_same_hierarchy": so}


# The paper's Tables 1 and 2 at h = 1/256 (Sec. 4.1; another mesh, so context only)
PAPER_TABLE_H256 = {1e-2: (8.9566e-6, 1.2731e-2), 1e-4: (8.4684e-6, 1.6453e-2)}


def paper_tables_sample(fa, torch, dev, n: int):
    """||u_rho - u_rho,h||_L2 and ||grad(u_rho - u_rho,h)||_L2 from GPU solves (FP64 V-cycle,
    tol 1e-10) with the device error norms, next to the paper's Tables 1 and 2."""
    import math
    import fem_workloads as W
    out = {"h": 1.0 / n, "rows": []}
    N = (n - 1) ** 3
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    for rho, (pl2, ph1) in PAPER_TABLE_H256.items():
        sys_ = fa.fem_assemble(n, rho, W.sine_target())
        h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP64)
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-10)[0]
        scale = 1.0 / (3.0 * rho * math.pi ** 2 + 1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fa.fem_errors(sys_, u, W.sine_target(), scale=scale, qlevel=1)
        te = time.perf_counter() - t0
        z = torch.empty_like(u)
        p = torch.empty_like(u)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fa.fem_recover(sys_, u, W.sine_target(), z, p)
        tr = time.perf_counter() - t1
        row = {"rho": rho, "iterations": res["iterations"], "l2": math.sqrt(r["l2sq"]),
               "h1": math.sqrt(r["h1sq"]), "paper_l2": pl2 if n == 256 else None,
               "paper_h1": ph1 if n == 256 else None, "errors_ms": te * 1e3,
               "recover_ms": tr * 1e3}
        out["rows"].append(row)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)
    return out


# Table 3 of the paper (Sec. 4.1): ||ubar - u_h||^2 in H^-1 and in L2 for ubar = sin sin sin at
# h = rho^(1/2); its L2 column is the continuous (1/8) (3 rho pi^2 / (3 rho pi^2 + 1))^2, its
# H^-1 column 0.030341 times that (the continuous dual norm gives 1 / (3 pi^2) = 0.033774 times)
PAPER_TABLE3 = {1.0: (3.54886e-3, 1.16966e-1), 1e-1: (2.11939e-3, 6.98529e-2),
                1e-2: (1.97952e-4, 6.52427e-3), 1e-3: (3.13686e-6, 1.03388e-4),
                1e-4: (3.30578e-8, 1.08962e-6)}


def table3_sample(fa, torch, dev, n: int):
    """||ubar - u_h||^2 in the discrete H^-1 norm (fem_error_hm1: r^T K^-1 r) and in L2
    (fem_errors) from GPU solves on one mesh (h = 1/n, FP64 V-cycle, tol 1e-10), next to the
    continuous values and the paper's Table 3 (its meshes follow h = rho^(1/2): context)."""
    import math
    import fem_workloads as W
    rows = []
    N = (n - 1) ** 3
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    for rho, (phm1, pl2) in PAPER_TABLE3.items():
        sys_ = fa.fem_assemble(n, rho, W.sine_target())
        h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP64)
        res = fa.pcg_solve(sys_, h, None, u, tol=1e-10)[0]
        fa.amg_hier_destroy(h)
        l2sq = fa.fem_errors(sys_, u, W.sine_target(), qlevel=0)["l2sq"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hm = fa.fem_error_hm1(sys_, u, W.sine_target(), tol=1e-10)
        thm = time.perf_counter() - t0
        a = 3.0 * rho * math.pi ** 2 / (3.0 * rho * math.pi ** 2 + 1.0)
        l2c = a * a / 8.0
        rows.append({"rho": rho, "iterations": res["iterations"], "hm1sq": hm["hm1sq"],
                     "l2sq": l2sq, "continuous_hm1sq": l2c / (3.0 * math.pi ** 2),
                     "continuous_l2sq": l2c, "paper_hm1sq": phm1, "paper_l2sq": pl2,
                     "hm1_ms": thm * 1e3, "hm1_stiffness_iterations": hm["solve"]["iterations"]})
        fa.fem_system_destroy(sys_)
    return {"h": 1.0 / n, "rows": rows}


# Table 4 of the paper (Sec. 4.1): AMG-PCG iterations and total coarsening + solving time on
# MACH-2 (cores not stated), stopped at a preconditioned relative residual of 1e-8; rows rho,
# columns h = 1/8 ... 1/256
PAPER_TABLE4 = {
    1.0: [(8, 0.01), (10, 0.06), (12, 0.72), (14, 8.29), (17, 127.06), (20, 1420.73)],
    1e-2: [(6, 0.01), (8, 0.05), (9, 0.56), (11, 6.83), (13, 94.28), (15, 910.77)],
    1e-4: [(5, 0.00), (4, 0.04), (4, 0.38), (5, 4.51), (7, 65.85), (8, 646.14)],
    1e-6: [(5, 0.00), (5, 0.04), (5, 0.41), (5, 4.46), (4, 52.90), (4, 499.10)],
    1e-8: [(5, 0.00), (5, 0.04), (5, 0.41), (5, 4.46), (5, 57.59), (5, 530.97)],
    1e-10: [(5, 0.00), (5, 0.04), (5, 0.41), (5, 4.43), (5, 57.04), (5, 560.33)],
    1e-12: [(5, 0.00), (5, 0.04), (5, 0.41), (5, 4.42), (5, 54.63), (5, 603.02)],
}
TABLE4_N = (8, 16, 32, 64, 128, 256)


def table4_sample(fa, torch, dev):
    """Table 4's whole grid: h = 1/8 ... 1/256 by rho = 1 ... 1e-12, for the paper's AMG
    (red-black coarsening, averaging interpolation, symmetric Gauss-Seidel; the split visiting
    the unknowns by hashed priority, and in index order with FP64 V-cycles) and smoothed
    aggregation with Chebyshev, with FP64 and with FP32 V-cycles in FP64 CG (flexible for
    FP32), stopped like the paper (preconditioned relative residual 1e-8).  Each entry:
    iterations and assemble + set-up + solve time (the second of two runs: the first also
    tunes launch shapes)."""
    import fem_workloads as W
    variants = {"red_black_sgs": dict(coarsening=fa.AMG_COARSEN_RED_BLACK,
                                      smoother=fa.AMG_SMOOTHER_SGS),
                "red_black_natural_sgs": dict(coarsening=fa.AMG_COARSEN_RED_BLACK,
                                              smoother=fa.AMG_SMOOTHER_SGS,
                                              order=fa.AMG_ORDER_NATURAL),
                "sa_chebyshev": dict(coarsening=fa.AMG_COARSEN_SA,
                                     smoother=fa.AMG_SMOOTHER_CHEBYSHEV)}
    precs = {"fp64": fa.AMG_PREC_FP64, "fp32": fa.AMG_PREC_FP32}
    grid = {}
    for name, opts in variants.items():
        for pname, prec in precs.items():
            if name == "red_black_natural_sgs" and pname == "fp32":
                continue
            key = name + "_" + pname
            grid[key] = {}
            for rho in PAPER_TABLE4:
                its, ms = [], []
                for n in TABLE4_N:
                    N = (n - 1) ** 3
                    u = torch.zeros(N, dtype=torch.float64, device=dev)
                    for rep in range(2 if n >= 64 else 1):
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        sys_ = fa.fem_assemble(n, rho, W.sine_target())
                        h = fa.amg_setup(sys_, precision=prec, **opts)
                        res = fa.pcg_solve(sys_, h, None, u, tol=1e-8,
                                           flexible=1 if pname == "fp32" else 0,
                                           stop=fa.PCG_STOP_PRECONDITIONED)[0]
                        torch.cuda.synchronize()
                        dt = time.perf_counter() - t0
                        fa.amg_hier_destroy(h)
                        fa.fem_system_destroy(sys_)
                    its.append(res["iterations"])
                    ms.append(round(dt * 1e3, 2))
                grid[key]["%g" % rho] = {"iterations": its, "total_ms": ms}
    paper = {"%g" % r: {"iterations": [v[0] for v in row], "setup_plus_solve_s": [v[1] for v in row]}
             for r, row in PAPER_TABLE4.items()}
    return {"h": [1.0 / n for n in TABLE4_N], "rho": ["%g" % r for r in PAPER_TABLE4],
            "stop": "preconditioned relative residual sqrt(<r,z>/<r0,z0>) <= 1e-8",
            "ours": grid, "paper_mach2": paper}


def config2_sample(fa, torch, dev, n: int = 128):
    """Config 2: the 128^3 Kuhn mesh (2,048,383 dofs) with FP64 AMG-PCG to 1e-8 for rho = 1,
    h^2, 1e-6, the sine and the discontinuous box target, on the uniform mesh (matrix-free)
    and on the mesh with interior vertices jittered by U(-0.2h, 0.2h) (CSR path)."""
    import fem_workloads as W
    N = (n - 1) ** 3
    xyz_j = W.jittered_xyz(n, 0.2, seed=0)
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    rows = []
    for rho in (1.0, 1.0 / n ** 2, 1e-6):
        for tname, t in (("sine", W.sine_target()), ("box", W.box_target())):
            for mesh, xyz in (("uniform", None), ("jittered", xyz_j)):
                for rep in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    sys_ = fa.fem_assemble(n, rho, t, xyz=xyz)
                    torch.cuda.synchronize()
                    t1 = time.perf_counter()
                    h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP64)
                    res = fa.pcg_solve(sys_, h, None, u, tol=TOL)[0]
                    torch.cuda.synchronize()
                    t2 = time.perf_counter()
                    info = fa.amg_hier_get_info(h)
                    fa.amg_hier_destroy(h)
                    fa.fem_system_destroy(sys_)
                rows.append({"rho": rho, "target": tname, "mesh": mesh,
                             "iterations": res["iterations"], "relres": res["relres"],
                             "assemble_ms": (t1 - t0) * 1e3, "setup_ms": info["setup_ms"],
                             "solve_ms": res["solve_ms"], "total_ms": (t2 - t0) * 1e3,
                             "dof_iters_per_s": N * res["iterations"] / (t2 - t0),
                             "solve_dof_iters_per_s": N * res["iterations"] / (res["solve_ms"] / 1e3)})
    return {"workload": "128^3 Kuhn mesh, 2,048,383 dofs, FP64 AMG-PCG (SA, Chebyshev 2) to 1e-8",
            "rows": rows}


# Table 5 of the paper (Sec. 4.1): BDDC-PCG iterations (time) at h = 1/128 on RADON-1 with p
# cores = subdomains (another partition: graph-partitioned subdomains; context)
PAPER_TABLE5 = {1.0: [34, 34, 35, 36], 1e-4: [27, 27, 28, 30], 1e-12: [20, 20, 21, 21]}
PAPER_TABLE5_P = [32, 64, 128, 256]


def bddc_sample(fa, torch, dev, n: int = 128, slabs=(4, 8, 16)):
    """BDDC-preconditioned interface CG (Sec. 3.2) on the 128^3 Kuhn mesh split into slabs of
    cube layers, for rho = 1, 1e-4, 1e-12, stopped at 1e-8 on the interface residual
    (subdomain AMG-PCG solves to 1e-12): iterations, set-up and solve time, and the global
    relative residual, next to the paper's Table 5 (graph-partitioned subdomains, one core
    each: context)."""
    import fem_workloads as W
    N = (n - 1) ** 3
    u = torch.zeros(N, dtype=torch.float64, device=dev)
    rows = []
    for rho in PAPER_TABLE5:
        sys_ = fa.fem_assemble(n, rho, W.sine_target())
        for p in slabs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b = fa.bddc_setup(sys_, p, inner_tol=1e-12)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            res = fa.bddc_solve(b, None, u, tol=1e-8, max_iter=200)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            fa.bddc_destroy(b)
            rows.append({"rho": rho, "slabs": p, "iterations": res["iterations"],
                         "relres": res["relres"], "setup_s": t1 - t0, "solve_s": t2 - t1})
        fa.fem_system_destroy(sys_)
    return {"workload": "128^3 Kuhn mesh (2,048,383 dofs), slabs of cube layers along z, plane-"
                        "average primal constraints, FP64 subdomain AMG-PCG to 1e-12, interface "
                        "CG to 1e-8", "rows": rows,
            "paper_table5_iterations": {"%g" % k: v for k, v in PAPER_TABLE5.items()},
            "paper_table5_p": PAPER_TABLE5_P}


def general_mesh_sample(fa, torch, dev, n: int = 32, refine: int = 2):
    """An unstructured mesh through fem_assemble_mesh: the unit cube split into 5 tets per cube
    (n^3 cubes), refined `refine` times by Bey's red refinement; FP32 V-cycle in FP64 flexible
    CG to 1e-8 at rho = h^2 of the refined mesh (h = 1 / (n 2^refine))."""
    import fem_workloads as W
    mesh = W.five_tet_mesh(n)
    for _ in range(refine):
        mesh = W.bey_refine(*mesh)
    xyz, tets, d = mesh
    h = 1.0 / (n * 2 ** refine)
    rho = h * h
    out = {}
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sys_ = fa.fem_assemble_mesh(xyz, tets, d, rho, W.sine_target())
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        hh = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
        info = fa.fem_system_get_info(sys_)
        u = torch.zeros(info["N"], dtype=torch.float64, device=dev)
        res = fa.pcg_solve(sys_, hh, None, u, tol=1e-8, flexible=1)[0]
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        hinfo = fa.amg_hier_get_info(hh)
        fa.amg_hier_destroy(hh)
        fa.fem_system_destroy(sys_)
        out = {"workload": "five-tet cube mesh, n = %d, %d Bey refinements: %d tets, %d unknowns, "
                           "rho = h^2, sine target, FP32 V-cycle, tol 1e-8" % (n, refine, len(tets),
                                                                              info["N"]),
               "value": info["N"] * res["iterations"] / (t2 - t0), "unit": "dof-iters/s",
               "assemble_ms": (t1 - t0) * 1e3, "setup_ms": hinfo["setup_ms"],
               "solve_ms": res["solve_ms"], "total_ms": (t2 - t0) * 1e3,
               "iterations": res["iterations"], "relres": res["relres"],
               "nnz_per_row": info["nnz"] / info["N"]}
    return out


# ||ubar - u_rho h||^2_{L2} on the paper's adaptive meshes (about 1.3-3.7M dofs): Table 6
# (discontinuous box target, Sec. 4.2) and Table 8 (1 + sin sin sin, Sec. 4.3), by rho
PAPER_TABLE6_L2SQ = {1e0: 1.2018e-1, 1e-1: 9.0747e-2, 1e-2: 3.6563e-2, 1e-3: 1.1894e-2,
                     1e-4: 3.8028e-3, 1e-5: 1.2075e-3, 1e-6: 3.7988e-4}
PAPER_TABLE8_L2SQ = {1e0: 1.5613e0, 1e-1: 1.0842e0, 1e-2: 3.2593e-1, 1e-3: 9.5243e-2,
                     1e-4: 3.0292e-2, 1e-5: 9.6709e-3}
# and the H^-1 columns of the same tables (the paper's discrete H^-1 norm is not stated)
PAPER_TABLE6_HM1SQ = {1e0: 2.1308e-3, 1e-1: 1.3401e-3, 1e-2: 1.9101e-4, 1e-3: 9.0010e-6,
                      1e-4: 3.1821e-7, 1e-5: 1.0474e-8, 1e-6: 3.3491e-10}
PAPER_TABLE8_HM1SQ = {1e0: 3.5241e-2, 1e-1: 2.1590e-2, 1e-2: 2.5430e-3, 1e-3: 8.8234e-5,
                      1e-4: 2.7302e-6, 1e-5: 8.5525e-8}


def adaptive_sample(fa, torch, dev, max_dofs: int = 1_000_000, theta: float = 0.5, n0: int = 8,
                    max_steps: int = 40):
    """The adaptive runs of Sec. 4.2-4.3 with the mesh on the device: from the Kuhn mesh with
    n0^3 cubes, solve (FP32 V-cycle in FP64 flexible CG to 1e-8) -> residual indicator ->
    bulk marking (theta) -> longest-edge bisection, until the mesh has max_dofs unknowns;
    then ||ubar - u_h||^2 in L2 and in the discrete H^-1 norm (fem_error_hm1 on the final
    mesh, outside the timed phases) against the paper's Tables 6 and 8 (its meshes come from
    another refinement rule and stop at 1.3-3.7M dofs)."""
    import fem_workloads as W
    cases = [("box (Table 6)", W.box_target(), PAPER_TABLE6_L2SQ, PAPER_TABLE6_HM1SQ),
             ("1 + sin sin sin (Table 8)", W.sine_plus_one_target(), PAPER_TABLE8_L2SQ,
              PAPER_TABLE8_HM1SQ)]
    out = []
    for name, target, paper, paper_hm1 in cases:
        for rho, pl2 in paper.items():
            m = fa.fem_mesh_create(*W.kuhn_mesh(n0))
            ph = {"assemble": 0.0, "setup": 0.0, "solve": 0.0, "estimate_mark": 0.0,
                  "refine": 0.0}
            its = []
            dofs = []
            step = 0
            torch.cuda.synchronize()
            t_start = time.perf_counter()
            while True:
                t0 = time.perf_counter()
                sys_ = fa.fem_assemble_on_mesh(m, rho, target)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                h = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                info = fa.fem_system_get_info(sys_)
                u = torch.zeros(info["N"], dtype=torch.float64, device=dev)
                res = fa.pcg_solve(sys_, h, None, u, tol=1e-8, flexible=1)[0]
                torch.cuda.synchronize()
                t3 = time.perf_counter()
                its.append(res["iterations"])
                dofs.append(info["N"])
                ph["assemble"] += t1 - t0
                ph["setup"] += t2 - t1
                ph["solve"] += t3 - t2
                nt = fa.fem_mesh_get_info(m)["nt"]
                if info["N"] >= max_dofs or step == max_steps:
                    err = fa.fem_errors(sys_, u, target, scale=1.0, qlevel=1)
                    fa.amg_hier_destroy(h)
                    fa.fem_system_destroy(sys_)
                    break
                eta = torch.empty(nt, dtype=torch.float64, device=dev)
                fa.fem_error_indicator(sys_, u, target, eta)
                mark = torch.empty(nt, dtype=torch.uint8, device=dev)
                fa.fem_mark_bulk(eta, theta, mark)
                fa.amg_hier_destroy(h)
                fa.fem_system_destroy(sys_)
                torch.cuda.synchronize()
                t4 = time.perf_counter()
                fa.fem_mesh_refine(m, mark)
                torch.cuda.synchronize()
                t5 = time.perf_counter()
                ph["estimate_mark"] += t4 - t3
                ph["refine"] += t5 - t4
                step += 1
            total = time.perf_counter() - t_start
            sys_p = fa.fem_assemble_on_mesh(m, rho, target, keep_pencil=True)
            hm = fa.fem_error_hm1(sys_p, u, target, tol=1e-10)
            fa.fem_system_destroy(sys_p)
            fa.fem_mesh_destroy(m)
            out.append({"target": name, "rho": rho, "steps": step, "dofs": info["N"], "tets": nt,
                        "iterations_min": min(its), "iterations_max": max(its),
                        "iterations_last": its[-1], "l2sq": err["l2sq"], "paper_l2sq": pl2,
                        "ratio_to_paper": err["l2sq"] / pl2, "hm1sq": hm["hm1sq"],
                        "paper_hm1sq": paper_hm1[rho], "hm1_ratio_to_paper":
                            hm["hm1sq"] / paper_hm1[rho],
                        "hm1_stiffness_iterations": hm["solve"]["iterations"], "total_s": total,
                        "phases_s": ph, "dofs_per_step": dofs, "iterations_per_step": its})
    return {"workload": "adaptive loop from the Kuhn mesh n = %d to >= %d dofs, theta = %.2f, "
                        "longest-edge bisection, FP32 V-cycle in FP64 flexible CG to 1e-8"
                        % (n0, max_dofs, theta), "rows": out}


def serving_sample(count: int, sizes=(32, 64, 96, 128, 192), fractions=(0.5, 0.8, 1.0)):
    """Config 5: Poisson streams of `count` solve requests through the continuous-batching
    service at fractions of the measured saturation rate."""
    import fem_workloads as W
    from paper_2102_03515_gb300 import serving as S

    def reqs(rate, seed):
        return [S.Request(id=r["id"], n=r["n"], rho=r["rho"], target=r["target"],
                          t_arrival=r["t"]) for r in W.request_stream(count, rate, seed, sizes)]

    # 4 slots per session and one CG iteration per tick: the latency-optimal setting of a
    # sweep over 4-16 slots and 1-3 iterations (p50/p99 at 0.8 x saturation)
    svc = S.SolveService(S.ServeConfig(slots=4, steps_per_tick=1))
    loads = []
    try:
        # warm the hierarchy cache and measure the saturation rate (all requests at once)
        sat = svc.run(reqs(1e9, 7), realtime=False)
        for i, frac in enumerate(fractions):
            rate = frac * sat["solves_per_s"]
            svc.done = []
            ld = svc.run(reqs(rate, 8 + i), realtime=True, time_limit=600)
            loads.append({"fraction_of_saturation": frac, "arrival_rate_per_s": rate,
                          "p50_ms": ld["p50_ms"], "p99_ms": ld["p99_ms"],
                          "mean_ms": ld.get("mean_ms"), "solves_per_s": ld["solves_per_s"],
                          "converged": ld["converged"], "solved": ld["solved"],
                          "cache_hit_rate": ld["cache_hit_rate"]})
    finally:
        svc.close()
    return {"workload": "Poisson streams of %d requests, n in %s, rho log-uniform in [1e-8, 1], "
                        "8-bump targets, tol 1e-8, at %s x the measured saturation rate"
                        % (count, list(sizes), list(fractions)),
            "saturation_solves_per_s": sat["solves_per_s"], "runs": loads}


def run_ours(args, rank: int, world: int):
    import torch
    import torch.distributed as dist

    import fem_workloads as W
    from paper_2102_03515_gb300 import build as B
    B.build()
    import paper_2102_03515_gb300 as fa

    cpu = None
    oref_proc = None
    oref_path = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # oracle first: no process is forked after the GPU is initialised
        try:
            cpu = oracle_subprocess(CPU_SAMPLE_N)
        except Exception as e:  # the GPU number stands on its own
            cpu = {"error": str(e)[:300]}
    if rank == 0 and world == 1 and not args.no_oracle_reference:
        # the oracle's own solution of the full system, computed beside the GPU work
        import tempfile
        oref_path = os.path.join(tempfile.mkdtemp(prefix="oracle_ref_"), "x.npy")
        oref_proc = oracle_reference_start(args.n, oref_path)

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n = args.n
    rho = 1.0 / n ** 2
    N = (n - 1) ** 3
    target = W.sine_target()

    def barrier():
        if world > 1:
            dist.barrier()

    def step(precision: int, u, tol=TOL, f=None):
        sys_ = fa.fem_assemble(n, rho, target)
        h = fa.amg_setup(sys_, precision=precision)
        res = fa.pcg_solve(sys_, h, f, u, tol=tol)[0]
        info = fa.amg_hier_get_info(h)
        fa.amg_hier_destroy(h)
        fa.fem_system_destroy(sys_)
        return res, info

    def timed(precision: int, steps: int, warmup: int, u):
        for _ in range(warmup):
            step(precision, u)
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = fa.fem_kernel_launches()
        results = []
        e0.record(stream)
        for _ in range(steps):
            results.append(step(precision, u))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        return ms, results, fa.fem_kernel_launches() - l0

    def max_over_ranks(x: float) -> float:
        return reduce_over_ranks(x, "max", world, dev)

    u = torch.zeros(N, dtype=torch.float64, device=dev)
    # ---- headline: FP32 V-cycle inside FP64 flexible CG
    with Clocks(local) as clk:
        ms, results, launches = timed(fa.AMG_PREC_FP32, args.steps, args.warmup, u)
    its = results[-1][0]["iterations"]
    relres = max(r[0]["relres"] for r in results)
    u_mixed = u.clone()
    value, ms = replica_throughput(N * its, ms, world, dev)
    solve_ms = statistics.mean(r[0]["solve_ms"] for r in results)
    setup_ms = statistics.mean(r[1]["setup_ms"] for r in results)

    # ---- FP64 V-cycle (plain FP64 AMG-PCG) and BF16-stored V-cycle on the same workload
    extra = {}
    for name, prec in (("fp64", fa.AMG_PREC_FP64), ("bf16", fa.AMG_PREC_BF16)):
        ms2, res2, _ = timed(prec, max(1, args.steps // 2), 1, u)
        it2 = res2[-1][0]["iterations"]
        v2, ms2 = replica_throughput(N * it2, ms2, world, dev)
        extra[name] = {"value": v2, "ms_per_step": ms2,
                       "iterations": it2, "relres": res2[-1][0]["relres"],
                       "solve_ms": res2[-1][0]["solve_ms"], "setup_ms": res2[-1][1]["setup_ms"]}
        if name == "fp64":
            u_fp64 = u.clone()
        else:
            u_bf16 = u.clone()
    # the FP64 V-cycle solve to 1e-13 (the parity bar's setting): compared with the oracle
    # below, together with the three solves above (tol 1e-8)
    step(fa.AMG_PREC_FP64, u, tol=1e-13)
    u_tight = u.clone()
    sols = {"fp32_tol1e-8": u_mixed, "fp64_tol1e-8": u_fp64, "bf16_tol1e-8": u_bf16,
            "fp64_tol1e-13": u_tight}

    # ---- end to end through the C ABI with host buffers: every step copies its right-hand
    # side in from pinned host memory (a caller's own load vector, here the sine target's)
    # and reads the solution back
    host_u = torch.empty(N, dtype=torch.float64, pin_memory=True)
    host_f = torch.empty(N, dtype=torch.float64, pin_memory=True)
    f_in = torch.empty(N, dtype=torch.float64, device=dev)
    sys0 = fa.fem_assemble(n, rho, target)
    fa.fem_system_get_rhs(sys0, f_in)
    fa.fem_system_destroy(sys0)
    host_f.copy_(f_in)
    f_in.zero_()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.steps // 2)
    for _ in range(e2e_steps):
        f_in.copy_(host_f, non_blocking=True)
        step(fa.AMG_PREC_FP32, u, f=f_in)
        host_u.copy_(u, non_blocking=True)
        torch.cuda.synchronize()
    e2e_value, e2e_ms = replica_throughput(N * its, (time.perf_counter() - t0) * 1e3 / e2e_steps,
                                           world, dev)

    hbm = _measured_hbm_gbs()
    # ---- dominant kernels of a step (launch list): the set-up's Galerkin product on the
    # finest level (A P by the brick kernel, the upper part of R (A P) by the merge kernel,
    # its mirror), recomputed from the hierarchy and timed with CUDA events on the stream it
    # runs on
    sys_ = fa.fem_assemble(n, rho, target)
    hg = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
    ginfo = fa.amg_hier_get_info(hg)
    gms, ap_entries = fa.amg_galerkin_timed(hg, 0, 5)
    fa.amg_hier_destroy(hg)
    # compulsory bytes of the two-stage product: P_0 and R_0 read once (12 bytes per stored
    # entry, 4 per row pointer; A_0 is the stencil, nothing to read), A_0 P_0 written and
    # read once (12 bytes per entry, 8 per row length, twice), A_1 written once (12 bytes per
    # entry, 4 per row pointer)
    rows0, rows1 = ginfo["rows"][0], ginfo["rows"][1]
    gbytes = (12.0 * (ginfo["pnnz"][0] + ginfo["rnnz"][0]) + 4.0 * (rows0 + 1 + 2 * (rows1 + 1)) +
              2 * (12.0 * ap_entries + 8.0 * rows0) + 12.0 * ginfo["nnz"][1])
    galerkin_roof = {"bound": "hbm", "achieved": gbytes / (gms * 1e-3) / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": gbytes / (gms * 1e-3) / 1e9 / hbm,
                     "traffic": TRAFFIC["galerkin_l0_n256"],
                     "kernel": "finest-level Galerkin product R (A P) (k_ap_brick, upper "
                               "part by k_mg, mirror k_u_*)",
                     "kernel_ms": gms, "algorithmic_bytes": gbytes, "ap_entries": ap_entries,
                     "peak_source": "measured copy rate"}
    # ---- CG's operator q = A p (double-float on the FP32 pipe), as CG launches it
    x = torch.randn(N, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    kms = fa.fem_spmv_timed(sys_, x, y, 20)
    fa.fem_system_destroy(sys_)
    # p as FP32 pairs (8 bytes) and p in FP64 for <p, q> (8 bytes) read, q written (8 bytes)
    obytes = 24.0 * N
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    op_roof = {"bound": "hbm", "achieved": obytes / (kms * 1e-3) / 1e9, "peak": hbm,
               "unit": "GB/s", "frac": obytes / (kms * 1e-3) / 1e9 / hbm,
               "traffic": TRAFFIC["cg_operator_n256"],
               "kernel": "CG operator q = A p, 15-point stencil in double-float arithmetic "
                         "(k_stencil_df)", "kernel_ms": kms, "algorithmic_bytes": obytes,
               "peak_source": "measured copy rate",
               "fp32_tflops": 131.0 * N / (kms * 1e-3) / 1e12,
               "fp32_peak_tflops_from_unit_counts": fp32_peak}
    # the FP64 ceiling measured on this GPU (independent FMA chains)
    fp64_measured = fa.fem_measure_fp64_rate(10)

    # ---- the V-cycle as a whole against the HBM roofline (FP32 hierarchy, warm, in situ)
    sys_ = fa.fem_assemble(n, rho, target)
    hv = fa.amg_setup(sys_, precision=fa.AMG_PREC_FP32)
    vinfo = fa.amg_hier_get_info(hv)
    rv = torch.randn(N, dtype=torch.float64, device=dev)
    zv = torch.empty_like(rv)
    fa.amg_vcycle_graph(hv, rv, zv, 3)                 # warm-up
    vms = fa.amg_vcycle_graph(hv, rv, zv, 20)          # CUDA events around 20 graph replays
    fa.amg_hier_destroy(hv)
    fa.fem_system_destroy(sys_)
    vbytes = vcycle_bytes(vinfo)
    vcycle_roof = {"bound": "hbm", "achieved": vbytes / (vms * 1e-3) / 1e9, "peak": hbm,
                   "unit": "GB/s", "frac": vbytes / (vms * 1e-3) / 1e9 / hbm,
                   "traffic": TRAFFIC["vcycle_fp32_n256"],
                   "kernel": "one FP32 V-cycle (all levels, replayed from a CUDA graph)",
                   "ms": vms, "algorithmic_bytes": vbytes, "peak_source": "measured copy rate"}

    batched = serving = tables = table3 = table4 = general = adaptive = config2 = bddc = None
    if not args.no_extras:
        tables = paper_tables_sample(fa, torch, dev, n)
        table3 = table3_sample(fa, torch, dev, n)
        table4 = table4_sample(fa, torch, dev)
        config2 = config2_sample(fa, torch, dev)
        general = general_mesh_sample(fa, torch, dev)
        bddc = bddc_sample(fa, torch, dev)
        adaptive = adaptive_sample(fa, torch, dev)
        batched = batched_sample(fa, torch, dev)
        serving = serving_sample(args.serve_requests)

    # ---- the solutions against the oracle's own solution of the full system
    err_vs_oracle = None
    oracle_full = None
    if oref_proc is not None:
        xo, oracle_full = oracle_reference_finish(oref_proc, oref_path)
        if xo is not None:
            xo_d = torch.as_tensor(xo, device=dev)
            no = torch.linalg.norm(xo_d).item()
            err_vs_oracle = {k: torch.linalg.norm(v - xo_d).item() / no for k, v in sols.items()}

    if rank != 0:
        return
    line = {
        "metric": "PCG dof-iters/s: assemble + AMG setup + PCG to ||r||/||f|| <= 1e-8 at "
                  "255^3 = 16,581,375 dofs",
        "value": value,
        "unit": "dof-iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64 CG + f32 V-cycle",
        "data": "synthetic (seeded, generated on the device)",
        "config": {"workload": "unit-cube Kuhn mesh 256^3, 16,581,375 interior dofs, rho=h^2, "
                               "sine target, SA-AMG V-cycle (Chebyshev 2) in flexible CG, "
                               "tol 1e-8, FP32 V-cycle",
                   "n": n, "rho": rho, "tol": TOL,
                   "l2": "inputs larger than L2 (about 10 GB of matrices and vectors)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "iterations": its,
        "relres": relres,
        "time_to_tol_ms": ms,
        "setup_ms": setup_ms,
        "solve_ms": solve_ms,
        "solve_dof_iters_per_s": N * its / (solve_ms / 1e3),
        "fp64": extra["fp64"],
        "bf16": extra["bf16"],
        "err_vs_oracle": err_vs_oracle,
        "oracle_reference": oracle_full,
        "e2e": {"value": e2e_value, "unit": "dof-iters/s",
                "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N,
                "ms_per_step": e2e_ms},
        "roofline": galerkin_roof,
        "roofline_cg_operator": op_roof,
        "roofline_vcycle": vcycle_roof,
        "fp64_fma_tflops_measured": fp64_measured,
        "clocks": clk.summary(),
        "gpu_launches": launches,
    }
    if tables is not None:
        line["paper_tables"] = tables
    if table3 is not None:
        line["paper_table3"] = table3
    if table4 is not None:
        line["paper_table4"] = table4
    if general is not None:
        line["general_mesh"] = general
    if adaptive is not None:
        line["adaptive"] = adaptive
    if config2 is not None:
        line["config2"] = config2
    if bddc is not None:
        line["bddc"] = bddc
    if batched is not None:
        line["batched"] = batched
    if serving is not None:
        line["serving"] = serving
    if cpu is not None:
        if "value" in cpu:
            line["cpu_baseline"] = {"value": cpu["value"], "unit": "dof-iters/s",
                                    "cores": round(cpu.get("cores_used", 1.0), 2),
                                    "kind": "oracle", **host_cpu(),
                                    "sample": "oracle assemble + SA hierarchy + AMG-PCG to 1e-8 "
                                              "on the %d^3 mesh (%d dofs, %d iterations, %.1f s)"
                                              % (cpu["n"], cpu["N"], cpu["iterations"],
                                                 cpu["seconds"])}
        else:
            line["cpu_baseline"] = {"value": None, "unit": "dof-iters/s", "cores": 1,
                                    "kind": "oracle", "sample": cpu.get("error", "")}
    print(json.dumps(line), flush=True)


def run_reference(args, rank: int):
    if rank != 0:
        return
    vals, samples = [], []
    for _ in range(args.warmup):
        oracle_sample(ORACLE_N)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s = oracle_sample(ORACLE_N)
        vals.append(s["value"])
        samples.append(s)
    dt = time.perf_counter() - t0
    value = statistics.mean(vals)
    line = {
        "impl": "reference",
        "metric": "PCG dof-iters/s: assemble + AMG setup + PCG to ||r||/||f|| <= 1e-8 at "
                  "255^3 = 16,581,375 dofs",
        "value": value,
        "unit": "dof-iters/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / max(1, args.steps),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "unit-cube Kuhn mesh, rho=h^2, sine target, SA-AMG V-cycle in "
                               "CG, tol 1e-8; each step a bounded sample on the %d^3 mesh "
                               "(%d dofs)" % (ORACLE_N, samples[0]["N"] if samples else 0),
                   "n": ORACLE_N},
        "cpu_baseline": {"value": value, "unit": "dof-iters/s",
                         "cores": round(statistics.mean(s["cores_used"] for s in samples), 2)
                         if samples else 1.0, "kind": "oracle", **host_cpu(),
                         "sample": "oracle full path on the %d^3 mesh per step" % ORACLE_N},
        "e2e": {"value": value, "unit": "dof-iters/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_CELLS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the tables, config 2, batched and serving samples")
    ap.add_argument("--no-oracle-reference", action="store_true",
                    help="skip the oracle's full-size solve (err_vs_oracle)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    args = ap.parse_args()
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
