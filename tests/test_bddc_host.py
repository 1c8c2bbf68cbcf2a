"""Host-side logic of the BDDC variant (no GPU): the slab split and its interface size, and
the all-reduce callback that sums the slabs' contributions over ranks, run as two gloo
processes on the CPU (the library calls it with host buffers for the coarse matrix and the
coarse right-hand sides)."""
import ctypes
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_partition_covers_the_layers():
    import paper_2102_03515_gb300 as fa
    for n, p in [(4, 2), (16, 4), (17, 3), (128, 8), (256, 7)]:
        lb, ni = fa.fem_bddc_partition(n, p)
        assert lb[0] == 0 and lb[-1] == n and len(lb) == p + 1
        assert all(lb[s + 1] - lb[s] >= 1 for s in range(p))
        assert max(lb[s + 1] - lb[s] for s in range(p)) - min(lb[s + 1] - lb[s] for s in range(p)) <= 1
        assert ni == (p - 1) * (n - 1) ** 2
    for n, p in [(3, 2), (16, 1), (16, 9)]:
        with pytest.raises(fa.FemError):
            fa.fem_bddc_partition(n, p)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import paper_2102_03515_gb300 as fa
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slabs = 5
        lb, _ = fa.fem_bddc_partition(40, slabs)
        # the slabs of this rank: a contiguous half of them
        s0, s1 = rank * slabs // world, (rank + 1) * slabs // world
        cb = fa.make_allreduce()
        # coarse matrix of the slab plane averages: each slab adds its 2x2 block (1/|s| here)
        nc = slabs - 1
        S = (ctypes.c_double * (nc * nc))()
        for s in range(s0, s1):
            faces = [f for f in (s - 1, s) if 0 <= f < nc]
            for a in faces:
                for b in faces:
                    S[a * nc + b] += 1.0 / (lb[s + 1] - lb[s]) + (1.0 if a == b else 0.0)
        cb(S, nc * nc, 0, None)
        q.put((rank, s0, s1, list(S)))
    finally:
        dist.destroy_process_group()


def test_allreduce_callback_sums_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, b0, S0), (r1, a1, b1, S1) = res
    assert (a0, b0, a1, b1) == (0, 2, 2, 5)     # every slab owned once
    assert S0 == S1                             # replicated after the sum
    # the sum equals the one-process assembly over all slabs
    import paper_2102_03515_gb300 as fa
    lb, _ = fa.fem_bddc_partition(40, 5)
    nc = 4
    ref = np.zeros((nc, nc))
    for s in range(5):
        faces = [f for f in (s - 1, s) if 0 <= f < nc]
        for a in faces:
            for b in faces:
                ref[a, b] += 1.0 / (lb[s + 1] - lb[s]) + (1.0 if a == b else 0.0)
    assert np.allclose(np.array(S0).reshape(nc, nc), ref, rtol=0, atol=1e-15)
