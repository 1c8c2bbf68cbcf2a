"""The multi-GPU path is replicas only (nothing is sharded): each rank runs its own steps and
the job's throughput is the units of all ranks over the slowest rank's time.  Two gloo
processes on the CPU check that reduction with unequal per-rank work and times."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = [1000.0, 3000.0][rank]
        ms = [10.0, 20.0][rank]
        value, ms_max = bench.replica_throughput(units, ms, world, "cpu")
        mx = bench.reduce_over_ranks(float(rank + 5), "max", world, "cpu")
        sm = bench.reduce_over_ranks(float(rank + 5), "sum", world, "cpu")
        out.put((rank, value, ms_max, mx, sm))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_over_two_gloo_ranks():
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
    for rank, value, ms_max, mx, sm in res:
        assert ms_max == 20.0
        assert value == pytest.approx(4000.0 / 0.020)
        assert mx == 6.0 and sm == 11.0


def test_single_rank_is_the_identity():
    import bench
    value, ms = bench.replica_throughput(500.0, 4.0, 1, "cpu")
    assert ms == 4.0 and value == pytest.approx(500.0 / 0.004)
