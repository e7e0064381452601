"""Host logic of bench.py's multi-GPU path, run as two gloo ranks on the CPU.

With N GPUs every rank solves its own seeded replica (independent problems,
no collective on the data path); the job's throughput is the units all ranks
processed divided by the slowest rank's time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [2.0, 3.0][rank]            # rank 1 is the slow one
    units = [1000.0, 1500.0][rank]   # replicas differ in size
    tms, value = bench.aggregate_ranks(ms, units, 10, dist, "cpu")
    out.put((rank, tms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, tms, value in res:
        assert tms == 3.0
        assert value == pytest.approx(10 * 2500.0 / 3e-3)


def test_single_process_aggregate():
    import bench
    ms, value = bench.aggregate_ranks(4.0, 100.0, 5)
    assert ms == 4.0 and value == pytest.approx(5 * 100.0 / 4e-3)


def test_replicas_are_distinct_seeded_problems():
    import bench
    (p0,), _ = bench.workload(1, rank=0)
    (p1,), _ = bench.workload(1, rank=1)
    assert p0.R == p1.R
    assert not all(np.array_equal(a, b) for a, b in zip(p0.q, p1.q))
