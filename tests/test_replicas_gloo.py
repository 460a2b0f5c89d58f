"""Multi-process (replica) path of bench.py on CPU with the gloo backend,
world size 2: the timed region is the maximum over ranks, the throughput
counts every rank's work, and every rank draws its own seeded replica."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        total, ms, value = bench.aggregate(100.0 * (rank + 1), 10, 1000, dist, "cpu")
        X = np.random.default_rng(0).uniform(-5, 5, (16, 3))
        field = bench.initial_field(X, bench.SEED + rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, field.tobytes())
        if rank == 0:
            out.put((total, ms, value, len(set(gathered))))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, ms, value, distinct = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert total == 200.0                      # max over ranks
    assert ms == 20.0
    assert value == pytest.approx(2 * 1000 * 4 / 0.020)
    assert distinct == 2                       # each rank steps its own replica


def test_single_process_aggregate():
    import bench
    total, ms, value = bench.aggregate(50.0, 5, 100)
    assert (total, ms) == (50.0, 10.0) and value == pytest.approx(100 * 4 / 0.010)
