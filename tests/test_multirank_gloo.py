"""The N > 1 host path of bench.py on the CPU: two gloo ranks (world_size 2).

Under torchrun every rank bootstraps its own flat level of independent gates (the
path shards by gate with no data-path collective); the whole-job figure is the units
all ranks processed over the slowest rank's time.  These tests run the bench's own
helpers for that on two spawned gloo processes, with no GPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [100.0, 125.0][rank]          # rank 1 is the slowest
        units = [4096 * 5, 4096 * 5][rank]
        q.put((rank,) + bench.reduce_max_sum(dist, ms, units, "cpu"))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, utot, rate in got:
        assert tmax == 125.0 and utot == 2 * 4096 * 5
        assert rate == pytest.approx(2 * 4096 * 5 / 0.125)


def test_rank_shards_are_distinct_problems():
    """Rank 0's shard is the 1-GPU workload; other ranks draw their own gates."""
    sys.path.insert(0, ROOT)
    import bench
    import tfhe_inputs as ti
    assert bench.shard_seed(ti.SEED_FLAT, 0) == ti.SEED_FLAT
    b0 = ti.flat_level(16, seed=bench.shard_seed(ti.SEED_FLAT, 0), p=ti.TOY)
    b1 = ti.flat_level(16, seed=bench.shard_seed(ti.SEED_FLAT, 1), p=ti.TOY)
    assert not np.array_equal(b0.inp, b1.inp)
    assert not np.array_equal(b0.types, b1.types) or not np.array_equal(b0.bits, b1.bits)
