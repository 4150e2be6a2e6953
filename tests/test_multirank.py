"""The multi-rank path of bench.py (one rank per GPU, rotation batches
sharded by rank, no collective on the data path, max-over-ranks timing),
run as world-size-2 gloo process groups on CPU."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q = bench.rank_rotations(rank, 16)
        my_time = 1.0 + rank  # rank 1 is the slow one
        slowest = bench.max_over_ranks(my_time, world, "cpu")
        out[rank] = (q, slowest, bench.job_throughput(16, world, slowest))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_rotations_and_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        q0, t0, v0 = out[0]
        q1, t1, v1 = out[1]
    assert not np.allclose(q0, q1)  # distinct rotation batches per rank
    assert np.allclose(np.linalg.norm(q0, axis=1), 1.0)
    assert t0 == t1 == 2.0  # both ranks see the slowest rank's time
    assert v0 == v1 == 2 * 16 / 2.0  # whole-job units over the slowest time


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert np.array_equal(bench.rank_rotations(0, 8), bench.rank_rotations(0, 8))
