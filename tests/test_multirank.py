"""The multi-rank paths, run as world-size-2 gloo process groups on CPU:
bench.py's (one rank per GPU, rotation batches sharded by rank, no
collective on the data path, max-over-ranks timing), and one rotation set
partitioned over ranks by SO(3) clusters with redundant torque halos
(paper_1711_05017_b300.shard)."""
import os
import socket

import numpy as np
import pytest
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


def _shard_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import oracle
    import synth
    from paper_1711_05017_b300 import shard as S
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        R, n = 160, 4
        q = synth.random_quaternions(21, R)
        mine = S.shard(q, world)[rank]  # every rank partitions the same set alike
        # ownership covers the set exactly once
        flags = torch.zeros(R, dtype=torch.int64)
        flags[torch.as_tensor(mine.owned)] = 1
        dist.all_reduce(flags)
        # the rank's torque for its owned rotations, from its build set alone,
        # equals the whole set's (stand-in energy fields: any values will do)
        E = np.random.default_rng(3).standard_normal((R, n, n, n))
        qn = q / np.linalg.norm(q, axis=1, keepdims=True)
        T_full, st_full = oracle.torque(qn, E, 6)
        T_mine, st_mine = oracle.torque(qn[mine.build], E[mine.build], 6)
        same = np.array_equal(T_mine[mine.local], T_full[mine.owned]) and np.array_equal(st_mine[mine.local],
                                                                                          st_full[mine.owned])
        out[rank] = (flags.numpy().tolist(), len(mine.owned), same)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_share_one_rotation_set_without_exchange():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] == [1] * 160 and r1[0] == [1] * 160  # each rotation owned by exactly one rank
    assert r0[1] + r1[1] == 160 and abs(r0[1] - r1[1]) <= 1
    assert r0[2] and r1[2]  # owned torque identical to the whole set's


def test_shard_neighbourhoods_and_query_routing():
    """Neighbour search inside a build set agrees with the oracle's over the
    whole set for every owned rotation; routed queries find their blend set
    on the chosen rank, and the route is exact for most poses."""
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    from paper_1711_05017_b300 import shard as S
    q = synth.random_quaternions(4, 300)
    qn = q / np.linalg.norm(q, axis=1, keepdims=True)
    shards = S.shard(q, 3)
    assert sorted(np.concatenate([s.owned for s in shards]).tolist()) == list(range(300))
    for s in shards:
        sub = qn[s.build]
        for g, l in zip(s.owned[::7], s.local[::7]):
            full, _ = oracle.nearest(qn, qn[g], 6, skip=int(g))
            loc, _ = oracle.nearest(sub, sub[l], 6, skip=int(l))
            assert np.array_equal(full, s.build[loc]), g
    # a complete rotation's 6 nearest all lie in the build set
    for s in shards:
        for g in s.complete[::5]:
            full, _ = oracle.nearest(qn, qn[g], 6, skip=int(g))
            assert np.isin(full, s.build).all(), g
    poses = synth.random_quaternions(8, 200)
    counts = {}
    for halo in (8, 16):
        sh = S.shard(q, 3, halo=halo)
        exact = 0
        for p in poses:
            r, ok = S.route(q, sh, p, k=4)
            want, _ = oracle.nearest(qn, p / np.linalg.norm(p), 4)
            if ok:
                assert np.isin(want, sh[r].complete).all()
            exact += ok
        counts[halo] = exact
    # a deeper halo makes more rotations complete and more routes exact
    assert counts[8] >= 120 and counts[16] >= 170 and counts[16] > counts[8]
    with pytest.raises(ValueError):
        S.shard(q, 2, halo=5)
