"""One rotation set partitioned over ranks (SO(3) clusters, redundant torque
halos): each rank's field set, built from its own build set, holds for its
owned rotations exactly the energy, force and torque fields of the field set
of the whole collection.  The ranks run one after the other on one GPU; they
share nothing."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch
    import paper_1711_05017_b300 as hf_
    from paper_1711_05017_b300 import build
    build.build()
    assert torch.cuda.is_available()
    return hf_


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_ranks_reproduce_the_whole_set(hf):
    from paper_1711_05017_b300 import shard as S
    n, R, world = 32, 96, 3
    ctx = hf.Context(0)
    s1, s2 = synth.c1_pair(9)
    r1 = oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    q = synth.random_quaternions(17, R).astype(np.float32)
    full = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
    full.compute(p1, p2, q)
    seen = np.zeros(R, dtype=int)
    shards = S.shard(q, world)
    for rank, s in enumerate(shards):
        fs = ctx.fieldset(n, len(s.build), hf.HF_E | hf.HF_F | hf.HF_T)
        fs.compute(p1, p2, q[s.build])
        for g, loc in zip(s.owned, s.local):
            for f in range(7):
                assert np.array_equal(host(fs.get(int(loc), f)), host(full.get(int(g), f))), (g, f)
            seen[g] += 1
        # a routed query answers as the whole set does when its route is exact
        t = np.array([0.05, -0.1, 0.02], dtype=np.float32)
        for p in synth.random_quaternions(30 + rank, 8).astype(np.float32):
            r, exact = S.route(q, shards, p, k=4)
            if exact and r == rank:
                np.testing.assert_array_equal(fs.query(t, p, k=4), full.query(t, p, k=4))
    assert (seen == 1).all()
