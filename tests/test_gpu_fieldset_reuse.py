"""A field set recomputed over changing rotation sets: the host preparation
(matrices, 6 nearest neighbours, least-squares operators) is reused only while
the quaternions are the same bytes, so every compute matches a fresh field
set bit for bit, torque included."""
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


def cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def fields(fs, R):
    import torch
    torch.cuda.synchronize()
    return np.stack([fs.get(r, f).cpu().numpy() for r in range(R) for f in range(7)])


def test_reused_set_matches_fresh_sets(hf):
    n, R = 32, 20
    ctx = hf.Context(0)
    s1, s2 = synth.c1_pair(3)
    r1 = oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    qa = synth.random_quaternions(41, R).astype(np.float32)
    qb = synth.random_quaternions(42, R).astype(np.float32)

    def fresh(q):
        fs = ctx.fieldset(n, R, flags)
        fs.compute(p1, p2, q, allow_rank_deficient=True)
        return fields(fs, R)

    reused = ctx.fieldset(n, R, flags)
    q = qa.copy()
    reused.compute(p1, p2, q, allow_rank_deficient=True)
    assert np.array_equal(fields(reused, R), fresh(qa), equal_nan=True)
    reused.compute(p1, p2, qb, allow_rank_deficient=True)
    assert np.array_equal(fields(reused, R), fresh(qb), equal_nan=True)
    reused.compute(p1, p2, q, allow_rank_deficient=True)  # back to the first set
    assert np.array_equal(fields(reused, R), fresh(qa), equal_nan=True)
    q[7] = synth.random_quaternions(43, 1)[0]  # one rotation changed in place
    reused.compute(p1, p2, q, allow_rank_deficient=True)
    assert np.array_equal(fields(reused, R), fresh(q), equal_nan=True)
