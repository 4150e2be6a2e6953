"""Analytic torque fields (HF_TA; the rotational gradient of Eq. 6b with the
moment on the stationary part) through the C ABI against the FP64 oracle.
Bar: max |gpu - oracle| <= 1e-5 * max |oracle field|, per component."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rot32(q):
    q = np.asarray(q, dtype=np.float32).astype(np.float64)
    return oracle.quat_to_rot(q / np.linalg.norm(q)).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("n,R", [(32, 4), (64, 2), (96, 1), (128, 1)])
def test_analytic_torque_matches_the_oracle(hf, n, R):
    ctx = hf.Context(0)
    s1, s2 = synth.c1_pair(5) if n == 32 else synth.c2_pair(5)
    k = min(len(s1.pts), 500)
    r1 = oracle.splat(n, s1.pts[:k], s1.sigma[:k]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[:k], s2.sigma[:k]).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    p1.moments()
    q = synth.random_quaternions(60 + n, R).astype(np.float32)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_TA)
    fs.compute(p1, p2, q)
    plain = ctx.fieldset(n, R, hf.HF_E | hf.HF_F)
    plain.compute(p1, p2, q)
    for r in range(R):
        r2r = oracle.resample(r2.astype(np.float64), rot32(q[r]))
        ref = oracle.torque_analytic(r1.astype(np.float64), r2r)
        for a in range(3):
            got = host(fs.get(r, 4 + a))
            assert np.abs(got - ref[a]).max() <= TOL * np.abs(ref[a]).max(), (r, a)
        for f in range(4):  # E and F are those of the plain set
            assert np.array_equal(host(fs.get(r, f)), host(plain.get(r, f))), (r, f)


def test_analytic_torque_flags_and_readiness(hf):
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    with pytest.raises(hf.HFError) as e:
        ctx.fieldset(32, 8, hf.HF_E | hf.HF_T | hf.HF_TA)
    assert e.value.status == B.HF_EINVAL
    with pytest.raises(hf.HFError) as e:
        ctx.fieldset(256, 2, hf.HF_E | hf.HF_TA)
    assert e.value.status == B.HF_EUNSUPPORTED
    s1, s2 = synth.c1_pair(6)
    n = 32
    r1 = oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    fs = ctx.fieldset(n, 2, hf.HF_E | hf.HF_TA)
    with pytest.raises(hf.HFError) as e:
        fs.compute(p1, p2, synth.random_quaternions(1, 2))
    assert e.value.status == B.HF_ENOTREADY
    with pytest.raises(hf.HFError) as e:
        p2.moments()
    assert e.value.status == B.HF_EINVAL
