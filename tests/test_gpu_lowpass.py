"""Single poses from truncated spectra (Section 4.2, "Truncated Inverse FFT"):
the CUDA path against the FP64 oracle, pose by pose.  Bar: per output
component, max |gpu - oracle| over the poses <= 1e-5 * max |oracle| over the
poses."""
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


def rot32(q):
    q = np.asarray(q, dtype=np.float32).astype(np.float64)
    return oracle.quat_to_rot(q / np.linalg.norm(q)).astype(np.float32).astype(np.float64)


def setup(hf, n, os_, seed):
    ctx = hf.Context(0)
    s1, s2 = synth.c1_pair(seed) if n == 32 else synth.c2_pair(seed)
    k = min(len(s1.pts), 800)
    r1 = oracle.splat(n, s1.pts[:k], s1.sigma[:k]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[:k], s2.sigma[:k]).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    p2.spectral(os_)
    table = oracle.spectral_table(r2.astype(np.float64), os_)
    return ctx, p1, p2, r1, table


@pytest.mark.parametrize("n,os_,K", [(32, 1, 4), (32, 2, 8), (64, 2, 8), (64, 1, 12)])
def test_single_and_batched_poses_match_the_oracle(hf, n, os_, K):
    import torch
    ctx, p1, p2, r1, table = setup(hf, n, os_, 2)
    P = 12
    rng = np.random.default_rng(n + K)
    t = rng.uniform(-0.6, 0.6, (P, 3)).astype(np.float32)
    q = synth.random_quaternions(100 + K, P).astype(np.float32)
    ref = np.stack([oracle.lowpass(r1.astype(np.float64), table, os_, K, rot32(q[i]), t[i].astype(np.float64))
                    for i in range(P)])
    one = np.stack([hf.lowpass_query(p1, p2, t[i], q[i], K=K) for i in range(P)])
    bat = hf.lowpass_query_batch(p1, p2, cuda(np.concatenate([t, q], 1)), K=K)
    torch.cuda.synchronize()
    bat = bat.cpu().numpy()
    for c in range(7):
        scale = np.abs(ref[:, c]).max()
        assert np.abs(one[:, c] - ref[:, c]).max() <= TOL * scale, c
        assert np.abs(bat[:, c] - ref[:, c]).max() <= TOL * scale, c


def test_all_modes_at_a_lattice_point_equal_the_spectral_field(hf):
    """With every non-Nyquist mode kept, a lattice translation reads the
    HF_SPECTRAL field set's value there."""
    n, os_ = 32, 2
    ctx, p1, p2, r1, table = setup(hf, n, os_, 3)
    q = synth.random_quaternions(7, 1).astype(np.float32)
    fs = ctx.fieldset(n, 1, hf.HF_E | hf.HF_F | hf.HF_SPECTRAL)
    fs.compute(p1, p2, q)
    h = 2.0 / n
    E = [fs.get(0, f).cpu().numpy() for f in range(4)]
    for j in [(0, 0, 0), (5, 17, 30)]:
        out = hf.lowpass_query(p1, p2, np.array(j, dtype=np.float32) * h, q[0], K=n // 2 - 1)
        for f in range(4):
            assert abs(out[f] - E[f][j[2], j[1], j[0]]) <= 2e-5 * np.abs(E[f]).max(), (j, f)


def test_lowpass_errors(hf):
    from paper_1711_05017_b300 import _binding as B
    n = 32
    ctx = hf.Context(0)
    s1, s2 = synth.c1_pair(4)
    r1 = oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    q = np.array([1, 0, 0, 0], dtype=np.float32)
    with pytest.raises(hf.HFError) as e:
        hf.lowpass_query(p1, p2, [0, 0, 0], q, K=4)
    assert e.value.status == B.HF_ENOTREADY
    p2.spectral(1)
    for K in (0, 16):
        with pytest.raises(hf.HFError) as e:
            hf.lowpass_query(p1, p2, [0, 0, 0], q, K=K)
        assert e.value.status == B.HF_EINVAL
    with pytest.raises(hf.HFError) as e:
        hf.lowpass_query(p1, p2, [0, 0, 0], np.zeros(4, dtype=np.float32), K=4)
    assert e.value.status == B.HF_EINVAL
