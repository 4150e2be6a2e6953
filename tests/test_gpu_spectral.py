"""Spectral mode (rotation in the frequency domain, Section 3.2 step 1): the
CUDA path against the FP64 oracle's spectral route, element by element.
Bar: max |gpu - oracle| <= 1e-5 * max |oracle field|, per field."""
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


def grids(n, seed, npts=None):
    s1, s2 = synth.c1_pair(seed) if n == 32 else synth.c2_pair(seed)
    k = npts or len(s1.pts)
    r1 = oracle.splat(n, s1.pts[:k], s1.sigma[:k]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[:k], s2.sigma[:k]).astype(np.float32)
    return r1, r2


def oracle_fields(r1, r2, q, os_):
    n = r1.shape[0]
    table = oracle.spectral_table(r2.astype(np.float64), os_)
    return np.stack(oracle.fields_spec(r1.astype(np.float64), oracle.spectral_rotate(table, n, rot32(q), os_)))


@pytest.mark.parametrize("n,os_,R", [(32, 1, 5), (32, 2, 5), (64, 1, 3), (64, 2, 3), (96, 1, 2)])
def test_spectral_fields_match_the_oracle(hf, n, os_, R):
    ctx = hf.Context(0)
    r1, r2 = grids(n, 1, npts=600 if n > 32 else None)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    p2.spectral(os_)
    q = synth.random_quaternions(40 + n + os_, R).astype(np.float32)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_SPECTRAL)
    fs.compute(p1, p2, q)
    for r in range(R):
        ref = oracle_fields(r1, r2, q[r], os_)
        for f in range(4):
            got = host(fs.get(r, f))
            assert np.abs(got - ref[f]).max() <= TOL * np.abs(ref[f]).max(), (r, f)


def test_spectral_128_padded_table_built_by_the_pencil_transform(hf):
    """os = 2 at 128^3 builds the table with the 256^3 pencil transform."""
    n, os_ = 128, 2
    ctx = hf.Context(0)
    r1, r2 = grids(n, 2, npts=300)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    p2.spectral(os_)
    q = synth.random_quaternions(77, 2).astype(np.float32)
    fs = ctx.fieldset(n, 2, hf.HF_E | hf.HF_F | hf.HF_SPECTRAL)
    fs.compute(p1, p2, q)
    ref = oracle_fields(r1, r2, q[1], os_)
    for f in range(4):
        got = host(fs.get(1, f))
        assert np.abs(got - ref[f]).max() <= TOL * np.abs(ref[f]).max(), f


def test_part_update_refreshes_the_table_and_errors(hf):
    from paper_1711_05017_b300 import _binding as B
    n = 32
    ctx = hf.Context(0)
    r1, r2 = grids(n, 3)
    _, r2b = grids(n, 4)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    q = synth.random_quaternions(9, 3).astype(np.float32)
    fs = ctx.fieldset(n, 3, hf.HF_E | hf.HF_F | hf.HF_SPECTRAL)
    with pytest.raises(hf.HFError) as e:  # no table yet
        fs.compute(p1, p2, q)
    assert e.value.status == B.HF_ENOTREADY
    with pytest.raises(hf.HFError) as e:
        p1.spectral(1)  # stationary parts keep their spectrum already
    assert e.value.status == B.HF_EINVAL
    p2.spectral(2)
    assert B.lib().hf_part_spectral_os(p2.handle) == 2
    p2.update(cuda(r2b))
    fs.compute(p1, p2, q)
    ref = oracle_fields(r1, r2b, q[2], 2)
    for f in range(4):
        got = host(fs.get(2, f))
        assert np.abs(got - ref[f]).max() <= TOL * np.abs(ref[f]).max(), f
