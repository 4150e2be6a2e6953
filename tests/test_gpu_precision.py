"""Precision variant at 256^3: the y-axis DFT stages on the tensor cores as
split hi/lo BF16 / FP16 DFT-matrix GEMMs with FP32 accumulation.

Bars: the plain FP32 path within 1e-5 of the FP64 oracle (max-abs error over
max |field|), the split variants within 2e-3 (the reduced-precision
tolerance); both split variants are also held against the FP32 path on
several rotations, and no tensor-core wait may have timed out."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

N = 256
TOL32, TOLSPLIT = 1e-5, 2e-3


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


def rel(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.fixture(scope="module")
def case(hf):
    """A 256^3 pair splatted by the oracle (a 400-point subset of the
    20000-point parts, same radius law), and its fields for 3 rotations in
    FP32 and both split variants."""
    ctx = hf.Context(0)
    s1, s2 = synth.c4_pair(0)
    sel = np.random.default_rng(3).choice(len(s1.pts), 400, replace=False)
    r1 = oracle.splat(N, s1.pts[sel], s1.sigma[sel]).astype(np.float32)
    r2 = oracle.splat(N, s2.pts[sel], s2.sigma[sel]).astype(np.float32)
    p = (ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING))
    q = synth.random_quaternions(0, 3).astype(np.float32)
    from paper_1711_05017_b300 import _binding as B
    B.lib().hf_tc_timeouts(1)
    out = {}
    for name, fl in (("fp32", 0), ("bf16", hf.HF_PREC_SPLIT_BF16), ("f16", hf.HF_PREC_SPLIT_F16)):
        fs = ctx.fieldset(N, 3, hf.HF_E | hf.HF_F | fl)
        fs.compute(p[0], p[1], q)
        out[name] = np.stack([np.stack([host(fs.get(r, f)) for f in range(4)]) for r in range(3)])
        fs.release()
    assert B.lib().hf_tc_timeouts(0) == 0
    return dict(r=(r1, r2), q=q, out=out)


def test_split_variants_track_the_fp32_path(case):
    ref = case["out"]["fp32"]
    for name in ("bf16", "f16"):
        for f in range(4):
            e = rel(case["out"][name][:, f], ref[:, f])
            assert e <= TOLSPLIT, (name, f, e)
    # FP16 hi + lo carries 22 significant bits against BF16's 16
    for f in range(4):
        assert rel(case["out"]["f16"][:, f], ref[:, f]) <= rel(case["out"]["bf16"][:, f], ref[:, f]) + 1e-7


def test_fields_against_the_oracle_at_256(case):
    r1, r2 = case["r"]
    q = case["q"][0].astype(np.float64)
    q /= np.linalg.norm(q)
    R = oracle.quat_to_rot(q).astype(np.float32).astype(np.float64)
    ref = np.stack(oracle.fields(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), R)))
    for f in range(4):
        assert rel(case["out"]["fp32"][0, f], ref[f]) <= TOL32, f
        for name in ("bf16", "f16"):
            assert rel(case["out"][name][0, f], ref[f]) <= TOLSPLIT, (name, f)


def test_precision_flag_errors(hf):
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    with pytest.raises(hf.HFError) as e:
        ctx.fieldset(128, 4, hf.HF_E | hf.HF_PREC_SPLIT_BF16)
    assert e.value.status == B.HF_EUNSUPPORTED
    with pytest.raises(hf.HFError) as e:
        ctx.fieldset(N, 4, hf.HF_E | hf.HF_PREC_SPLIT_BF16 | hf.HF_PREC_SPLIT_F16)
    assert e.value.status == B.HF_EINVAL
