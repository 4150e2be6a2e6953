"""The moving part's support (per axis, the circular range of slabs that hold
a nonzero node): the rotated resample reads no texels for samples in cells
outside it.  Those cells' corners are all zero, so every field of a field set
must be the same, bit for bit, as that of a part built without a support
(HF_SUPPORT=0), for supports in the middle of the grid, across the period,
a single node, the whole torus and an empty grid, on both pipelines."""
import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def ctx(hf):
    return hf.Context(0)


def cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def fields(hf, ctx, n, g1, g2, q, monkeypatch, support):
    import torch
    if support:
        monkeypatch.delenv("HF_SUPPORT", raising=False)
    else:
        monkeypatch.setenv("HF_SUPPORT", "0")
    p1, p2 = ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)
    monkeypatch.delenv("HF_SUPPORT", raising=False)
    fs = ctx.fieldset(n, len(q), hf.HF_E | hf.HF_F)
    fs.compute(p1, p2, q)
    torch.cuda.synchronize()
    return np.stack([fs.get(r, f).cpu().numpy() for r in range(len(q)) for f in range(4)])


def moving_grid(hf, ctx, n, kind):
    """Moving densities whose supports take every shape the box handles."""
    import torch
    rng = np.random.default_rng(n)
    if kind == "centred":  # the peg, inside the grid
        s = synth.c2_pair(0)[1]
        return ctx.density_build(n, cuda(s.pts[:1500]), cuda(s.sigma[:1500]))
    if kind == "wrapping":  # a cluster across the corner of the period on all three axes
        pts = np.array([0.96, -0.97, 0.93]) + rng.normal(0, 0.03, (200, 3))
        pts = (pts + 1.0) % 2.0 - 1.0
        return ctx.density_build(n, cuda(pts), cuda(rng.uniform(0.02, 0.05, 200)))
    if kind == "node":  # one nonzero node
        g = torch.zeros((n, n, n), device="cuda")
        g[n // 3, 0, n - 1] = 1.0
        return g
    if kind == "full":  # no zero anywhere
        return cuda(rng.uniform(0.5, 1.5, (n, n, n)))
    assert kind == "empty"
    return torch.zeros((n, n, n), device="cuda")


@pytest.mark.parametrize("n,kind", [(64, "centred"), (64, "wrapping"), (64, "node"), (64, "full"),
                                    (64, "empty"), (96, "wrapping"), (128, "centred"), (256, "wrapping")])
def test_support_skip_is_exact(hf, ctx, n, kind, monkeypatch):
    s = synth.c2_pair(0)[0]
    g1 = ctx.density_build(n, cuda(s.pts[:1500]), cuda(s.sigma[:1500]))
    g2 = moving_grid(hf, ctx, n, kind)
    q = synth.random_quaternions(500 + n, 2 if n == 256 else 5).astype(np.float32)
    with_box = fields(hf, ctx, n, g1, g2, q, monkeypatch, True)
    without = fields(hf, ctx, n, g1, g2, q, monkeypatch, False)
    assert np.array_equal(with_box, without)
    if kind == "empty":
        assert not with_box.any()


def test_update_refreshes_the_support(hf, ctx, monkeypatch):
    """A part made from a centred grid and updated to one across the period
    skips by the new grid's support."""
    import torch
    n = 64
    s = synth.c2_pair(0)[0]
    g1 = ctx.density_build(n, cuda(s.pts[:1500]), cuda(s.sigma[:1500]))
    q = synth.random_quaternions(600, 4).astype(np.float32)
    p1 = ctx.part(g1, hf.HF_STATIONARY)
    p2 = ctx.part(moving_grid(hf, ctx, n, "centred"), hf.HF_MOVING)
    g2 = moving_grid(hf, ctx, n, "wrapping")
    p2.update(g2)
    fs = ctx.fieldset(n, len(q), hf.HF_E | hf.HF_F)
    fs.compute(p1, p2, q)
    torch.cuda.synchronize()
    got = np.stack([fs.get(r, f).cpu().numpy() for r in range(len(q)) for f in range(4)])
    assert np.array_equal(got, fields(hf, ctx, n, g1, g2, q, monkeypatch, False))
