"""Object lifetimes across the C ABI: parts, field sets, batches and servers
hold a reference to their context, so the context's handle can be dropped
first (as a garbage collector finalising a reference cycle may do) and the
objects still work and release cleanly, leaving no stale CUDA error for the
next call."""
import gc

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import paper_1711_05017_b300 as hf_
    from paper_1711_05017_b300 import build
    build.build()
    return hf_


def _parts(hf, ctx, n=64, seed=3):
    import torch
    s1, s2 = synth.c2_pair(seed)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a[:800], dtype=np.float32)).cuda()  # noqa: E731
    return (ctx.part(ctx.density_build(n, cu(s1.pts), cu(s1.sigma)), hf.HF_STATIONARY),
            ctx.part(ctx.density_build(n, cu(s2.pts), cu(s2.sigma)), hf.HF_MOVING))


def test_context_handle_dropped_before_its_objects(hf):
    ctx = hf.Context(0)
    p1, p2 = _parts(hf, ctx)
    q = synth.random_quaternions(5, 8).astype(np.float32)
    fs = ctx.fieldset(64, 8, hf.HF_E | hf.HF_F)
    fs.compute(p1, p2, q)
    ref = fs.get(3, 0).cpu().numpy()
    srv = hf.Server(ctx, max_inflight=1, query_lanes=1)
    ctx.close()  # the caller's handle goes first
    assert np.array_equal(fs.get(3, 0).cpu().numpy(), ref)  # the objects keep working
    assert np.isfinite(fs.query([0.1, 0.0, -0.2], q[3])).all()
    sid = srv.open(p1, p2)
    rid = srv.submit(sid, q, hf.HF_E | hf.HF_F)
    assert srv.wait([rid])[rid][0] == "done"
    srv.close()
    fs.release()
    p1.release()
    p2.release()  # the last reference: the context goes now
    # a cycle holding a context and its objects, collected by the GC
    ctx2 = hf.Context(0)
    box = {"ctx": ctx2, "parts": _parts(hf, ctx2, seed=4)}
    box["self"] = box
    del ctx2, box
    gc.collect()
    # the next calls see no stale error
    ctx3 = hf.Context(0)
    a, b = _parts(hf, ctx3, seed=5)
    fs3 = ctx3.fieldset(64, 8, hf.HF_E | hf.HF_F)
    fs3.compute(a, b, q)
    assert np.isfinite(fs3.get(0, 0).cpu().numpy()).all()
