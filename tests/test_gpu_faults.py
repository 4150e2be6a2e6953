"""Host-side fault injection: every allocation an operation makes is failed
in turn (hf_inject_alloc_failure).  Each failure must come back as an error
status, leave the context's reserved bytes where they were, and leave the
device usable: the same operation run again right after gives bitwise the
result of a run that never failed.  No GPU fault is involved: the failing
call is a fake of the allocator's out-of-memory answer."""
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


def cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def env(hf):
    ctx = hf.Context(0)
    grids = {}
    for n in (32, 64):
        s1, s2 = synth.c2_pair(n) if n >= 64 else synth.c1_pair(n)
        grids[n] = tuple(ctx.density_build(n, cuda(s.pts[:1200]), cuda(s.sigma[:1200])) for s in (s1, s2))
    parts = {n: (ctx.part(g[0], hf.HF_STATIONARY), ctx.part(g[1], hf.HF_MOVING)) for n, g in grids.items()}
    return ctx, grids, parts


class Made:
    """Handles an operation creates, released on every exit path."""

    def __init__(self):
        self.items = []

    def __call__(self, h):
        self.items.append(h)
        return h

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        for h in reversed(self.items):
            h.release()
        self.items.clear()
        return False


def op_moving_part(hf, env):
    ctx, grids, parts = env
    with Made() as made:
        p2 = made(ctx.part(grids[64][1], hf.HF_MOVING))
        E = cuda(np.zeros((64,) * 3))
        ctx.fields(parts[64][0], p2, synth.random_quaternions(3, 1)[0], E)
        return host(E)


def op_stationary_part(hf, env):
    ctx, grids, parts = env
    with Made() as made:
        p1 = made(ctx.part(grids[64][0], hf.HF_STATIONARY))
        E = cuda(np.zeros((64,) * 3))
        ctx.fields(p1, parts[64][1], synth.random_quaternions(4, 1)[0], E)
        return host(E)


def op_fieldset(hf, env):
    ctx, grids, parts = env
    with Made() as made:
        fs = made(ctx.fieldset(64, 10, hf.HF_E | hf.HF_F | hf.HF_T))
        fs.compute(*parts[64], synth.random_quaternions(5, 10))
        return np.stack([host(fs.get(r, f)) for r in (0, 9) for f in (0, 1, 4)])


def op_torque(hf, env):
    ctx, grids, parts = env
    q = synth.random_quaternions(6, 8).astype(np.float32)
    with Made() as made:
        fs = made(ctx.fieldset(32, 8, hf.HF_E | hf.HF_F))
        fs.compute(*parts[32], q)
        E = cuda(np.stack([host(fs.get(r, 0)) for r in range(8)]))
    T = cuda(np.zeros((8, 3, 32, 32, 32)))
    ctx.torque(32, q, E, T)
    return host(T)


def op_spectral_lowpass(hf, env):
    ctx, grids, parts = env
    rng = np.random.default_rng(7)
    tq = cuda(np.concatenate([rng.uniform(-0.5, 0.5, (6, 3)), synth.random_quaternions(7, 6)], 1))
    with Made() as made:
        p2 = made(ctx.part(grids[32][1], hf.HF_MOVING))
        p2.spectral(2)
        return host(hf.lowpass_query_batch(parts[32][0], p2, tq, K=6))


def op_moments(hf, env):
    ctx, grids, parts = env
    with Made() as made:
        p1 = made(ctx.part(grids[32][0], hf.HF_STATIONARY))
        p1.moments()
        fs = made(ctx.fieldset(32, 2, hf.HF_E | hf.HF_F | hf.HF_TA))
        fs.compute(p1, parts[32][1], synth.random_quaternions(8, 2))
        return np.stack([host(fs.get(1, f)) for f in (0, 4, 6)])


def op_batch_graph(hf, env):
    ctx, grids, parts = env
    with Made() as made:
        b = made(hf.Batch(ctx, [parts[64], parts[32]], [8, 7], hf.HF_E | hf.HF_F | hf.HF_T))
        b.set_rotations(0, synth.random_quaternions(9, 8))
        b.set_rotations(1, synth.random_quaternions(10, 7))
        b.capture()
        b.launch()
        return np.stack([host(b.fieldset(0).get(7, 5))[:32, :32, :32], host(b.fieldset(1).get(6, 0))])


def op_batch_queue(hf, env):
    ctx, grids, parts = env
    with Made() as made:
        b = made(hf.Batch(ctx, [parts[64], parts[64]], [12, 9], hf.HF_E | hf.HF_F))
        b.set_rotations(0, synth.random_quaternions(11, 12))
        b.set_rotations(1, synth.random_quaternions(12, 9))
        b.capture_queue(chunk=8)
        b.launch()
        b.status()
        return np.stack([host(b.fieldset(0).get(11, 2)), host(b.fieldset(1).get(3, 0))])


def op_checkpoints(hf, env, tmp):
    ctx, grids, parts = env
    with Made() as made:
        p1 = made(hf.Part.load(ctx, tmp / "p1.npy"))
        p2 = made(hf.Part.load(ctx, tmp / "p2.npy"))
        fl = made(hf.FieldSet.load(ctx, tmp / "fs.npy"))
        fs = made(ctx.fieldset(64, 7, hf.HF_E | hf.HF_F))
        fs.compute(p1, p2, synth.random_quaternions(13, 7))
        return np.stack([host(fs.get(6, 1)), host(fl.get(2, 3))])


OPS = {"moving_part": op_moving_part, "stationary_part": op_stationary_part, "fieldset": op_fieldset,
       "torque": op_torque, "spectral_lowpass": op_spectral_lowpass, "moments": op_moments,
       "batch_graph": op_batch_graph, "batch_queue": op_batch_queue, "checkpoints": op_checkpoints}


@pytest.mark.parametrize("name", list(OPS))
def test_each_failed_allocation_is_reported_and_leaves_no_trace(hf, env, name, tmp_path):
    import torch
    from paper_1711_05017_b300 import _binding as B
    ctx, grids, parts = env
    if name == "checkpoints":
        parts[64][0].save(tmp_path / "p1.npy")
        parts[64][1].save(tmp_path / "p2.npy")
        fs = ctx.fieldset(64, 7, hf.HF_E | hf.HF_F)
        fs.compute(*parts[64], synth.random_quaternions(14, 7))
        fs.save(tmp_path / "fs.npy")
        fs.release()
        op = lambda: op_checkpoints(hf, env, tmp_path)  # noqa: E731
    else:
        op = lambda: OPS[name](hf, env)  # noqa: E731
    hf.inject_alloc_failure(0)
    ref = op()  # also makes any per-context scratch the operation keeps
    torch.cuda.synchronize()
    base = ctx.reserved_bytes()
    c0 = hf.inject_alloc_failure(0)
    assert np.array_equal(op(), ref)
    count = hf.inject_alloc_failure(0) - c0
    assert count >= 1
    for k in range(1, count + 1):
        hf.inject_alloc_failure(k)
        try:
            with pytest.raises(hf.HFError) as e:
                op()
        finally:
            hf.inject_alloc_failure(0)
        assert e.value.status in (B.HF_ENOMEM, B.HF_ECUDA), (k, str(e.value))
        del e
        torch.cuda.synchronize()
        assert ctx.reserved_bytes() == base, (k, ctx.reserved_bytes(), base)
        assert np.array_equal(op(), ref), k


def test_bulk_copy_wait_is_bounded_and_reported(hf, env):
    """The bounded wait of the bulk-staged kernels, in one block: a wait
    that cannot complete (the mbarrier expects more bytes than the copy
    brings) gives up after its bound, counts itself and returns; the device
    stays usable and the next build is exact."""
    import ctypes
    from paper_1711_05017_b300 import _binding as B
    L = B.lib()
    t = ctypes.c_int(-1)
    assert L.hf_bulk_selftest(0, 0, ctypes.byref(t)) == B.HF_OK and t.value == 0
    ref = op_fieldset(hf, env)
    assert L.hf_bulk_selftest(0, 1, ctypes.byref(t)) == B.HF_ETIMEOUT and t.value == 1
    assert L.hf_bulk_timeouts(1) >= 1
    assert L.hf_bulk_timeouts(0) == 0
    assert np.array_equal(op_fieldset(hf, env), ref)
    assert L.hf_bulk_timeouts(0) == 0
