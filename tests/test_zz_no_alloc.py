"""hf_fields_noalloc: the energy/force entry point for callers that may not
allocate device memory while they run (a 1 kHz haptic loop that cannot
afford a cudaMalloc stall, a plug-in whose host application owns all device
memory).  It must give what the allocating entry point hf_fields gives, and
what the FP64 oracle gives, and keep doing so on back-to-back calls that
share its static scratch; after its first (set-up) call on a device, calls
must not change the device's free memory.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # max |noalloc - reference| <= TOL * max |reference|, per field


def _setup():
    import torch
    import paper_1711_05017_b300 as hf
    from paper_1711_05017_b300 import _binding as B
    from paper_1711_05017_b300 import build

    build.build()
    stream = torch.cuda.current_stream()
    return torch, hf, B, B.lib(), ctypes.c_void_p(stream.cuda_stream)


def _call(L, B, n, g1, g2, q, outs, sp):
    return L.hf_fields_noalloc(n, ctypes.c_void_p(g1.data_ptr()), ctypes.c_void_p(g2.data_ptr()), B.fptr(q),
                               *[ctypes.c_void_p(t.data_ptr()) for t in outs], sp)


def test_noalloc_matches_hf_fields_on_consecutive_calls():
    torch, hf, B, L, sp = _setup()
    ctx = hf.Context(0)
    for n, seed in ((64, 0), (64, 1), (32, 2)):  # back-to-back calls, sizes mixed
        s1, s2 = synth.c1_pair(seed)
        g1 = ctx.density_build(n, torch.as_tensor(s1.pts, dtype=torch.float32).cuda(),
                               torch.as_tensor(s1.sigma, dtype=torch.float32).cuda())
        g2 = ctx.density_build(n, torch.as_tensor(s2.pts, dtype=torch.float32).cuda(),
                               torch.as_tensor(s2.sigma, dtype=torch.float32).cuda())
        q = synth.random_quaternions(50 + seed, 1)[0].astype(np.float32)
        ref = [torch.empty((n, n, n), device="cuda") for _ in range(4)]
        ctx.fields(ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING), q, *ref)
        got = [torch.full((n, n, n), float("nan"), device="cuda") for _ in range(4)]
        rc = _call(L, B, n, g1, g2, q, got, sp)
        assert rc == B.HF_OK, L.hf_last_error()
        torch.cuda.synchronize()
        for f, (a, b) in enumerate(zip(got, ref)):
            b = b.double()
            err = float((a.double() - b).abs().max()) / float(b.abs().max())
            assert err <= TOL, (n, seed, f, err)


@pytest.mark.parametrize("n", [32, 64])
def test_noalloc_matches_the_oracle(n):
    """Oracle-splatted float32 grids of the c1 pair, one random rotation: the
    four fields against the oracle's resample + fields, twice in a row."""
    torch, hf, B, L, sp = _setup()
    s1, s2 = synth.c1_pair(5)
    r1 = oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)
    g1, g2 = torch.as_tensor(r1).cuda(), torch.as_tensor(r2).cuda()
    for seed in (60, 61):
        q = synth.random_quaternions(seed, 1)[0].astype(np.float32)
        qq = q.astype(np.float64) / np.linalg.norm(q.astype(np.float64))
        Rm = oracle.quat_to_rot(qq).astype(np.float32).astype(np.float64)
        ref = oracle.fields(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), Rm))
        got = [torch.full((n, n, n), float("nan"), device="cuda") for _ in range(4)]
        assert _call(L, B, n, g1, g2, q, got, sp) == B.HF_OK, L.hf_last_error()
        torch.cuda.synchronize()
        for f in range(4):
            a = got[f].cpu().numpy().astype(np.float64)
            assert np.abs(a - ref[f]).max() <= TOL * np.abs(ref[f]).max(), (n, seed, f)


def test_noalloc_calls_after_the_first_leave_free_memory_unchanged():
    """After a warm-up call (the per-device set-up), further calls change the
    device's free memory by nothing: no allocation, by the library or by a
    lazily loaded module."""
    torch, hf, B, L, sp = _setup()
    n = 64
    s1, s2 = synth.c1_pair(3)
    g1 = torch.as_tensor(oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)).cuda()
    g2 = torch.as_tensor(oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)).cuda()
    outs = [torch.empty((n, n, n), device="cuda") for _ in range(4)]
    q = synth.random_quaternions(70, 3).astype(np.float32)
    assert _call(L, B, n, g1, g2, q[0], outs, sp) == B.HF_OK, L.hf_last_error()  # set-up call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for i in (1, 2):
        assert _call(L, B, n, g1, g2, q[i], outs, sp) == B.HF_OK, L.hf_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    torch, hf, B, L, sp = _setup()
    x = torch.zeros((128, 128, 128), device="cuda")
    q = np.array([1, 0, 0, 0], dtype=np.float32)
    p = ctypes.c_void_p(x.data_ptr())
    rc = L.hf_fields_noalloc(128, p, p, B.fptr(q), p, p, p, p, None)
    assert rc == B.HF_EINVAL
    assert b"maximum N=64" in L.hf_last_error()
