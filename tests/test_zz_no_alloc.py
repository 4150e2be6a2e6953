"""hf_fields_noalloc: the energy/force entry point for callers that may not
allocate device memory while they run (a 1 kHz haptic loop that cannot
afford a cudaMalloc stall, a plug-in whose host application owns all device
memory).  It must give what the allocating entry point hf_fields gives, and
keep doing so on back-to-back calls that share its static scratch.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # max |noalloc - hf_fields| <= TOL * max |hf_fields|, per field


def test_noalloc_matches_hf_fields_on_consecutive_calls():
    import torch
    import paper_1711_05017_b300 as hf
    from paper_1711_05017_b300 import _binding as B
    from paper_1711_05017_b300 import build

    build.build()
    L = B.lib()
    ctx = hf.Context(0)
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
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
        rc = L.hf_fields_noalloc(n, ctypes.c_void_p(g1.data_ptr()), ctypes.c_void_p(g2.data_ptr()), B.fptr(q),
                                 *[ctypes.c_void_p(t.data_ptr()) for t in got], sp)
        assert rc == B.HF_OK, L.hf_last_error()
        torch.cuda.synchronize()
        for f, (a, b) in enumerate(zip(got, ref)):
            b = b.double()
            err = float((a.double() - b).abs().max()) / float(b.abs().max())
            assert err <= TOL, (n, seed, f, err)


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    import torch
    from paper_1711_05017_b300 import _binding as B
    from paper_1711_05017_b300 import build

    build.build()
    L = B.lib()
    x = torch.zeros((128, 128, 128), device="cuda")
    q = np.array([1, 0, 0, 0], dtype=np.float32)
    p = ctypes.c_void_p(x.data_ptr())
    rc = L.hf_fields_noalloc(128, p, p, B.fptr(q), p, p, p, p, None)
    assert rc == B.HF_EINVAL
    assert b"maximum N=64" in L.hf_last_error()
