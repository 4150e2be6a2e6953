"""Mesh descriptor (Eq. 2 on closed triangle meshes) on the GPU against the
FP64 oracle, node by node, and fed through the field pipeline.  Outputs are
float32: max |gpu - oracle| <= 1e-6 * max |oracle| per output."""
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


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def meshes():
    n = 16
    h = 2.0 / n
    hole, peg = synth.peg_hole_pair(24)
    return [("box", synth.box(np.full(3, -0.3 + h / 4), np.full(3, 0.3 + h / 4))), ("peg", peg), ("hole", hole)]


@pytest.mark.parametrize("n", [16, 32])
@pytest.mark.parametrize("which", [0, 1, 2])
def test_mesh_descriptor_matches_the_oracle(hf, n, which):
    import torch
    name, (V, T) = meshes()[which]
    ctx = hf.Context(0)
    sigma, gmax, dmax = 0.5, 0.02, 10
    aux = torch.empty((2, n, n, n), dtype=torch.float32, device="cuda")
    rho = ctx.density_mesh(n, V, T, sigma, gmax, dmax, aux=aux)
    W, XI, RHO = oracle.mesh_sdf(n, V, T, sigma, gmax, dmax)
    got_rho, got_aux = host(rho), host(aux)
    assert np.abs(got_rho - RHO).max() <= 1e-6 * np.abs(RHO).max(), name
    assert np.abs(got_aux[0] - W).max() <= 1e-6, name
    assert np.abs(got_aux[1] - XI).max() <= 1e-6 * np.abs(XI).max(), name


def test_mesh_descriptors_through_the_field_pipeline(hf):
    """Peg and holed block as mesh descriptors at 64^3.  The GPU descriptors
    equal the oracle's (float32-rounded) within 1e-6; the field set built
    from those same float32 grids equals the oracle's fields of them within
    the float32 bar, 1e-5 per field."""
    import torch
    n, R = 64, 2
    hole, peg = synth.peg_hole_pair(24)
    ctx = hf.Context(0)
    g1 = ctx.density_mesh(n, *hole, 0.5, 0.05, 8)
    g2 = ctx.density_mesh(n, *peg, 0.5, 0.05, 8)
    r1 = oracle.mesh_sdf(n, *hole, 0.5, 0.05, 8)[2].astype(np.float32)
    r2 = oracle.mesh_sdf(n, *peg, 0.5, 0.05, 8)[2].astype(np.float32)
    assert np.abs(host(g1) - r1).max() <= 1e-6 * np.abs(r1).max()
    assert np.abs(host(g2) - r2).max() <= 1e-6 * np.abs(r2).max()
    # both sides start from the identical float32 grids
    p1 = ctx.part(torch.as_tensor(r1).cuda(), hf.HF_STATIONARY)
    p2 = ctx.part(torch.as_tensor(r2).cuda(), hf.HF_MOVING)
    q = synth.random_quaternions(31, R).astype(np.float32)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F)
    fs.compute(p1, p2, q)
    for r in range(R):
        qq = q[r].astype(np.float64)
        Rm = oracle.quat_to_rot(qq / np.linalg.norm(qq)).astype(np.float32).astype(np.float64)
        ref = oracle.fields(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), Rm))
        for f in range(4):
            got = host(fs.get(r, f))
            assert np.abs(got - ref[f]).max() <= 1e-5 * np.abs(ref[f]).max(), (r, f)


def test_mesh_errors(hf):
    import torch
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    V, T = synth.box(np.full(3, -0.3), np.full(3, 0.3))
    bad = T.copy()
    bad[3, 1] = len(V)
    with pytest.raises(hf.HFError) as e:
        ctx.density_mesh(16, V, bad)
    assert e.value.status == B.HF_EINVAL
    with pytest.raises(hf.HFError) as e:
        ctx.density_mesh(16, V, T, max_depth=13)
    assert e.value.status == B.HF_EINVAL
    torch.cuda.synchronize()
