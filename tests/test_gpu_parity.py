"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element
by element, on seeded synthetic inputs.  Tolerance (the float32 bar):
max |gpu - oracle| <= 1e-5 * max |oracle field|, per field."""
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


@pytest.fixture(scope="module")
def ctx(hf):
    return hf.Context(0)


def cuda(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rel_err(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def norm_quats(q32):
    q = np.asarray(q32, dtype=np.float32).astype(np.float64).reshape(-1, 4)
    return q / np.linalg.norm(q, axis=1, keepdims=True)


# ------------------------------------------------------------------ splat

@pytest.mark.parametrize("n,which", [(32, "c1"), (64, "c2"), (96, "c2")])
def test_splat_parity(ctx, n, which):
    s1, s2 = synth.c1_pair(0) if which == "c1" else synth.c2_pair(0)
    for part in (s1, s2):
        pts32 = part.pts.astype(np.float32)
        sig32 = part.sigma.astype(np.float32)
        got = host(ctx.density_build(n, cuda(pts32), cuda(sig32)))
        ref = oracle.splat(n, pts32.astype(np.float64), sig32.astype(np.float64))
        assert rel_err(got, ref) <= TOL


@pytest.mark.parametrize("n", [64, 128])
def test_splat_wide_and_narrow_cutoffs(ctx, n):
    """Radii up to 0.17 put some cutoff spheres (6 sigma) within a tile's
    half-width of half the period, where the nearest image to a tile's
    centre is not the minimum image of every node: those chunks take the
    per-node minimum image, the rest the direct offsets."""
    rng = np.random.default_rng(11)
    pts = rng.uniform(-1, 1, (1500, 3)).astype(np.float32)
    # the first 20 points wide: the first chunk of 512 takes the minimum
    # image, later chunks of the same tile the direct offsets
    sig = np.where(np.arange(1500) < 20, rng.uniform(0.15, 0.17, 1500),
                   rng.uniform(0.01, 0.05, 1500)).astype(np.float32)
    got = host(ctx.density_build(n, cuda(pts), cuda(sig)))
    ref = oracle.splat(n, pts.astype(np.float64), sig.astype(np.float64))
    assert rel_err(got, ref) <= TOL


def test_splat_signed_amplitudes_and_empty(ctx):
    import torch
    rng = np.random.default_rng(4)
    pts = rng.uniform(-1, 1, (300, 3)).astype(np.float32)
    sig = rng.uniform(0.03, 0.12, 300).astype(np.float32)
    amp = rng.uniform(-2, 2, 300).astype(np.float32)
    got = host(ctx.density_build(64, cuda(pts), cuda(sig), cuda(amp)))
    ref = oracle.splat(64, pts.astype(np.float64), sig.astype(np.float64), amp.astype(np.float64))
    assert rel_err(got, ref) <= TOL
    out = torch.full((32, 32, 32), 7.0, device="cuda")
    e = torch.empty(0, device="cuda")
    ctx.density_build(32, e.reshape(0, 3), e, out=out)
    assert float(out.abs().max()) == 0.0


# --------------------------------------------------------------- resample

@pytest.mark.parametrize("n", [32, 64, 96, 128])
def test_resample_parity(hf, n):
    rng = np.random.default_rng(n)
    rho = rng.standard_normal((n, n, n)).astype(np.float32)
    d = cuda(rho)
    assert np.array_equal(host(hf.resample(d, np.eye(3))), rho.astype(np.float64))  # identity: exact copy
    for q in synth.random_quaternions(100 + n, 3):
        R = oracle.quat_to_rot(q)
        got = host(hf.resample(d, R))
        ref = oracle.resample(rho.astype(np.float64), R.astype(np.float32).astype(np.float64))
        assert rel_err(got, ref) <= TOL


# -------------------------------------------------------------------- FFT

@pytest.mark.parametrize("n", [32, 64, 96, 128])
def test_rfft3d_parity(hf, n):
    rng = np.random.default_rng(200 + n)
    x = rng.standard_normal((n, n, n)).astype(np.float32)
    got = hf.rfft3d(cuda(x))
    import torch
    torch.cuda.synchronize()
    g = got.cpu().numpy().astype(np.complex128)
    ref = oracle.fft3d(x.astype(np.float64), -1)[:, :, : n // 2 + 1]
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max()


# ----------------------------------------------------------------- fields

def gpu_fields(hf, ctx, rho1, rho2, q):
    import torch
    n = rho1.shape[0]
    s1 = ctx.part(cuda(rho1), hf.HF_STATIONARY)
    s2 = ctx.part(cuda(rho2), hf.HF_MOVING)
    out = [torch.empty((n, n, n), device="cuda") for _ in range(4)]
    ctx.fields(s1, s2, q, *out)
    return [host(o) for o in out]


def test_fields_c1_identity_vs_direct_sum(hf, ctx):
    """32^3 ring/peg workload, identity rotation: E against the direct O(N^6)
    correlation sum, F against the oracle's spectral force."""
    s1, s2 = synth.c1_pair(0)
    r1 = oracle.splat(32, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(32, s2.pts, s2.sigma).astype(np.float32)
    E, Fx, Fy, Fz = gpu_fields(hf, ctx, r1, r2, [1, 0, 0, 0])
    r1d, r2d = r1.astype(np.float64), r2.astype(np.float64)
    assert rel_err(E, oracle.correlate_direct(r1d, r2d)) <= TOL
    ref = oracle.fields(r1d, r2d)
    for g, r in zip((E, Fx, Fy, Fz), ref):
        assert rel_err(g, r) <= TOL


@pytest.mark.parametrize("n", [32, 64, 96, 128])
def test_fields_rotated_parity(hf, ctx, n):
    s1, s2 = synth.c2_pair(0) if n >= 64 else synth.c1_pair(0)
    r1 = oracle.splat(n, s1.pts[:1500], s1.sigma[:1500]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[:1500], s2.sigma[:1500]).astype(np.float32)
    for q in synth.random_quaternions(300 + n, 2 if n < 128 else 1):
        got = gpu_fields(hf, ctx, r1, r2, q)
        qn = norm_quats(q.astype(np.float32))[0]
        R = oracle.quat_to_rot(qn).astype(np.float32).astype(np.float64)
        ref = oracle.fields(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), R))
        for g, r in zip(got, ref):
            assert rel_err(g, r) <= TOL


def test_fields_ragged_odd_size_and_gaussian_closed_form(hf, ctx):
    """96 = 2^5 * 3 (radix-3 stages) with single Gaussians: the GPU energy
    also sits on the continuous closed form within the float32 bar."""
    n = 96
    h = 2.0 / n
    s1, s2 = 3 * h, 3.5 * h
    c1, c2 = np.array([0.11, -0.23, 0.05]), np.array([-0.3, 0.17, 0.2])
    r1 = oracle.splat(n, c1[None], np.array([s1]), cutoff=10.0).astype(np.float32)
    r2 = oracle.splat(n, c2[None], np.array([s2]), cutoff=10.0).astype(np.float32)
    E, *_ = gpu_fields(hf, ctx, r1, r2, [1, 0, 0, 0])
    S = s1**2 + s2**2
    pref = (2 * np.pi * s1**2 * s2**2 / S) ** 1.5
    j = np.arange(n)
    z, y, x = np.meshgrid(j, j, j, indexing="ij")
    t = np.stack([x, y, z], -1) * h
    Ec = np.zeros((n, n, n))
    for m in np.ndindex(3, 3, 3):
        r = c1 - c2 - (t + 2.0 * (np.array(m) - 1))
        Ec += pref * np.exp(-(r**2).sum(-1) / (2 * S))
    assert rel_err(E, Ec) <= TOL


# ------------------------------------------------------ field set, torque, query

@pytest.fixture(scope="module")
def small_set(hf, ctx):
    n, R = 32, 24
    s1, s2 = synth.c1_pair(1)
    r1 = oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)
    q = synth.random_quaternions(77, R).astype(np.float32)
    p1 = ctx.part(cuda(r1), hf.HF_STATIONARY)
    p2 = ctx.part(cuda(r2), hf.HF_MOVING)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
    fs.compute(p1, p2, q)
    qn = norm_quats(q)
    ref = np.stack([np.stack(oracle.fields(r1.astype(np.float64), oracle.resample(
        r2.astype(np.float64), oracle.quat_to_rot(qq).astype(np.float32).astype(np.float64)))) for qq in qn])
    T, st = oracle.torque(qn, ref[:, 0], 6)
    assert (st == 0).all()
    return dict(n=n, R=R, q=q, qn=qn, fs=fs, ref=ref, T=T, p=(p1, p2), r=(r1, r2))


def test_fieldset_energy_force_torque(hf, small_set):
    fs, ref, T = small_set["fs"], small_set["ref"], small_set["T"]
    for f in range(4):
        got = np.stack([host(fs.get(r, f)) for r in range(small_set["R"])])
        assert rel_err(got, ref[:, f]) <= TOL, f
    for d in range(3):
        got = np.stack([host(fs.get(r, 4 + d)) for r in range(small_set["R"])])
        assert rel_err(got, T[:, d]) <= TOL, d


def test_torque_float64_variant(hf, ctx, small_set):
    import torch
    n, R = small_set["n"], small_set["R"]
    fs = small_set["fs"]
    E = torch.stack([fs.get(r, 0) for r in range(R)]).contiguous()
    got = {}
    for flags in (0, hf.HF_TORQUE_F64, hf.HF_TORQUE_C):
        T = torch.empty((R, 3, n, n, n), device="cuda")
        st = ctx.torque(n, small_set["q"], E, T, flags=flags)
        assert (st == 0).all()
        assert rel_err(host(T), small_set["T"]) <= TOL
        got[flags] = host(T).astype(np.float32)
    # the compensated float32 product is as accurate as the float64 one before
    # the final rounding: the same float32 results but where the exact value
    # lies within about 2^-44 of a rounding boundary, and never more than one
    # float32 step apart
    a, b = got[hf.HF_TORQUE_C], got[hf.HF_TORQUE_F64]
    assert np.mean(a == b) >= 0.999
    step = np.spacing(np.maximum(np.abs(a), np.abs(b)).astype(np.float32))
    assert (np.abs(a.astype(np.float64) - b.astype(np.float64)) <= step).all()
    with pytest.raises(hf.HFError):
        ctx.torque(n, small_set["q"], E, torch.empty((R, 3, n, n, n), device="cuda"),
                   flags=hf.HF_TORQUE_F64 | hf.HF_TORQUE_C)
    # the same products through a field set's flags
    p1, p2 = small_set["p"]
    for flags in (hf.HF_TORQUE_F64, hf.HF_TORQUE_C):
        fs2 = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T | flags)
        fs2.compute(p1, p2, small_set["q"])
        T2 = np.stack([np.stack([host(fs2.get(r, 4 + d)) for d in range(3)]) for r in range(R)])
        assert np.array_equal(T2.astype(np.float32), got[flags]), flags
        fs2.release()
    with pytest.raises(hf.HFError):
        ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T | hf.HF_TORQUE_F64 | hf.HF_TORQUE_C)


def test_query_batch_and_single(hf, small_set):
    import torch
    fs, qn, n = small_set["fs"], small_set["qn"], small_set["n"]
    fields7 = np.concatenate([small_set["ref"], np.moveaxis(small_set["T"], 1, 1)], axis=1)
    rng = np.random.default_rng(5)
    Q = 64
    t = rng.uniform(-1.5, 1.5, (Q, 3))
    qs = synth.random_quaternions(91, Q)
    qs[:4] = small_set["q"][:4]  # exact member rotations
    t[4:8] = np.array([[3, 5, 7], [0, 0, 0], [31, 1, 2], [-1, -2, 40]]) * (2.0 / n)  # nodes
    tq = np.concatenate([t, qs], axis=1).astype(np.float32)
    scale = np.abs(fields7).reshape(len(qn), 7, -1).max(axis=(0, 2))
    for k in (1, 4, 6):
        got = host(fs.query_batch(cuda(tq), k=k))
        ref = np.stack([oracle.query(qn, fields7, tq[i, :3].astype(np.float64),
                                     tq[i, 3:].astype(np.float64), k) for i in range(Q)])
        assert (np.abs(got - ref) / scale).max() <= TOL, k
    one = fs.query(tq[10, :3], tq[10, 3:], k=4)
    ref = oracle.query(qn, fields7, tq[10, :3].astype(np.float64), tq[10, 3:].astype(np.float64), 4)
    assert (np.abs(one - ref) / scale).max() <= TOL
    del torch


# ----------------------------------------------------------------- errors

def test_errors_are_status_codes(hf, ctx, small_set):
    import torch
    from paper_1711_05017_b300 import _binding as B
    with pytest.raises(hf.HFError) as e:
        ctx.density_build(48, torch.zeros((1, 3), device="cuda"), torch.ones(1, device="cuda"))
    assert e.value.status == B.HF_EUNSUPPORTED
    with pytest.raises(hf.HFError) as e:
        ctx.fieldset(32, 5, hf.HF_E | hf.HF_F | hf.HF_T)
    assert e.value.status == B.HF_EINVAL
    with pytest.raises(hf.HFError) as e:
        small_set["fs"].query([0, 0, 0], [1, 0, 0, 0], k=9)
    assert e.value.status == B.HF_EINVAL
    fs2 = ctx.fieldset(32, 8)
    with pytest.raises(hf.HFError) as e:
        fs2.query([0, 0, 0], [1, 0, 0, 0])
    assert e.value.status == B.HF_ENOTREADY
    small = hf.Context(0, hbm_budget_bytes=1 << 20)
    with pytest.raises(hf.HFError) as e:
        small.fieldset(64, 4)
    assert e.value.status == B.HF_EBUDGET
    # degenerate inputs: a zero or non-finite quaternion is refused before any
    # launch; an empty query batch is a no-op
    fs = small_set["fs"]
    p1, p2 = small_set["p"]
    bad = small_set["q"].copy()
    bad[3] = 0.0
    with pytest.raises(hf.HFError) as e:
        fs.compute(p1, p2, bad)
    assert e.value.status == B.HF_EINVAL
    bad[3] = [np.nan, 0, 0, 1]
    with pytest.raises(hf.HFError) as e:
        fs.compute(p1, p2, bad)
    assert e.value.status == B.HF_EINVAL
    empty = torch.zeros((0, 7), device="cuda")
    assert fs.query_batch(empty).shape == (0, 7)
    torch.cuda.synchronize()


def test_rank_deficient_rotation_set_flags_nan(hf, ctx, small_set):
    """All rotations about one axis: the torque neighbourhood has rank 1."""
    n = 32
    angs = np.linspace(-0.6, 0.6, 9)
    q = np.array([[np.cos(a / 2), 0, 0, np.sin(a / 2)] for a in angs], dtype=np.float32)
    p1, p2 = small_set["p"]
    for prec in (0, hf.HF_TORQUE_F64, hf.HF_TORQUE_C):
        fs = ctx.fieldset(n, len(q), hf.HF_E | hf.HF_F | hf.HF_T | prec)
        rc = fs.compute(p1, p2, q, allow_rank_deficient=True)
        assert rc == 1  # HF_EINVAL after computing everything else
        assert np.isnan(host(fs.get(0, 4))).all(), prec
        assert np.isfinite(host(fs.get(0, 0))).all()
        fs.release()


# ------------------------------------------- full-size workload, sampled

@pytest.mark.slow
def test_c2_full_size_sampled(hf, ctx):
    """128^3, 1024 rotations in the benchmark's launch configuration; sampled
    rotations against the oracle one by one, torque of a sampled rotation
    from the oracle's least squares over its 6 neighbours."""
    import torch
    n, R = 128, 1024
    s1, s2 = synth.c2_pair(0)
    g1 = ctx.density_build(n, cuda(s1.pts), cuda(s1.sigma))
    g2 = ctx.density_build(n, cuda(s2.pts), cuda(s2.sigma))
    q = synth.random_quaternions(0, R).astype(np.float32)
    p1, p2 = ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
    fs.compute(p1, p2, q)
    r1, r2 = host(g1), host(g2)
    qn = norm_quats(q)
    cache = {}

    def ofields(i):
        if i not in cache:
            R_ = oracle.quat_to_rot(qn[i]).astype(np.float32).astype(np.float64)
            cache[i] = np.stack(oracle.fields(r1, oracle.resample(r2, R_)))
        return cache[i]

    for i in (0, 1023):
        ref = ofields(i)
        for f in range(4):
            assert rel_err(host(fs.get(i, f)), ref[f]) <= TOL, (i, f)
    nb, _ = oracle.nearest(qn, qn[0], 6, skip=0)
    sub = [0] + list(nb)
    T, st = oracle.torque(qn[sub], np.stack([ofields(i)[0] for i in sub]), 6)
    assert st[0] == 0
    for d in range(3):
        assert rel_err(host(fs.get(0, 4 + d)), T[0, d]) <= TOL, d
    del torch


@pytest.mark.parametrize("pencil", [False, True])
def test_ragged_last_chunk(hf, pencil):
    """11 rotations launched 4 at a time (chunks 4, 4, 3) on either
    pipeline: every rotation, those of the short last chunk included, matches
    the oracle, and so does the torque of a rotation in that chunk (its
    neighbours lie in other chunks)."""
    n, R = 64, 11
    ctx = hf.Context(0)
    ctx.tune_set(n, 4, pencil=pencil)
    s1, s2 = synth.c2_pair(12)
    k = 800
    r1 = oracle.splat(n, s1.pts[:k], s1.sigma[:k]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[:k], s2.sigma[:k]).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    q = synth.random_quaternions(13, R).astype(np.float32)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
    fs.compute(p1, p2, q)
    qn = norm_quats(q)
    ref = np.stack([np.stack(oracle.fields(r1.astype(np.float64), oracle.resample(
        r2.astype(np.float64), oracle.quat_to_rot(qq).astype(np.float32).astype(np.float64)))) for qq in qn])
    for r in range(R):
        for f in range(4):
            assert rel_err(host(fs.get(r, f)), ref[r, f]) <= TOL, (r, f)
    T, st = oracle.torque(qn, ref[:, 0], 6)
    for r in (8, 10):  # both in the last chunk
        assert st[r] == 0
        for d in range(3):
            assert rel_err(host(fs.get(r, 4 + d)), T[r, d]) <= TOL, (r, d)


# ------------------------------------------------ 256^3 (pencil pipeline)

@pytest.mark.slow
def test_rfft3d_and_fields_256(hf, ctx):
    """256^3 runs the pencil pipeline (planes exceed one CTA's shared memory)."""
    import torch
    n = 256
    rng = np.random.default_rng(256)
    x = rng.standard_normal((n, n, n)).astype(np.float32)
    got = hf.rfft3d(cuda(x))
    torch.cuda.synchronize()
    ref = np.fft.rfftn(x.astype(np.float64))
    assert np.abs(got.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()
    del got, x
    s1, s2 = synth.c4_pair(0)
    r1 = oracle.splat(n, s1.pts[:300], s1.sigma[:300]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[:300], s2.sigma[:300]).astype(np.float32)
    q = synth.random_quaternions(4, 1)[0]
    got = gpu_fields(hf, ctx, r1, r2, q)
    qn = norm_quats(q.astype(np.float32))[0]
    R = oracle.quat_to_rot(qn).astype(np.float32).astype(np.float64)
    ref = oracle.fields(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), R))
    for g, r in zip(got, ref):
        assert rel_err(g, r) <= TOL


@pytest.mark.slow
def test_fieldset_256_batched_matches_oracle(hf):
    """The batched 256^3 field set (pencil pipeline, 3 rotations per launch,
    so that launches hold several rotations and the last one is short)
    against the oracle, element by element, on rotations in the first,
    middle and short last launch.  The parts are 400-point subsets splatted
    by the oracle; the reference is the oracle's resample and its
    library-DFT fields route."""
    n, R = 256, 8
    ctx = hf.Context(0)
    ctx.tune_set(n, 3, pencil=True)
    s1, s2 = synth.c4_pair(2)
    sel = np.random.default_rng(7).choice(len(s1.pts), 400, replace=False)
    r1 = oracle.splat(n, s1.pts[sel], s1.sigma[sel]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[sel], s2.sigma[sel]).astype(np.float32)
    p1, p2 = ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING)
    q = synth.random_quaternions(17, R).astype(np.float32)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F)
    fs.compute(p1, p2, q)
    qn = norm_quats(q)
    for r in (0, 4, 7):
        Rm = oracle.quat_to_rot(qn[r]).astype(np.float32).astype(np.float64)
        ref = oracle.fields_lib(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), Rm))
        for f in range(4):
            assert rel_err(host(fs.get(r, f)), ref[f]) <= TOL, (r, f)
    fs.release()


def test_fieldset_256_matches_single_rotation_path(hf, ctx):
    """The batched 256^3 field set equals the one-rotation entry point."""
    import torch
    n, R = 256, 8
    s1, s2 = synth.c4_pair(1)
    g1 = ctx.density_build(n, cuda(s1.pts), cuda(s1.sigma))
    g2 = ctx.density_build(n, cuda(s2.pts), cuda(s2.sigma))
    q = synth.random_quaternions(8, R).astype(np.float32)
    p1, p2 = ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)
    fs = ctx.fieldset(n, R, hf.HF_E | hf.HF_F | hf.HF_T)
    fs.compute(p1, p2, q)
    out = [torch.empty((n, n, n), device="cuda") for _ in range(4)]
    for i in (0, 5):
        ctx.fields(p1, p2, q[i], *out)
        for f in range(4):
            a, b = host(fs.get(i, f)), host(out[f])
            assert rel_err(a, b) <= 1e-6, (i, f)
    assert np.isfinite(host(fs.get(3, 4))).all()


def test_no_bulk_copy_wait_gave_up(hf):
    """Every bulk-staged pass C block of the tests above saw its planes
    arrive: no bounded wait ran out."""
    from paper_1711_05017_b300 import _binding as B
    assert B.lib().hf_bulk_timeouts(0) == 0


def test_query_selection_near_ties(hf, tmp_path):
    """The pose query's choice of the k nearest rotations, exactly as the
    oracle ranks them, where the float32 pass of the launched kernels cannot
    tell rotations apart: clusters of rotations 2e-4 to 1e-3 rad apart, exact
    duplicates (ties go to the lower index), and a query at a stored rotation
    (an exact hit).  A set whose energy field of rotation j is the constant
    j + 1 (written as a checkpoint with numpy) makes every answer the weighted
    sum of the chosen indices; the launched query, the batched one and the
    resident one are compared with the oracle's blend of the same fields.
    (No query sits exactly on a clustered rotation: there one ulp of |dot|,
    from the two sides normalising the quaternions in different rounding
    orders, decides the exact-hit rule and moves the 1/theta blend by up to
    5e-3; exact member rotations are tested apart from clusters.)"""
    import torch
    from scipy.spatial.transform import Rotation
    n = 32
    rng = np.random.default_rng(7)
    base = synth.random_quaternions(70, 8)
    quats = []
    for b in base:
        quats.append(b)
        for ang in (2e-4, 5e-4, 1e-3):
            ax = rng.normal(size=3)
            dq = Rotation.from_rotvec(ax / np.linalg.norm(ax) * ang).as_quat()  # x, y, z, w
            r = Rotation.from_quat([b[1], b[2], b[3], b[0]]) * Rotation.from_quat(dq)
            x, y, z, w = r.as_quat()
            quats.append([w, x, y, z])
    quats += [quats[1], quats[5], quats[2]]  # exact duplicates at higher indices
    q32 = np.asarray(quats, dtype=np.float32)
    R = len(q32)
    fields = np.zeros((R, 4, n, n, n), dtype=np.float32)
    for j in range(R):
        fields[j, 0] = j + 1.0
    path = tmp_path / "ties.hfc"
    with open(path, "wb") as f:
        np.lib.format.write_array(f, np.array([0x31504B4348465348, 1, hf.HF_CKPT_FIELDSET, n, R, hf.HF_E | hf.HF_F, 4,
                                                0, 1, 2, 3, -1, -1, -1, 0, 0], dtype=np.int64))
        np.lib.format.write_array(f, q32)
        np.lib.format.write_array(f, fields)
    ctx = hf.Context(0)
    fs = hf.FieldSet.load(ctx, path)
    torch.cuda.synchronize()
    # queries: near each cluster (inside the float32 ambiguity), and at stored rotations
    poses = []
    for i, b in enumerate(base):
        for ang in (1e-4, 3e-4, 2e-3):
            ax = rng.normal(size=3)
            dq = Rotation.from_rotvec(ax / np.linalg.norm(ax) * ang).as_quat()
            r = Rotation.from_quat([b[1], b[2], b[3], b[0]]) * Rotation.from_quat(dq)
            x, y, z, w = r.as_quat()
            poses.append((rng.uniform(-0.9, 0.9, 3).astype(np.float32), np.array([w, x, y, z], dtype=np.float32)))
    f64 = fields[:, :1].astype(np.float64)
    ks = (1, 2, 4, 5, 8)
    tq = cuda(np.stack([np.concatenate([t, qq]) for t, qq in poses]))
    qn = norm_quats(q32)
    for k in ks:
        ref = np.array([oracle.query(qn, f64, t.astype(np.float64), qq.astype(np.float64), k)[0]
                        for t, qq in poses])
        one = np.array([fs.query(t, qq, k=k)[0] for t, qq in poses])
        bat = fs.query_batch(tq, k=k)[:, 0].cpu().numpy()
        assert np.abs(one - ref).max() <= 1e-5 * np.abs(ref).max(), k
        assert np.array_equal(one, bat), k
        ctx.resident_queries(True)
        res = np.array([fs.query(t, qq, k=k)[0] for t, qq in poses])
        ctx.resident_queries(False)
        assert np.array_equal(one, res), k
    fs.release()
