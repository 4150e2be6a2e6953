"""Many part pairs of uneven grid sizes built by one CUDA graph (hf_batch_*),
and the launch-shape autotuner (hf_autotune / hf_tune_*).

The batch runs the same kernels in the same order per pair as a plain
field-set compute, so its fields must equal that compute's bitwise; one pair
is also checked against the FP64 oracle directly (max-abs error at most
1e-5 of the field's largest magnitude)."""
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
    return t.detach().cpu().numpy()


def make_pair(hf, ctx, n, seed, npts=1200):
    s1, s2 = synth.c2_pair(seed) if n >= 64 else synth.c1_pair(seed)
    g1 = ctx.density_build(n, cuda(s1.pts[:npts]), cuda(s1.sigma[:npts]))
    g2 = ctx.density_build(n, cuda(s2.pts[:npts]), cuda(s2.sigma[:npts]))
    return ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING), (g1, g2)


def all_fields(fs, R, nf):
    return np.stack([np.stack([host(fs.get(r, f)) for f in range(nf)]) for r in range(R)])


def plain(hf, ctx, pair, q, flags):
    fs = ctx.fieldset(pair[0].n, len(q), flags)
    fs.compute(pair[0], pair[1], q)
    return fs


def test_batch_equals_per_pair_builds_and_relaunches(hf):
    import torch
    ctx = hf.Context(0)
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    sizes = [32, 64, 96, 64, 128, 32]
    Rs = [12, 9, 8, 20, 7, 40]
    pairs = [make_pair(hf, ctx, n, 10 + i)[:2] for i, n in enumerate(sizes)]
    batch = hf.Batch(ctx, pairs, Rs, flags)
    assert batch.slots() == len(pairs)
    qs = [synth.random_quaternions(100 + i, r).astype(np.float32) for i, r in enumerate(Rs)]
    for i, q in enumerate(qs):
        batch.set_rotations(i, q)
    batch.capture()
    batch.launch()
    torch.cuda.synchronize()
    for i, q in enumerate(qs):
        ref = all_fields(plain(hf, ctx, pairs[i], q, flags), Rs[i], 7)
        got = all_fields(batch.fieldset(i), Rs[i], 7)
        assert np.array_equal(got, ref), i
    # new rotations for two pairs, replayed without a new capture
    qs[1] = synth.random_quaternions(200, Rs[1]).astype(np.float32)
    qs[4] = synth.random_quaternions(201, Rs[4]).astype(np.float32)
    batch.set_rotations(1, qs[1])
    batch.set_rotations(4, qs[4])
    batch.launch()
    torch.cuda.synchronize()
    for i in (1, 4, 5):
        ref = all_fields(plain(hf, ctx, pairs[i], qs[i], flags), Rs[i], 7)
        assert np.array_equal(all_fields(batch.fieldset(i), Rs[i], 7), ref), i
    # recorded again on two branches (slots 0, 2, 4 on one, 1, 3, 5 on the other)
    batch.capture(lanes=2)
    batch.launch()
    torch.cuda.synchronize()
    for i in (0, 3):
        ref = all_fields(plain(hf, ctx, pairs[i], qs[i], flags), Rs[i], 7)
        assert np.array_equal(all_fields(batch.fieldset(i), Rs[i], 7), ref), i
    # the batch's sets answer queries: a lattice node at a member rotation
    # reads that rotation's stored values
    fs = batch.fieldset(1)
    n, h = 64, 2.0 / 64
    E = all_fields(fs, Rs[1], 4)
    for r, j in ((0, (3, 17, 60)), (5, (32, 0, 9))):
        out = fs.query(np.array(j) * h, qs[1][r], k=4)
        ref = E[r, :, j[2], j[1], j[0]]
        assert np.abs(out[:4] - ref).max() <= 1e-6 * np.abs(E[r]).max()
    batch.release()


def test_batch_pair_matches_the_oracle(hf):
    import torch
    ctx = hf.Context(0)
    n, R = 32, 3
    s1, s2 = synth.c1_pair(4)
    r1 = oracle.splat(n, s1.pts, s1.sigma).astype(np.float32)
    r2 = oracle.splat(n, s2.pts, s2.sigma).astype(np.float32)
    p = (ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING))
    other = make_pair(hf, ctx, 64, 5)[:2]
    batch = hf.Batch(ctx, [other, p], [4, R])
    q = synth.random_quaternions(9, R).astype(np.float32)
    batch.set_rotations(0, synth.random_quaternions(8, 4))
    batch.set_rotations(1, q)
    batch.capture()
    batch.launch()
    torch.cuda.synchronize()
    got = all_fields(batch.fieldset(1), R, 4)
    qn = q.astype(np.float64)
    qn /= np.linalg.norm(qn, axis=1, keepdims=True)
    for r in range(R):
        Rm = oracle.quat_to_rot(qn[r]).astype(np.float32).astype(np.float64)
        ref = np.stack(oracle.fields(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), Rm)))
        for f in range(4):
            assert np.abs(got[r, f] - ref[f]).max() <= TOL * np.abs(ref[f]).max(), (r, f)


def test_streaming_slots_hold_the_last_pair(hf):
    """slots_per_size=1: three pairs of one size and rotation count share one
    set; after a launch it holds the last pair's fields, and asking for an
    earlier pair's set is refused."""
    import torch
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    pairs = [make_pair(hf, ctx, 64, 20 + i)[:2] for i in range(3)] + [make_pair(hf, ctx, 32, 30)[:2]]
    Rs = [16, 16, 16, 8]
    batch = hf.Batch(ctx, pairs, Rs, hf.HF_E | hf.HF_F, slots_per_size=1)
    assert batch.slots() == 2
    qs = [synth.random_quaternions(300 + i, r).astype(np.float32) for i, r in enumerate(Rs)]
    for i, q in enumerate(qs):
        batch.set_rotations(i, q)
    batch.capture()
    batch.launch()
    torch.cuda.synchronize()
    with pytest.raises(hf.HFError) as e:
        batch.fieldset(0)
    assert e.value.status == B.HF_ENOTREADY
    for i in (2, 3):
        ref = all_fields(plain(hf, ctx, pairs[i], qs[i], hf.HF_E | hf.HF_F), Rs[i], 4)
        assert np.array_equal(all_fields(batch.fieldset(i), Rs[i], 4), ref), i
    batch.release()


def test_batch_errors(hf):
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    a = make_pair(hf, ctx, 32, 40)[:2]
    b = make_pair(hf, ctx, 64, 41)[:2]
    with pytest.raises(hf.HFError) as e:  # parts of different sizes in one pair
        hf.Batch(ctx, [(a[0], b[1])], [8])
    assert e.value.status == B.HF_EINVAL
    with pytest.raises(hf.HFError):  # torque with fewer than 7 rotations
        hf.Batch(ctx, [a], [6], hf.HF_E | hf.HF_F | hf.HF_T)
    batch = hf.Batch(ctx, [a, b], [8, 8])
    batch.set_rotations(0, synth.random_quaternions(1, 8))
    with pytest.raises(hf.HFError) as e:  # pair 1 has no rotations yet
        batch.capture()
    assert e.value.status == B.HF_ENOTREADY
    with pytest.raises(hf.HFError) as e:
        batch.launch()
    assert e.value.status == B.HF_ENOTREADY
    bad = synth.random_quaternions(2, 8)
    bad[3] = 0
    with pytest.raises(hf.HFError) as e:
        batch.set_rotations(1, bad)
    assert e.value.status == B.HF_EINVAL
    batch.release()


def test_autotune_choice_cache_and_results(hf, tmp_path):
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    import json
    path = tmp_path / "tune.json"
    chunk, pencil, rps = ctx.autotune(64, path)
    assert chunk > 0 and pencil in (0, 1) and rps > 0
    assert ctx.tune_get(64)[:2] == (chunk, pencil)
    doc = json.loads(path.read_text())  # the cache is JSON: one entry per (device, N)
    (ent,) = [e for e in doc["tune"] if e["n"] == 64]
    assert ent["chunk"] == chunk and ent["pipeline"] == ("pencil" if pencil else "slab")
    assert ent["radix"] == "yz 8x8, x inverse 8x8" and ent["passB_columns_per_cta"] in (16, 32)
    assert (ent["tile_b"], ent["tile_c"]) == ctx.tune_tiles(64)
    # a second context reads the cache instead of timing
    ctx2 = hf.Context(0)
    assert ctx2.autotune(64, path) == (chunk, pencil, pytest.approx(rps, rel=1e-5))
    # the tuned shape gives the same fields as the built-in one (independent
    # per-rotation arithmetic; the pipelines may round differently)
    pair = make_pair(hf, ctx, 64, 50)[:2]
    q = synth.random_quaternions(51, 40).astype(np.float32)
    tuned = all_fields(plain(hf, ctx2, pair, q, hf.HF_E | hf.HF_F), 40, 4)
    ctx2.tune_set(64, 0)
    base = all_fields(plain(hf, ctx2, pair, q, hf.HF_E | hf.HF_F), 40, 4)
    for f in range(4):
        assert np.abs(tuned[:, f] - base[:, f]).max() <= 2e-6 * np.abs(base[:, f]).max()
    # hand-set shapes, the pencil pipeline at 64^3 included
    ctx2.tune_set(64, 8, pencil=True)
    assert ctx2.tune_get(64)[:2] == (8, 1)
    pen = all_fields(plain(hf, ctx2, pair, q, hf.HF_E | hf.HF_F), 40, 4)
    for f in range(4):
        assert np.abs(pen[:, f] - base[:, f]).max() <= 2e-6 * np.abs(base[:, f]).max()
    with pytest.raises(hf.HFError) as e:
        ctx2.tune_set(256, 4, pencil=False)
    assert e.value.status == B.HF_EUNSUPPORTED


@pytest.mark.parametrize("n", [64, 96, 128])
def test_tile_candidates_give_the_same_fields(hf, n):
    """Every compiled launch-shape candidate of passes B and C (the
    autotuner's choices) gives the built-in shape's fields bit for bit: the
    per-item arithmetic is the same, only the blocks' tiling differs."""
    ctx = hf.Context(0)
    pair = make_pair(hf, ctx, n, 60)[:2]
    q = synth.random_quaternions(61, 10).astype(np.float32)
    base = all_fields(plain(hf, ctx, pair, q, hf.HF_E | hf.HF_F), 10, 4)
    for tb in (0, 1):
        for tc in ((0, 1, 2, 3, 4, 5, 6) if n == 128 else (0, 1, 5)):
            ctx.tune_tiles(n, (tb, tc))
            assert ctx.tune_tiles(n) == (tb, tc)
            got = all_fields(plain(hf, ctx, pair, q, hf.HF_E | hf.HF_F), 10, 4)
            assert np.array_equal(got, base), (tb, tc)
    if n == 128:
        # the x inverse with its digits in the other order: the same sums in
        # another order, so equal to rounding (and bit for bit run to run)
        ctx.tune_tiles(n, (0, 7))
        got = all_fields(plain(hf, ctx, pair, q, hf.HF_E | hf.HF_F), 10, 4)
        for f in range(4):
            assert np.abs(got[:, f] - base[:, f]).max() <= 1e-6 * np.abs(base[:, f]).max(), f
        assert np.array_equal(all_fields(plain(hf, ctx, pair, q, hf.HF_E | hf.HF_F), 10, 4), got)
    with pytest.raises(hf.HFError):
        ctx.tune_tiles(n, (0, 2) if n != 128 else (2, 0))
    # two pipelines alternating chunks on two streams: the same fields
    ctx.tune_tiles(n, (0, 0))
    ctx.tune_set(n, 4)
    assert ctx.tune_lanes(n, 2) == 2 and ctx.tune_lanes(n) == 2
    got = all_fields(plain(hf, ctx, pair, q, hf.HF_E | hf.HF_F), 10, 4)
    assert np.array_equal(got, base)


# ------------------------------------------------ one launch over a work queue

def _queue_pairs(hf, ctx, spec):
    pairs, quats = [], []
    for i, (n, R) in enumerate(spec):
        p1, p2, _ = make_pair(hf, ctx, n, 70 + i)
        pairs.append((p1, p2))
        quats.append(synth.random_quaternions(80 + i, R).astype(np.float32))
    return pairs, quats


def test_one_launch_queue_equals_per_pair_builds(hf):
    """Pairs of 64^3, 96^3 and 128^3 with ragged rotation counts, built by
    ONE launch of the work-queue kernel: every field of every rotation equals
    the pair's own per-pass build bit for bit, on two launches in a row."""
    ctx = hf.Context(0)
    flags = hf.HF_E | hf.HF_F
    spec = [(64, 40), (128, 24), (96, 33), (64, 17), (128, 20)]
    pairs, quats = _queue_pairs(hf, ctx, spec)
    b = hf.Batch(ctx, pairs, [R for _, R in spec], flags)
    for i, q in enumerate(quats):
        b.set_rotations(i, q)
    b.capture_queue(chunk=16)
    for launch in range(2):
        b.launch()
        items, runs = b.status()
        assert items > 0 and runs > 0
        for i, (pr, q) in enumerate(zip(pairs, quats)):
            ref = plain(hf, ctx, pr, q, flags)
            got = b.fieldset(i)
            assert np.array_equal(all_fields(got, len(q), 4), all_fields(ref, len(q), 4)), (launch, i)
            ref.release()
    b.release()


def test_one_launch_queue_matches_the_oracle(hf):
    """One 64^3 pair of the one-launch build against the FP64 oracle."""
    ctx = hf.Context(0)
    n, R = 64, 12
    s1, s2 = synth.c2_pair(91)
    r1 = oracle.splat(n, s1.pts[:600], s1.sigma[:600]).astype(np.float32)
    r2 = oracle.splat(n, s2.pts[:600], s2.sigma[:600]).astype(np.float32)
    p = (ctx.part(cuda(r1), hf.HF_STATIONARY), ctx.part(cuda(r2), hf.HF_MOVING))
    q = synth.random_quaternions(92, R).astype(np.float32)
    b = hf.Batch(ctx, [p], [R], hf.HF_E | hf.HF_F)
    b.set_rotations(0, q)
    b.capture_queue(chunk=5)
    b.launch()
    b.status()
    fs = b.fieldset(0)
    for r in (0, 6, 11):
        qq = q[r].astype(np.float64)
        Rm = oracle.quat_to_rot(qq / np.linalg.norm(qq)).astype(np.float32).astype(np.float64)
        ref = oracle.fields(r1.astype(np.float64), oracle.resample(r2.astype(np.float64), Rm))
        for f in range(4):
            got = host(fs.get(r, f)).astype(np.float64)
            assert np.abs(got - ref[f]).max() <= TOL * np.abs(ref[f]).max(), (r, f)
    b.release()


def test_one_launch_shared_output_sets_hold_the_last_pair(hf):
    """Three 64^3 pairs sharing one output set: items of a later pair wait
    for the earlier pair's same rotations, so after the launch the set holds
    the last pair's fields exactly."""
    ctx = hf.Context(0)
    flags = hf.HF_E | hf.HF_F
    spec = [(64, 20), (64, 20), (64, 20)]
    pairs, quats = _queue_pairs(hf, ctx, spec)
    b = hf.Batch(ctx, pairs, [20, 20, 20], flags, slots_per_size=1)
    assert b.slots() == 1
    for i, q in enumerate(quats):
        b.set_rotations(i, q)
    b.capture_queue(chunk=8)
    b.launch()
    b.status()
    ref = plain(hf, ctx, pairs[2], quats[2], flags)
    assert np.array_equal(all_fields(b.fieldset(2), 20, 4), all_fields(ref, 20, 4))
    ref.release()
    b.release()


def test_one_launch_bounded_wait_reports_timeout(hf):
    """A planted wait that nothing satisfies runs out its bounded poll count:
    the launch stops early, the status says HF_ETIMEOUT, and the same context
    then builds correctly."""
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    flags = hf.HF_E | hf.HF_F
    spec = [(64, 16), (96, 16)]
    pairs, quats = _queue_pairs(hf, ctx, spec)
    b = hf.Batch(ctx, pairs, [16, 16], flags)
    for i, q in enumerate(quats):
        b.set_rotations(i, q)
    b.capture_queue(chunk=8, spin_limit=20000, self_test=1)
    b.launch()
    with pytest.raises(hf.HFError) as e:
        b.status()
    assert e.value.status == B.HF_ETIMEOUT
    b.capture_queue(chunk=8)
    b.launch()
    b.status()
    ref = plain(hf, ctx, pairs[1], quats[1], flags)
    assert np.array_equal(all_fields(b.fieldset(1), 16, 4), all_fields(ref, 16, 4))
    ref.release()
    b.release()
