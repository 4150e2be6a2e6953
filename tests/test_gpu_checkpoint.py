"""Checkpoint / resume on the GPU: parts, computed field sets and a served
session saved to files and loaded back give the saved state bit for bit --
field sets built from loaded parts, loaded fields, queries against them, and
a restarted server's answers; numpy reads every array of the files on its
own (the files are NPY arrays in the documented layout)."""
import os

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


def parts(hf, ctx, n, seed, npts=1500):
    import torch
    s1, s2 = synth.c2_pair(seed)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    g1 = ctx.density_build(n, cu(s1.pts[:npts]), cu(s1.sigma[:npts]))
    g2 = ctx.density_build(n, cu(s2.pts[:npts]), cu(s2.sigma[:npts]))
    return ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING), g2


def read_all(path):
    out = []
    with open(path, "rb") as f:
        while f.peek(1) if hasattr(f, "peek") else f.read(1):
            out.append(np.lib.format.read_array(f))
    return out


def all_fields(fs, R):
    return np.stack([np.stack([fs.get(r, f).cpu().numpy() for f in range(7)]) for r in range(R)])


def test_parts_and_field_sets_round_trip_bitwise(hf, tmp_path):
    n, R = 64, 12
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    ctx = hf.Context(0)
    p1, p2, g2 = parts(hf, ctx, n, 30)
    q = synth.random_quaternions(31, R).astype(np.float32)
    fs = ctx.fieldset(n, R, flags)
    fs.compute(p1, p2, q)
    ref = all_fields(fs, R)
    a, b, c = (os.path.join(tmp_path, x) for x in ("s1.hfc", "s2.hfc", "set.hfc"))
    p1.save(a)
    p2.save(b)
    fs.save(c)
    assert hf.checkpoint_info(a)[:2] == (hf.HF_CKPT_PART, n)
    assert hf.checkpoint_info(c) == (hf.HF_CKPT_FIELDSET, n, R, flags)
    # numpy reads the files on its own: the moving grid, the rotations, the fields
    arrs = read_all(b)
    assert np.array_equal(arrs[1], g2.cpu().numpy())
    arrs = read_all(c)
    assert np.array_equal(arrs[1], q)
    assert arrs[2].shape == (R, 7, n, n, n) and np.array_equal(arrs[2], ref)
    # parts loaded back build the same fields; the loaded set holds them
    l1, l2 = hf.Part.load(ctx, a), hf.Part.load(ctx, b)
    fs2 = ctx.fieldset(n, R, flags)
    fs2.compute(l1, l2, q)
    assert np.array_equal(all_fields(fs2, R), ref)
    fl = hf.FieldSet.load(ctx, c)
    assert (fl.n, fl.R) == (n, R)
    assert np.array_equal(all_fields(fl, R), ref)
    rng = np.random.default_rng(3)
    for _ in range(8):
        t, qq = rng.uniform(-1, 1, 3), synth.random_quaternions(int(rng.integers(1 << 30)), 1)[0]
        assert np.array_equal(fl.query(t, qq), fs.query(t, qq))
    for x in (fs, fs2, fl):
        x.release()


def test_uncomputed_set_and_bad_files_are_refused(hf, tmp_path):
    from paper_1711_05017_b300 import _binding as B
    ctx = hf.Context(0)
    fs = ctx.fieldset(32, 8, hf.HF_E | hf.HF_F)
    with pytest.raises(hf.HFError) as e:
        fs.save(os.path.join(tmp_path, "never.hfc"))
    assert e.value.status == B.HF_ENOTREADY
    p1, p2, _ = parts(hf, ctx, 32, 32, npts=300)
    pp = os.path.join(tmp_path, "p.hfc")
    p1.save(pp)
    with pytest.raises(hf.HFError):
        hf.FieldSet.load(ctx, pp)  # a part file is not a field set
    fs.release()


def test_server_session_restored_after_restart(hf, tmp_path):
    """A session with a chunked request is saved, the server and parts are
    dropped, and a new server over reloaded parts restores it: every field
    of every rotation and queries at member rotations are the same bits."""
    from paper_1711_05017_b300 import _binding as B
    n, R = 64, 40
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    ctx = hf.Context(0)
    p1, p2, _ = parts(hf, ctx, n, 33)
    srv = hf.Server(ctx, max_inflight=2, query_lanes=2)
    srv.set_chunk_bytes(B.lib().hf_fieldset_bytes(n, 20, flags))
    sid = srv.open(p1, p2)
    q = synth.random_quaternions(34, R).astype(np.float32)
    rid = srv.submit(sid, q, flags)
    assert srv.wait([rid])[rid][0] == "done"
    assert srv.request_chunks(rid, R)[0] > 1
    ref = np.stack([np.stack([srv.field(sid, r, f, n).cpu().numpy() for f in range(7)]) for r in range(R)])
    t = np.array([0.1, -0.2, 0.3])
    qref = [srv.query(sid, t, q[r], k=4) for r in (0, 17, 39)]
    pa, pb, ps = (os.path.join(tmp_path, x) for x in ("p1.hfc", "p2.hfc", "session.hfc"))
    p1.save(pa)
    p2.save(pb)
    srv.session_save(sid, ps)
    assert hf.checkpoint_info(ps)[:3] == (hf.HF_CKPT_SESSION, n, R)
    srv.close()
    del p1, p2
    # restart: new parts from the files, a new server, the session restored
    l1, l2 = hf.Part.load(ctx, pa), hf.Part.load(ctx, pb)
    srv2 = hf.Server(ctx, max_inflight=2, query_lanes=2)
    sid2 = srv2.open(l1, l2)
    with pytest.raises(hf.HFError):
        srv2.query(sid2, t, q[0])  # nothing published yet
    srv2.session_restore(sid2, ps)
    got = np.stack([np.stack([srv2.field(sid2, r, f, n).cpu().numpy() for f in range(7)]) for r in range(R)])
    assert np.array_equal(got, ref)
    for r, a in zip((0, 17, 39), qref):
        assert np.array_equal(srv2.query(sid2, t, q[r], k=4), a)
    srv2.close()
