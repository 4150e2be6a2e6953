"""The serving runtime (hf_server_*): sessions with resident field sets,
budget-admitted continuous batching of builds, supersede, eviction, and pose
queries on high-priority lanes while builds run."""
import threading
import time

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


def make_parts(hf, ctx, n, seed, npts=1500):
    import torch
    s1, s2 = synth.c2_pair(seed) if n >= 64 else synth.c1_pair(seed)
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()  # noqa: E731
    g1 = ctx.density_build(n, cu(s1.pts[:npts]), cu(s1.sigma[:npts]))
    g2 = ctx.density_build(n, cu(s2.pts[:npts]), cu(s2.sigma[:npts]))
    return ctx.part(g1, hf.HF_STATIONARY), ctx.part(g2, hf.HF_MOVING)


def fields_of(srv, sid, rots, n):
    return np.stack([np.stack([srv.field(sid, r, f, n).cpu().numpy() for f in range(7)]) for r in rots])


def test_result_is_the_same_alone_and_in_the_mix(hf):
    """Each build gives the same fields whether it runs alone or overlapped
    with other sessions' builds on the device (bitwise: same kernels, same
    order of arithmetic)."""
    ctx = hf.Context(0)
    srv = hf.Server(ctx, max_inflight=4, query_lanes=4)
    pa = make_parts(hf, ctx, 64, 0)
    pb = make_parts(hf, ctx, 32, 1)
    pc = make_parts(hf, ctx, 96, 2)
    a, b, c = srv.open(*pa), srv.open(*pb), srv.open(*pc)
    qa = synth.random_quaternions(11, 24)
    r = srv.submit(a, qa)
    assert srv.wait([r])[r][0] == "done"
    alone = fields_of(srv, a, (0, 7, 23), 64)
    # the same request again, now in a mix submitted together
    rids = [srv.submit(b, synth.random_quaternions(12, 40)), srv.submit(a, qa),
            srv.submit(c, synth.random_quaternions(13, 16)), srv.submit(b, synth.random_quaternions(14, 48))]
    res = srv.wait(rids)
    assert res[rids[1]][0] == "done" and res[rids[2]][0] == "done"
    mixed = fields_of(srv, a, (0, 7, 23), 64)
    assert np.array_equal(alone, mixed)
    st = srv.stats()
    assert st["completed"] >= 4 and st["failed"] == 0
    srv.close()


def test_budget_admission_and_rejection(hf):
    n = 64
    need = None
    from paper_1711_05017_b300 import _binding as B
    one = B.lib().hf_fieldset_bytes(n, 32, hf.HF_E | hf.HF_F | hf.HF_T)
    ctx = hf.Context(0, hbm_budget_bytes=int(2.5 * one) + (64 << 20))
    parts = make_parts(hf, ctx, n, 3)
    srv = hf.Server(ctx, max_inflight=4, query_lanes=2)
    srv.set_chunk_bytes(0)  # whole sets only: an oversized request is rejected, not split
    sids = [srv.open(*parts) for _ in range(3)]
    # a set larger than the whole budget is rejected at once
    with pytest.raises(hf.HFError) as e:
        srv.submit(sids[0], synth.random_quaternions(5, 96))
    assert e.value.status == B.HF_EBUDGET
    # three sets of which only two fit at a time: admission waits, all finish,
    # and the reserved bytes never exceed the budget
    rids = [srv.submit(s, synth.random_quaternions(20 + i, 32)) for i, s in enumerate(sids)]
    peak = 0
    t0 = time.time()
    while time.time() - t0 < 60:
        st = srv.stats()
        peak = max(peak, st["reserved_bytes"])
        if all(srv.state(r)[0] in ("done", "failed") for r in rids):
            break
        time.sleep(0.0005)
    assert all(srv.state(r)[0] == "done" for r in rids)
    assert peak <= ctx.reserved_bytes() + st["budget_bytes"]
    assert peak <= st["budget_bytes"]
    assert st["evicted"] >= 1  # published sets had to make room for the third
    del need
    srv.close()


def test_newer_request_supersedes_a_queued_one(hf):
    ctx = hf.Context(0)
    srv = hf.Server(ctx, max_inflight=1, query_lanes=1)
    big = make_parts(hf, ctx, 128, 4)
    small = make_parts(hf, ctx, 32, 5)
    s_big, s_small = srv.open(*big), srv.open(*small)
    r0 = srv.submit(s_big, synth.random_quaternions(30, 64))  # occupies the only slot
    r1 = srv.submit(s_small, synth.random_quaternions(31, 8))
    r2 = srv.submit(s_small, synth.random_quaternions(32, 8))  # supersedes r1 while it waits
    res = srv.wait([r0, r1, r2])
    assert res[r1][0] == "superseded" and res[r2][0] == "done" and res[r0][0] == "done"
    srv.close()


def test_queries_during_builds_are_exact_at_nodes_and_member_rotations(hf):
    """While other sessions build, queries at lattice nodes with a member
    rotation return that rotation's stored values (exact trilinear weights,
    exact rotation hit)."""
    n = 64
    h = 2.0 / n
    ctx = hf.Context(0)
    srv = hf.Server(ctx, max_inflight=3, query_lanes=8)
    pq = make_parts(hf, ctx, n, 6)
    sq = srv.open(*pq)
    q = synth.random_quaternions(40, 16).astype(np.float32)
    r = srv.submit(sq, q)
    assert srv.wait([r])[r][0] == "done"
    ref = fields_of(srv, sq, range(16), n)
    others = [srv.open(*make_parts(hf, ctx, 128, 7 + i)) for i in range(2)]
    busy = [srv.submit(o, synth.random_quaternions(50 + i, 128)) for i, o in enumerate(others)]
    errs, lat = [], []

    def worker(seed):
        rng = np.random.default_rng(seed)
        for _ in range(200):
            i = int(rng.integers(16))
            j = rng.integers(0, n, 3)
            t0 = time.perf_counter()
            out = srv.query(sq, j * h, q[i], k=4)
            lat.append(time.perf_counter() - t0)
            errs.append(np.abs(out - ref[i, :, j[2], j[1], j[0]]).max() / (np.abs(ref[i]).max() + 1e-30))

    th = [threading.Thread(target=worker, args=(s,)) for s in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    srv.wait(busy)
    assert max(errs) <= 1e-6
    assert srv.stats()["queries"] >= 800
    srv.close()


def test_native_query_driver_meets_the_rate(hf):
    """Two sessions replayed at 1 kHz from native threads while a third
    session builds: every query answered, latencies recorded per query."""
    ctx = hf.Context(0)
    srv = hf.Server(ctx, max_inflight=2, query_lanes=4)
    a = srv.open(*make_parts(hf, ctx, 64, 8))
    b = srv.open(*make_parts(hf, ctx, 32, 9))
    c = srv.open(*make_parts(hf, ctx, 128, 10))
    r = [srv.submit(a, synth.random_quaternions(60, 16)), srv.submit(b, synth.random_quaternions(61, 16))]
    res = srv.wait(r)
    from paper_1711_05017_b300 import _binding as B
    for rid in r:
        st, _ = srv.state(rid)
        assert st == "done", B.lib().hf_last_error()
    assert np.isfinite(srv.query(a, [0.1, 0.2, 0.3], synth.random_quaternions(63, 1)[0])).all()
    busy = srv.submit(c, synth.random_quaternions(62, 96))
    steps = 300
    poses = np.stack([np.concatenate([synth.translation_walk(70 + i, steps), synth.quaternion_walk(80 + i, steps)], 1)
                      for i in range(2)])
    srv.query_latencies()
    t0 = time.perf_counter()
    answered, not_ready, late = srv.drive_queries([a, b], poses, rate_hz=1000.0)
    took = time.perf_counter() - t0
    lat = srv.query_latencies()
    srv.wait([busy])
    assert answered == 2 * steps and not_ready == 0
    assert lat.size == 2 * steps and np.isfinite(lat).all()
    assert took >= 0.29  # paced, not burst
    srv.close()


def test_chunked_request_equals_single_shot_bitwise(hf):
    """A request split into rotation chunks (each built with its torque
    neighbours) gives, for every rotation of the request, the same E, F and
    least-squares T as one build of the whole set, bit for bit; a query at a
    member rotation is routed to the chunk that owns it."""
    from paper_1711_05017_b300 import _binding as B
    n, R = 64, 60
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    ctx = hf.Context(0)
    p1, p2 = make_parts(hf, ctx, n, 21)
    srv = hf.Server(ctx, max_inflight=3, query_lanes=2)
    srv.set_chunk_bytes(B.lib().hf_fieldset_bytes(n, 24, flags))
    sid = srv.open(p1, p2)
    q = synth.random_quaternions(90, R).astype(np.float32)
    rid = srv.submit(sid, q, flags)
    assert srv.wait([rid])[rid][0] == "done"
    nchunks, owner = srv.request_chunks(rid, R)
    assert nchunks > 1 and set(owner) == set(range(nchunks))
    fs = ctx.fieldset(n, R, flags)
    fs.compute(p1, p2, q)
    for r in range(R):
        for f in range(7):
            a = srv.field(sid, r, f, n).cpu().numpy()
            b = fs.get(r, f).cpu().numpy()
            assert np.array_equal(a, b), (r, f, owner[r])
    h = 2.0 / n
    for r in (0, R // 2, R - 1):
        t = np.array([3, 5, 7]) * h
        got = srv.query(sid, t, q[r], k=1)
        ref = fs.query(t, q[r], k=1)
        assert np.array_equal(got, ref), r
    st = srv.stats()
    assert st["chunks_completed"] == nchunks and st["chunks_resident"] == nchunks
    fs.release()
    srv.close()


def test_chunks_admitted_as_memory_frees_and_evicted_least_recent_first(hf):
    """A request four times larger than the budget is built chunk by chunk:
    the reserved bytes stay within the budget, earlier chunks are evicted to
    admit later ones, the request completes, and a query that routes to an
    evicted chunk is refused as not ready while one that routes to a
    resident chunk is answered."""
    from paper_1711_05017_b300 import _binding as B
    n, R = 64, 96
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    one = B.lib().hf_fieldset_bytes(n, 24, flags)
    ctx = hf.Context(0, hbm_budget_bytes=int(2.2 * one) + (64 << 20))
    p1, p2 = make_parts(hf, ctx, n, 22)
    srv = hf.Server(ctx, max_inflight=2, query_lanes=2)
    srv.set_chunk_bytes(one)
    sid = srv.open(p1, p2)
    q = synth.random_quaternions(91, R).astype(np.float32)
    rid = srv.submit(sid, q, flags)
    peak = 0
    t0 = time.time()
    while time.time() - t0 < 120 and srv.state(rid)[0] not in ("done", "failed"):
        peak = max(peak, srv.stats()["reserved_bytes"])
        time.sleep(0.0005)
    assert srv.state(rid)[0] == "done", B.lib().hf_last_error()
    nchunks, owner = srv.request_chunks(rid, R)
    st = srv.stats()
    assert nchunks >= 4
    assert peak <= st["budget_bytes"]
    assert st["evicted"] >= 1 and st["chunks_resident"] < nchunks
    resident, refused = 0, 0
    for r in range(R):
        try:
            srv.query(sid, [0.0, 0.0, 0.0], q[r], k=1)
            resident += 1
        except hf.HFError as e:
            assert e.status == B.HF_ENOTREADY
            refused += 1
    assert resident > 0 and refused > 0
    srv.close()


def test_closing_a_session_mid_build_leaves_the_others_exact(hf):
    """A session closed while its builds are queued and running: its
    requests end failed, its parts stay alive for the build in flight even
    after the caller drops them, and the other sessions' results are bitwise
    those of a run without it."""
    import gc
    ctx = hf.Context(0)
    srv = hf.Server(ctx, max_inflight=2, query_lanes=2)
    keep = make_parts(hf, ctx, 64, 0)
    other = srv.open(*keep)
    q = synth.random_quaternions(31, 40)
    r = srv.submit(other, q)
    assert srv.wait([r])[r][0] == "done"
    alone = fields_of(srv, other, (0, 13, 39), 64)
    cancelled = 0
    for round_ in range(3):
        gone = srv.open(*make_parts(hf, ctx, 128, 5 + round_))  # the test keeps no handle to these parts
        gc.collect()
        # builds of tens of milliseconds: the close lands while they run or wait
        doomed = [srv.submit(gone, synth.random_quaternions(40 + round_, 192)) for _ in range(2)]
        rid = srv.submit(other, q)
        time.sleep(0.002 * round_)
        srv.close_session(gone)
        gc.collect()
        res = srv.wait(doomed + [rid])
        assert res[rid][0] == "done"
        states = [res[d][0] for d in doomed]
        assert all(x in ("failed", "superseded", "done") for x in states), states
        cancelled += states.count("failed")
        assert np.array_equal(fields_of(srv, other, (0, 13, 39), 64), alone)
    assert cancelled >= 1
    with pytest.raises(hf.HFError):
        srv.submit(gone, q)
    st = srv.stats()
    assert st["sessions"] == 1
    srv.close()


def test_metrics_log_lines_account_for_every_query_and_build(hf, tmp_path):
    """The JSON-lines metrics log: one parsable line per period and a last
    one at close; the per-period query and build counts add up to what the
    server answered and finished while it was open, the counters only grow,
    and each period's percentiles are ordered and bound the exact latencies
    the library recorded."""
    import json
    ctx = hf.Context(0)
    srv = hf.Server(ctx, max_inflight=2, query_lanes=4)
    a = srv.open(*make_parts(hf, ctx, 64, 8))
    b = srv.open(*make_parts(hf, ctx, 32, 9))
    r = [srv.submit(a, synth.random_quaternions(60, 16)), srv.submit(b, synth.random_quaternions(61, 16))]
    assert all(v[0] == "done" for v in srv.wait(r).values())
    path = tmp_path / "metrics.jsonl"
    srv.query_latencies()
    before = srv.stats()
    srv.log_open(path, period_ms=50)
    steps = 400
    poses = np.stack([np.concatenate([synth.translation_walk(90 + i, steps), synth.quaternion_walk(95 + i, steps)], 1)
                      for i in range(2)])
    builds = [srv.submit(a, synth.random_quaternions(64 + i, 24)) for i in range(3)]
    answered, not_ready, _ = srv.drive_queries([a, b], poses, rate_hz=1000.0)
    assert srv.wait(builds)
    lat = srv.query_latencies()
    time.sleep(0.12)
    srv.log_close()
    after = srv.stats()
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert len(lines) >= 6  # 0.4 s of queries at 50 ms per line, plus the last
    assert all(y["t_s"] > x["t_s"] for x, y in zip(lines, lines[1:]))
    for key in ("completed", "queries", "rotations_completed", "submitted"):
        seq = [x[key] for x in lines]
        assert seq == sorted(seq) and before[key] <= seq[0] and seq[-1] == after[key], key
    assert sum(x["query"]["n"] for x in lines) == answered == lat.size
    assert sum(x["build"]["n"] for x in lines) == after["completed"] - before["completed"]
    top = 0.0
    for x in lines:
        qn = x["query"]
        if qn["n"]:
            assert qn["p50_us"] <= qn["p99_us"] <= qn["p999_us"] <= qn["max_us"] * 1.0905
            top = max(top, qn["max_us"])
        else:
            assert qn["p50_us"] is None
    assert abs(top - float(lat.max())) <= 1e-3 * top + 1e-3
    last = {s: (ans, nr) for s, ans, nr in lines[-1]["session_queries"]}
    assert sorted(last) == [a, b]
    assert sum(v[0] for v in last.values()) >= answered
    srv.close()


def test_preload_loads_the_kernel_modules_once(hf):
    """hf_ctx_preload loads every kernel of the builds, torque and queries;
    a second call finds the same modules and loads nothing new."""
    ctx = hf.Context(0)
    n1 = ctx.preload()
    n2 = ctx.preload()
    assert n1 == n2 and n1 > 50


def test_budgeted_server_builds_in_its_arena_bitwise(hf):
    """With a budget the server carves its field sets from one device arena:
    while sets are resident the arena has less free, the fields are bitwise
    those of a standalone field-set build of the same rotations, and once
    every set is evicted and released the arena is one free range again."""
    from paper_1711_05017_b300 import _binding as B
    n, R = 64, 24
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    one = B.lib().hf_fieldset_bytes(n, R, flags)
    ctx = hf.Context(0, hbm_budget_bytes=int(3.5 * one) + (64 << 20))
    p1, p2 = make_parts(hf, ctx, n, 31)
    srv = hf.Server(ctx, max_inflight=2, query_lanes=2)
    st0 = srv.stats()
    assert st0["arena_bytes"] >= 3 * one
    assert st0["arena_free_bytes"] == st0["arena_bytes"]
    sid = srv.open(p1, p2)
    q = synth.random_quaternions(77, R)
    rid = srv.submit(sid, q, flags)
    assert srv.wait([rid])[rid][0] == "done"
    st1 = srv.stats()
    assert st1["arena_free_bytes"] <= st1["arena_bytes"] - one
    got = fields_of(srv, sid, (0, 11, 23), n)
    fs = ctx.fieldset(n, R, flags)
    fs.compute(p1, p2, q)
    ref = np.stack([np.stack([fs.get(r, f).cpu().numpy() for f in range(7)]) for r in (0, 11, 23)])
    assert np.array_equal(got, ref)
    fs.release()
    # a second request of the same session replaces the first set, which is
    # retired and returned to the arena
    rid2 = srv.submit(sid, synth.random_quaternions(78, R), flags)
    assert srv.wait([rid2])[rid2][0] == "done"
    t0 = time.time()
    while time.time() - t0 < 10 and srv.stats()["arena_free_bytes"] < st1["arena_free_bytes"]:
        time.sleep(0.01)
    st2 = srv.stats()
    assert st2["arena_free_bytes"] == st1["arena_free_bytes"]
    assert st2["arena_largest_free"] >= st2["arena_free_bytes"] - 2 * one
    srv.close()


def _poses(seed, m):
    rng = np.random.default_rng(seed)
    t = rng.uniform(-0.6, 0.6, size=(m, 3)).astype(np.float32)
    return t, synth.random_quaternions(seed + 1, m).astype(np.float32)


@pytest.mark.parametrize("n", [64, 96])
def test_resident_queries_equal_launched_ones(hf, n, monkeypatch):
    """Queries answered by the resident query kernel (no launch) equal, bit
    for bit, those of a launched query kernel on the same field set, from one
    thread and from several at once; with HF_RESIDENT_QUERIES=0 the server
    launches every query and gives the same answers."""
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    R = 24
    ctx = hf.Context(0)
    p1, p2 = make_parts(hf, ctx, n, 41)
    q = synth.random_quaternions(101, R)
    fs = ctx.fieldset(n, R, flags)
    fs.compute(p1, p2, q)
    import torch
    torch.cuda.synchronize()  # hf_query runs on its own stream, not ordered after the build
    t, qq = _poses(7, 120)
    ks = [1 + (i % 8) for i in range(len(t))]
    ref = np.stack([fs.query(t[i], qq[i], k=ks[i]) for i in range(len(t))])
    for resident in (True, False):
        if not resident:
            monkeypatch.setenv("HF_RESIDENT_QUERIES", "0")
        srv = hf.Server(ctx, max_inflight=1, query_lanes=20)  # two blocks of lanes
        sid = srv.open(p1, p2)
        rid = srv.submit(sid, q, flags)
        assert srv.wait([rid])[rid][0] == "done"
        got = np.stack([srv.query(sid, t[i], qq[i], k=ks[i]) for i in range(len(t))])
        assert np.array_equal(got, ref), resident
        outs = {}

        def worker(w):
            outs[w] = np.stack([srv.query(sid, t[i], qq[i], k=ks[i]) for i in range(w, len(t), 6)])

        th = [threading.Thread(target=worker, args=(w,)) for w in range(6)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for w in range(6):
            assert np.array_equal(outs[w], ref[w::6]), (resident, w)
        st = srv.stats()
        if resident:
            assert st["resident_live"] == 1
            assert st["resident_queries"] >= 2 * len(t) and st["resident_timeouts"] == 0
        else:
            assert st["resident_live"] == 0 and st["resident_queries"] == 0
        srv.close()
    fs.release()


def test_context_resident_queries_equal_launched_ones(hf):
    """hf_ctx_resident_queries: FieldSet.query through the resident query
    kernel gives the launched kernel's answers bit for bit; turning it off
    and on again (twice on is a no-op) keeps them."""
    import torch
    flags = hf.HF_E | hf.HF_F | hf.HF_T
    n, R = 64, 24
    ctx = hf.Context(0)
    p1, p2 = make_parts(hf, ctx, n, 43)
    q = synth.random_quaternions(103, R)
    fs = ctx.fieldset(n, R, flags)
    fs.compute(p1, p2, q)
    torch.cuda.synchronize()
    t, qq = _poses(9, 100)
    ks = [1 + (i % 8) for i in range(len(t))]

    def run():
        return np.stack([fs.query(t[i], qq[i], k=ks[i]) for i in range(len(t))])

    ref = run()
    ctx.resident_queries(True)
    ctx.resident_queries(True)
    assert np.array_equal(run(), ref)
    ctx.resident_queries(False)
    assert np.array_equal(run(), ref)
    ctx.resident_queries(True)
    assert np.array_equal(run(), ref)
    ctx.resident_queries(False)
    fs.release()
