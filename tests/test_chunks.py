"""Host logic of the serving runtime's rotation-set chunking
(hf_rotation_chunks, no GPU): every rotation is owned once, build sets
respect the limit and are in ascending global order, and -- checked with the
oracle's own nearest-rotation search -- each owned rotation's 6 nearest
within its chunk's build set are its 6 nearest in the whole set, so the
least-squares torque (Section 2.4's rotational gradient by finite
differences) that a chunk computes equals the whole set's; and on a tiny
case with fields linear in the log map, the oracle's torque of each chunk
equals the whole set's, exactly."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def hf():
    from paper_1711_05017_b300 import build
    build.build()
    import paper_1711_05017_b300 as hf_
    return hf_


@pytest.mark.parametrize("R,max_build", [(64, 24), (200, 40), (512, 90), (512, 7)])
def test_chunks_cover_and_keep_torque_neighbours(hf, R, max_build):
    q = synth.random_quaternions(100 + R, R).astype(np.float32)
    owner, builds = hf.rotation_chunks(q, max_build)
    qd = q.astype(np.float64)
    qd /= np.linalg.norm(qd, axis=1, keepdims=True)
    assert owner.shape == (R,) and owner.min() == 0 and owner.max() == len(builds) - 1
    for c, b in enumerate(builds):
        assert len(b) <= max_build
        assert np.all(np.diff(b) > 0)  # ascending global order
        owned = np.flatnonzero(owner == c)
        assert len(owned) >= 1 and np.isin(owned, b).all()
        for i in owned:
            glob, _ = oracle.nearest(qd, qd[i], 6, skip=int(i))
            assert np.isin(glob, b).all(), (c, i)
            li = int(np.searchsorted(b, i))
            loc, _ = oracle.nearest(qd[b], qd[i], 6, skip=li)
            assert np.array_equal(b[loc], glob), (c, i)


def test_chunks_without_halo_partition_the_set(hf):
    R = 100
    q = synth.random_quaternions(7, R).astype(np.float32)
    owner, builds = hf.rotation_chunks(q, 16, halo=False)
    allm = np.concatenate(builds)
    assert np.array_equal(np.sort(allm), np.arange(R))
    for c, b in enumerate(builds):
        assert np.array_equal(np.flatnonzero(owner == c), b)


def test_chunked_oracle_torque_equals_whole_set(hf):
    """Fields E_r = a . Log(R_r) + b on a 2^3 grid: the oracle's torque of each
    owned rotation, computed from its chunk's build set alone, is the whole
    set's, bit for bit (same neighbours, same order)."""
    R, n = 60, 2
    q = synth.random_quaternions(11, R).astype(np.float32)
    qd = q.astype(np.float64)
    qd /= np.linalg.norm(qd, axis=1, keepdims=True)
    rng = np.random.default_rng(3)
    a, b0 = rng.standard_normal((n, n, n, 3)), rng.standard_normal((n, n, n))
    logs = np.stack([oracle.so3_log(oracle.quat_to_rot(x)) for x in qd])
    E = np.einsum("zyxa,ra->rzyx", a, logs) + b0
    T, st = oracle.torque(qd, E, 6)
    owner, builds = hf.rotation_chunks(q, 20)
    assert len(builds) > 1
    for c, bset in enumerate(builds):
        Tc, stc = oracle.torque(qd[bset], E[bset], 6)
        for m, g in enumerate(bset):
            if owner[g] == c:
                assert stc[m] == st[g]
                assert np.array_equal(Tc[m], T[g]), (c, g)


def test_chunk_errors(hf):
    q = synth.random_quaternions(1, 10).astype(np.float32)
    with pytest.raises(hf.HFError):
        hf.rotation_chunks(q, 6)  # a torque halo needs 7 rotations per build
    with pytest.raises(hf.HFError):
        hf.rotation_chunks(q[:5], 10)  # fewer than 7 rotations cannot carry a torque
    bad = q.copy()
    bad[3] = 0
    with pytest.raises(hf.HFError):
        hf.rotation_chunks(bad, 10)
