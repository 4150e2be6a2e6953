"""Pins of the oracle's torque (least-squares finite differences across the
nearest sampled rotations, standing in for Eq. 6b) and of its pose query
(restricted-orientation mode, Section 4.2) against scipy's independent
rotation routines, exactly linear fields, the analytic torque of a Gaussian
pair, and the exactness / linear precision of trilinear interpolation."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import synth


def sp_rot(q):
    return Rotation.from_quat([q[1], q[2], q[3], q[0]])


def test_so3_log_vs_scipy():
    for q in synth.random_quaternions(11, 50):
        R = sp_rot(q)
        if R.magnitude() > np.pi - 1e-3:
            continue
        assert np.abs(oracle.so3_log(R.as_matrix()) - R.as_rotvec()).max() <= 1e-10


def test_so3_log_near_identity_and_near_pi():
    v = np.array([1e-9, -2e-9, 3e-9])
    assert np.abs(oracle.so3_log(Rotation.from_rotvec(v).as_matrix()) - v).max() <= 1e-15
    ax = np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])
    v = (np.pi - 1e-8) * ax
    got = oracle.so3_log(Rotation.from_rotvec(v).as_matrix())
    assert min(np.abs(got - v).max(), np.abs(got + v).max()) <= 1e-6


def test_nearest_vs_scipy_angles():
    Q = synth.random_quaternions(3, 200)
    rots = [sp_rot(q) for q in Q]
    for i in (0, 17, 199):
        ang = np.array([(rots[j] * rots[i].inv()).magnitude() for j in range(len(Q))])
        ang[i] = np.inf
        ref = np.argsort(ang, kind="stable")[:6]
        idx, a = oracle.nearest(Q, Q[i], 6, skip=i)
        assert list(idx) == list(ref)
        assert np.abs(a - ang[ref]).max() <= 1e-7


def test_torque_exact_on_fields_linear_in_the_log_map():
    """E_j = c + g . Log(R_j R_0^T) makes the least-squares gradient at
    rotation 0 exact, so T_0 = -g to rounding (pins the Log map, the normal
    equations, the neighbour set and the sign)."""
    n = 4
    rng = np.random.default_rng(1)
    Q = synth.random_quaternions(21, 40)
    c = rng.standard_normal((n, n, n))
    g = rng.standard_normal((3, n, n, n))
    r0 = sp_rot(Q[0])
    E = np.stack([c + np.einsum("a,azyx->zyx", (sp_rot(q) * r0.inv()).as_rotvec(), g) for q in Q])
    T, st = oracle.torque(Q, E, 6)
    assert st[0] == 0
    assert np.abs(T[0] + g).max() <= 1e-9 * np.abs(g).max()


def test_torque_rank_deficient_neighbourhood_is_flagged():
    """All rotations about one axis: the 6 x 3 difference matrix has rank 1."""
    n = 4
    angs = [0.0, 0.1, -0.1, 0.2, -0.2, 0.3, -0.3]
    Q = np.array([[np.cos(a / 2), 0, 0, np.sin(a / 2)] for a in angs])
    E = np.random.default_rng(2).standard_normal((len(Q), n, n, n))
    T, st = oracle.torque(Q, E, 6)
    assert st[0] == 1 and np.isnan(T[0]).all()


def test_torque_matches_analytic_gaussian_torque():
    """Two Gaussians, the moving one off its reference point: with the 6
    neighbours at +-delta about each axis the least-squares gradient is a
    central difference (O(delta^2)); E(R, t) = A exp(-|c1 - R c2 - t|^2/2S)
    gives T = -E (R c2 x d) / S, d = c1 - R c2 - t.  Trilinear resampling
    (sigma = 6h) adds an error well below the 5% allowed on strong cells."""
    n = 48
    h = 2.0 / n
    s1 = s2 = 6 * h
    c1 = np.array([0.25, 0.0, 0.1])
    c2 = np.array([0.3, 0.05, -0.1])
    d = 0.03
    qs = [np.array([1.0, 0, 0, 0])]
    for ax in range(3):
        for sgn in (1, -1):
            v = np.zeros(3)
            v[ax] = sgn * d
            r = Rotation.from_rotvec(v).as_quat()
            qs.append(np.array([r[3], r[0], r[1], r[2]]))
    Q = np.stack(qs)
    r1 = oracle.splat(n, c1[None], np.array([s1]))
    r2 = oracle.splat(n, c2[None], np.array([s2]))
    E = np.stack([oracle.fields(r1, oracle.resample(r2, oracle.quat_to_rot(q)))[0] for q in Q])
    T, st = oracle.torque(Q, E, 6)
    assert st[0] == 0
    S = s1**2 + s2**2
    pref = (2 * np.pi * s1**2 * s2**2 / S) ** 1.5
    j = np.arange(n)
    z, y, x = np.meshgrid(j, j, j, indexing="ij")
    t = np.stack([x, y, z], -1) * h
    t = np.where(t >= 1.0, t - 2.0, t)  # wrapped lags
    dd = c1 - c2 - t
    Ea = pref * np.exp(-(dd**2).sum(-1) / (2 * S))
    Ta = -Ea[..., None] * np.cross(c2, dd) / S
    mag = np.linalg.norm(Ta, axis=-1)
    strong = mag > 0.5 * mag.max()
    Tg = np.moveaxis(T[0], 0, -1)
    err = np.linalg.norm(Tg - Ta, axis=-1)[strong].max()
    assert err <= 0.05 * mag.max()


def _fields_for_query(nrot, nf, n, seed):
    return np.random.default_rng(seed).standard_normal((nrot, nf, n, n, n))


def test_query_exact_at_nodes_and_member_rotations():
    n = 8
    h = 2.0 / n
    Q = synth.random_quaternions(31, 12)
    Fd = _fields_for_query(len(Q), 7, n, 4)
    for i, jx, jy, jz in [(0, 0, 0, 0), (5, 3, 7, 1), (11, 6, 2, 5)]:
        out = oracle.query(Q, Fd, np.array([jx, jy, jz]) * h, Q[i], k=4)
        assert np.abs(out - Fd[i, :, jz, jy, jx]).max() <= 1e-12
    # a lag beyond the box wraps periodically
    out = oracle.query(Q, Fd, np.array([n + 1, -1, 2 * n + 3]) * h, Q[2], k=4)
    assert np.abs(out - Fd[2, :, 3, n - 1, 1]).max() <= 1e-12


def test_query_reproduces_affine_fields():
    """Trilinear interpolation has linear precision; rotation weights sum to 1."""
    n = 8
    h = 2.0 / n
    Q = synth.random_quaternions(32, 10)
    j = np.arange(n, dtype=float)
    z, y, x = np.meshgrid(j, j, j, indexing="ij")
    Fd = np.empty((len(Q), 2, n, n, n))
    for r in range(len(Q)):
        Fd[r, 0] = 1.5 + 0.25 * x - 0.5 * y + 0.125 * z
        Fd[r, 1] = -2.0 + x + y + z
    rng = np.random.default_rng(9)
    for _ in range(10):
        u = rng.uniform(0.5, n - 1.5, 3)
        q = synth.random_quaternions(int(rng.integers(1000)), 1)[0]
        out = oracle.query(Q, Fd, u * h, q, k=4)
        assert abs(out[0] - (1.5 + 0.25 * u[0] - 0.5 * u[1] + 0.125 * u[2])) <= 1e-12
        assert abs(out[1] - (-2.0 + u.sum())) <= 1e-12


def test_query_rotation_weights_inverse_angle():
    """Per-rotation constant fields expose the blend: sum_j w_j v_j with
    w_j proportional to 1/theta_j over the k nearest (scipy angles)."""
    n = 4
    Q = synth.random_quaternions(33, 30)
    vals = np.arange(len(Q), dtype=float) * 1.7 - 3.0
    Fd = np.broadcast_to(vals[:, None, None, None, None], (len(Q), 1, n, n, n)).copy()
    q = synth.random_quaternions(34, 1)[0]
    ang = np.array([(sp_rot(p) * sp_rot(q).inv()).magnitude() for p in Q])
    for k in (1, 4, 6):
        sel = np.argsort(ang, kind="stable")[:k]
        w = 1 / ang[sel]
        w /= w.sum()
        out = oracle.query(Q, Fd, np.array([0.1, 0.2, -0.3]), q, k=k)
        assert abs(out[0] - (w * vals[sel]).sum()) <= 1e-9
