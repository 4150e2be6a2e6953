"""Skeleton-sample generators for the synthetic workloads.

All positions live in the periodic box [-1, 1)^3.  A part is P points with
centre (x, y, z), ball radius sigma and amplitude a (1 unless stated).

Workloads (sizes, counts and distributions of the benchmark configurations):

  c1  32^3, identity rotation: ring of 200 points (radius 0.4, plane z = 0)
      against a peg of 200 points on the z-axis segment [-0.4, 0.4];
      radii U(0.05, 0.15).
  c2  128^3, 1024 random rotations: a "hole" of 5000 points on 3 coaxial
      rings (r = 0.30, 0.30, 0.45 at z = -0.3, +0.3, 0) and 2 square sheets
      (side 0.9, z = +-0.45); a "peg" of 5000 points on 2 axis segments
      (x = -0.1, z in [-0.4, 0]; x = +0.1, z in [0.05, 0.4]) and 1 ring
      (r = 0.25, z = 0); radii U(0.02, 0.08).
  c3  64 pairs with N from {64: 24, 96: 24, 128: 16} (shuffled), 1000-8000
      points per part of the same primitive mix, parameters jittered +-10%,
      256 rotations per pair.
  c4  256^3, 20000 points per part (rings, segments, sheets),
      radii U(0.01, 0.05), 512 rotations.
  c5  16 serving sessions, N uniform over {64, 128, 256}, Poisson build
      requests (2/s per session, 64-512 rotations), 1 kHz pose random walks.

Points are split over primitives in proportion to their measure (length for
curves, area for sheets); the rounding remainder goes to the first primitive.
Random rotations: 4 standard normals from numpy's PCG64, normalised, sign
chosen so that w >= 0.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class Part:
    pts: np.ndarray  # (P, 3) float64
    sigma: np.ndarray  # (P,) float64
    amp: np.ndarray = field(default=None)  # (P,) float64 or None (= 1)

    @property
    def n_points(self) -> int:
        return len(self.sigma)


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def ring(rng, n, radius, z=0.0, center=(0.0, 0.0)):
    """n points uniform in angle on a circle of the given radius in plane z."""
    th = rng.uniform(0.0, 2.0 * np.pi, n)
    return np.stack([center[0] + radius * np.cos(th), center[1] + radius * np.sin(th),
                     np.full(n, z)], axis=1)


def segment(rng, n, a, b):
    """n points uniform on the straight segment from a to b."""
    s = rng.uniform(0.0, 1.0, n)[:, None]
    a, b = np.asarray(a, float), np.asarray(b, float)
    return a[None, :] + s * (b - a)[None, :]


def sheet(rng, n, side, z):
    """n points uniform on an axis-aligned square of the given side, plane z."""
    xy = rng.uniform(-side / 2, side / 2, (n, 2))
    return np.concatenate([xy, np.full((n, 1), z)], axis=1)


def _split(total, measures):
    w = np.asarray(measures, float)
    cnt = np.floor(total * w / w.sum()).astype(int)
    cnt[0] += total - cnt.sum()
    return cnt


def _primitive_points(rng, total, prims):
    """prims: list of (kind, params, measure)."""
    counts = _split(total, [p[2] for p in prims])
    out = []
    for (kind, par, _), c in zip(prims, counts):
        if kind == "ring":
            out.append(ring(rng, c, par["r"], par["z"]))
        elif kind == "segment":
            out.append(segment(rng, c, par["a"], par["b"]))
        elif kind == "sheet":
            out.append(sheet(rng, c, par["side"], par["z"]))
    return np.concatenate(out, axis=0)


def _hole_prims(j=None):
    """3 coaxial rings + 2 sheets; j(x) jitters a parameter (identity if None)."""
    j = j or (lambda x: x)
    prims = []
    for r, z in ((0.30, -0.3), (0.30, 0.3), (0.45, 0.0)):
        r, z = j(r), j(z)
        prims.append(("ring", {"r": r, "z": z}, 2 * np.pi * r))
    for z in (-0.45, 0.45):
        s, z = j(0.9), j(z)
        prims.append(("sheet", {"side": s, "z": z}, s * s))
    return prims


def _peg_prims(j=None):
    """2 axis segments + 1 ring."""
    j = j or (lambda x: x)
    xa, xb = j(-0.1), j(0.1)
    za0, za1, zb0, zb1 = j(-0.4), j(0.0), j(0.05), j(0.4)
    r = j(0.25)
    return [
        ("segment", {"a": (xa, 0.0, za0), "b": (xa, 0.0, za1)}, abs(za1 - za0)),
        ("segment", {"a": (xb, 0.0, zb0), "b": (xb, 0.0, zb1)}, abs(zb1 - zb0)),
        ("ring", {"r": r, "z": 0.0}, 2 * np.pi * r),
    ]


def mixed_part(rng, n_points, kind, rmin, rmax, jitter=0.0):
    """A hole-like ('hole') or peg-like ('peg') part, optionally with every
    primitive parameter jittered by a uniform factor in [1-jitter, 1+jitter]."""
    j = None
    if jitter:
        j = lambda x: x * rng.uniform(1 - jitter, 1 + jitter)  # noqa: E731
    prims = _hole_prims(j) if kind == "hole" else _peg_prims(j)
    pts = _primitive_points(rng, n_points, prims)
    sigma = rng.uniform(rmin, rmax, n_points)
    return Part(pts, sigma)


def random_quaternions(seed, count):
    """Uniform random unit quaternions (w, x, y, z), w >= 0."""
    g = _rng(seed)
    q = g.standard_normal((count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q[q[:, 0] < 0] *= -1.0
    return q


def c1_pair(seed=0):
    """Ring (stationary) and straight peg (moving), 200 points each, 32^3."""
    g = _rng(seed)
    s1 = Part(ring(g, 200, 0.4, 0.0), g.uniform(0.05, 0.15, 200))
    s2 = Part(segment(g, 200, (0, 0, -0.4), (0, 0, 0.4)), g.uniform(0.05, 0.15, 200))
    return s1, s2


def c2_pair(seed=0):
    """Hole (3 rings + 2 sheets) and peg (2 segments + ring), 5000 points each."""
    g = _rng(seed)
    s1 = mixed_part(g, 5000, "hole", 0.02, 0.08)
    s2 = mixed_part(g, 5000, "peg", 0.02, 0.08)
    return s1, s2


def c4_pair(seed=0):
    """20000 points per part, radii U(0.01, 0.05): rings, segments and sheets."""
    g = _rng(seed)
    s1 = mixed_part(g, 20000, "hole", 0.01, 0.05)
    s2 = mixed_part(g, 20000, "peg", 0.01, 0.05)
    return s1, s2


@dataclass
class PairSpec:
    n: int
    s1: Part
    s2: Part
    quat_seed: int
    n_rot: int


def c3_pairs(seed=0, n_rot=256, sizes=((64, 24), (96, 24), (128, 16))) -> List[PairSpec]:
    """Uneven batch: grid sizes in the stated counts, order shuffled by seed."""
    g = _rng(seed)
    ns = np.concatenate([np.full(c, n) for n, c in sizes])
    g.shuffle(ns)
    out = []
    for i, n in enumerate(ns):
        p1, p2 = g.integers(1000, 8001, 2)
        s1 = mixed_part(g, int(p1), "hole", 0.02, 0.08, jitter=0.1)
        s2 = mixed_part(g, int(p2), "peg", 0.02, 0.08, jitter=0.1)
        out.append(PairSpec(int(n), s1, s2, quat_seed=seed * 1000 + i + 1, n_rot=n_rot))
    return out


@dataclass
class Session:
    n: int
    s1: Part
    s2: Part
    arrivals: np.ndarray  # request times, seconds
    n_rot: np.ndarray  # rotations per request
    quat_seeds: np.ndarray


def c5_sessions(seed=0, n_sessions=16, duration_s=60.0, rate_hz=2.0,
                sizes=(64, 128, 256), rot_range=(64, 512)) -> List[Session]:
    """Serving workload: per session a grid size, a part pair and a Poisson
    stream of field-build requests."""
    g = _rng(seed)
    out = []
    for s in range(n_sessions):
        n = int(g.choice(sizes))
        rmin, rmax = (0.01, 0.05) if n == 256 else (0.02, 0.08)
        p1, p2 = g.integers(1000, 8001, 2)
        s1 = mixed_part(g, int(p1), "hole", rmin, rmax, jitter=0.1)
        s2 = mixed_part(g, int(p2), "peg", rmin, rmax, jitter=0.1)
        gaps = g.exponential(1.0 / rate_hz, int(duration_s * rate_hz * 3) + 8)
        t = np.cumsum(gaps)
        t = t[t < duration_s]
        nr = g.integers(rot_range[0], rot_range[1] + 1, len(t))
        qs = g.integers(0, 2**31 - 1, len(t))
        out.append(Session(n, s1, s2, t, nr, qs))
    return out


def translation_walk(seed, steps, step_sigma=0.002, start=None):
    """Random-walk translations (one step per ms), wrapped to [-1, 1)."""
    g = _rng(seed)
    t0 = np.zeros(3) if start is None else np.asarray(start, float)
    t = t0 + np.cumsum(g.normal(0.0, step_sigma, (steps, 3)), axis=0)
    return (t + 1.0) % 2.0 - 1.0


def quaternion_walk(seed, steps, step_sigma=0.002, start=None):
    """Random-walk orientations, one step per ms: axis-angle increments with
    N(0, step_sigma^2) components, accumulated; the orientation at step k is
    exp(sum of increments) applied on the left of the start orientation."""
    g = _rng(seed)
    v = np.cumsum(g.normal(0.0, step_sigma, (steps, 3)), axis=0)
    th = np.linalg.norm(v, axis=1, keepdims=True)
    safe = np.where(th > 0, th, 1.0)
    dq = np.concatenate([np.cos(th / 2), np.sin(th / 2) * v / safe], axis=1)
    q0 = np.array([1.0, 0, 0, 0]) if start is None else np.asarray(start, float)
    w1, x1, y1, z1 = dq.T
    w2, x2, y2, z2 = q0
    q = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                  w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                  w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                  w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=1)
    return q / np.linalg.norm(q, axis=1, keepdims=True)
