"""Partition one rotation set over ranks with no exchange on the data path.

Rotations are the units of the field build: each one's energy and force
fields depend on that rotation alone.  The finite-difference torque of a
rotation also needs the energy fields of its 6 nearest sampled rotations
(geodesic angle, ties to the lower index).  So a rank that owns a cluster
of rotations also builds the nearest neighbours of its owned rotations that
another rank owns (a halo, recomputed redundantly).  Its torque for every
owned rotation is then the full set's, and no rank ever reads another's
fields.

  - clusters: balanced k-means on SO(3) (distance 1 - |q . c|, so that q and
    -q are the same rotation), deterministic from the input;
  - build set of a rank: its owned rotations and their `halo` nearest
    rotations (halo >= 6; the default 8 keeps a margin over the torque's 6
    so that a tie resolved differently by rounding cannot drop a neighbour),
    in global index order, so that a neighbour search inside the build set
    breaks ties exactly as one over the whole set;
  - queries: a pose blends the fields of its k nearest sampled rotations,
    torque included, so it is exact on a rank whose set of complete
    rotations holds all k: rotations whose 6 nearest are all in the rank's
    build set (the owned ones and part of the halo).  A pose goes to the
    owner of its nearest rotation when that rank qualifies, else to the
    first rank that does; when none does, the route says so (exact False)
    and the owner answers with its own nearest k.

This is host logic only (which rotations each rank builds); every field is
computed by the library's kernels on the rank's own GPU.
"""
import numpy as np


def _unit(quats):
    q = np.asarray(quats, dtype=np.float64).reshape(-1, 4)
    n = np.linalg.norm(q, axis=1, keepdims=True)
    if not np.all(n > 0):
        raise ValueError("a quaternion is zero")
    return q / n


def nearest(quats, k, q=None, skip_self=True):
    """Indices of the k nearest rotations of quats to each of q (default: to
    each rotation of quats, itself excluded), by geodesic angle, ties to the
    lower index.  (R or Q) x k int array."""
    Q = _unit(quats)
    P = Q if q is None else _unit(q)
    cos = np.abs(P @ Q.T)  # cos of half the geodesic angle: larger is nearer
    if q is None and skip_self:
        np.fill_diagonal(cos, -1.0)
    k = min(k, Q.shape[0] - (1 if (q is None and skip_self) else 0))
    # stable sort on -cos keeps equal angles in index order
    order = np.argsort(-cos, axis=1, kind="stable")
    return order[:, :k]


def cluster(quats, world, iters=8):
    """Balanced clusters of a rotation set: owner rank of every rotation
    (int array of R), each rank owning floor(R/world) or ceil(R/world)."""
    Q = _unit(quats)
    R = Q.shape[0]
    if world < 1 or world > R:
        raise ValueError(f"world={world} for {R} rotations")
    # farthest-point initial centres, from rotation 0
    centres = [0]
    dist = 1.0 - np.abs(Q @ Q[0])
    for _ in range(1, world):
        i = int(np.argmax(dist))
        centres.append(i)
        dist = np.minimum(dist, 1.0 - np.abs(Q @ Q[i]))
    C = Q[centres].copy()
    cap = -(-R // world)
    owner = np.zeros(R, dtype=np.int64)
    for _ in range(iters):
        d = 1.0 - np.abs(Q @ C.T)  # R x world
        # capacity-limited assignment: rotations in order of how strongly
        # they prefer their best centre take it while it has room
        best = np.argsort(d, axis=1, kind="stable")
        margin = np.take_along_axis(d, best[:, 1:2], 1)[:, 0] - d[np.arange(R), best[:, 0]] if world > 1 else np.zeros(R)
        load = np.zeros(world, dtype=np.int64)
        for i in np.argsort(-margin, kind="stable"):
            for c in best[i]:
                if load[c] < cap:
                    owner[i] = c
                    load[c] += 1
                    break
        # new centres: the principal eigenvector of each cluster's q q^T
        # (sign-free mean of unit quaternions)
        for c in range(world):
            M = Q[owner == c]
            w, v = np.linalg.eigh(M.T @ M)
            C[c] = v[:, -1]
    return owner


class Shard:
    """One rank's share of a rotation set.

    owned    -- global indices this rank reports (torque included), ascending
    build    -- global indices this rank builds fields for, ascending: owned
                plus the halo; its field set holds them in this order
    local    -- position in `build` of each owned rotation
    complete -- global indices in `build` whose 6 nearest are all in `build`
                (their torque is the whole set's), ascending
    """

    def __init__(self, owned, build, complete):
        self.owned = np.asarray(owned, dtype=np.int64)
        self.build = np.asarray(build, dtype=np.int64)
        self.complete = np.asarray(complete, dtype=np.int64)
        pos = {int(g): i for i, g in enumerate(self.build)}
        self.local = np.array([pos[int(g)] for g in self.owned], dtype=np.int64)


def shard(quats, world, halo=8):
    """Partition quats over `world` ranks: a list of Shard, one per rank."""
    if halo < 6:
        raise ValueError("the torque needs the 6 nearest rotations: halo >= 6")
    Q = _unit(quats)
    owner = cluster(Q, world)
    nb = nearest(Q, halo)
    out = []
    for r in range(world):
        owned = np.flatnonzero(owner == r)
        build = np.union1d(owned, nb[owned].ravel())
        complete = build[np.isin(nb[build, :6], build).all(axis=1)]
        out.append(Shard(owned, build, complete))
    return out


def route(quats, shards, q, k=4):
    """Rank for a pose query with rotation q blending k sampled rotations:
    (rank, exact).  exact is True when the k rotations the query blends over
    the whole set are complete rotations of that rank."""
    want = nearest(quats, k, q=np.asarray(q).reshape(1, 4), skip_self=False)[0]
    owner_of_nearest = next(r for r, s in enumerate(shards) if np.isin(want[0], s.owned))
    order = [owner_of_nearest] + [r for r in range(len(shards)) if r != owner_of_nearest]
    for r in order:
        if np.isin(want, shards[r].complete).all():
            return r, True
    return owner_of_nearest, False
