"""Procedural closed triangle meshes standing in for the paper's CAD parts
(its Fig. 4 zero-clearance peg and hole): a box, a capped cylinder (peg)
and a tube (a block's cylindrical hole: outer wall, inner wall, two annular
caps).  Every mesh is closed and oriented with outward normals
(counter-clockwise seen from outside).  Vertices float64 (V, 3), triangles
int32 (T, 3).  No arithmetic of the method lives here."""
import numpy as np


def box(lo, hi):
    """Axis-aligned box [lo, hi] as 12 triangles."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    V = np.array([[x, y, z] for z in (lo[2], hi[2]) for y in (lo[1], hi[1]) for x in (lo[0], hi[0])])
    # vertex index = x + 2 y + 4 z (bits)
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    T = []
    for a, b, c, d in quads:
        T += [(a, b, c), (a, c, d)]
    return V, np.asarray(T, dtype=np.int32)


def _ring(r, z, seg, phase=0.0):
    th = 2 * np.pi * (np.arange(seg) + phase) / seg
    return np.stack([r * np.cos(th), r * np.sin(th), np.full(seg, z)], 1)


def cylinder(r, z0, z1, seg=24, center=(0.0, 0.0)):
    """Capped cylinder of radius r along z in [z0, z1] (a peg)."""
    c = np.array([center[0], center[1], 0.0])
    bot, top = _ring(r, z0, seg) + c, _ring(r, z1, seg) + c
    V = np.concatenate([bot, top, [[c[0], c[1], z0], [c[0], c[1], z1]]])
    cb, ct = 2 * seg, 2 * seg + 1
    T = []
    for i in range(seg):
        j = (i + 1) % seg
        T += [(i, j, seg + j), (i, seg + j, seg + i)]  # side, outward
        T += [(cb, j, i)]                              # bottom cap, normal -z
        T += [(ct, seg + i, seg + j)]                  # top cap, normal +z
    return V, np.asarray(T, dtype=np.int32)


def tube(r_in, r_out, z0, z1, seg=24, center=(0.0, 0.0)):
    """Thick-walled tube (a hole of radius r_in through a round block of
    radius r_out) along z in [z0, z1]."""
    c = np.array([center[0], center[1], 0.0])
    ob, ot = _ring(r_out, z0, seg) + c, _ring(r_out, z1, seg) + c
    ib, it = _ring(r_in, z0, seg) + c, _ring(r_in, z1, seg) + c
    V = np.concatenate([ob, ot, ib, it])
    OB, OT, IB, IT = 0, seg, 2 * seg, 3 * seg
    T = []
    for i in range(seg):
        j = (i + 1) % seg
        T += [(OB + i, OB + j, OT + j), (OB + i, OT + j, OT + i)]  # outer wall, normal outward
        T += [(IB + i, IT + j, IB + j), (IB + i, IT + i, IT + j)]  # inner wall, normal toward the axis
        T += [(OB + i, IB + j, OB + j), (OB + i, IB + i, IB + j)]  # bottom annulus, normal -z
        T += [(OT + i, OT + j, IT + j), (OT + i, IT + j, IT + i)]  # top annulus, normal +z
    return V, np.asarray(T, dtype=np.int32)


def peg_hole_pair(seg=32):
    """A round peg and a block with a matching round hole (small clearance),
    the peg's axis along z, both centred at the origin of their frames."""
    hole = tube(0.21, 0.52, -0.33, 0.33, seg)
    peg = cylinder(0.19, -0.43, 0.43, seg)
    return hole, peg
