"""Pins of the oracle's mesh descriptor (Eq. 2 on closed triangle meshes).

Against what geometry fixes: the winding number of a closed mesh is exactly
1 inside and 0 outside (checked against exact box and polygonal-prism
inclusion); the signed distance to an axis-aligned box has a closed form;
as sigma grows the Gaussian weight tends to 1 and, solid angles being
additive over any subdivision, the descriptor becomes the winding number
(the indicator, Section 2.3); the skeletal density of a cube peaks at its
centre (the medial axis meets there); the adaptive Riemann sum converges
as the solid-angle threshold shrinks."""
import numpy as np
import pytest

import oracle
import synth

N = 16
H = 2.0 / N


def node_grid(n):
    c = -1.0 + np.arange(n) * (2.0 / n)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([x, y, z], -1)


def box_mesh():
    lo, hi = np.full(3, -0.3 + H / 4), np.full(3, 0.3 + H / 4)  # faces between nodes
    return synth.box(lo, hi), lo, hi


def test_winding_number_and_distance_of_a_box():
    (V, T), lo, hi = box_mesh()
    W, XI, _ = oracle.mesh_sdf(N, V, T, 0.5, 0.05, 8)
    p = node_grid(N)
    inside = ((p > lo) & (p < hi)).all(-1)
    assert np.abs(W - inside).max() <= 1e-12
    out = np.linalg.norm(np.maximum(np.maximum(lo - p, p - hi), 0.0), axis=-1)
    inn = np.minimum(p - lo, hi - p).min(-1)
    ref = np.where(inside, -inn, out)
    assert np.abs(XI - ref).max() <= 1e-12


def test_winding_number_of_a_polygonal_peg_and_tube():
    n = 24
    p = node_grid(n)
    seg, r, z0, z1 = 16, 0.43, -0.52, 0.47
    V, T = synth.cylinder(r, z0, z1, seg)
    W = oracle.mesh_sdf(n, V, T, 0.5, 0.05, 6)[0]
    # inside the convex polygon of the cross-section: on the inner side of every edge
    th = 2 * np.pi * np.arange(seg) / seg
    P = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    inside_poly = np.ones(p.shape[:3], bool)
    for i in range(seg):
        a, b = P[i], P[(i + 1) % seg]
        e = b - a
        inside_poly &= (e[0] * (p[..., 1] - a[1]) - e[1] * (p[..., 0] - a[0])) > 0
    inside = inside_poly & (p[..., 2] > z0) & (p[..., 2] < z1)
    assert np.abs(W - inside).max() <= 1e-10
    Vt, Tt = synth.tube(0.21, 0.52, -0.33, 0.33, 16)
    Wt = oracle.mesh_sdf(n, Vt, Tt, 0.5, 0.05, 6)[0]
    assert np.abs(Wt * (1 - Wt)).max() <= 1e-10  # 0 or 1 everywhere
    assert Wt[n // 2, n // 2, n // 2] < 0.5        # the hole's axis is outside the part


def test_large_sigma_gives_the_indicator():
    (V, T), _, _ = box_mesh()
    W, _, RHO = oracle.mesh_sdf(N, V, T, 1e9, 0.05, 8)
    assert np.abs(RHO - W).max() <= 1e-12


def test_skeletal_density_peaks_at_the_cube_centre():
    n = 16
    V, T = synth.box(np.full(3, -0.375), np.full(3, 0.375))  # centred on node n/2, faces between nodes
    W, _, RHO = oracle.mesh_sdf(n, V, T, 0.5, 0.02, 10)
    k = np.unravel_index(np.argmax(np.where(W > 0.5, RHO, -np.inf)), RHO.shape)
    assert k == (n // 2, n // 2, n // 2)
    assert RHO[k] > 0 and RHO.min() < 0  # positive inside, negative outside


def test_subdivision_converges():
    (V, T), _, _ = box_mesh()
    coarse = oracle.mesh_sdf(N, V, T, 0.5, 0.02, 10)[2]
    fine = oracle.mesh_sdf(N, V, T, 0.5, 0.005, 12)[2]
    assert np.abs(coarse - fine).max() <= 5e-3 * np.abs(fine).max()
