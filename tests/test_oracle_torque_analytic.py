"""Pins of the oracle's analytic torque field (the rotational gradient of
Eq. 6b, moment moved onto the stationary part by integration by parts).

Two isotropic Gaussians give a closed form: with S = s1^2 + s2^2 and
d = c1 - R c2 - t, E = A exp(-|d|^2 / 2S) and the world-frame rotational
derivative about the moving part's reference point is
T = -dE/dtheta = -(E / S) (R c2) x d.  Compared at every lag where the
periodic images do not reach (|t| <= 0.5 per axis)."""
import numpy as np
import pytest

import oracle


def closed_form(n, c1, c2, s1, s2, R):
    h = 2.0 / n
    S = s1 * s1 + s2 * s2
    pref = (2 * np.pi * s1 * s1 * s2 * s2 / S) ** 1.5
    j = np.fft.fftfreq(n, d=1.0 / n)
    tz, ty, tx = np.meshgrid(j * h, j * h, j * h, indexing="ij")
    t = np.stack([tx, ty, tz], -1)
    d = c1 - R @ c2 - t
    E = pref * np.exp(-(d ** 2).sum(-1) / (2 * S))
    T = -(E / S)[..., None] * np.cross(R @ c2, d)
    near = (np.abs(t) <= 0.5 + 1e-12).all(-1)
    return E, T, near


@pytest.mark.parametrize("n,q", [(32, (0.9, 0.2, -0.3, 0.25)), (48, (0.3, -0.7, 0.5, 0.4))])
def test_gaussian_pair_torque_matches_the_closed_form(n, q):
    c1 = np.array([0.1, -0.05, 0.2])
    c2 = np.array([0.15, 0.1, -0.1])
    s1, s2 = 0.12, 0.1
    q = np.asarray(q) / np.linalg.norm(q)
    R = oracle.quat_to_rot(q)
    r1 = oracle.splat(n, c1[None], np.array([s1]))
    r2r = oracle.splat(n, (R @ c2)[None], np.array([s2]))  # isotropic: rotating the density moves its centre
    T = np.stack(oracle.torque_analytic(r1, r2r), -1)
    E, Tc, near = closed_form(n, c1, c2, s1, s2, R)
    scale = np.abs(Tc[near]).max()
    assert np.abs(T[near] - Tc[near]).max() <= 1e-5 * scale


def test_torque_vanishes_for_centred_isotropic_pair():
    """Two Gaussians centred at the origins of their parts: rotating the
    moving part about its own centre changes nothing, so T = 0 at every lag
    the periodic images do not reach."""
    n = 32
    r1 = oracle.splat(n, np.array([[0.2, -0.1, 0.05]]), np.array([0.1]))
    r2 = oracle.splat(n, np.zeros((1, 3)), np.array([0.12]))
    T = np.stack(oracle.torque_analytic(r1, r2), -1)
    E = oracle.fields(r1, r2)[0]
    _, _, near = closed_form(n, np.zeros(3), np.zeros(3), 0.1, 0.12, np.eye(3))
    assert np.abs(T[near]).max() <= 1e-7 * np.abs(E).max()
