"""Pins of the oracle's single-pose evaluation with truncated spectra
(Section 4.2, "Truncated Inverse FFT"; Section 3.3, low-pass filtering).

With every non-Nyquist mode kept and a lattice translation, the one-point
sum is the inverse transform at that lattice point, so it must equal the
spectral-route field there (identity rotation, and an exact quarter turn).
With fewer modes and the identity, it equals numpy's transform of the
masked spectrum product.  Force and torque must be the derivatives of the
energy in translation and in world-frame rotation (central differences)."""
import numpy as np
import pytest

import oracle

N = 16


def rz90():
    return np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])


def rodrigues(w):
    th = np.linalg.norm(w)
    if th == 0:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx


@pytest.fixture(scope="module")
def dens():
    rng = np.random.default_rng(11)
    return rng.random((N, N, N)), rng.random((N, N, N))


@pytest.mark.parametrize("R", [np.eye(3), rz90()], ids=["identity", "quarter_turn"])
@pytest.mark.parametrize("os_", [1, 2])
def test_all_modes_at_lattice_points_equal_the_field(dens, R, os_):
    r1, r2 = dens
    T = oracle.spectral_table(r2, os_)
    ref = oracle.fields_spec(r1, oracle.spectral_rotate(T, N, R, os_))
    h = 2.0 / N
    for j in [(0, 0, 0), (3, 5, 14), (8, 1, 9)]:  # (jx, jy, jz)
        out = oracle.lowpass(r1, T, os_, N // 2 - 1, R, np.array(j) * h)
        for f in range(4):
            scale = np.abs(ref[f]).max()
            assert abs(out[f] - ref[f][j[2], j[1], j[0]]) <= 1e-11 * scale, (j, f)


def test_truncation_is_the_masked_transform(dens):
    r1, r2 = dens
    K = 3
    T = oracle.spectral_table(r2, 1)
    h = 2.0 / N
    A, B = np.fft.fftn(r1), np.fft.fftn(r2)
    k = np.fft.fftfreq(N, d=1.0 / N)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    mask = (np.abs(kx) <= K) & (np.abs(ky) <= K) & (np.abs(kz) <= K)
    E = np.real(np.fft.ifftn(np.where(mask, A * np.conj(B), 0))) * h**3
    for j in [(0, 0, 0), (2, 7, 11)]:
        out = oracle.lowpass(r1, T, 1, K, np.eye(3), np.array(j) * h)
        assert abs(out[0] - E[j[2], j[1], j[0]]) <= 1e-12 * np.abs(E).max()


def test_force_and_torque_are_the_derivatives(dens):
    r1, r2 = dens
    K, os_ = 3, 2
    T = oracle.spectral_table(r2, os_)
    rng = np.random.default_rng(5)
    for _ in range(3):
        q = rng.normal(size=4)
        R = oracle.quat_to_rot(q / np.linalg.norm(q))
        t = rng.uniform(-1, 1, 3)
        out = oracle.lowpass(r1, T, os_, K, R, t)
        dt = 1e-6
        for d in range(3):
            e = np.zeros(3)
            e[d] = dt
            g = (oracle.lowpass(r1, T, os_, K, R, t + e)[0] - oracle.lowpass(r1, T, os_, K, R, t - e)[0]) / (2 * dt)
            assert abs(out[1 + d] + g) <= 1e-6 * (abs(g) + np.abs(out[1:4]).max())
        dth = 1e-7
        for a in range(3):
            w = np.zeros(3)
            w[a] = dth
            Ep = oracle.lowpass(r1, T, os_, K, rodrigues(w) @ R, t)[0]
            Em = oracle.lowpass(r1, T, os_, K, rodrigues(-w) @ R, t)[0]
            g = (Ep - Em) / (2 * dth)
            assert abs(out[4 + a] + g) <= 1e-5 * (abs(g) + np.abs(out[4:7]).max())
