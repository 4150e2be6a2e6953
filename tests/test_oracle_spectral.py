"""Pins of the oracle's frequency-domain rotation (Section 3.2, step 1:
interpolate the precomputed moving spectrum at R^T omega).

Checked against what the mathematics fixes, not against the oracle itself:
the spectrum of an origin-centred Gaussian is real and positive and an
offset one carries the phase exp(-2 pi i omega.c) (pins the centring and the
frequency scale omega = k'/(2 os)); zero padding samples the same continuous
transform at twice the rate; the identity and exact 90-degree rotations land
on table nodes, where interpolation is exact, so the rotated spectrum equals
the DFT of the exactly rotated grid; for a generic rotation the interpolated
spectrum converges to the DFT of the rotated density as the padding grows."""
import numpy as np
import pytest

import oracle

N = 16


def gaussian(n, c, sigma):
    return oracle.splat(n, np.asarray([c], dtype=np.float64), np.asarray([sigma], dtype=np.float64))


def nyquist_zeroed(b):
    b = b.copy()
    h = b.shape[0] // 2
    b[h, :, :] = 0
    b[:, h, :] = 0
    b[:, :, h] = 0
    return b


def rot_z90():
    return np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])


@pytest.mark.parametrize("os_", [1, 2])
def test_centred_gaussian_has_a_real_positive_table(os_):
    t = oracle.spectral_table(gaussian(N, (0.0, 0.0, 0.0), 0.12), os_)
    assert np.abs(t.imag).max() <= 1e-12 * np.abs(t).max()
    assert (t.real > 0).all()


def test_offset_gaussian_carries_the_translation_phase():
    # on nodes, so the sampled density is an exact shift; 6 sigma + |c| < 1,
    # so neither copy wraps around the period
    c = np.array([0.25, -0.125, 0.375])
    os_ = 2
    t0 = oracle.spectral_table(gaussian(N, (0.0, 0.0, 0.0), 0.08), os_)
    t = oracle.spectral_table(gaussian(N, c, 0.08), os_)
    k = np.fft.fftfreq(os_ * N, d=1.0 / (os_ * N))  # signed indices
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    omega = np.stack([kx, ky, kz], -1) / (2.0 * os_)
    phase = np.exp(-2j * np.pi * (omega @ c))
    assert np.abs(t - t0 * phase).max() <= 1e-10 * np.abs(t0).max()


def test_zero_padding_samples_the_same_transform():
    rng = np.random.default_rng(0)
    rho = rng.random((N, N, N))
    t1 = oracle.spectral_table(rho, 1)
    t2 = oracle.spectral_table(rho, 2)
    assert np.abs(t2[::2, ::2, ::2] - t1).max() <= 1e-11 * np.abs(t1).max()


@pytest.mark.parametrize("os_", [1, 2])
def test_identity_rotation_reproduces_the_dft(os_):
    rng = np.random.default_rng(1)
    rho = rng.random((N, N, N))
    b = oracle.spectral_rotate(oracle.spectral_table(rho, os_), N, np.eye(3), os_)
    ref = nyquist_zeroed(np.fft.fftn(rho))
    assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("os_", [1, 2])
def test_quarter_turn_equals_the_dft_of_the_turned_grid(os_):
    rng = np.random.default_rng(2)
    rho = rng.random((N, N, N))
    R = rot_z90()
    b = oracle.spectral_rotate(oracle.spectral_table(rho, os_), N, R, os_)
    ref = nyquist_zeroed(np.fft.fftn(oracle.resample(rho, R)))
    assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()


def test_generic_rotation_converges_with_padding():
    """An offset Gaussian rotated by a generic R: the interpolated spectrum
    approaches the DFT of the Gaussian placed at R c, faster with padding."""
    n = 32
    c = np.array([0.3, -0.1, 0.2])
    q = np.array([0.9, 0.2, -0.3, 0.25])
    R = oracle.quat_to_rot(q / np.linalg.norm(q))
    sig = 0.15
    ref = nyquist_zeroed(np.fft.fftn(gaussian(n, R @ c, sig)))
    errs = []
    for os_ in (1, 2, 4):
        b = oracle.spectral_rotate(oracle.spectral_table(gaussian(n, c, sig), os_), n, R, os_)
        errs.append(np.abs(b - ref).max() / np.abs(ref).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.25 * errs[0]


def test_fields_from_the_spectrum_match_the_grid_route():
    rng = np.random.default_rng(3)
    r1, r2 = rng.random((N, N, N)), rng.random((N, N, N))
    a = oracle.fields(r1, r2)
    b = oracle.fields_spec(r1, np.fft.fftn(r2))
    for f in range(4):
        assert np.abs(a[f] - b[f]).max() <= 1e-12 * np.abs(a[f]).max()
