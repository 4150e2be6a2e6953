"""Pins of the oracle's own DFT (Eqs. 7a/7b, Section 3.2) against the brute
force sum and against numpy's pocketfft, an independent library."""
import numpy as np
import pytest

import oracle


def brute_dft(x, sign):
    n = len(x)
    k = np.arange(n)
    W = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
    return W @ x


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft1d_vs_brute_force(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    got = oracle.fft1d(x, sign)
    ref = brute_dft(x, sign)
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("n", [32, 64, 96, 128, 256])
def test_fft1d_vs_numpy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(oracle.fft1d(x, -1), np.fft.fft(x), rtol=0, atol=1e-12 * np.sqrt(n) * 4)
    assert np.allclose(oracle.fft1d(x, +1), n * np.fft.ifft(x), rtol=0, atol=1e-12 * np.sqrt(n) * 4)


@pytest.mark.parametrize("n", [6, 8, 12, 16])
def test_fft3d_vs_numpy(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    F = oracle.fft3d(x, -1)
    ref = np.fft.fftn(x)
    assert np.abs(F - ref).max() <= 1e-12 * np.abs(ref).max()
    B = oracle.fft3d(F, +1) / n**3
    assert np.abs(B - x).max() <= 1e-12


def test_parseval():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((16, 16, 16))
    X = oracle.fft3d(x, -1)
    assert abs((np.abs(x) ** 2).sum() - (np.abs(X) ** 2).sum() / 16**3) <= 1e-10 * (x**2).sum()


def test_real_input_is_hermitian():
    rng = np.random.default_rng(8)
    n = 8
    x = rng.standard_normal((n, n, n))
    X = oracle.fft3d(x, -1)
    neg = (-np.arange(n)) % n
    Xm = X[np.ix_(neg, neg, neg)]
    assert np.abs(X - np.conj(Xm)).max() <= 1e-12 * np.abs(X).max()
