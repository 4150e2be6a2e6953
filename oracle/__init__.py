"""FP64 CPU oracle for the skeletal-density energy / force / torque fields.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the package smoke
check and by the benchmark's CPU-baseline leg, never by the product path.
It shares no code with the CUDA library; the only module both sides use is
the seeded input generator package ``synth``.

Each function wraps one routine of ``hf_oracle.c`` (plain C, double
precision) and cites the passage of Behandish & Ilies (2016) it follows.
Arrays are numpy float64, grids are (N, N, N) indexed [z, y, x].

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (brute force, closed forms, numpy's
pocketfft, scipy's rotation routines, exact invariants); see tests/.
"""
import ctypes
import os

import numpy as np

from .build import build_oracle

_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build_oracle())
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.or_splat.argtypes = [i, i, d, d, d, ctypes.c_double, d]
        _lib.or_quat_to_rot.argtypes = [d, d]
        _lib.or_resample.argtypes = [i, d, d, d]
        _lib.or_fft1d.argtypes = [i, d, d, i]
        _lib.or_fft3d.argtypes = [i, d, i]
        _lib.or_correlate_direct.argtypes = [i, d, d, d]
        _lib.or_fields.argtypes = [i, d, d, d, d, d, d]
        _lib.or_torque.argtypes = [i, i, d, d, i, d, ip]
        _lib.or_query.argtypes = [i, i, d, d, i, d, d, i, d]
        _lib.or_nearest.argtypes = [i, d, d, i, i, ip, d]
        _lib.or_so3_log.argtypes = [d, d]
        _lib.or_fields_spec.argtypes = [i, d, d, d, d, d, d]
        _lib.or_spectral_table.argtypes = [i, i, d, d]
        _lib.or_spectral_rotate.argtypes = [i, i, d, d, d]
        _lib.or_lowpass.argtypes = [i, d, d, i, i, d, d, d]
        _lib.or_torque_analytic.argtypes = [i, d, d, d, d, d]
        _lib.or_mesh_sdf.argtypes = [i, i, d, i, ip, ctypes.c_double, ctypes.c_double, i, d, d, d]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def splat(n, pts, sigma, amp=None, cutoff=6.0):
    """Skeletal density on the N^3 grid: sum of peak-normalised Gaussians
    exp(-r^2 / 2 sigma_i^2), truncated at r <= cutoff*sigma_i, minimum-image
    distance on the period-2 torus.  Stand-in for the skeletal density of
    Section 2.3 (the Gaussian kernel g_sigma highlighting skeleton branches)."""
    pts, sigma = _f64(pts).reshape(-1, 3), _f64(sigma).reshape(-1)
    a = None if amp is None else _f64(amp).reshape(-1)
    out = np.empty((n, n, n))
    _L().or_splat(n, len(sigma), _p(pts), _p(sigma), None if a is None else _p(a), float(cutoff), _p(out))
    return out


def quat_to_rot(q):
    """Unit quaternion (w, x, y, z) -> rotation matrix R in SO(3) (Section 2.2)."""
    q = _f64(q).reshape(4)
    R = np.empty((3, 3))
    _L().or_quat_to_rot(_p(q), _p(R))
    return R


def resample(rho, R):
    """rho^R[n] = rho(R^T x_n) by periodic trilinear interpolation
    (Section 2.4, motion decomposition feeding Eq. 3)."""
    rho = _f64(rho)
    n = rho.shape[0]
    R = _f64(R).reshape(3, 3)
    out = np.empty_like(rho)
    _L().or_resample(n, _p(rho), _p(R), _p(out))
    return out


def fft1d(x, sign=-1):
    """Unscaled 1D DFT (Eq. 7a for sign=-1, Eq. 7b without 1/N for +1)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    _L().or_fft1d(len(x), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(sign))
    return out


def fft3d(x, sign=-1):
    """Unscaled 3D DFT over all three axes (Eqs. 7a/7b)."""
    a = np.array(x, dtype=np.complex128, order="C", copy=True)
    _L().or_fft3d(a.shape[0], a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(sign))
    return a


def correlate_direct(rho1, rho2r):
    """E[j] = h^3 sum_n rho1[n] rho2r[(n - j) mod N] -- Eqs. 1/3 as a direct
    Riemann sum over the periodic grid, O(N^6)."""
    rho1, rho2r = _f64(rho1), _f64(rho2r)
    n = rho1.shape[0]
    E = np.empty_like(rho1)
    _L().or_correlate_direct(n, _p(rho1), _p(rho2r), _p(E))
    return E


def fields(rho1, rho2r):
    """(E, Fx, Fy, Fz) over all lags by the convolution theorem, Eq. 5, and
    the gradient multiplier 2 pi i omega of Eq. 6a (Nyquist multiplier 0);
    F = -grad_t E."""
    rho1, rho2r = _f64(rho1), _f64(rho2r)
    n = rho1.shape[0]
    outs = [np.empty_like(rho1) for _ in range(4)]
    _L().or_fields(n, _p(rho1), _p(rho2r), *[_p(o) for o in outs])
    return tuple(outs)


def fields_lib(rho1, rho2r, workers=None):
    """fields() with the DFT step done by a library (scipy's pocketfft,
    double precision, multithreaded) instead of the oracle's own recursive
    transform: the same definition in the same order -- S = h^3 rho1^
    conj(rho2R^) (Eq. 5, reflection as conjugation), E = IDFT(S) / N^3,
    F_d = -IDFT(2 pi i omega_d S) / N^3 with omega = k~ / (N h) and each
    axis' Nyquist multiplier 0 (Eq. 6a).  For grids (256^3) where the own
    transform takes tens of seconds per rotation; pinned against fields()
    and the direct sum."""
    import scipy.fft as sf
    rho1, rho2r = _f64(rho1), _f64(rho2r)
    n = rho1.shape[0]
    w = workers if workers is not None else (os.cpu_count() or 1)
    h = 2.0 / n
    S = sf.fftn(rho1, workers=w)
    S *= np.conj(sf.fftn(rho2r, workers=w))
    S *= h**3
    E = sf.ifftn(S, workers=w).real.copy()  # ifftn carries the 1/N^3
    k = np.arange(n, dtype=np.float64)
    k = np.where(k < (n + 1) // 2, k, k - n)
    if n % 2 == 0:
        k[n // 2] = 0.0
    omega = k / (n * h)
    F = []
    for shape in ((1, 1, n), (1, n, 1), (n, 1, 1)):  # x, y, z on arrays [z, y, x]
        G = S * (2.0j * np.pi * omega.reshape(shape))
        F.append(-sf.ifftn(G, workers=w).real)
        del G
    return (E, *F)


def fields_spec(rho1, b):
    """fields() given the moving density's rotated spectrum b = DFT(rho2R)
    (complex, natural order) instead of the rotated grid (Eqs. 5, 6a)."""
    rho1 = _f64(rho1)
    b = np.ascontiguousarray(b, dtype=np.complex128)
    n = rho1.shape[0]
    outs = [np.empty_like(rho1) for _ in range(4)]
    _L().or_fields_spec(n, _p(rho1), b.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), *[_p(o) for o in outs])
    return tuple(outs)


def spectral_table(rho2, os=1):
    """Centred spectrum of rho2 zero-padded to os*N nodes per axis (Section
    3.2, the precomputed moving spectrum): (-1)^(kx+ky+kz) DFT(pad rho2),
    complex (os N)^3, natural order."""
    rho2 = _f64(rho2)
    n = rho2.shape[0]
    t = np.empty((os * n,) * 3, dtype=np.complex128)
    _L().or_spectral_table(n, int(os), _p(rho2), t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return t


def spectral_rotate(table, n, R, os=1):
    """Spectrum of the rotated moving density on the N grid by trilinear
    interpolation of the table at os R^T k (Section 3.2, step 1); zero on the
    Nyquist planes."""
    table = np.ascontiguousarray(table, dtype=np.complex128)
    assert table.shape == (os * n,) * 3
    out = np.empty((n, n, n), dtype=np.complex128)
    _L().or_spectral_rotate(n, int(os), table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _p(_f64(R)),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def torque_analytic(rho1, rho2r):
    """Torque fields (Tx, Ty, Tz) over all lags by the rotational gradient of
    Eq. 6b, with the moment moved onto the stationary part by integrating by
    parts: T = C(-u x grad rho1, rho2R) - t x F (T = -grad_theta E for world
    perturbations about the moving part's reference point)."""
    rho1, rho2r = _f64(rho1), _f64(rho2r)
    n = rho1.shape[0]
    outs = [np.empty_like(rho1) for _ in range(3)]
    _L().or_torque_analytic(n, _p(rho1), _p(rho2r), *[_p(o) for o in outs])
    return tuple(outs)


def mesh_sdf(n, V, T, sigma=0.5, gamma_max=0.05, dmax=8):
    """Mesh descriptor of Eq. 2 on the N^3 nodes for a closed, outward
    oriented triangle mesh: (W, xi, rho) = winding number (PMC), signed
    distance (negative inside), and the skeletal density (1/4pi) integral of
    exp(-(eta/|xi| - 1)^2 / 2 sigma^2) d gamma (solid-angle element), by
    adaptive subdivision down to gamma_max per piece (depth <= dmax)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.int32)
    outs = [np.empty((n, n, n)) for _ in range(3)]
    _L().or_mesh_sdf(int(n), len(V), _p(V), len(T), T.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), float(sigma),
                     float(gamma_max), int(dmax), *[_p(o) for o in outs])
    return tuple(outs)


def lowpass(rho1, table, os, K, R, t):
    """Single-pose (E, Fx, Fy, Fz, Tx, Ty, Tz) from spectra truncated to
    |k~_a| <= K, the inverse transform summed at the one translation t
    (Section 4.2, "Truncated Inverse FFT"; Section 3.3 low-pass filtering);
    T is the exact rotational derivative of the interpolated model."""
    rho1 = _f64(rho1)
    table = np.ascontiguousarray(table, dtype=np.complex128)
    n = rho1.shape[0]
    out = np.empty(7)
    _L().or_lowpass(n, _p(rho1), table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(os), int(K),
                    _p(_f64(R)), _p(_f64(np.asarray(t, dtype=np.float64).reshape(3))), _p(out))
    return out


def torque(quats, E, knn=6):
    """T = -dE/dtheta per rotation by least squares over the knn nearest
    sampled rotations (left perturbations), the finite-difference stand-in
    for Eq. 6b.  E: (R, N, N, N).  Returns (T (R, 3, N, N, N), status (R,))."""
    quats = _f64(quats).reshape(-1, 4)
    E = _f64(E)
    nrot, n = E.shape[0], E.shape[1]
    T = np.empty((nrot, 3, n, n, n))
    st = np.zeros(nrot, dtype=np.int32)
    _L().or_torque(n, nrot, _p(quats), _p(E), int(knn), _p(T),
                   st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return T, st


def query(quats, fields_, t, q, k=4):
    """Pose query (Section 4.2, restricted motion DOF): blend of the k nearest
    sampled rotations (weights 1/theta) of periodic trilinear samples at
    u = t/h.  fields_: (R, F, N, N, N).  Returns (F,) values."""
    quats = _f64(quats).reshape(-1, 4)
    fl = _f64(fields_)
    nrot, nf, n = fl.shape[0], fl.shape[1], fl.shape[2]
    t, q = _f64(t).reshape(3), _f64(q).reshape(4)
    out = np.empty(nf)
    _L().or_query(n, nrot, _p(quats), _p(fl), nf, _p(t), _p(q), int(k), _p(out))
    return out


def nearest(quats, q, k, skip=-1):
    """k nearest sampled rotations to q by geodesic angle, ties to lower index."""
    quats = _f64(quats).reshape(-1, 4)
    q = _f64(q).reshape(4)
    idx = np.empty(k, dtype=np.int32)
    ang = np.empty(k)
    _L().or_nearest(len(quats), _p(quats), _p(q), int(skip), int(k),
                    idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(ang))
    return idx, ang


def so3_log(M):
    """Axis-angle vector of a rotation matrix."""
    M = _f64(M).reshape(3, 3)
    v = np.empty(3)
    _L().or_so3_log(_p(M), _p(v))
    return v


def pose_fields(rho1, rho2, quats):
    """Convenience: for each quaternion, resample rho2 and return the stacked
    (R, 4, N, N, N) array of (E, Fx, Fy, Fz)."""
    out = []
    for q in _f64(quats).reshape(-1, 4):
        out.append(np.stack(fields(rho1, resample(rho2, quat_to_rot(q)))))
    return np.stack(out)
