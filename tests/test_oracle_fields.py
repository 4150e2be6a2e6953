"""Pins of the oracle's density, resampling and energy/force fields against
what the paper and the mathematics fix: the direct correlation sum (Eqs. 1/3),
the correlation theorem (Eq. 5), the closed-form overlap of two Gaussian
kernels, exact 90-degree and integer-shift equivariance, the indicator
special case (intersection volume, Section 2.2), finite differences of the
band-limited interpolant against the spectral force (Eq. 6a), and scipy's
independent periodic trilinear interpolation and rotation routines."""
import numpy as np
import pytest
from scipy import ndimage
from scipy.spatial.transform import Rotation

import oracle
import synth


def rand_density(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, n, n))


# ----------------------------------------------------------------- splat ----

def test_splat_single_point_peak_and_mass():
    n = 64
    h = 2.0 / n
    c = np.array([[-1 + 10 * h, -1 + 7 * h, -1 + 20 * h]])  # on a node
    sig = np.array([3 * h])
    rho = oracle.splat(n, c, sig)
    assert rho[20, 7, 10] == 1.0  # peak amplitude 1 at the node
    # Gaussian integral (2 pi)^{3/2} sigma^3 minus the tail cut at r > 6 sigma:
    # P(chi_3 > 6) = erfc(6/sqrt 2) + sqrt(2/pi) 6 e^{-18}.  The Riemann sum
    # adds the Poisson error ~exp(-2 pi^2 sigma^2 / h^2) = e^-177 and the
    # lattice error of the jump at the cut, below e^-18 x (shell nodes) / mass
    # ~ 1.5e-7 x (lattice discrepancy of the shell); a 5- or 7-sigma cut
    # would move the mass by >= 7e-8, well outside the 2e-8 allowed here.
    from math import erfc, exp, pi, sqrt
    tail = erfc(6 / sqrt(2)) + sqrt(2 / pi) * 6 * exp(-18)
    mass = rho.sum() * h**3
    exact = (2 * np.pi) ** 1.5 * sig[0] ** 3 * (1 - tail)
    assert abs(mass - exact) <= 2e-8 * exact


def test_splat_minimum_image_and_cutoff():
    n = 16
    h = 2.0 / n
    sig = 0.1
    c = np.array([[0.98, 0.0, 0.0]])  # near the +x face: wraps to x ~ -1
    rho = oracle.splat(n, c, np.array([sig]))
    x = -1 + np.arange(n) * h
    dx = x - 0.98
    dx -= 2 * np.round(dx / 2)
    y0 = n // 2  # y = 0, z = 0 nodes
    expect = np.where(np.abs(dx) <= 6 * sig, np.exp(-dx**2 / (2 * sig**2)), 0.0)
    assert np.allclose(rho[y0, y0, :], expect, rtol=1e-14, atol=1e-300)
    assert rho[y0, y0, 0] > 0.5  # the wrapped node x = -1 is 0.02 away


def test_splat_amplitudes_are_linear():
    n = 16
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1, 1, (5, 3))
    sig = rng.uniform(0.1, 0.15, 5)
    amp = rng.uniform(-2, 2, 5)
    total = oracle.splat(n, pts, sig, amp)
    parts = sum(a * oracle.splat(n, p[None], s[None]) for p, s, a in zip(pts, sig, amp))
    assert np.allclose(total, parts, rtol=0, atol=1e-13)


# ----------------------------------------------------------- rotations ----

def test_quat_to_rot_vs_scipy():
    q = synth.random_quaternions(5, 20)
    for qq in q:
        ref = Rotation.from_quat([qq[1], qq[2], qq[3], qq[0]]).as_matrix()
        assert np.abs(oracle.quat_to_rot(qq) - ref).max() <= 1e-14


def test_identity_resample_is_bitwise_copy():
    rho = rand_density(16, 1)
    assert np.array_equal(oracle.resample(rho, np.eye(3)), rho)


def test_resample_vs_scipy_map_coordinates():
    """Periodic trilinear interpolation at R^T x_n, against scipy's
    order-1 spline with grid-wrap boundary (an independent implementation)."""
    n = 16
    h = 2.0 / n
    rho = rand_density(n, 2)
    R = oracle.quat_to_rot(synth.random_quaternions(9, 1)[0])
    got = oracle.resample(rho, R)
    ii = np.arange(n)
    z, y, x = np.meshgrid(ii, ii, ii, indexing="ij")
    P = np.stack([-1 + x * h, -1 + y * h, -1 + z * h], -1).reshape(-1, 3)
    Q = P @ R  # row p -> (R^T p)^T
    U = (Q + 1) / h  # index coordinates (x, y, z)
    ref = ndimage.map_coordinates(rho, [U[:, 2], U[:, 1], U[:, 0]], order=1, mode="grid-wrap")
    assert np.abs(got.reshape(-1) - ref).max() <= 1e-12


R90Z = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
R90X = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])


def perm_by_rotation(g, R):
    """Index-level image of a grid under p -> R^T p about the origin node N/2:
    out[n] = g[R^T (n - N/2) + N/2 mod N]."""
    n = g.shape[0]
    ii = np.arange(n)
    z, y, x = np.meshgrid(ii, ii, ii, indexing="ij")
    c = np.stack([x, y, z], -1) - n // 2
    src = (c @ R.astype(int)) + n // 2  # row c -> (R^T c)^T
    src %= n
    return g[src[..., 2], src[..., 1], src[..., 0]]


@pytest.mark.parametrize("R", [R90Z, R90X, R90Z @ R90X])
def test_resample_90deg_is_exact_permutation(R):
    rho = rand_density(16, 4)
    assert np.array_equal(oracle.resample(rho, R), perm_by_rotation(rho, R))


# ------------------------------------------------------- correlation ----

@pytest.mark.parametrize("n", [4, 8, 16])
def test_direct_equals_fft_path(n):
    r1, r2 = rand_density(n, 10 + n), rand_density(n, 20 + n)
    Ed = oracle.correlate_direct(r1, r2)
    E, *_ = oracle.fields(r1, r2)
    assert np.abs(E - Ed).max() <= 1e-12 * np.abs(Ed).max()


def test_direct_equals_fft_path_c1():
    """32^3 workload densities (ring vs peg), identity rotation."""
    s1, s2 = synth.c1_pair(0)
    r1 = oracle.splat(32, s1.pts, s1.sigma)
    r2 = oracle.splat(32, s2.pts, s2.sigma)
    Ed = oracle.correlate_direct(r1, r2)
    E, *_ = oracle.fields(r1, r2)
    assert np.abs(E - Ed).max() <= 1e-12 * np.abs(Ed).max()


def test_dc_sum_rule_and_force_sums_vanish():
    n = 16
    h = 2.0 / n
    r1, r2 = rand_density(n, 31), rand_density(n, 32)
    E, Fx, Fy, Fz = oracle.fields(r1, r2)
    assert abs(E.sum() - h**3 * r1.sum() * r2.sum()) <= 1e-11 * h**3 * np.abs(r1).sum() * np.abs(r2).sum()
    for F in (Fx, Fy, Fz):
        assert abs(F.sum()) <= 1e-11 * np.abs(F).sum()


def test_fields_real_input_sanity():
    n = 8
    r1, r2 = rand_density(n, 41), rand_density(n, 42)
    out = oracle.fields(r1, r2)
    for f in out:
        assert np.isfinite(f).all()


def gaussian_pair_closed_form(n, c1, s1, c2, s2):
    """E(t) and F(t) = -grad E for two peak-1 Gaussians on the period-2 torus:
    E(t) = (2 pi s1^2 s2^2 / S)^{3/2} exp(-|c1 - c2 - t|^2 / (2 S)),  S = s1^2 + s2^2,
    summed over the periodic images of t."""
    h = 2.0 / n
    S = s1**2 + s2**2
    pref = (2 * np.pi * s1**2 * s2**2 / S) ** 1.5
    j = np.arange(n)
    z, y, x = np.meshgrid(j, j, j, indexing="ij")
    t = np.stack([x, y, z], -1) * h
    d = np.asarray(c1) - np.asarray(c2)
    E = np.zeros((n, n, n))
    G = np.zeros((n, n, n, 3))
    for mx in (-2, -1, 0, 1):
        for my in (-2, -1, 0, 1):
            for mz in (-2, -1, 0, 1):
                r = d - (t + 2.0 * np.array([mx, my, mz]))
                e = pref * np.exp(-(r**2).sum(-1) / (2 * S))
                E += e
                G += e[..., None] * r / S  # grad_t E
    return E, -G[..., 0], -G[..., 1], -G[..., 2]


def test_gaussian_closed_form_exact():
    """Single Gaussians of width 3h, cutoff beyond the half period: Riemann-sum
    (Poisson) error e^-89 and image truncation e^-57 -- the FFT path equals the
    continuous closed form to rounding."""
    n = 64
    h = 2.0 / n
    s1, s2 = 3 * h, 3.5 * h
    c1, c2 = np.array([0.11, -0.23, 0.05]), np.array([-0.3, 0.17, 0.2])
    r1 = oracle.splat(n, c1[None], np.array([s1]), cutoff=10.0)
    r2 = oracle.splat(n, c2[None], np.array([s2]), cutoff=10.0)
    E, Fx, Fy, Fz = oracle.fields(r1, r2)
    Ec, Fxc, Fyc, Fzc = gaussian_pair_closed_form(n, c1, s1, c2, s2)
    m = np.abs(Ec).max()
    assert np.abs(E - Ec).max() <= 1e-12 * m
    mf = max(np.abs(Fxc).max(), np.abs(Fyc).max(), np.abs(Fzc).max())
    for F, Fc in ((Fx, Fxc), (Fy, Fyc), (Fz, Fzc)):
        assert np.abs(F - Fc).max() <= 1e-10 * mf


def test_gaussian_closed_form_with_6sigma_cutoff():
    """With the 6-sigma truncation of the definition the error is bounded by
    the discarded tail mass, P(chi_3 > 6) < 1e-7 of the kernel mass."""
    n = 64
    h = 2.0 / n
    s1, s2 = 3 * h, 3 * h
    c1, c2 = np.array([0.0, 0.1, -0.1]), np.array([0.2, -0.1, 0.0])
    r1 = oracle.splat(n, c1[None], np.array([s1]))
    r2 = oracle.splat(n, c2[None], np.array([s2]))
    E, *_ = oracle.fields(r1, r2)
    Ec, *_ = gaussian_pair_closed_form(n, c1, s1, c2, s2)
    assert np.abs(E - Ec).max() <= 2e-7 * np.abs(Ec).max()


@pytest.mark.parametrize("R", [R90Z, R90X])
def test_rotated_part_equals_permuted_grid(R):
    n = 16
    r1, r2 = rand_density(n, 51), rand_density(n, 52)
    a = oracle.fields(r1, oracle.resample(r2, R))
    b = oracle.fields(r1, perm_by_rotation(r2, R))
    for u, v in zip(a, b):
        assert np.abs(u - v).max() <= 1e-12 * np.abs(v).max()


def test_rotating_both_parts_rotates_the_energy():
    """E'[R j] = E[j] for a 90-degree R applied to both parts."""
    n = 16
    R = R90Z
    r1, r2 = rand_density(n, 61), rand_density(n, 62)
    E, *_ = oracle.fields(r1, r2)
    E2, *_ = oracle.fields(oracle.resample(r1, R), oracle.resample(r2, R))
    # lag j (wrapped, centred at 0) maps to R j
    j = np.arange(n)
    z, y, x = np.meshgrid(j, j, j, indexing="ij")
    J = np.stack([x, y, z], -1)
    RJ = (J @ R.T.astype(int)) % n  # row j -> (R j)^T
    assert np.abs(E2[RJ[..., 2], RJ[..., 1], RJ[..., 0]] - E).max() <= 1e-12 * np.abs(E).max()


def test_integer_shift_shifts_the_fields():
    n = 16
    s = (3, -5, 7)  # (z, y, x) cells
    r1, r2 = rand_density(n, 71), rand_density(n, 72)
    a = oracle.fields(r1, r2)
    b = oracle.fields(r1, np.roll(r2, s, axis=(0, 1, 2)))
    for u, v in zip(a, b):  # rho2'[n] = rho2[n - s]  =>  E'[j] = E[j + s]
        assert np.abs(np.roll(u, tuple(-k for k in s), axis=(0, 1, 2)) - v).max() <= 1e-12 * np.abs(u).max()


def test_indicator_boxes_give_overlap_volume():
    """Indicator densities make Eq. 1 the intersection volume (Section 2.2);
    on the grid: h^3 x (number of common nodes), a product of 1D counts."""
    n = 16
    h = 2.0 / n
    A = [(2, 9), (4, 8), (0, 5)]  # [lo, hi) per axis (x, y, z)
    B = [(5, 12), (1, 3), (3, 14)]
    def box(lims):
        g = np.zeros((n, n, n))
        (x0, x1), (y0, y1), (z0, z1) = lims
        g[z0:z1, y0:y1, x0:x1] = 1.0
        return g
    E, *_ = oracle.fields(box(A), box(B))
    idx = np.arange(n)
    def count1d(a, b, j):  # #{m in a : (m - j) mod n in b}
        return sum(1 for m in range(*a) if b[0] <= (m - j) % n < b[1])
    cx = np.array([count1d(A[0], B[0], j) for j in idx])
    cy = np.array([count1d(A[1], B[1], j) for j in idx])
    cz = np.array([count1d(A[2], B[2], j) for j in idx])
    expect = h**3 * cz[:, None, None] * cy[None, :, None] * cx[None, None, :]
    assert np.abs(E - expect).max() <= 1e-12


def test_force_equals_fd_of_band_limited_interpolant():
    """Central finite differences of the trigonometric interpolant of E
    (numpy FFT, Nyquist term in its symmetric cosine form) reproduce the
    spectral force of Eq. 6a: pins the multiplier, its sign and the Nyquist
    rule."""
    n = 8
    h = 2.0 / n
    r1, r2 = rand_density(n, 81), rand_density(n, 82)
    E, Fx, Fy, Fz = oracle.fields(r1, r2)
    Ehat = np.fft.fftn(E)
    k = np.arange(n)

    def basis(u):  # per-axis values of the interpolant's modes at index coord u
        b = np.exp(2j * np.pi * np.where(k < n // 2, k, k - n) * u / n)
        b[n // 2] = np.cos(np.pi * u)
        return b

    def interp(u):  # u = (x, y, z) index coordinates
        bx, by, bz = basis(u[0]), basis(u[1]), basis(u[2])
        return np.real(np.einsum("zyx,z,y,x->", Ehat, bz, by, bx)) / n**3

    rng = np.random.default_rng(5)
    d = 1e-5
    scale = max(np.abs(Fx).max(), np.abs(Fy).max(), np.abs(Fz).max())
    for _ in range(12):
        j = rng.integers(0, n, 3)  # (x, y, z)
        assert abs(interp(j.astype(float)) - E[j[2], j[1], j[0]]) <= 1e-12 * np.abs(E).max()
        for ax, F in enumerate((Fx, Fy, Fz)):
            up, dn = j.astype(float), j.astype(float)
            up[ax] += d
            dn[ax] -= d
            fd = -(interp(up) - interp(dn)) / (2 * d * h)
            assert abs(fd - F[j[2], j[1], j[0]]) <= 1e-6 * scale


# ------------------------------------- library-transform route (large grids) ----

@pytest.mark.parametrize("n", [8, 12, 16])
def test_fields_lib_equals_direct_sum_and_own_transform(n):
    """The library-DFT route gives the direct Riemann sum (Eqs. 1/3) and the
    own-transform fields element by element, even and non-power-of-two N."""
    r1, r2 = rand_density(n, 300 + n), rand_density(n, 400 + n)
    Ed = oracle.correlate_direct(r1, r2)
    lib = oracle.fields_lib(r1, r2, workers=2)
    own = oracle.fields(r1, r2)
    assert np.abs(lib[0] - Ed).max() <= 1e-12 * np.abs(Ed).max()
    for a, b in zip(lib, own):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_fields_lib_gaussian_closed_form():
    """Energy and force of two Gaussians (variance s1^2 + s2^2) in closed
    form: a dropped term, a sign or an axis swap in the multiplier fails."""
    n = 64
    h = 2.0 / n
    s1, s2 = 3 * h, 3.5 * h
    c1, c2 = np.array([0.11, -0.23, 0.05]), np.array([-0.3, 0.17, 0.2])
    r1 = oracle.splat(n, c1[None], np.array([s1]), cutoff=10.0)
    r2 = oracle.splat(n, c2[None], np.array([s2]), cutoff=10.0)
    E, Fx, Fy, Fz = oracle.fields_lib(r1, r2)
    Ec, Fxc, Fyc, Fzc = gaussian_pair_closed_form(n, c1, s1, c2, s2)
    assert np.abs(E - Ec).max() <= 1e-12 * np.abs(Ec).max()
    mf = max(np.abs(Fxc).max(), np.abs(Fyc).max(), np.abs(Fzc).max())
    for F, Fc in ((Fx, Fxc), (Fy, Fyc), (Fz, Fzc)):
        assert np.abs(F - Fc).max() <= 1e-10 * mf
