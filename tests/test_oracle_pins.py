"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to an independent fact: numerical
quadrature of Eq. G along the beam, scipy's quaternion rotations, numpy's FFT,
closed forms (peak of an isotropic Gaussian, total mass, Parseval), symmetry
(image rotation, quaternion sign), published electron wavelengths, and central
differences of the oracle's own loss.  A dropped term, a wrong sign, a
transposed operand or a swapped image axis in the oracle fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

import oracle
from paper_2509_25075_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cov_world(theta):
    """Sigma = R_q S S^T R_q^T with scipy's rotation (scalar-last quaternion)."""
    w, x, y, z = theta[6:10]
    Rq = Rotation.from_quat([x, y, z, w]).as_matrix()
    return Rq @ np.diag(np.asarray(theta[3:6], dtype=np.float64) ** 2) @ Rq.T


def _random_theta(rng, n):
    th = np.zeros((n, 11))
    th[:, 0:3] = rng.normal(scale=6.0, size=(n, 3))
    th[:, 3:6] = rng.uniform(1.5, 4.0, size=(n, 3))
    th[:, 6:10] = rng.normal(size=(n, 4))
    th[:, 10] = rng.uniform(0.5, 1.5, size=n)
    return th


def _line_integral(theta, Rv, tv, x, y):
    """Integral over z' of Eq. G along the ray through (x, y) of view (Rv, tv)."""
    p = theta[0:3]
    Si = np.linalg.inv(_cov_world(theta))
    rho = theta[10]

    def f(z):
        xc = np.array([x - tv[0], y - tv[1], z])
        xw = Rv.T @ xc          # camera x' = R x + (t, 0)  =>  x = R^T (x' - (t, 0))
        e = xw - p
        return rho * math.exp(-0.5 * e @ Si @ e)

    zc = (Rv @ p)[2]
    val, err = integrate.quad(f, zc - 60.0, zc + 60.0, epsabs=1e-14, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_marginalisation_matches_quadrature(seed):
    """Eq. render / appendix: projecting Eq. G along the beam gives the 2D
    Gaussian with the top-left block of the viewed covariance."""
    rng = np.random.default_rng(seed)
    th = _random_theta(rng, 1)
    Rv = syn.rotations(1, rng)
    tv = rng.normal(scale=2.0, size=(1, 2))
    d, apix = 32, 1.0
    pix = rng.integers(0, d * d, size=6)
    got1 = oracle.project_pixels(th, Rv, tv, d, apix, 0.0, pix, norm_mode=1)
    got0 = oracle.project_pixels(th, Rv, tv, d, apix, 0.0, pix, norm_mode=0)
    detS = np.linalg.det(_cov_world(th[0]))
    for i, pi in enumerate(pix):
        v, u = divmod(int(pi), d)
        x, y = (u - d / 2) * apix, (v - d / 2) * apix
        ref = _line_integral(th[0], Rv[0], tv[0], x, y)
        assert abs(got1[i] - ref) <= 1e-9 * max(ref, 1e-6), (got1[i], ref)
        # norm_mode 0 = Eq. render: rho is the mass, i.e. the line integral of
        # Eq. G divided by the 3D normalisation (2 pi)^3/2 |Sigma|^1/2
        ref0 = ref / ((2 * math.pi) ** 1.5 * math.sqrt(detS))
        assert abs(got0[i] - ref0) <= 1e-9 * max(ref0, 1e-9)


def test_isotropic_peak_closed_form():
    """Eq. render at the centre of an isotropic Gaussian: rho / (2 pi sigma^2)."""
    d, apix, sigma, rho = 16, 1.3, 2.1, 0.7
    u, v = 5, 11
    th = np.array([[(u - d / 2) * apix, (v - d / 2) * apix, 3.0, sigma, sigma, sigma, 0.3, -0.2, 0.9, 0.1, rho]])
    img = oracle.project(th, np.eye(3)[None], np.zeros((1, 2)), d, apix, 0.0)
    assert img[0, v, u] == pytest.approx(rho / (2 * math.pi * sigma ** 2), rel=1e-14)
    # one pixel to the right: exp(-apix^2 / (2 sigma^2)) lower
    assert img[0, v, u + 1] == pytest.approx(
        rho / (2 * math.pi * sigma ** 2) * math.exp(-apix ** 2 / (2 * sigma ** 2)), rel=1e-13)


@pytest.mark.parametrize("seed", [3, 4])
def test_mass_conservation(seed):
    """apix^2 * sum of pixels = sum of rho (norm_mode 0, tau = 0), any view."""
    rng = np.random.default_rng(seed)
    d, apix = 64, 1.0
    th = _random_theta(rng, 5)
    th[:, 0:3] = rng.uniform(-5, 5, size=(5, 3))
    th[:, 3:6] = rng.uniform(1.6, 3.0, size=(5, 3))
    Rv = syn.rotations(2, rng)
    img = oracle.project(th, Rv, np.zeros((2, 2)), d, apix, 0.0)
    for b in range(2):
        assert img[b].sum() * apix ** 2 == pytest.approx(th[:, 10].sum(), rel=1e-10)


def test_rotation_invariance_of_isotropic_at_origin():
    rng = np.random.default_rng(5)
    th = np.zeros((3, 11))
    th[:, 3:6] = np.array([[1.5] * 3, [2.0] * 3, [3.0] * 3])
    th[:, 6:10] = rng.normal(size=(3, 4))
    th[:, 10] = [1.0, 0.5, 2.0]
    Rv = syn.rotations(3, rng)
    img = oracle.project(th, Rv, np.zeros((3, 2)), 24, 1.1, 0.0)
    np.testing.assert_allclose(img[1], img[0], rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(img[2], img[0], rtol=1e-12, atol=1e-16)


def test_view_rotation_about_beam_permutes_pixels():
    """R_z(90 deg): x' = (-x_y, x_x), so image[v][u] = identity image[d-u][v].
    Pins the axis convention (row = y, column = x) and the sign of R."""
    rng = np.random.default_rng(6)
    d = 20
    th = _random_theta(rng, 4)
    th[:, 0:3] = rng.uniform(-4, 4, size=(4, 3))
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    img = oracle.project(th, np.stack([np.eye(3), Rz]), np.zeros((2, 2)), d, 1.0, 0.0)
    for v in range(d):
        for u in range(1, d):
            assert img[1, v, u] == pytest.approx(img[0, d - u, v], rel=1e-12, abs=1e-15)


def test_rotation_about_y_shows_z_extent():
    """R_y(90 deg) maps the Gaussian's z-axis onto the image x-axis."""
    d, apix = 32, 1.0
    th = np.array([[0.0, 0.0, 0.0, 1.7, 2.3, 3.4, 1.0, 0.0, 0.0, 0.0, 1.0]])
    Ry = np.array([[0.0, 0.0, 1.0], [0.0, 1.0, 0.0], [-1.0, 0.0, 0.0]])
    img_y = oracle.project(th, Ry[None], np.zeros((1, 2)), d, apix, 0.0)
    th2 = th.copy()
    th2[0, 3:6] = [3.4, 2.3, 1.7]
    img_ref = oracle.project(th2, np.eye(3)[None], np.zeros((1, 2)), d, apix, 0.0)
    np.testing.assert_allclose(img_y, img_ref, rtol=1e-13, atol=1e-17)
    pre = oracle.preprocess(th, Ry[None], np.zeros((1, 2)))
    assert pre[0, 0, 2] == pytest.approx(3.4 ** 2, rel=1e-14)
    assert pre[0, 0, 4] == pytest.approx(2.3 ** 2, rel=1e-14)


def test_quaternion_sign_and_scale():
    rng = np.random.default_rng(7)
    th = _random_theta(rng, 3)
    Rv = syn.rotations(2, rng)
    t = rng.normal(size=(2, 2))
    a = oracle.project(th, Rv, t, 16, 1.0, 1e-4)
    th2 = th.copy()
    th2[:, 6:10] *= -2.5
    b = oracle.project(th2, Rv, t, 16, 1.0, 1e-4)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-17)


def test_preprocess_against_scipy():
    """Mean, covariance, amplitude and depth of one viewed Gaussian."""
    rng = np.random.default_rng(8)
    th = _random_theta(rng, 4)
    Rv = syn.rotations(3, rng)
    t = rng.normal(size=(3, 2))
    for mode in (0, 1):
        pre = oracle.preprocess(th, Rv, t, norm_mode=mode)
        for b in range(3):
            for j in range(4):
                S = Rv[b] @ _cov_world(th[j]) @ Rv[b].T
                m = Rv[b] @ th[j, 0:3]
                C = S[:2, :2]
                np.testing.assert_allclose(pre[b, j, 0:2], m[:2] + t[b], rtol=1e-13, atol=1e-13)
                np.testing.assert_allclose(pre[b, j, [2, 3, 4]], [C[0, 0], C[0, 1], C[1, 1]], rtol=1e-12)
                assert pre[b, j, 6] == pytest.approx(m[2], rel=1e-12, abs=1e-12)
                if mode == 0:
                    amp = th[j, 10] / (2 * math.pi * math.sqrt(np.linalg.det(C)))
                else:
                    amp = th[j, 10] * math.sqrt(2 * math.pi) * math.sqrt(np.linalg.det(S) / np.linalg.det(C))
                assert pre[b, j, 5] == pytest.approx(amp, rel=1e-12)


def test_degenerate_gaussians_contribute_nothing():
    th = np.array([
        [0, 0, 0, 2, 2, 2, 0, 0, 0, 0, 1.0],       # zero quaternion
        [0, 0, 0, 2, 2, 2, 1, 0, 0, 0, -1.0],      # negative rho
        [0, 0, 0, 0, 0, 2, 1, 0, 0, 0, 1.0],       # singular projected covariance
    ])
    img = oracle.project(th, np.eye(3)[None], np.zeros((1, 2)), 16, 1.0, 0.0)
    assert np.all(img == 0.0)


def test_tile_hits_match_single_gaussian_images():
    rng = np.random.default_rng(9)
    d, tile, apix, tau = 32, 8, 1.0, 2e-3
    th = _random_theta(rng, 6)
    th[:, 0:3] = rng.uniform(-12, 12, size=(6, 3))
    th[:, 3:6] = rng.uniform(0.8, 3.0, size=(6, 3))
    Rv = syn.rotations(2, rng)
    t = rng.normal(size=(2, 2))
    hits = oracle.tile_hits(th, Rv, t, d, apix, tau, tile)
    nt = d // tile
    for j in range(6):
        img = oracle.project(th[j:j + 1], Rv, t, d, apix, tau)
        for b in range(2):
            for tt in range(nt * nt):
                ty, tx = divmod(tt, nt)
                block = img[b, ty * tile:(ty + 1) * tile, tx * tile:(tx + 1) * tile]
                assert hits[b, j, tt] == (1 if np.any(block > 0) else 0)


# ---------------------------------------------------------------- CTF -----

def _numpy_conv(hhalf, x):
    """irfft2(Hs . rfft2(x)) with Hs = H symmetrised on the self-conjugate
    columns (kx = 0 and kx = d/2)."""
    d = x.shape[-1]
    hs = hhalf.copy()
    neg = (-np.arange(d)) % d
    for c in (0, d // 2):
        hs[..., :, c] = 0.5 * (hhalf[..., :, c] + hhalf[..., neg, c])
    return np.fft.irfft2(hs * np.fft.rfft2(x), s=(d, d))


def test_ctf_identity():
    rng = np.random.default_rng(10)
    x = rng.normal(size=(2, 16, 16))
    y = oracle.ctf_apply(np.ones((2, 16, 16)), x)
    np.testing.assert_allclose(y, x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d", [8, 12, 16])
def test_ctf_matches_numpy_fft(d):
    rng = np.random.default_rng(11 + d)
    x = rng.normal(size=(3, d, d))
    hhalf = rng.uniform(-1, 1, size=(3, d, d // 2 + 1))
    y = oracle.ctf_apply(oracle.ctf_grid_from_half(hhalf), x)
    np.testing.assert_allclose(y, _numpy_conv(hhalf, x), rtol=0, atol=1e-12)
    # delta image -> point-spread function
    delta = np.zeros((3, d, d))
    delta[:, 0, 0] = 1.0
    psf = oracle.ctf_apply(oracle.ctf_grid_from_half(hhalf), delta)
    np.testing.assert_allclose(psf, _numpy_conv(hhalf, delta), rtol=0, atol=1e-13)


def test_ctf_operator_is_self_adjoint():
    rng = np.random.default_rng(12)
    d = 16
    x, y = rng.normal(size=(2, 1, d, d))
    H = oracle.ctf_grid_from_half(rng.uniform(-1, 1, size=(1, d, d // 2 + 1)))
    lhs = np.sum(oracle.ctf_apply(H, x) * y)
    rhs = np.sum(x * oracle.ctf_apply(H, y))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_loss_and_adjoint_against_numpy():
    rng = np.random.default_rng(13)
    B, d = 3, 12
    proj = rng.normal(size=(B, d, d))
    imgs = rng.normal(size=(B, d, d))
    hhalf = rng.uniform(-1, 1, size=(B, d, d // 2 + 1))
    L, pred, li, g = oracle.loss(oracle.ctf_grid_from_half(hhalf), proj, imgs)
    ref_pred = _numpy_conv(hhalf, proj)
    np.testing.assert_allclose(pred, ref_pred, atol=1e-12)
    r = ref_pred - imgs
    np.testing.assert_allclose(li, np.mean(r ** 2, axis=(1, 2)), rtol=1e-12)
    assert L == pytest.approx(np.mean(r ** 2), rel=1e-12)
    np.testing.assert_allclose(g, _numpy_conv(hhalf, 2 * r / (B * d * d)), atol=1e-13)
    # Parseval on the residual
    assert np.sum(r ** 2) == pytest.approx(np.sum(np.abs(np.fft.fft2(r)) ** 2) / d ** 2, rel=1e-12)


def test_loss_gradient_wrt_projection_by_differences():
    rng = np.random.default_rng(14)
    B, d = 2, 8
    proj = rng.normal(size=(B, d, d))
    imgs = rng.normal(size=(B, d, d))
    H = oracle.ctf_grid_from_half(rng.uniform(-1, 1, size=(B, d, d // 2 + 1)))
    _, _, _, g = oracle.loss(H, proj, imgs)
    for (b, v, u) in [(0, 0, 0), (1, 3, 5), (0, 7, 2)]:
        h = 1e-5
        pp, pm = proj.copy(), proj.copy()
        pp[b, v, u] += h
        pm[b, v, u] -= h
        fd = (oracle.loss(H, pp, imgs)[0] - oracle.loss(H, pm, imgs)[0]) / (2 * h)
        assert fd == pytest.approx(g[b, v, u], rel=1e-8, abs=1e-14)


def test_electron_wavelength_and_ctf_zeros():
    with open(os.path.join(GOLDEN, "electron_wavelength.json")) as f:
        table = json.load(f)
    for row in table["rows"]:
        kv, lam = row["kV"], row["lambda_A"]
        # with w = 0, Cs = 0, no phase, no envelope: H = -sin(pi lambda dF k^2);
        # its first zero away from k = 0 is at k^2 = 1 / (lambda dF)
        df = 15000.0
        prm = [df, df, 0.0, kv, 0.0, 0.0, 0.0, 0.0]
        k1 = math.sqrt(1.0 / (lam * df))
        # tabulated wavelengths carry 4-5 digits: the zero sits where
        # the phase pi lambda dF k^2 is pi to that accuracy
        assert abs(oracle.ctf_value(prm, k1, 0.0)) < 5e-3 * math.pi
        # quarter period: H = -sin(pi/2) = -1
        assert oracle.ctf_value(prm, math.sqrt(0.5 / (lam * df)), 0.0) == pytest.approx(-1.0, abs=2e-4)


def test_ctf_formula_terms():
    kv = 300.0
    volt = kv * 1e3
    lam = 12.2643247 / math.sqrt(volt * (1 + 0.978466e-6 * volt))
    # amplitude contrast at k = 0
    assert oracle.ctf_value([1e4, 1e4, 0, kv, 2.7, 0.1, 0, 0], 0.0, 0.0) == pytest.approx(-0.1, abs=1e-15)
    # spherical aberration alone: chi = -pi/2 Cs lambda^3 k^4
    k = 0.3
    chi = -0.5 * math.pi * 2.7e7 * lam ** 3 * k ** 4
    assert oracle.ctf_value([0, 0, 0, kv, 2.7, 0, 0, 0], k, 0) == pytest.approx(-math.sin(chi), rel=1e-12)
    # astigmatism: defocus U along the astigmatism angle, V across it
    ang = 0.4
    prm = [2e4, 1e4, ang, kv, 0, 0, 0, 0]
    k = 0.05
    along = oracle.ctf_value(prm, k * math.cos(ang), k * math.sin(ang))
    across = oracle.ctf_value(prm, -k * math.sin(ang), k * math.cos(ang))
    assert along == pytest.approx(-math.sin(math.pi * lam * 2e4 * k * k), rel=1e-11)
    assert across == pytest.approx(-math.sin(math.pi * lam * 1e4 * k * k), rel=1e-11)
    # B-factor envelope and phase shift
    base = oracle.ctf_value([1.2e4, 1.2e4, 0, kv, 2.7, 0.07, 0.3, 0], 0.1, 0.05)
    damp = oracle.ctf_value([1.2e4, 1.2e4, 0, kv, 2.7, 0.07, 0.3, 80.0], 0.1, 0.05)
    assert damp == pytest.approx(base * math.exp(-80.0 * (0.1 ** 2 + 0.05 ** 2) / 4), rel=1e-13)


def test_ctf_grid_from_params_is_symmetric():
    prm = syn.ctf_params(syn.WORKLOADS["A1"], B=2)
    H = oracle.ctf_grid_from_params(prm, 16, 1.2)
    neg = (-np.arange(16)) % 16
    np.testing.assert_allclose(H, H[:, neg][:, :, neg], rtol=0, atol=1e-15)
    assert H[0, 0, 0] == pytest.approx(-float(prm[0, 5]), rel=1e-6)


@pytest.mark.parametrize("d,apix", [(32, 1.3), (24, 0.9)])
def test_ctf_grid_maps_bins_to_physical_frequencies(d, apix):
    """Eq. loss applies the transfer function in Fourier space.  A real
    grating with an integer number of periods across the box, along x (the
    column index u), along y (the row index v) or a diagonal, is an
    eigenfunction of that operator: the CTF grid built from parameters must
    scale it by the transfer function evaluated at the grating's physical
    frequency (n_x / (d apix), n_y / (d apix)) in 1/Angstrom.  The CTF is
    astigmatic at an angle that is neither 0 nor a multiple of pi/4, so a
    swapped axis, a dropped apix, a missing 1/d or an unsigned bin index each
    change the value."""
    prm = np.array([[1.6e4, 1.1e4, 0.61, 300.0, 2.7, 0.1, 0.2, 15.0]])
    H = oracle.ctf_grid_from_params(prm, d, apix)
    v, u = np.meshgrid(np.arange(d), np.arange(d), indexing="ij")
    for nx, ny in [(3, 0), (0, 5), (4, -7), (-6, 2), (5, 5), (1, -3)]:
        for phase in (0.0, 0.7):
            grating = np.cos(2 * np.pi * (nx * u + ny * v) / d + phase)[None]
            out = oracle.ctf_apply(H, grating)
            h = oracle.ctf_value(prm[0], nx / (d * apix), ny / (d * apix))
            np.testing.assert_allclose(out, h * grating, rtol=0, atol=1e-12)
    # the pin discriminates: the swapped-axis and unsigned-bin readings give
    # other values at the gratings used above
    assert abs(oracle.ctf_value(prm[0], 4 / (d * apix), -7 / (d * apix))
               - oracle.ctf_value(prm[0], -7 / (d * apix), 4 / (d * apix))) > 1e-3
    assert abs(oracle.ctf_value(prm[0], 4 / (d * apix), -7 / (d * apix))
               - oracle.ctf_value(prm[0], 4 / (d * apix), (d - 7) / (d * apix))) > 1e-3


# ------------------------------------------------------------ gradients -----

def _case(seed, M=3, B=2, d=8):
    rng = np.random.default_rng(seed)
    apix = 1.0
    th = _random_theta(rng, M)
    th[:, 0:3] = rng.uniform(-2.5, 2.5, size=(M, 3))
    th[:, 3:6] = rng.uniform(0.9, 2.2, size=(M, 3))
    Rv = syn.rotations(B, rng)
    t = rng.normal(scale=0.5, size=(B, 2))
    imgs = rng.normal(scale=0.02, size=(B, d, d))
    H = oracle.ctf_grid_from_half(rng.uniform(-1, 1, size=(B, d, d // 2 + 1)))
    return th, Rv, t, imgs, H, d, apix


@pytest.mark.parametrize("norm_mode", [0, 1])
@pytest.mark.parametrize("seed", [20, 21])
def test_gradient_central_differences(norm_mode, seed):
    th, Rv, t, imgs, H, d, apix = _case(seed)
    tau = 0.0
    proj = oracle.project(th, Rv, t, d, apix, tau, norm_mode)
    _, _, _, g = oracle.loss(H, proj, imgs)
    G = oracle.grad(th, Rv, t, d, apix, tau, g, norm_mode)
    scale = np.max(np.abs(G))
    for j in range(th.shape[0]):
        for m in range(11):
            h = 1e-6 * max(1.0, abs(th[j, m]))
            tp, tm = th.copy(), th.copy()
            tp[j, m] += h
            tm[j, m] -= h
            fd = (oracle.forward_loss(tp, Rv, t, H, imgs, d, apix, tau, norm_mode)
                  - oracle.forward_loss(tm, Rv, t, H, imgs, d, apix, tau, norm_mode)) / (2 * h)
            assert abs(fd - G[j, m]) <= 1e-7 * scale + 1e-6 * abs(fd), (j, m, fd, G[j, m])


def test_gradient_with_threshold_away_from_boundary():
    """With tau > 0 the pair set is fixed under small steps unless a pair sits
    on the threshold; central differences then still hold."""
    th, Rv, t, imgs, H, d, apix = _case(22)
    tau = 1e-3
    proj = oracle.project(th, Rv, t, d, apix, tau)
    _, _, _, g = oracle.loss(H, proj, imgs)
    G = oracle.grad(th, Rv, t, d, apix, tau, g)
    scale = np.max(np.abs(G))
    for j in range(th.shape[0]):
        for m in range(11):
            h = 1e-7 * max(1.0, abs(th[j, m]))
            tp, tm = th.copy(), th.copy()
            tp[j, m] += h
            tm[j, m] -= h
            fd = (oracle.forward_loss(tp, Rv, t, H, imgs, d, apix, tau)
                  - oracle.forward_loss(tm, Rv, t, H, imgs, d, apix, tau)) / (2 * h)
            assert abs(fd - G[j, m]) <= 1e-6 * scale + 1e-5 * abs(fd), (j, m, fd, G[j, m])


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_rho_gradient_is_linear(norm_mode):
    """dL/drho_j = <g, image_j / rho_j> exactly (the value is linear in rho)."""
    th, Rv, t, imgs, H, d, apix = _case(23, M=4)
    tau = 2e-3
    proj = oracle.project(th, Rv, t, d, apix, tau, norm_mode)
    _, _, _, g = oracle.loss(H, proj, imgs)
    G = oracle.grad(th, Rv, t, d, apix, tau, g, norm_mode)
    for j in range(4):
        img_j = oracle.project(th[j:j + 1], Rv, t, d, apix, tau, norm_mode)
        assert G[j, 10] == pytest.approx(np.sum(g * img_j) / th[j, 10], rel=1e-12, abs=1e-18)


def test_absolute_gradient_terms():
    """The absolute sums (the error scale of a float32 gradient) bound the
    gradient, and for rho, whose per-pixel terms are g * value / rho, equal
    <|g|, image_j> / rho_j exactly."""
    th, Rv, t, imgs, H, d, apix = _case(25, M=4)
    tau = 2e-3
    proj = oracle.project(th, Rv, t, d, apix, tau)
    _, _, _, g = oracle.loss(H, proj, imgs)
    G = oracle.grad(th, Rv, t, d, apix, tau, g)
    A = oracle.grad(th, Rv, t, d, apix, tau, g, absolute=True)
    assert np.all(A >= np.abs(G) * (1 - 1e-12))
    assert np.any(A > 2 * np.abs(G))  # the smooth-field terms do cancel
    for j in range(4):
        img_j = oracle.project(th[j:j + 1], Rv, t, d, apix, tau)
        assert A[j, 10] == pytest.approx(np.sum(np.abs(g) * img_j) / th[j, 10], rel=1e-12, abs=1e-18)


def test_borderline_gradient_terms():
    """grad_border sums |g dvalue/dtheta| over exactly the pairs whose value
    lies within rel * tau of tau, on either side.  With tau set to the value
    of one pixel of a single-Gaussian, single-view case, that pixel alone
    qualifies, so the sum equals the absolute gradient of a unit upstream
    gradient at that pixel (computed with tau = 0, where every pair counts);
    a band wide enough to hold every value gives the tau = 0 absolute sums,
    and a Gaussian whose peak stays below the band gives zero."""
    th, Rv, t, imgs, H, d, apix = _case(26, M=3, B=1)
    rng = np.random.default_rng(5)
    g = rng.normal(size=(1, d, d))
    for j in range(3):
        one = th[j:j + 1]
        img = oracle.project(one, Rv, t, d, apix, 0.0)[0]
        v, u = np.unravel_index(np.argsort(img, axis=None)[-5], img.shape)  # a pixel below the peak
        tau = img[v, u]
        others = np.abs(img - tau) <= 1e-9 * tau
        assert others.sum() == 1  # that pixel alone sits in the band
        delta = np.zeros((1, d, d))
        delta[0, v, u] = abs(g[0, v, u])
        want = np.abs(oracle.grad(one, Rv, t, d, apix, 0.0, delta * np.sign(g[0, v, u])))
        got = oracle.grad_border(one, Rv, t, d, apix, tau, g, rel=1e-9)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
    everything = oracle.grad_border(th, Rv, t, d, apix, 1e-6, g, rel=1e300)
    np.testing.assert_allclose(everything, oracle.grad(th, Rv, t, d, apix, 0.0, g, absolute=True),
                               rtol=1e-13, atol=0)
    peak = oracle.project(th[:1], Rv, t, d, apix, 0.0).max()
    assert np.all(oracle.grad_border(th[:1], Rv, t, d, apix, 2 * peak, g, rel=1e-5) == 0)


def test_gradient_selection_matches_full():
    th, Rv, t, imgs, H, d, apix = _case(24, M=5)
    proj = oracle.project(th, Rv, t, d, apix, 1e-3)
    _, _, _, g = oracle.loss(H, proj, imgs)
    full = oracle.grad(th, Rv, t, d, apix, 1e-3, g)
    part = oracle.grad(th, Rv, t, d, apix, 1e-3, g, sel=[3, 0])
    np.testing.assert_array_equal(part, full[[3, 0]])


def test_golden_regression_case():
    """Stored oracle outputs of one small seeded case (written by
    tests/golden/make_golden.py, which calls only the oracle)."""
    path = os.path.join(GOLDEN, "oracle_small_case.json")
    with open(path) as f:
        gold = json.load(f)
    w = syn.Workload("golden", d=16, M=12, B=2, apix=1.2)
    params = syn.gaussians(w)
    R, t = syn.views(w)
    prm = syn.ctf_params(w)
    imgs = syn.images(w)
    proj = oracle.project(params, R, t, w.d, w.apix, w.tau)
    H = oracle.ctf_grid_from_params(prm, w.d, w.apix)
    L, _, _, g = oracle.loss(H, proj, imgs)
    G = oracle.grad(params, R, t, w.d, w.apix, w.tau, g)
    assert L == pytest.approx(gold["loss"], rel=1e-12)
    np.testing.assert_allclose(proj.sum(axis=(1, 2)), gold["proj_sums"], rtol=1e-12)
    np.testing.assert_allclose(G, np.array(gold["grad"]), rtol=1e-10, atol=1e-12 * np.max(np.abs(G)))
