"""Pins of the oracle's ablation constraints and nearest-neighbour distances
(Sec. 4, Design Choices of 3DGS for cryo-EM) against closed forms, symmetry,
central differences and an independent k-d tree."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_2509_25075_gb300 import synthetic as syn

from test_oracle_pins import _case, _random_theta


def test_no_rotation_ignores_the_quaternion_and_keeps_axes():
    """R_j = I: the world covariance is diag(s^2); under the identity view the
    2D Gaussian is axis-aligned with variances s0^2, s1^2 (closed form), and
    any quaternion (even zero) gives the same image."""
    d, apix = 32, 1.0
    th = np.zeros((1, 11))
    th[0, 3:6] = (1.7, 2.6, 0.9)
    th[0, 6:10] = (0.3, -0.8, 0.2, 0.5)
    th[0, 10] = 1.3
    Rv, tv = np.eye(3)[None], np.zeros((1, 2))
    img = oracle.project(th, Rv, tv, d, apix, 0.0, no_rotation=True)
    u = np.arange(d) - d / 2
    want = th[0, 10] / (2 * np.pi * 1.7 * 2.6) * np.exp(-0.5 * (u[None, :] / 1.7) ** 2
                                                        - 0.5 * (u[:, None] / 2.6) ** 2)
    np.testing.assert_allclose(img[0], want, rtol=1e-13, atol=1e-16)
    th2 = th.copy()
    th2[0, 6:10] = 0.0
    np.testing.assert_array_equal(oracle.project(th2, Rv, tv, d, apix, 0.0, no_rotation=True), img)


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_isotropic_closed_form_and_invariance(norm_mode):
    """S_j = s_j I: the peak at a pixel-centred Gaussian is rho / (2 pi s0^2)
    (mode 0) or rho sqrt(2 pi) s0 (mode 1, line integral of a spherical
    Gaussian of peak rho), whatever s1, s2, q and the view are."""
    d, apix = 32, 1.0
    rng = np.random.default_rng(5)
    th = np.zeros((1, 11))
    th[0, 3:6] = (2.2, 0.4, 7.0)
    th[0, 6:10] = rng.normal(size=4)
    th[0, 10] = 0.8
    Rv = syn.rotations(3, rng)
    tv = np.zeros((3, 2))
    img = oracle.project(th, Rv, tv, d, apix, 0.0, norm_mode, isotropic=True)
    peak = 0.8 / (2 * np.pi * 2.2 ** 2) if norm_mode == 0 else 0.8 * np.sqrt(2 * np.pi) * 2.2
    for b in range(3):
        assert img[b, d // 2, d // 2] == pytest.approx(peak, rel=1e-12)
        np.testing.assert_allclose(img[b], img[0], rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("flags", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("norm_mode", [0, 1])
def test_constrained_gradient_central_differences(flags, norm_mode):
    """The folded gradient is the derivative of the constrained loss with
    respect to the free parameters: zero for the fixed quaternion and for
    the unused scale entries, the total for the shared scale."""
    no_rot, iso = flags
    th, Rv, t, imgs, H, d, apix = _case(30 + norm_mode)
    proj = oracle.project(th, Rv, t, d, apix, 0.0, norm_mode, no_rot, iso)
    _, _, _, g = oracle.loss(H, proj, imgs)
    G = oracle.grad(th, Rv, t, d, apix, 0.0, g, norm_mode, no_rotation=no_rot, isotropic=iso)
    scale = np.max(np.abs(G))
    for j in range(th.shape[0]):
        for m in range(11):
            h = 1e-6 * max(1.0, abs(th[j, m]))
            tp, tm = th.copy(), th.copy()
            tp[j, m] += h
            tm[j, m] -= h
            fd = (oracle.forward_loss(tp, Rv, t, H, imgs, d, apix, 0.0, norm_mode, no_rot, iso)
                  - oracle.forward_loss(tm, Rv, t, H, imgs, d, apix, 0.0, norm_mode, no_rot, iso)) / (2 * h)
            assert abs(fd - G[j, m]) <= 1e-7 * scale + 1e-6 * abs(fd), (j, m, fd, G[j, m])
    if no_rot:
        assert np.all(G[:, 6:10] == 0.0)
    if iso:
        assert np.all(G[:, 4:6] == 0.0)


def test_nn_lattice():
    """A cubic lattice of spacing 0.5 (exact in float32): every point's
    nearest neighbour is 0.5 away; an interior point has six at 0.5, the
    next twelve at 0.5 sqrt 2, and equal distances list smaller indices first."""
    g = np.arange(5, dtype=np.float32) * 0.5
    pts = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    dist, idx = oracle.nn_distance(pts, 16)
    assert np.all(dist[:, 0] == np.float32(0.5))
    c = 62  # (2, 2, 2)
    assert np.all(dist[c, :6] == np.float32(0.5))
    assert np.all(dist[c, 6:16] == np.float32(np.sqrt(np.float32(0.5))))
    assert list(idx[c, :6]) == sorted(idx[c, :6])
    assert set(idx[c, :6]) == {c - 25, c - 5, c - 1, c + 1, c + 5, c + 25}


def test_nn_against_kdtree():
    rng = np.random.default_rng(7)
    pts = (rng.normal(size=(3000, 3)) * 20).astype(np.float32)
    dist, idx = oracle.nn_distance(pts, 5)
    dd, ii = cKDTree(pts.astype(np.float64)).query(pts.astype(np.float64), 6)
    np.testing.assert_allclose(dist, dd[:, 1:], rtol=2e-7)
    assert np.mean(idx == ii[:, 1:]) > 0.999  # float32 vs float64 near-ties may swap


def test_nn_degenerate_inputs():
    pts = np.array([[0, 0, 0], [3, 4, 0], [np.nan, 0, 0]], dtype=np.float32)
    dist, idx = oracle.nn_distance(pts, 2)
    assert dist[0, 0] == 5.0 and idx[0, 0] == 1
    assert np.isinf(dist[0, 1]) and idx[0, 1] == -1
    assert np.all(np.isinf(dist[2])) and np.all(idx[2] == -1)
