"""Pins of the oracle's density query (Eq. query) against scipy's Gaussian
density, closed forms, the mass, and the oracle's independently pinned
projection (integrating the volume along z must give the image)."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.stats import multivariate_normal

import oracle

from test_oracle_pins import _random_theta


def _sigma(theta):
    w, x, y, z = theta[6:10]
    Rq = Rotation.from_quat([x, y, z, w]).as_matrix()
    return Rq @ np.diag(np.asarray(theta[3:6], dtype=np.float64) ** 2) @ Rq.T


def test_query_matches_scipy_density():
    rng = np.random.default_rng(40)
    d, apix = 16, 1.3
    th = _random_theta(rng, 4)
    th[:, 0:3] = rng.uniform(-5, 5, size=(4, 3))
    vox = rng.integers(0, d ** 3, 300)
    got0 = oracle.query_voxels(th, d, apix, 0.0, vox, norm_mode=0)
    got1 = oracle.query_voxels(th, d, apix, 0.0, vox, norm_mode=1)
    x, y, z = vox % d, (vox // d) % d, vox // (d * d)
    X = np.stack([x, y, z], 1) * apix - d / 2 * apix
    want0 = np.zeros(len(vox))
    want1 = np.zeros(len(vox))
    for t in th:
        S = _sigma(t)
        pdf = multivariate_normal(mean=t[0:3], cov=S).pdf(X)
        want0 += t[10] * pdf
        want1 += t[10] * pdf * (2 * np.pi) ** 1.5 * np.sqrt(np.linalg.det(S))
    np.testing.assert_allclose(got0, want0, rtol=1e-10, atol=1e-300)
    np.testing.assert_allclose(got1, want1, rtol=1e-10, atol=1e-300)


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_query_peak_closed_form(norm_mode):
    d, apix, s = 16, 0.9, 1.7
    th = np.zeros((1, 11))
    th[0, 0:3] = (1 * apix, -2 * apix, 3 * apix)  # on a voxel centre
    th[0, 3:6] = s
    th[0, 6:10] = (0.2, 0.9, -0.1, 0.4)
    th[0, 10] = 1.4
    vol = oracle.query(th, d, apix, 0.0, norm_mode)
    peak = vol[d // 2 + 3, d // 2 - 2, d // 2 + 1]
    want = 1.4 if norm_mode == 1 else 1.4 / ((2 * np.pi) ** 1.5 * s ** 3)
    assert peak == pytest.approx(want, rel=1e-14)
    assert peak == vol.max()


def test_query_mass():
    """apix^3 * sum of voxels = sum of rho (mode 0, well-sampled Gaussians
    inside the box; the grid sum of a Gaussian is exact to e^(-2 pi^2 s^2))."""
    rng = np.random.default_rng(41)
    d, apix = 48, 1.0  # centres 8 sigma or more from the faces
    th = _random_theta(rng, 5)
    th[:, 0:3] = rng.uniform(-4, 4, size=(5, 3))
    th[:, 3:6] = rng.uniform(1.5, 2.5, size=(5, 3))
    vol = oracle.query(th, d, apix, 0.0, 0)
    assert apix ** 3 * vol.sum() == pytest.approx(th[:, 10].sum(), rel=1e-10)


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_query_integrates_to_the_projection(norm_mode):
    """Summing the volume along z (times apix) gives the identity-view image
    of Eq. render (mode 0) or of the exact line integral (mode 1)."""
    rng = np.random.default_rng(42 + norm_mode)
    d, apix = 48, 1.1  # every Gaussian 7 sigma or more inside the faces
    th = _random_theta(rng, 6)
    th[:, 0:3] = rng.uniform(-5, 5, size=(6, 3))
    th[:, 3:6] = rng.uniform(1.6, 3.0, size=(6, 3))
    vol = oracle.query(th, d, apix, 0.0, norm_mode)
    img = oracle.project(th, np.eye(3)[None], np.zeros((1, 2)), d, apix, 0.0, norm_mode)[0]
    np.testing.assert_allclose(apix * vol.sum(axis=0), img, rtol=1e-9, atol=1e-12 * img.max())


def test_query_threshold_keeps_only_values_above_tau():
    rng = np.random.default_rng(44)
    d, apix = 16, 1.0
    th = _random_theta(rng, 1)
    th[0, 0:3] = (0.3, -0.2, 0.1)
    full = oracle.query(th, d, apix, 0.0, 1)
    tau = 0.37 * full.max()
    cut = oracle.query(th, d, apix, tau, 1)
    np.testing.assert_array_equal(cut, np.where(full > tau, full, 0.0))
    assert np.all(oracle.query(th, d, apix, 2 * full.max(), 1) == 0.0)


def test_query_ablation_flags():
    """Isotropic + no rotation: a spherical Gaussian of radius s0 whatever
    s1, s2 and q are."""
    d, apix = 16, 1.0
    th = np.zeros((1, 11))
    th[0, 3:6] = (2.0, 0.3, 9.0)
    th[0, 6:10] = (0.0, 0.0, 0.0, 0.0)
    th[0, 10] = 1.0
    vol = oracle.query(th, d, apix, 0.0, 1, no_rotation=True, isotropic=True)
    c = np.arange(d) - d / 2
    r2 = c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2
    np.testing.assert_allclose(vol, np.exp(-0.5 * r2 / 4.0), rtol=1e-13)
