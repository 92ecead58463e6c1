"""Pins of the oracle's Fourier shell correlation (Eq. fsc) against a
brute-force DFT, Parseval, the identities FSC(X, aX) = sign(a), and
hand-computed threshold crossings."""
import numpy as np
import pytest

import oracle


def _dft3(X):
    """3D DFT by explicit sums over all voxels (tiny grids only)."""
    d = X.shape[0]
    n = np.arange(d)
    W = np.exp(-2j * np.pi * np.outer(n, n) / d)
    out = np.zeros((d, d, d), dtype=complex)
    for kz in range(d):
        for ky in range(d):
            for kx in range(d):
                out[kz, ky, kx] = np.sum(X * W[kz][:, None, None] * W[ky][None, :, None] * W[kx][None, None, :])
    return out


def test_shell_sums_match_brute_force_dft():
    rng = np.random.default_rng(70)
    d = 6
    X1, X2 = rng.normal(size=(2, d, d, d))
    num, p1, p2 = oracle.fsc_shell_sums(X1, X2)
    F1, F2 = _dft3(X1), _dft3(X2)
    want = np.zeros((3, len(num)))
    for kz in range(d):
        for ky in range(d):
            for kx in range(d):
                s = [k if k < d / 2 else k - d for k in (kz, ky, kx)]
                sh = int(np.floor(np.sqrt(sum(v * v for v in s)) + 0.5))
                want[0, sh] += (F1[kz, ky, kx] * np.conj(F2[kz, ky, kx])).real
                want[1, sh] += abs(F1[kz, ky, kx]) ** 2
                want[2, sh] += abs(F2[kz, ky, kx]) ** 2
    np.testing.assert_allclose(num, want[0], rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(p1, want[1], rtol=1e-10)
    np.testing.assert_allclose(p2, want[2], rtol=1e-10)


def test_parseval_over_all_shells():
    rng = np.random.default_rng(71)
    d = 12
    X1, X2 = rng.normal(size=(2, d, d, d))
    num, p1, p2 = oracle.fsc_shell_sums(X1, X2)
    assert p1.sum() == pytest.approx(d ** 3 * np.sum(X1 ** 2), rel=1e-12)
    assert num.sum() == pytest.approx(d ** 3 * np.sum(X1 * X2), rel=1e-10, abs=1e-8)
    # shell populations: shell 0 holds only k = 0, shell 1 the 6 axis neighbours
    _, cnt, _ = oracle.fsc_shell_sums(np.ones((d, d, d)), np.ones((d, d, d)))
    assert cnt[0] == pytest.approx(d ** 6) and np.all(cnt[1:] == 0)


def test_fsc_identities():
    rng = np.random.default_rng(72)
    X = rng.normal(size=(16, 16, 16))
    c, _, res = oracle.fsc(X, X, 1.3)
    np.testing.assert_allclose(c, 1.0, rtol=1e-12)
    assert res == pytest.approx(2 * 1.3)  # never crosses: Nyquist
    c2, _, _ = oracle.fsc(X, -2.5 * X, 1.3)
    np.testing.assert_allclose(c2, -1.0, rtol=1e-12)
    c3, _, _ = oracle.fsc(X, 0.1 * X + 7.0, 1.3)  # offset only moves shell 0
    np.testing.assert_allclose(c3[1:], 1.0, rtol=1e-12)


def test_fsc_of_independent_noise_is_small():
    rng = np.random.default_rng(73)
    X1, X2 = rng.normal(size=(2, 32, 32, 32))
    c, (num, p1, p2), _ = oracle.fsc(X1, X2, 1.0)
    # shell i of a 32^3 grid holds ~4 pi i^2 frequencies: |FSC| ~ 1/sqrt(that)
    i = np.arange(4, 17)
    assert np.all(np.abs(c[i]) < 5.0 / np.sqrt(2 * np.pi * i ** 2))


@pytest.mark.parametrize("curve,kstar", [
    ([1.0, 0.9, 0.5, 0.1, 0.0], 2 + (0.5 - 0.143) / 0.4),
    ([1.0, 0.1, 0.0], (1.0 - 0.143) / 0.9),
    ([1.0, 0.9, 0.8, 0.7], 3.0),
    ([1.0, 0.95, 0.143, 0.0], 2.0),  # exactly at the threshold is not below it
])
def test_crossing_hand_computed(curve, kstar):
    assert oracle.fsc_crossing(curve, 64, 1.25) == pytest.approx(64 * 1.25 / kstar, rel=1e-12)
