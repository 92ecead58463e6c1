"""GPU parity of the Fourier shell correlation (Eq. fsc) through the C ABI
against the oracle: random and correlated maps on several grid sizes, maps
made by the density query, and the threshold crossing."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _ctx(d, apix=1.2):
    return gt.context(syn.Workload("fsc", d=d, M=16, B=1, apix=apix, seed=1))


def _compare(ctx, X1, X2, thr=0.143):
    fsc, sums, res = ctx.gem_fsc(gt.to_dev(X1), gt.to_dev(X2), thr)
    assert ctx.gem_status() == 0
    c, (num, p1, p2), r = oracle.fsc(X1.astype(np.float32), X2.astype(np.float32), ctx.apix, thr)
    got = sums.cpu().numpy()
    # sums: relative to the shell's power scale
    scale = np.sqrt(p1 * p2)
    np.testing.assert_allclose(got[1], p1, rtol=2e-5, atol=1e-6 * p1.max())
    np.testing.assert_allclose(got[2], p2, rtol=2e-5, atol=1e-6 * p2.max())
    assert np.all(np.abs(got[0] - num) <= 2e-5 * scale + 1e-6 * scale.max())
    np.testing.assert_allclose(fsc.cpu().numpy(), c, atol=5e-5)
    return float(res.item()), r, c


@pytest.mark.parametrize("d", [16, 48, 96])
def test_fsc_random_maps(d):
    rng = np.random.default_rng(d)
    X1 = rng.normal(size=(d, d, d)).astype(np.float32)
    X2 = (0.7 * X1 + 0.5 * rng.normal(size=(d, d, d))).astype(np.float32)
    _compare(_ctx(d), X1, X2)


def test_fsc_crossing_of_correlated_maps():
    """Two noisy copies of a smooth map: the FSC falls with frequency and
    crosses 0.143; the GPU crossing agrees with the oracle's."""
    d = 64
    rng = np.random.default_rng(80)
    k = np.fft.fftfreq(d)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    signal = np.real(np.fft.ifftn(np.fft.fftn(rng.normal(size=(d, d, d))) * np.exp(-k2 / (2 * 0.08 ** 2))))
    signal /= signal.std()
    X1 = (signal + 0.3 * rng.normal(size=(d, d, d))).astype(np.float32)
    X2 = (signal + 0.3 * rng.normal(size=(d, d, d))).astype(np.float32)
    ctx = _ctx(d, apix=1.3)
    res, r, c = _compare(ctx, X1, X2)
    assert c[1] > 0.9 and c[-1] < 0.143
    assert 2 * 1.3 < r < d * 1.3
    assert res == pytest.approx(r, rel=1e-4)


@pytest.mark.parametrize("name", ["A2", "A3"])
def test_fsc_of_query_maps(name):
    """Half-maps in the GSFSC sense: the density of the Gaussians and of a
    perturbed copy, both from the density query."""
    w = syn.WORKLOADS[name]
    th = syn.gaussians(w)
    rng = np.random.default_rng(81)
    th2 = th.copy()
    th2[:, 0:3] += rng.normal(scale=0.3 * w.apix, size=(w.M, 3)).astype(np.float32)
    ctx = gt.context(w)
    v1 = ctx.gem_query(gt.to_dev(th), w.tau_query).clone()
    v2 = ctx.gem_query(gt.to_dev(th2), w.tau_query).clone()
    X1, X2 = v1.cpu().numpy(), v2.cpu().numpy()
    res, r, _ = _compare(ctx, X1, X2)
    assert res == pytest.approx(r, rel=1e-4)


def test_fsc_rejects_bad_threshold():
    from paper_2509_25075_gb300 import binding
    ctx = _ctx(16)
    X = torch.zeros(16, 16, 16, device=gt.DEV)
    with pytest.raises(binding.GemError) as ei:
        ctx.gem_fsc(X, X, 1.5)
    assert ei.value.code == binding.GEM_EINVAL
