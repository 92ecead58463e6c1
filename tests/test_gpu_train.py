"""GPU tests of the training loop: the Adam step against the oracle, a fit
to images the oracle rendered from known Gaussians, checkpoint / resume, and
the isotropic ablation with nearest-neighbour scales."""
import os

import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import synthetic as syn
from paper_2509_25075_gb300 import train

pytestmark = pytest.mark.gpu


def _raw(rng, M):
    raw = np.zeros((M, 11), dtype=np.float32)
    raw[:, 0:3] = rng.normal(size=(M, 3))
    raw[:, 3:6] = np.log(rng.uniform(1.0, 3.0, size=(M, 3)))
    raw[:, 6:10] = rng.normal(size=(M, 4))
    raw[:, 10] = np.log(rng.uniform(0.5, 1.5, size=M))
    return raw


@pytest.mark.parametrize("iso", [False, True])
def test_adam_step_matches_oracle(iso):
    rng = np.random.default_rng(100)
    M = 777
    raw = _raw(rng, M)
    m = np.zeros_like(raw)
    v = np.zeros_like(raw)
    ctx = gt.context(syn.Workload("adam", d=32, M=M, B=1, seed=1))
    R, Mm, V = gt.to_dev(raw), gt.to_dev(m), gt.to_dev(v)
    P = torch.empty_like(R)
    lr = (0.05, 0.01, 0.002, 0.02)
    iso_s = rng.uniform(0.5, 2.0, size=M).astype(np.float32) if iso else None
    ro, mo, vo = raw.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 5):
        g = rng.normal(size=raw.shape).astype(np.float32)
        g[3, 4] = np.nan  # non-finite entries count as zero
        ctx.gem_adam_step(R, Mm, V, gt.to_dev(g), P, lr, t, iso_scale=None if iso_s is None else gt.to_dev(iso_s))
        ro, mo, vo, po = oracle.adam_step(ro, mo, vo, g, lr, t, iso_scale=iso_s)
    np.testing.assert_allclose(R.cpu().numpy(), ro, rtol=2e-6, atol=2e-6)
    np.testing.assert_allclose(Mm.cpu().numpy(), mo, rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(V.cpu().numpy(), vo, rtol=2e-5, atol=1e-9)
    np.testing.assert_allclose(P.cpu().numpy(), po, rtol=4e-6, atol=2e-6)


def _problem(seed=110, M=40, N=96, d=32, apix=1.5):
    """Images the oracle renders (FP64) from known Gaussians, no noise."""
    w = syn.Workload("fit", d=d, M=M, B=N, apix=apix, s_lo=1.2, s_hi=2.2, n_clusters=6, seed=seed)
    truth = syn.gaussians(w).astype(np.float64)
    R, t = syn.views(w)
    prm = syn.ctf_params(w)
    proj = oracle.project(truth, R, t, d, w.apix, 0.0)
    H = oracle.ctf_grid_from_params(prm, d, w.apix)
    images = oracle.ctf_apply(H, proj)
    rng = np.random.default_rng(seed + 1)
    init = truth.copy()
    init[:, 0:3] += rng.normal(scale=0.6 * w.apix, size=(M, 3))
    init[:, 3:6] *= 1.25
    init[:, 10] *= 0.8
    data = {"images": images, "R": R, "t": t, "ctf_params": prm}
    model = train.ModelConfig(d=d, apix=w.apix, M=M, tau=0.0)
    return truth, init, data, model


def test_training_fits_oracle_rendered_images():
    truth, init, data, model = _problem()
    cfg = train.TrainConfig(batch=32, lr=(0.02, 0.01, 0.005, 0.01), seed=3)
    tr = train.Trainer(model, cfg, init, data)
    hist = tr.run(300, record_every=1)
    first, last = np.mean(hist[:5]), np.mean(hist[-5:])
    assert last < first / 10, (first, last)
    # the map (Eq. query) approaches the truth's; individual Gaussians may
    # trade places, so compare densities, not parameters
    fit = tr.params.cpu().numpy().astype(np.float64)
    d, apix = model.d, model.apix
    vt = oracle.query(truth, d, apix, 0.0)
    e0 = np.linalg.norm(oracle.query(init, d, apix, 0.0) - vt) / np.linalg.norm(vt)
    e1 = np.linalg.norm(oracle.query(fit, d, apix, 0.0) - vt) / np.linalg.norm(vt)
    assert e1 < 0.5 * e0, (e0, e1)
    tr.close()


def test_checkpoint_resume_continues_the_run(tmp_path):
    truth, init, data, model = _problem(seed=120)
    path = str(tmp_path / "ckpt.pt")
    cfg = train.TrainConfig(batch=16, seed=5, checkpoint_every=4, checkpoint_path=path)
    a = train.Trainer(model, cfg, init, data)
    a.run(8)
    # the checkpoint holds step 8; a fresh trainer resumed from step 4 must
    # reproduce steps 5..8 (same batches; gradients equal up to the float
    # atomics' summation order)
    b_cfg = train.TrainConfig(batch=16, seed=999)
    a4 = train.Trainer(model, cfg, init, data)
    a4.run(4)
    a4.save(path)
    b = train.Trainer(model, b_cfg, init, data)
    b.load(path)
    assert b.step_count == 4
    b.run(4)
    ra, rb = a.raw.cpu().numpy(), b.raw.cpu().numpy()
    np.testing.assert_allclose(rb, ra, rtol=1e-4, atol=1e-5)
    assert a.history[4:] == pytest.approx(b.history[4:], rel=1e-5)
    with pytest.raises(ValueError):
        other = train.Trainer(train.ModelConfig(d=32, apix=model.apix, M=model.M, tau=1e-3), b_cfg, init, data)
        other.load(path)
    for x in (a, a4, b):
        x.close()


def test_isotropic_ablation_uses_nearest_neighbour_scales():
    truth, init, data, model = _problem(seed=130)
    model = train.ModelConfig(d=model.d, apix=model.apix, M=model.M, isotropic=1, no_rotation=1)
    cfg = train.TrainConfig(batch=16, seed=7, iso_nn=True)
    tr = train.Trainer(model, cfg, init, data)
    tr.run(5)
    p = tr.params.cpu().numpy()
    # the scales of the last step are the nearest-neighbour distances of the
    # centres before that step's update (one step behind), all three equal
    assert np.all(p[:, 3] == p[:, 4]) and np.all(p[:, 3] == p[:, 5])
    assert np.all(np.isfinite(p)) and np.all(p[:, 3] > 0)
    tr.close()
