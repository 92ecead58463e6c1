"""Edge cases of the float path against the oracle: empty tile lists, a
single Gaussian and a single view, Gaussians that cannot contribute mixed
with ones that do, one tile whose list spans many windows, the smallest and
largest image sides, and images whose sides need a radix-3 FFT stage."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _run(w, th, R, t, g=None, **ctx_kw):
    ctx = gt.context(w, **ctx_kw)
    args = [gt.to_dev(th), gt.to_dev(R), gt.to_dev(t)]
    proj = torch.empty(R.shape[0], w.d, w.d, device=gt.DEV)
    ctx.gem_project(*args, proj)
    grad = None
    if g is not None:
        grad = torch.empty(th.shape[0], 11, device=gt.DEV)
        ctx.gem_project_backward(gt.to_dev(g), grad)
    assert ctx.gem_status() == 0
    return ctx, proj.cpu().numpy(), None if grad is None else grad.cpu().numpy()


def test_gaussians_outside_every_view_give_empty_lists():
    w = syn.Workload("out", d=32, M=40, B=3, seed=71)
    inp = gt.inputs(w)
    th = inp["params"].copy()
    th[:, 0] += 500.0  # far beyond the image, in every view's x or y
    th[:, 1] += 500.0
    th[:, 2] += 500.0
    g = np.ones((w.B, w.d, w.d), dtype=np.float32)
    ctx, proj, grad = _run(w, th, inp["R"], inp["t"], g)
    assert ctx.gem_pair_count() == 0
    assert np.all(proj == 0.0)
    assert np.all(grad == 0.0)


def test_single_gaussian_single_view():
    w = syn.Workload("one", d=32, M=1, B=1, seed=72)
    th = np.array([[0.7, -1.1, 0.4, 2.0, 3.1, 1.4, 0.9, 0.2, -0.3, 0.1, 1.3]], dtype=np.float32)
    R = np.eye(3, dtype=np.float32)[None]
    t = np.array([[0.5, -0.25]], dtype=np.float32)
    g = syn.smooth_field(w) * 1e-2
    _, proj, grad = _run(w, th, R, t, g)
    ref = oracle.project(th, R, t, w.d, w.apix, w.tau)
    gt.assert_proj_close(proj, ref)
    gt.assert_grad_close(grad, oracle.grad(th, R, t, w.d, w.apix, w.tau, g))


def test_degenerate_gaussians_contribute_nothing():
    """rho <= 0, a zero quaternion, zero scales, NaN and infinite parameters:
    no contribution and zero gradient; the valid Gaussians are unaffected."""
    w = syn.Workload("degen", d=48, M=60, B=2, seed=73)
    inp = gt.inputs(w)
    th = inp["params"].copy()
    th[0, 10] = 0.0
    th[1, 10] = -1.0
    th[2, 6:10] = 0.0
    th[3, 3:6] = 0.0
    th[4, 0] = np.nan
    th[5, 3] = np.inf
    bad = [0, 1, 2, 3, 4, 5]
    g = syn.smooth_field(w) * 1e-3
    _, proj, grad = _run(w, th, inp["R"], inp["t"], g)
    assert np.all(np.isfinite(proj)) and np.all(np.isfinite(grad))
    keep = np.ones(w.M, bool)
    keep[bad] = False
    good = {"params": th[keep], "R": inp["R"], "t": inp["t"]}
    ref = oracle.project(th[keep], inp["R"], inp["t"], w.d, w.apix, w.tau)
    gt.assert_proj_close(proj, ref, w.tau, gt.borderline_pairs(good, w, w.tau))
    assert np.all(grad[bad] == 0.0)
    G = oracle.grad(th[keep], inp["R"], inp["t"], w.d, w.apix, w.tau, g)
    gt.assert_grad_close(grad[keep], G)


def test_one_tile_list_spanning_many_windows():
    """Every Gaussian on the same spot: one tile's list holds thousands of
    entries (many staging windows), in depth order."""
    w = syn.Workload("pile", d=32, M=3000, B=2, s_lo=0.6, s_hi=1.2, seed=74)
    inp = gt.inputs(w)
    th = inp["params"].copy()
    rng = np.random.default_rng(75)
    th[:, 0:3] = rng.normal(scale=0.5, size=(w.M, 3)) + np.array([3.0, -2.0, 0.0])
    g = syn.smooth_field(w) * 1e-3
    ctx, proj, grad = _run(w, th, inp["R"], inp["t"], g)
    ts = ctx.gem_inspect_bins()[0].cpu().numpy()
    assert np.max(np.diff(ts)) > 1000
    ref = oracle.project(th, inp["R"], inp["t"], w.d, w.apix, w.tau)
    border = gt.borderline_pairs({"params": th, "R": inp["R"], "t": inp["t"]}, w, w.tau)
    gt.assert_proj_close(proj, ref, w.tau, border)
    gt.assert_grad_close(grad, oracle.grad(th, inp["R"], inp["t"], w.d, w.apix, w.tau, g))


@pytest.mark.parametrize("d", [16, 144, 768])
def test_smallest_radix3_and_largest_sides(d):
    w = syn.Workload(f"d{d}", d=d, M=150, B=2, apix=1.1, seed=76)
    inp = gt.inputs(w)
    g = syn.smooth_field(w) * 1e-3
    ctx, proj, grad = _run(w, inp["params"], inp["R"], inp["t"], g)
    if d <= 144:
        ref = oracle.project(inp["params"], inp["R"], inp["t"], d, w.apix, w.tau)
        border = gt.borderline_pairs(inp, w, w.tau)
        gt.assert_proj_close(proj, ref, w.tau, border)
        gt.assert_grad_close(grad, oracle.grad(inp["params"], inp["R"], inp["t"], d, w.apix, w.tau, g))
    else:
        rng = np.random.default_rng(77)
        pix = rng.integers(0, w.B * d * d, 200)
        ref = oracle.project_pixels(inp["params"], inp["R"], inp["t"], d, w.apix, w.tau, pix)
        assert np.max(np.abs(proj.reshape(-1)[pix] - ref)) <= 1e-5 * np.max(np.abs(proj)) + 8 * w.tau
        sel = rng.choice(w.M, 10, replace=False)
        G = oracle.grad(inp["params"], inp["R"], inp["t"], d, w.apix, w.tau, g, sel=sel)
        for k, j in enumerate(sel):
            n = np.linalg.norm(G[k])
            assert np.linalg.norm(grad[j] - G[k]) <= 1e-4 * n + 1e-12
    # the CTF step at this side
    prm = syn.ctf_params(w)
    imgs = syn.images(w)
    loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
    dproj = torch.empty(w.B, d, d, device=gt.DEV)
    ctx.gem_ctf_loss(gt.to_dev(proj), gt.to_dev(imgs), ctf_params=gt.to_dev(prm), dproj=dproj, loss=loss)
    if d <= 144:
        L, _, _, og = oracle.loss(oracle.ctf_grid_from_params(prm, d, w.apix), proj, imgs)
        assert loss.item() == pytest.approx(L, rel=1e-5)
        assert np.max(np.abs(dproj.cpu().numpy() - og)) <= 2e-6 * np.max(np.abs(og))
    else:
        sel = np.array([1])
        L, _, oli, og = oracle.loss(oracle.ctf_grid_from_params(prm[sel], d, w.apix), proj[sel], imgs[sel])
        og = og * len(sel) / w.B
        assert np.max(np.abs(dproj.cpu().numpy()[sel] - og)) <= 2e-6 * np.max(np.abs(og))
