"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (same context settings, and the rasteriser configurations the
autotuner picks for the shape, as bench.py picks them), on outputs the
oracle can compute one by one: sampled projected pixels, the loss and
adjoint of sampled images, and the gradient of sampled Gaussians for a
seeded upstream gradient."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

FULL = ["A2", "A3", "A4", "A5"]


def _ctx(w):
    return gt.context(w, zsort=1)


def _tuned(ctx, args):
    """The autotuner's choice for this shape, as bench.py makes it; the
    context then runs it (no configuration named)."""
    f, b = ctx.gem_autotune(*args, reps=2)
    M, B = args[0].shape[0], args[1].shape[0]
    assert ctx.gem_get_raster_config(B, M) == (f, b)
    return f, b


@pytest.mark.parametrize("name", FULL)
def test_fullsize_projection_sampled_pixels(name):
    w = syn.WORKLOADS[name]
    inp = gt.inputs(w)
    ctx = _ctx(w)
    proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    args = [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
    _tuned(ctx, args)
    ctx.gem_project(*args, proj)
    assert ctx.gem_status() == 0
    rng = np.random.default_rng(100)
    # half the samples near the particle (the image centre), half anywhere
    n = 96
    b = rng.integers(0, w.B, n)
    c = w.d // 2
    r = int(0.3 * w.d)
    v = np.where(np.arange(n) < n // 2, rng.integers(c - r, c + r, n), rng.integers(0, w.d, n))
    u = np.where(np.arange(n) < n // 2, rng.integers(c - r, c + r, n), rng.integers(0, w.d, n))
    pix = (b * w.d + v) * w.d + u
    ref = oracle.project_pixels(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, pix)
    got = proj.cpu().numpy().reshape(-1)[pix].astype(np.float64)
    scale = float(proj.abs().max().item())
    # within 1e-5 of the image maximum, plus tau per pair that float32 and
    # float64 may put on different sides of the threshold (at most a few per
    # pixel here)
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale + 8 * w.tau
    ctx.close()


@pytest.mark.parametrize("name", FULL)
def test_fullsize_ctf_loss_sampled_images(name):
    w = syn.WORKLOADS[name]
    proj = syn.smooth_field(w)
    imgs = syn.images(w)
    prm = syn.ctf_params(w)
    ctx = _ctx(w)
    pred = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    dproj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    li = torch.empty(w.B, dtype=torch.float64, device=gt.DEV)
    loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
    ctx.gem_ctf_loss(gt.to_dev(proj), gt.to_dev(imgs), ctf_params=gt.to_dev(prm), pred=pred, dproj=dproj,
                     loss_img=li, loss=loss)
    sel = np.array([0, w.B // 3, w.B - 1])
    H = oracle.ctf_grid_from_params(prm[sel], w.d, w.apix)
    _, opred, oli, og = oracle.loss(H, proj[sel], imgs[sel])
    np.testing.assert_allclose(li.cpu().numpy()[sel], oli, rtol=1e-5)
    # the oracle's adjoint of the 3-image batch carries 2 / (3 d^2)
    og = og * len(sel) / w.B
    p = pred.cpu().numpy()[sel]
    assert np.max(np.abs(p - opred)) <= 1e-5 * np.max(np.abs(opred))
    g = dproj.cpu().numpy()[sel]
    assert np.max(np.abs(g - og)) <= 2e-6 * np.max(np.abs(og))
    # the batch loss is the mean of the per-image losses
    assert loss.item() == pytest.approx(float(li.double().mean().item()), rel=1e-12)
    ctx.close()


@pytest.mark.parametrize("upstream", ["smooth", "noise"])
@pytest.mark.parametrize("name", FULL)
def test_fullsize_gradient_sampled_gaussians(name, upstream):
    """The gradient of sampled Gaussians at full size, each held to the
    contract's 1e-4 of its own gradient (per entry 1e-3 where significant),
    plus the terms of its pairs that sit within 1e-5 relative of tau; for a
    smooth upstream gradient and for one that is noise (as the adjoint of a
    loss against noisy images is)."""
    w = syn.WORKLOADS[name]
    inp = gt.inputs(w)
    if upstream == "smooth":
        g = syn.smooth_field(w) * 1e-3
    else:
        g = np.random.default_rng(102).normal(size=(w.B, w.d, w.d)).astype(np.float32) * 1e-3
    ctx = _ctx(w)
    proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    # params, R and t stay referenced: the backward reads them again
    args = [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
    _tuned(ctx, args)
    ctx.gem_project(*args, proj)
    grad = torch.empty(w.M, 11, device=gt.DEV)
    ctx.gem_project_backward(gt.to_dev(g), grad)
    assert ctx.gem_status() == 0
    rng = np.random.default_rng(101)
    sel = rng.choice(w.M, size=12, replace=False)
    ref = oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g, sel=sel)
    border = oracle.grad_border(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g, rel=1e-5, sel=sel)
    gt.assert_grad_per_gaussian(grad.cpu().numpy()[sel], ref, border)
    ctx.close()
