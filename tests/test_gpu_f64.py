"""FP64 check mode against the FP64 oracle (agreement to ~1e-12), and the
float path against the FP64 check mode over whole images at the largest
workload (d = 384, M = 500 000, one view)."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

F8 = torch.float64


def _d(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=F8).to(gt.DEV)


CASES = [
    (syn.Workload("f32", d=32, M=60, B=3, apix=1.2, seed=61), 0, 0.0, (0, 0)),
    (syn.Workload("f48", d=48, M=90, B=2, apix=1.0, s_lo=0.4, s_hi=5.0, seed=62), 1, 1.0, (0, 0)),
    (syn.Workload("f32a", d=32, M=50, B=2, apix=1.3, seed=63), 0, 1.0, (1, 1)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0].name)
def test_f64_step_matches_oracle(case):
    w, norm_mode, tf, (no_rot, iso) = case
    inp = gt.inputs(w)
    th = inp["params"].astype(np.float64)
    tau = tf * w.tau
    ctx = gt.context(w, tau=tau, norm_mode=norm_mode, no_rotation=no_rot, isotropic=iso)
    proj = torch.empty(w.B, w.d, w.d, dtype=F8, device=gt.DEV)
    args = [_d(th), _d(inp["R"]), _d(inp["t"])]  # read again by the backward: keep alive
    ctx.gem_project_f64(*args, proj)
    flags = dict(no_rotation=bool(no_rot), isotropic=bool(iso))
    ref = oracle.project(th, inp["R"], inp["t"], w.d, w.apix, tau, norm_mode, **flags)
    got = proj.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # CTF, loss and adjoint: parameter form
    H = oracle.ctf_grid_from_params(inp["ctf_params"], w.d, w.apix)
    L, opred, oli, og = oracle.loss(H, ref, inp["images"])
    pred = torch.empty_like(proj)
    dproj = torch.empty_like(proj)
    li = torch.empty(w.B, dtype=F8, device=gt.DEV)
    loss = torch.empty(1, dtype=F8, device=gt.DEV)
    ctx.gem_ctf_loss_f64(proj, _d(inp["images"]), ctf_params=_d(inp["ctf_params"]), pred=pred,
                         dproj=dproj, loss_img=li, loss=loss)
    assert loss.item() == pytest.approx(L, rel=1e-12)
    np.testing.assert_allclose(li.cpu().numpy(), oli, rtol=1e-12)
    assert np.max(np.abs(pred.cpu().numpy() - opred)) <= 1e-12 * np.max(np.abs(opred))
    assert np.max(np.abs(dproj.cpu().numpy() - og)) <= 1e-12 * np.max(np.abs(og))
    # a5-a6
    grad = torch.empty(w.M, 11, dtype=F8, device=gt.DEV)
    ctx.gem_project_backward_f64(dproj, grad)
    G = oracle.grad(th, inp["R"], inp["t"], w.d, w.apix, tau, og, norm_mode, **flags)
    got = grad.cpu().numpy()
    assert np.linalg.norm(got - G) <= 1e-11 * np.linalg.norm(G)
    big = np.abs(G) > 1e-3 * np.max(np.abs(G))
    assert np.max(np.abs(got[big] - G[big]) / np.abs(G[big])) <= 1e-9
    assert ctx.gem_status() == 0


def test_f64_ctf_array_form():
    w = syn.Workload("fa", d=48, M=10, B=2, seed=64)
    rng = np.random.default_rng(65)
    half = rng.uniform(-1, 1, size=(w.B, w.d, w.d // 2 + 1))
    proj = rng.normal(size=(w.B, w.d, w.d))
    imgs = rng.normal(size=(w.B, w.d, w.d))
    ctx = gt.context(w)
    pred = torch.empty(w.B, w.d, w.d, dtype=F8, device=gt.DEV)
    dproj = torch.empty_like(pred)
    loss = torch.empty(1, dtype=F8, device=gt.DEV)
    ctx.gem_ctf_loss_f64(_d(proj), _d(imgs), ctf=_d(half), pred=pred, dproj=dproj, loss=loss)
    L, opred, _, og = oracle.loss(oracle.ctf_grid_from_half(half), proj, imgs)
    assert loss.item() == pytest.approx(L, rel=1e-12)
    assert np.max(np.abs(pred.cpu().numpy() - opred)) <= 1e-12 * np.max(np.abs(opred))
    assert np.max(np.abs(dproj.cpu().numpy() - og)) <= 1e-12 * np.max(np.abs(og))


def test_float_path_against_f64_check_at_full_size():
    """A5 (d = 384, M = 500 000), one view: the float tiled projection and
    gradient over whole images against the FP64 check mode, which is itself
    pinned to the oracle on sampled pixels."""
    w = syn.WORKLOADS["A5"]
    inp = gt.inputs(w)
    R, t = inp["R"][:1], inp["t"][:1]
    th = inp["params"]
    ctx = gt.context(w, zsort=1)
    p64 = torch.empty(1, w.d, w.d, dtype=F8, device=gt.DEV)
    a64 = [_d(th), _d(R), _d(t)]  # read again by the backward passes: keep alive
    ctx.gem_project_f64(*a64, p64)
    p32 = torch.empty(1, w.d, w.d, device=gt.DEV)
    a32 = [gt.to_dev(th), gt.to_dev(R), gt.to_dev(t)]
    ctx.gem_project(*a32, p32)
    g = syn.smooth_field(w, B=1) * 1e-3
    g64 = torch.empty(w.M, 11, dtype=F8, device=gt.DEV)
    ctx.gem_project_backward_f64(_d(g), g64)
    g32 = torch.empty(w.M, 11, device=gt.DEV)
    ctx.gem_project_backward(gt.to_dev(g), g32)
    assert ctx.gem_status() == 0
    img64 = p64.cpu().numpy()
    rng = np.random.default_rng(66)
    pix = rng.integers(0, w.d * w.d, 48)
    ref = oracle.project_pixels(th, R, t, w.d, w.apix, w.tau, pix)
    assert np.max(np.abs(img64.reshape(-1)[pix] - ref)) <= 1e-12 * np.max(np.abs(img64))
    # float32 against FP64 over the whole image: 1e-5 of the maximum plus
    # tau per pair float32 may put on the other side of the threshold
    err = np.abs(p32.cpu().numpy().astype(np.float64) - img64)
    assert np.max(err) <= 1e-5 * np.max(np.abs(img64)) + 8 * w.tau
    G64, G32 = g64.cpu().numpy(), g32.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(G32 - G64) <= 1e-4 * np.linalg.norm(G64)
