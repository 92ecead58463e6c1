"""GPU parity: every step of the hot path through the C ABI against the FP64
oracle on the same seeded inputs (tolerances in gemtest.py)."""
import math

import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import binding
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

# small cases: several tiles, M and B not multiples of any chunk or group size
SMALL = [
    syn.Workload("s48", d=48, M=1037, B=5, apix=1.2, seed=11),
    syn.Workload("s64", d=64, M=733, B=3, apix=1.3, seed=12),
    syn.Workload("s32w", d=32, M=301, B=2, apix=1.0, s_lo=0.3, s_hi=6.0, n_clusters=4, seed=13),
]
# Gaussians so large that the first chunk of 256 (depth order) has more block
# rows (big96: about 3100, big128: 3900) and more candidate tiles (3600,
# 5100) than the tile count stages (2048 of each), while the second chunk
# fits both: the staged and the unstaged paths run in one binning.
# Their lists need more than the default 16 entries per (image, Gaussian)
# (big128: about 17), so their contexts get 64.
LARGE = [
    syn.Workload("big96", d=96, M=300, B=2, apix=1.2, s_lo=3.0, s_hi=10.0, n_clusters=3, seed=14),
    syn.Workload("big128", d=128, M=300, B=2, apix=1.2, s_lo=4.0, s_hi=12.0, n_clusters=3, seed=14),
]
LARGE_PAIRS = {w.name: 64 * w.B * w.M for w in LARGE}
# elongated Gaussians: scales drawn independently per axis over 0.3-12 px,
# so many are needles up to 40 times longer than wide, seen at every angle
NEEDLES = syn.Workload("needles", d=64, M=400, B=6, apix=1.2, s_lo=0.3, s_hi=12.0, n_clusters=4, seed=15)


def _project(w, inp, dense=False, **kw):
    if w.name in LARGE_PAIRS:
        kw.setdefault("max_pairs", LARGE_PAIRS[w.name])
    ctx = gt.context(w, **kw)
    proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    args = [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
    if dense:
        ctx.gem_project_dense(*args, proj)
    else:
        ctx.gem_project(*args, proj)
    assert ctx.gem_status() == 0
    return ctx, args, proj


@pytest.mark.parametrize("w", SMALL, ids=lambda w: w.name)
def test_records_match_oracle(w):
    inp = gt.inputs(w)
    ctx, _, _ = _project(w, inp)
    rec = ctx.gem_inspect_records().cpu().numpy().astype(np.float64)
    ref = oracle.preprocess(inp["params"], inp["R"], inp["t"], w.norm_mode)
    valid = ref[..., 7] == 1
    np.testing.assert_array_equal(rec[..., 7] == 1, valid)
    px = ref[..., 0] / w.apix + w.d / 2
    py = ref[..., 1] / w.apix + w.d / 2
    np.testing.assert_allclose(rec[..., 0][valid], px[valid], rtol=0, atol=2e-5 * w.d)
    np.testing.assert_allclose(rec[..., 1][valid], py[valid], rtol=0, atol=2e-5 * w.d)
    cov = np.stack([ref[..., 2], ref[..., 3], ref[..., 3], ref[..., 4]], -1).reshape(*ref.shape[:2], 2, 2)
    con = np.linalg.inv(cov[valid] / w.apix ** 2)
    scale = np.max(np.abs(con), axis=(1, 2))
    got = rec[..., 2:5][valid]
    for k, (a, b) in enumerate([(0, 0), (0, 1), (1, 1)]):
        np.testing.assert_array_less(np.abs(got[:, k] - con[:, a, b]), 1e-5 * scale + 1e-30)
    np.testing.assert_allclose(rec[..., 5][valid], np.log2(ref[..., 5][valid]), rtol=0, atol=2e-6 * 30)
    np.testing.assert_allclose(rec[..., 6][valid], ref[..., 6][valid], rtol=0, atol=1e-5 * w.d * w.apix)


@pytest.mark.parametrize("zsort", [1, 0])
@pytest.mark.parametrize("w", SMALL + LARGE + [NEEDLES], ids=lambda w: w.name)
def test_bins_cover_exact_pairs_and_are_ordered(w, zsort):
    """Each tile list holds every Gaussian with a pixel above tau in that tile
    (brute force), only Gaussians whose extent box meets the tile, no
    duplicates, in ascending depth (zsort 1) or slot order (zsort 0: the
    3D Morton key of the mean, then the index)."""
    inp = gt.inputs(w)
    ctx, _, _ = _project(w, inp, zsort=zsort)
    ts, lst = ctx.gem_inspect_bins()
    ts, lst = ts.cpu().numpy(), lst.cpu().numpy()
    hits = oracle.tile_hits(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, 16, w.norm_mode)
    pre = oracle.preprocess(inp["params"], inp["R"], inp["t"], w.norm_mode)
    nt = w.d // 16
    T = nt * nt
    depth = pre[..., 6]
    qstep = 2.0 * w.d * w.apix / 65536
    # extent box of value > tau * exp(-margin) (FP64), in pixel coordinates
    amp = pre[..., 5]
    with np.errstate(divide="ignore", invalid="ignore"):
        kappa = 2.0 * (np.log(np.maximum(amp, 1e-300) / w.tau) + 1e-3 / math.log2(math.e) * 2)
    rx = np.sqrt(np.maximum(kappa, 0) * pre[..., 2]) / w.apix
    ry = np.sqrt(np.maximum(kappa, 0) * pre[..., 4]) / w.apix
    cx = pre[..., 0] / w.apix + w.d / 2
    cy = pre[..., 1] / w.apix + w.d / 2
    mkey = gt.morton_keys(inp["params"], w.d, w.apix)
    assert ts[-1] == len(lst) == ctx.gem_pair_count()
    for b in range(w.B):
        for t in range(T):
            ent = lst[ts[b * T + t]:ts[b * T + t + 1]]
            assert len(np.unique(ent)) == len(ent)
            want = set(np.nonzero(hits[b, :, t])[0].tolist())
            have = set(ent.tolist())
            assert want <= have, (b, t, sorted(want - have)[:5])
            ty, tx = divmod(t, nt)
            x0, y0 = 16 * tx, 16 * ty
            for j in have - want:
                assert cx[b, j] + rx[b, j] + 1e-3 >= x0 and cx[b, j] - rx[b, j] - 1e-3 <= x0 + 15
                assert cy[b, j] + ry[b, j] + 1e-3 >= y0 and cy[b, j] - ry[b, j] - 1e-3 <= y0 + 15
            if zsort:
                dz = np.diff(depth[b, ent])
                assert np.all(dz >= -qstep), (b, t, dz.min())
            else:
                order = mkey[ent].astype(np.int64) * w.M + ent
                assert np.all(np.diff(order) > 0)


@pytest.mark.parametrize("w", SMALL + LARGE, ids=lambda w: w.name)
def test_kept_pair_count_matches_brute_force(w):
    """The rasteriser's walk (tile lists + 4x4 block masks) finds every pair
    whose value exceeds tau: its kept count equals the oracle's brute-force
    count up to pairs within float32 reach of tau."""
    inp = gt.inputs(w)
    ctx, _, _ = _project(w, inp)
    kept, evaluated = ctx.gem_pair_stats()
    ref, border = gt.kept_pairs(inp, w, w.tau)
    assert abs(kept - ref) <= border, (kept, ref, border)
    assert evaluated >= kept


@pytest.mark.parametrize("w", SMALL, ids=lambda w: w.name)
def test_bins_are_deterministic(w):
    inp = gt.inputs(w)
    ctx, args, proj = _project(w, inp)
    ts1, l1 = [x.cpu().clone() for x in ctx.gem_inspect_bins()]
    p1 = proj.cpu().clone()
    proj2 = torch.empty_like(proj)
    ctx.gem_project(*args, proj2)
    ts2, l2 = [x.cpu() for x in ctx.gem_inspect_bins()]
    assert torch.equal(ts1, ts2) and torch.equal(l1, l2)
    assert torch.equal(p1, proj2.cpu())


@pytest.mark.parametrize("norm_mode", [0, 1])
@pytest.mark.parametrize("dense", [False, True], ids=["tiled", "dense"])
@pytest.mark.parametrize("w", SMALL, ids=lambda w: w.name)
def test_projection_matches_oracle(w, dense, norm_mode):
    inp = gt.inputs(w)
    tau = w.tau if norm_mode == 0 else w.tau * 50
    _, _, proj = _project(w, inp, dense=dense, norm_mode=norm_mode, tau=tau)
    ref = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, tau, norm_mode)
    border = gt.borderline_pairs(inp, w, tau, norm_mode)
    gt.assert_proj_close(proj.cpu().numpy(), ref, tau, border)


@pytest.mark.parametrize("w", LARGE, ids=lambda w: w.name)
def test_large_gaussians_projection_and_gradient(w):
    """Projection and gradient when the binning's chunk staging overflows.
    A wide Gaussian's gradient entries are sums of thousands of per-pixel
    terms of both signs; every Gaussian is held to 1e-4 of its own gradient
    (1e-3 per significant entry), plus the terms of its pairs within 1e-5
    relative of tau, and the whole to the usual norm tolerance."""
    inp = gt.inputs(w)
    ctx, _, proj = _project(w, inp)
    ref = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau)
    gt.assert_proj_close(proj.cpu().numpy(), ref, w.tau, gt.borderline_pairs(inp, w, w.tau))
    g = syn.smooth_field(w) * 1e-3
    grad = torch.empty(w.M, 11, device=gt.DEV)
    ctx.gem_project_backward(gt.to_dev(g), grad)
    assert ctx.gem_status() == 0
    ref = oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g)
    border = oracle.grad_border(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g, rel=1e-5)
    got = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref) + np.linalg.norm(border)
    gt.assert_grad_per_gaussian(got, ref, border)


def test_needles_projection_and_gradient_under_noise():
    """Elongated Gaussians under a noise upstream gradient (the adjoint of a
    loss against noisy images is mostly noise).  Every term of a needle's
    gradient then has both signs, and its rotation entries come from the
    small mixed moments across and along the needle; each Gaussian is still
    held to 1e-4 of its own gradient (1e-3 per significant entry) plus the
    terms of its pairs within 1e-5 relative of tau."""
    w = NEEDLES
    inp = gt.inputs(w)
    ctx, _, proj = _project(w, inp)
    ref = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau)
    gt.assert_proj_close(proj.cpu().numpy(), ref, w.tau, gt.borderline_pairs(inp, w, w.tau))
    g = np.random.default_rng(16).normal(size=(w.B, w.d, w.d)) * 1e-3
    grad = torch.empty(w.M, 11, device=gt.DEV)
    ctx.gem_project_backward(gt.to_dev(g), grad)
    assert ctx.gem_status() == 0
    ref = oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g)
    border = oracle.grad_border(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g, rel=1e-5)
    gt.assert_grad_per_gaussian(grad.cpu().numpy(), ref, border)


def test_projection_tau_zero_every_pair():
    w = syn.Workload("t0", d=32, M=97, B=3, apix=1.1, seed=21)
    inp = gt.inputs(w)
    for dense in (False, True):
        _, _, proj = _project(w, inp, dense=dense, tau=0.0)
        ref = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, 0.0)
        gt.assert_proj_close(proj.cpu().numpy(), ref)


@pytest.mark.parametrize("form", ["params", "array"])
@pytest.mark.parametrize("d,B", [(16, 3), (48, 2), (64, 3), (96, 2), (128, 1)])
def test_ctf_loss_matches_oracle(d, B, form):
    w = syn.Workload("ctf", d=d, M=10, B=B, apix=1.2, seed=31 + d)
    proj = syn.smooth_field(w)
    imgs = syn.images(w)
    ctx = gt.context(w)
    kw = {}
    if form == "params":
        prm = syn.ctf_params(w)
        kw["ctf_params"] = gt.to_dev(prm)
        H = oracle.ctf_grid_from_params(prm, d, w.apix)
    else:
        arr = syn.ctf_array(w)
        kw["ctf"] = gt.to_dev(arr)
        H = oracle.ctf_grid_from_half(arr)
    pred = torch.empty(B, d, d, device=gt.DEV)
    dproj = torch.empty(B, d, d, device=gt.DEV)
    li = torch.empty(B, dtype=torch.float64, device=gt.DEV)
    loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
    ctx.gem_ctf_loss(gt.to_dev(proj), gt.to_dev(imgs), pred=pred, dproj=dproj, loss_img=li, loss=loss, **kw)
    L, opred, oli, og = oracle.loss(H, proj, imgs)
    assert loss.item() == pytest.approx(L, rel=1e-5)
    np.testing.assert_allclose(li.cpu().numpy(), oli, rtol=1e-5)
    p = pred.cpu().numpy()
    assert np.max(np.abs(p - opred)) <= 1e-5 * np.max(np.abs(opred))
    # dL/dproj feeds sums with heavy cancellation in the gradient, whose
    # per-entry check needs it to about 1e-6 of its maximum
    g = dproj.cpu().numpy()
    assert np.max(np.abs(g - og)) <= 2e-6 * np.max(np.abs(og))


@pytest.mark.parametrize("norm_mode", [0, 1])
@pytest.mark.parametrize("dense", [False, True], ids=["tiled", "dense"])
@pytest.mark.parametrize("w", SMALL, ids=lambda w: w.name)
def test_backward_matches_oracle(w, dense, norm_mode):
    inp = gt.inputs(w)
    g = syn.smooth_field(w) * 1e-3
    ctx, args, proj = _project(w, inp, dense=dense, norm_mode=norm_mode)
    grad = torch.empty(w.M, 11, device=gt.DEV)
    if dense:
        ctx.gem_project_backward_dense(gt.to_dev(g), grad)
    else:
        ctx.gem_project_backward(gt.to_dev(g), grad)
    assert ctx.gem_status() == 0
    ref = oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g, norm_mode)
    gt.assert_grad_close(grad.cpu().numpy(), ref)


@pytest.mark.parametrize("w", SMALL[:2], ids=lambda w: w.name)
def test_full_step_matches_oracle(w):
    inp = gt.inputs(w)
    ctx = gt.context(w)
    T = {k: gt.to_dev(v) for k, v in inp.items()}
    loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
    pred = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    ctx.gem_forward(T["params"], T["R"], T["t"], T["images"], loss, ctf_params=T["ctf_params"], pred=pred)
    grad = torch.empty(w.M, 11, device=gt.DEV)
    ctx.gem_backward(grad)
    assert ctx.gem_status() == 0
    proj = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau)
    H = oracle.ctf_grid_from_params(inp["ctf_params"], w.d, w.apix)
    L, opred, _, og = oracle.loss(H, proj, inp["images"])
    assert loss.item() == pytest.approx(L, rel=1e-5)
    G = oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, og)
    gt.assert_grad_close(grad.cpu().numpy(), G)
    # the autograd wrapper gives the same gradient (up to the order in which
    # float atomics add the per-tile moments: the last bits may differ)
    p = T["params"].clone().requires_grad_(True)
    lt = binding.GemLoss.apply(p, T["R"], T["t"], T["ctf_params"], T["images"], ctx)
    lt.backward()
    assert lt.item() == loss.item()
    gt.assert_grad_close(p.grad.double().cpu().numpy(), grad.double().cpu().numpy(),
                         norm_tol=1e-6, entry_tol=1e-4)


def test_forward_is_deterministic():
    w = SMALL[0]
    inp = gt.inputs(w)
    ctx = gt.context(w)
    T = {k: gt.to_dev(v) for k, v in inp.items()}
    out = []
    for _ in range(2):
        loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
        pred = torch.empty(w.B, w.d, w.d, device=gt.DEV)
        ctx.gem_forward(T["params"], T["R"], T["t"], T["images"], loss, ctf_params=T["ctf_params"], pred=pred)
        out.append((loss.item(), pred.cpu()))
    assert out[0][0] == out[1][0]
    assert torch.equal(out[0][1], out[1][1])
