"""The hot path's C boundary as a user drives it (Eq. recon: images, known
poses and CTFs in, the Gaussians' gradient out): gem_set_gaussians with
gem_forward(params = NULL), and a context created with fp64_check, whose
gem_forward / gem_backward compute in float64 on the same float arrays."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import binding
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

W = syn.Workload("bnd", d=48, M=411, B=3, apix=1.2, seed=41)


def _step(ctx, T, params, pred=True):
    loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
    p = torch.empty(W.B, W.d, W.d, device=gt.DEV) if pred else None
    ctx.gem_forward(params, T["R"], T["t"], T["images"], loss, ctf_params=T["ctf_params"], pred=p)
    grad = torch.empty(W.M, 11, device=gt.DEV)
    ctx.gem_backward(grad)
    assert ctx.gem_status() == 0
    return loss.item(), (p.cpu().numpy() if pred else None), grad.cpu().numpy()


def test_set_gaussians_equals_explicit_params():
    inp = gt.inputs(W)
    T = {k: gt.to_dev(v) for k, v in inp.items()}
    ctx = gt.context(W)
    l1, p1, g1 = _step(ctx, T, T["params"])
    ctx.gem_set_gaussians(T["params"])
    l2, p2, g2 = _step(ctx, T, None)
    assert l1 == l2
    np.testing.assert_array_equal(p1, p2)
    np.testing.assert_array_equal(g1, g2)
    ctx.close()


def test_forward_without_set_gaussians_is_a_state_error():
    inp = gt.inputs(W)
    T = {k: gt.to_dev(v) for k, v in inp.items()}
    ctx = gt.context(W)
    loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
    rc = ctx.lib.gem_forward(ctx.h, None, W.M, W.B, binding._ptr(T["R"]), binding._ptr(T["t"]), None,
                             binding._ptr(T["ctf_params"]), binding._ptr(T["images"]), None, binding._ptr(loss))
    assert rc == binding.GEM_ESTATE
    ctx.close()


@pytest.mark.parametrize("norm_mode", [0, 1])
def test_fp64_check_context_matches_oracle(norm_mode):
    inp = gt.inputs(W)
    T = {k: gt.to_dev(v) for k, v in inp.items()}
    tau = W.tau if norm_mode == 0 else 50 * W.tau
    ctx = gt.context(W, fp64_check=1, norm_mode=norm_mode, tau=tau)
    loss, pred, grad = _step(ctx, T, T["params"])
    proj = oracle.project(inp["params"], inp["R"], inp["t"], W.d, W.apix, tau, norm_mode)
    H = oracle.ctf_grid_from_params(inp["ctf_params"], W.d, W.apix)
    L, opred, _, g = oracle.loss(H, proj, inp["images"])
    G = oracle.grad(inp["params"], inp["R"], inp["t"], W.d, W.apix, tau, g, norm_mode)
    # float64 arithmetic throughout: the loss to 1e-12; pred and grad carry
    # only the final rounding to float32
    assert loss == pytest.approx(L, rel=1e-12)
    assert np.max(np.abs(pred - opred)) <= 1e-7 * np.max(np.abs(opred))
    assert np.linalg.norm(grad - G) <= 1e-7 * np.linalg.norm(G)
    big = np.abs(G) > 1e-3 * np.max(np.abs(G))
    assert np.max(np.abs(grad - G)[big] / np.abs(G)[big]) <= 1e-6
    ctx.close()
