"""GPU parity of the ablation constraints (no rotation, isotropic scaling) and
of the nearest-neighbour distances (Sec. 4, Design Choices of 3DGS for
cryo-EM), through the C ABI, against the oracle."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

W = syn.Workload("abl48", d=48, M=900, B=4, apix=1.2, seed=21)
FLAGS = [(1, 0), (0, 1), (1, 1)]


@pytest.mark.parametrize("flags", FLAGS, ids=["norot", "iso", "both"])
@pytest.mark.parametrize("norm_mode", [0, 1])
def test_constrained_projection_and_gradient(flags, norm_mode):
    no_rot, iso = flags
    inp = gt.inputs(W)
    th = inp["params"].copy()
    th[:7, 6:10] = 0.0  # a zero quaternion is legal when rotation is fixed
    if not no_rot:
        th[:7, 6] = 1.0
    ctx = gt.context(W, norm_mode=norm_mode, no_rotation=no_rot, isotropic=iso)
    proj = torch.empty(W.B, W.d, W.d, device=gt.DEV)
    args = [gt.to_dev(th), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
    ctx.gem_project(*args, proj)
    ref = oracle.project(th, inp["R"], inp["t"], W.d, W.apix, W.tau, norm_mode,
                         no_rotation=bool(no_rot), isotropic=bool(iso))
    c = oracle.constrained(th, bool(no_rot), bool(iso))
    border = gt.borderline_pairs({"params": c, "R": inp["R"], "t": inp["t"]}, W, W.tau, norm_mode)
    gt.assert_proj_close(proj.cpu().numpy(), ref, W.tau, border)
    g = syn.smooth_field(W) * 1e-3
    grad = torch.empty(W.M, 11, device=gt.DEV)
    ctx.gem_project_backward(gt.to_dev(g), grad)
    assert ctx.gem_status() == 0
    G = oracle.grad(th, inp["R"], inp["t"], W.d, W.apix, W.tau, g, norm_mode,
                    no_rotation=bool(no_rot), isotropic=bool(iso))
    got = grad.cpu().numpy()
    gt.assert_grad_close(got, G)
    if no_rot:
        assert np.all(got[:, 6:10] == 0.0)
    if iso:
        assert np.all(got[:, 4:6] == 0.0)


def test_constrained_equals_explicit_parameters():
    """The flags give exactly what the same Gaussians written out with
    q = (1, 0, 0, 0) and three equal scales give (same kernels, same bits)."""
    inp = gt.inputs(W)
    th = inp["params"]
    out = []
    for flags, params in (((1, 1), th), ((0, 0), oracle.constrained(th, True, True))):
        ctx = gt.context(W, no_rotation=flags[0], isotropic=flags[1])
        proj = torch.empty(W.B, W.d, W.d, device=gt.DEV)
        ctx.gem_project(gt.to_dev(params), gt.to_dev(inp["R"]), gt.to_dev(inp["t"]), proj)
        out.append(proj.cpu())
    assert torch.equal(out[0], out[1])


def _clustered(M, seed, spread=30.0):
    rng = np.random.default_rng(seed)
    c = rng.normal(scale=spread, size=(16, 3))
    p = c[rng.integers(0, 16, M)] + rng.normal(scale=spread / 10, size=(M, 3))
    th = np.zeros((M, 11), dtype=np.float32)
    th[:, 0:3] = p
    th[:, 3:6] = 1.0
    th[:, 6] = 1.0
    th[:, 10] = 1.0
    return th


@pytest.mark.parametrize("M,k", [(1, 1), (2, 3), (17, 4), (5000, 1), (5000, 8), (20011, 16)])
def test_nn_distance_bit_exact(M, k):
    th = _clustered(M, seed=M + k)
    if M > 100:
        th[5, 0] = np.nan       # a centre that is not finite
        th[6, 0:3] = th[7, 0:3]  # two coincident centres
        th[8, 0:3] = (500.0, -400.0, 900.0)  # an outlier far from everything
    ctx = gt.context(syn.Workload("nn", d=32, M=M, B=1, seed=1))
    dist, idx = ctx.gem_nn_distance(gt.to_dev(th), k)
    rd, ri = oracle.nn_distance(th[:, 0:3], k)
    np.testing.assert_array_equal(dist.cpu().numpy(), rd)
    np.testing.assert_array_equal(idx.cpu().numpy().astype(np.int64), ri)


def test_nn_distance_degenerate_layouts():
    """All centres on a line, or all equal: the grid stays bounded and the
    result exact."""
    M = 3000
    for kind in ("line", "same"):
        th = _clustered(M, seed=3)
        if kind == "line":
            th[:, 1] = 0.0
            th[:, 2] = 0.0
        else:
            th[:, 0:3] = 1.5
        ctx = gt.context(syn.Workload("nn", d=32, M=M, B=1, seed=1))
        dist, idx = ctx.gem_nn_distance(gt.to_dev(th), 2)
        rd, ri = oracle.nn_distance(th[:, 0:3], 2)
        np.testing.assert_array_equal(dist.cpu().numpy(), rd)
        np.testing.assert_array_equal(idx.cpu().numpy().astype(np.int64), ri)
