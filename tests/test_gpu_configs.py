"""Every kernel configuration of the two rasterisers (the autotuner's search
space) against the FP64 oracle, and the autotuner itself.  A configuration
changes how the work of Eq. render / Eq. accu (forward) and of the sparse
gradient (backward) is spread over the GPU, never what is computed."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import binding
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

CASES = [
    syn.Workload("c48", d=48, M=1037, B=5, apix=1.2, seed=11),
    syn.Workload("c32w", d=32, M=301, B=2, apix=1.0, s_lo=0.3, s_hi=6.0, n_clusters=4, seed=13),
    # long lists (several windows per tile) and wide Gaussians
    syn.Workload("c64big", d=64, M=900, B=3, apix=1.2, s_lo=1.0, s_hi=8.0, n_clusters=2, seed=15),
]


def _n_configs():
    return binding.raster_configs()


def _fwd_ids():
    return list(range(len(_n_configs()[0])))


def _bwd_ids():
    return list(range(len(_n_configs()[1])))


def _ctx(w, **kw):
    return gt.context(w, max_pairs=64 * w.B * w.M, **kw)


@pytest.mark.parametrize("fwd", _fwd_ids())
@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_every_forward_config_matches_oracle(w, fwd):
    inp = gt.inputs(w)
    ctx = _ctx(w)
    ctx.gem_set_raster_config(fwd, -1)
    proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    args = [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
    ctx.gem_project(*args, proj)
    assert ctx.gem_status() == 0
    ref = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau)
    gt.assert_proj_close(proj.cpu().numpy(), ref, w.tau, gt.borderline_pairs(inp, w, w.tau))
    # the pair statistics do not depend on the configuration
    kept, evaluated = ctx.gem_pair_stats()
    ctx.gem_set_raster_config(0, -1)
    assert ctx.gem_pair_stats() == (kept, evaluated)
    ctx.close()


def test_persistent_forward_is_bitwise_the_per_tile_forward():
    """The persistent forms run the same tile code in another order: the
    same bits (the persistent grids of 6 and 7 CTAs per SM run the kernel
    built for 8)."""
    w = CASES[2]
    inp = gt.inputs(w)
    names = _n_configs()[0]
    out = {}
    for i, name in enumerate(names):
        ctx = _ctx(w)
        ctx.gem_set_raster_config(i, -1)
        proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
        args = [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
        ctx.gem_project(*args, proj)
        assert ctx.gem_status() == 0
        out[name] = proj.cpu().numpy()
        ctx.close()
    for name, img in out.items():
        if "persistent" in name:
            base = name.split(", persistent")[0]
            if base not in out:
                base = "aligned, 256-record windows, 8 CTAs/SM"
            np.testing.assert_array_equal(img, out[base])


@pytest.mark.parametrize("bwd", _bwd_ids())
@pytest.mark.parametrize("w", CASES, ids=lambda w: w.name)
def test_every_backward_config_matches_oracle(w, bwd):
    inp = gt.inputs(w)
    ctx = _ctx(w)
    ctx.gem_set_raster_config(-1, bwd)
    proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    # params, R and t stay referenced: the backward reads them again
    args = [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
    ctx.gem_project(*args, proj)
    g = syn.smooth_field(w) * 1e-3
    grad = torch.empty(w.M, 11, device=gt.DEV)
    ctx.gem_project_backward(gt.to_dev(g), grad)
    assert ctx.gem_status() == 0
    ref = oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g)
    border = oracle.grad_border(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g, rel=1e-5)
    gt.assert_grad_per_gaussian(grad.cpu().numpy(), ref, border)
    ctx.close()


def test_autotune_records_a_choice_that_computes_the_same_step():
    w = syn.Workload("tune", d=48, M=700, B=4, apix=1.2, seed=17)
    inp = gt.inputs(w)
    T = {k: gt.to_dev(v) for k, v in inp.items()}
    ctx = _ctx(w)
    f, b = ctx.gem_autotune(T["params"], T["R"], T["t"], reps=2)
    nf, nb = (len(x) for x in ctx.raster_configs())
    assert 0 <= f < nf and 0 <= b < nb
    # a context that names no configuration uses the recorded choice for
    # this shape (another context included), and the default elsewhere
    other = _ctx(w)
    assert other.gem_get_raster_config(w.B, w.M) == (f, b)
    assert ctx.gem_get_raster_config(w.B, w.M) == (f, b)
    # after autotuning the step still matches the oracle
    loss = torch.empty(1, dtype=torch.float64, device=gt.DEV)
    ctx.gem_forward(T["params"], T["R"], T["t"], T["images"], loss, ctf_params=T["ctf_params"])
    grad = torch.empty(w.M, 11, device=gt.DEV)
    ctx.gem_backward(grad)
    assert ctx.gem_status() == 0
    proj = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau)
    H = oracle.ctf_grid_from_params(inp["ctf_params"], w.d, w.apix)
    L, _, _, g = oracle.loss(H, proj, inp["images"])
    assert loss.item() == pytest.approx(L, rel=1e-5)
    G = oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g)
    gt.assert_grad_close(grad.cpu().numpy(), G)
    # an explicit configuration wins over the recorded one; bad indices fail
    ctx.gem_set_raster_config(0, 0)
    assert ctx.gem_get_raster_config(w.B, w.M) == (0, 0)
    with pytest.raises(binding.GemError):
        ctx.gem_set_raster_config(nf, 0)
    ctx.close()
    other.close()


def test_persistent_backward_matches_the_per_tile_backward():
    """The persistent backward runs the same tile code in another order, and
    its window size only regroups the records into rounds (each (tile,
    Gaussian) partial is one lane's sum over the record's blocks either way);
    the float64 moments are sums of the same partials in another order, so
    the gradients agree with the per-tile grid's with as many lanes per
    record to float rounding of float64 sums (here: 1e-6)."""
    w = CASES[2]
    inp = gt.inputs(w)
    names = _n_configs()[1]
    g = gt.to_dev(syn.smooth_field(w) * 1e-3)
    out = {}
    for i, name in enumerate(names):
        ctx = _ctx(w)
        ctx.gem_set_raster_config(-1, i)
        proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
        args = [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])]
        ctx.gem_project(*args, proj)
        grad = torch.empty(w.M, 11, device=gt.DEV)
        ctx.gem_project_backward(g, grad)
        assert ctx.gem_status() == 0
        out[name] = grad.cpu().numpy().astype(np.float64)
        ctx.close()
    for name, gr in out.items():
        if "persistent" in name:
            lanes = name.split(" per record")[0]
            base = out[lanes + " per record, 128-record warp windows"]
            assert np.linalg.norm(gr - base) <= 1e-6 * np.linalg.norm(base), name
