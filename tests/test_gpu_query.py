"""GPU parity of the density query (Eq. query) through the C ABI: whole
volumes against the oracle on small grids (ragged slice batches, both
normalisations, threshold, ablation flags), sampled voxels at full size, and
consistency with the projection."""
import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _border(params, d, apix, tau, norm_mode, rel=1e-5):
    """Per-voxel count of pairs whose FP64 value lies within rel * tau of tau."""
    if tau <= 0:
        return np.zeros((d, d, d))
    cnt = np.zeros((d, d, d))
    for j in range(params.shape[0]):
        v = oracle.query(params[j:j + 1], d, apix, 0.0, norm_mode)
        cnt += np.abs(v - tau) <= rel * tau
    return cnt


CASES = [
    # (workload, max_B, tau factor, norm_mode, no_rotation, isotropic)
    (syn.Workload("q32", d=32, M=150, B=1, apix=1.2, seed=51), 32, 0.0, 0, 0, 0),
    (syn.Workload("q48", d=48, M=220, B=1, apix=1.0, seed=52), 5, 1.0, 0, 0, 0),
    (syn.Workload("q48w", d=48, M=120, B=1, apix=1.3, s_lo=0.3, s_hi=6.0, seed=53), 7, 1.0, 1, 0, 0),
    (syn.Workload("q32f", d=32, M=100, B=1, apix=1.1, seed=54), 16, 1.0, 0, 1, 1),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0].name}-B{c[1]}-t{c[2]}-n{c[3]}-f{c[4]}{c[5]}")
def test_query_volume_matches_oracle(case):
    w, max_B, tf, norm_mode, no_rot, iso = case
    th = syn.gaussians(w)
    full = oracle.query(th, w.d, w.apix, 0.0, norm_mode, bool(no_rot), bool(iso))
    tau = tf * 1e-3 * float(full.max())  # cuts the outer shell of every Gaussian
    ctx = gt.context(syn.Workload(w.name, d=w.d, M=w.M, B=max_B, apix=w.apix, seed=1),
                     norm_mode=norm_mode, no_rotation=no_rot, isotropic=iso)
    vol = ctx.gem_query(gt.to_dev(th), tau)
    assert ctx.gem_status() == 0
    ref = oracle.query(th, w.d, w.apix, tau, norm_mode, bool(no_rot), bool(iso)) if tau > 0 else full
    border = _border(oracle.constrained(th, bool(no_rot), bool(iso)), w.d, w.apix, tau, norm_mode)
    gt.assert_proj_close(vol.cpu().numpy(), ref, tau, border)


@pytest.mark.parametrize("name", ["A2", "A3"])
def test_query_fullsize_sampled_voxels(name):
    w = syn.WORKLOADS[name]
    th = syn.gaussians(w)
    ctx = gt.context(w)
    tau = w.tau_query
    vol = ctx.gem_query(gt.to_dev(th), tau)
    assert ctx.gem_status() == 0
    rng = np.random.default_rng(60)
    n = 64
    c, r = w.d // 2, int(0.3 * w.d)
    near = rng.integers(c - r, c + r, size=(n // 2, 3))
    anywhere = rng.integers(0, w.d, size=(n // 2, 3))
    zyx = np.concatenate([near, anywhere])
    vox = (zyx[:, 0] * w.d + zyx[:, 1]) * w.d + zyx[:, 2]
    ref = oracle.query_voxels(th, w.d, w.apix, tau, vox)
    got = vol.cpu().numpy().reshape(-1)[vox].astype(np.float64)
    scale = float(vol.max().item())
    # plus tau per pair that float32 and float64 may put on different sides
    # of the threshold (a few per voxel at most)
    assert np.max(np.abs(got - ref)) <= 1e-5 * scale + 8 * tau


def test_query_integrates_to_the_identity_projection():
    """apix * (sum over z of the GPU volume) equals the GPU projection at the
    identity view (Eq. render is the line integral of the mode-0 density)."""
    w = syn.Workload("qp", d=64, M=400, B=1, apix=1.2, s_lo=1.5, s_hi=3.0, seed=55)
    th = syn.gaussians(w)
    th[:, 0:3] *= 0.5  # keep every Gaussian 6 sigma inside the z faces
    ctx = gt.context(w, tau=0.0)
    vol = ctx.gem_query(gt.to_dev(th), 0.0)
    proj = torch.empty(1, w.d, w.d, device=gt.DEV)
    ctx.gem_project(gt.to_dev(th), gt.to_dev(np.eye(3)[None]), gt.to_dev(np.zeros((1, 2))), proj)
    got = (vol.double().sum(0) * w.apix).cpu().numpy()
    ref = proj[0].double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_query_ends_the_backward_state():
    w = syn.Workload("qs", d=32, M=50, B=2, seed=56)
    inp = gt.inputs(w)
    ctx = gt.context(w)
    proj = torch.empty(w.B, w.d, w.d, device=gt.DEV)
    ctx.gem_project(gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"]), proj)
    ctx.gem_query(gt.to_dev(inp["params"]), 0.0)
    from paper_2509_25075_gb300 import binding
    lib = binding.load()
    g = torch.zeros(w.B, w.d, w.d, device=gt.DEV)
    grad = torch.zeros(w.M, 11, device=gt.DEV)
    assert lib.gem_project_backward(ctx.h, binding._ptr(g), binding._ptr(grad)) == binding.GEM_ESTATE
