"""Error paths on a real context: call order, bad arguments, and a pair list
that overflows its capacity.  None of them faults the GPU: the library checks
arguments on the host, and the overflow is caught on the device (entries past
the capacity are dropped) and reported through the status word."""
import numpy as np
import pytest
import torch

import gemtest as gt
from paper_2509_25075_gb300 import binding
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu

W = syn.Workload("err", d=32, M=200, B=2, apix=1.2, seed=41)


def _inputs():
    inp = gt.inputs(W)
    return [gt.to_dev(inp["params"]), gt.to_dev(inp["R"]), gt.to_dev(inp["t"])], inp


def test_backward_before_projection_is_a_state_error():
    ctx = gt.context(W)
    g = torch.zeros(W.B, W.d, W.d, device=gt.DEV)
    grad = torch.zeros(W.M, 11, device=gt.DEV)
    ctx.M, ctx.B = W.M, W.B
    with pytest.raises(binding.GemError) as ei:
        ctx.gem_project_backward(g, grad)
    assert ei.value.code == binding.GEM_ESTATE
    with pytest.raises(binding.GemError) as ei:
        ctx.gem_backward(grad)
    assert ei.value.code == binding.GEM_ESTATE


def test_sizes_beyond_the_context_are_rejected():
    ctx = gt.context(W)
    args, _ = _inputs()
    lib = binding.load()
    proj = torch.zeros(W.B + 1, W.d, W.d, device=gt.DEV)
    # B above max_B, M above max_M: rejected before any launch
    rc = lib.gem_project(ctx.h, binding._ptr(args[0]), W.M, W.B + 1, binding._ptr(args[1]),
                         binding._ptr(args[2]), binding._ptr(proj))
    assert rc == binding.GEM_EINVAL
    assert b"max_B" in lib.gem_last_error(ctx.h)
    rc = lib.gem_project(ctx.h, binding._ptr(args[0]), W.M + 1, W.B, binding._ptr(args[1]),
                         binding._ptr(args[2]), binding._ptr(proj))
    assert rc == binding.GEM_EINVAL
    # misaligned image pointer
    rc = lib.gem_project(ctx.h, binding._ptr(args[0]), W.M, W.B, binding._ptr(args[1]),
                         binding._ptr(args[2]), proj.data_ptr() + 4)
    assert rc == binding.GEM_EINVAL
    assert b"aligned" in lib.gem_last_error(ctx.h)
    # both CTF forms at once
    imgs = torch.zeros(W.B, W.d, W.d, device=gt.DEV)
    with pytest.raises(binding.GemError):
        ctx.gem_ctf_loss(imgs, imgs, ctf=torch.zeros(W.B, W.d, W.d // 2 + 1, device=gt.DEV),
                         ctf_params=torch.zeros(W.B, 8, device=gt.DEV))
    assert ctx.gem_status() == binding.GEM_OK


def test_capacity_overflow_is_reported_not_faulted():
    args, inp = _inputs()
    full = gt.context(W)
    proj_full = torch.empty(W.B, W.d, W.d, device=gt.DEV)
    full.gem_project(*args, proj_full)
    need = full.gem_pair_count()
    assert need > 8
    small = gt.context(W, max_pairs=need // 2)
    proj = torch.empty(W.B, W.d, W.d, device=gt.DEV)
    small.gem_project(*args, proj)
    assert small.gem_status() == binding.GEM_ECAPACITY
    # the status word is cleared by the read; the context stays usable
    assert small.gem_status() == binding.GEM_OK
    grad = torch.empty(W.M, 11, device=gt.DEV)
    small.gem_project_backward(torch.zeros_like(proj), grad)
    assert small.gem_status() in (binding.GEM_OK, binding.GEM_ECAPACITY)
    torch.cuda.synchronize()
    # an overflowed call reads no list entry: its outputs are zero
    assert np.all(proj.cpu().numpy() == 0.0)
    assert np.all(grad.cpu().numpy() == 0.0)
    # a context with enough room gives the full result again
    full.gem_project(*args, proj)
    assert full.gem_status() == binding.GEM_OK
    assert torch.equal(proj, proj_full)


def test_tiled_backward_after_dense_projection_is_a_state_error():
    args, _ = _inputs()
    ctx = gt.context(W)
    proj = torch.empty(W.B, W.d, W.d, device=gt.DEV)
    ctx.gem_project(*args, proj)
    ctx.gem_project_dense(*args, proj)  # replaces the records; its lists are stale
    grad = torch.empty(W.M, 11, device=gt.DEV)
    with pytest.raises(binding.GemError) as ei:
        ctx.gem_project_backward(torch.zeros_like(proj), grad)
    assert ei.value.code == binding.GEM_ESTATE
    ctx.gem_project_backward_dense(torch.zeros_like(proj), grad)
    assert torch.count_nonzero(grad).item() == 0
