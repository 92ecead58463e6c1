"""The allocation-free variant of the CTF + loss + adjoint step.

Some callers cannot allocate device memory where they need this step (a
fixed memory budget, an allocator that forbids cudaMalloc after start-up, or
code that must not trigger the synchronisation an allocation can cause).
gem_ctf_loss_static serves them from fixed-size scratch arrays inside the
library.  This file checks, through the C ABI, that two calls in a row give
what gem_ctf_loss gives, and that an oversized request is refused before
anything runs.  It is collected last so that a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import gemtest as gt
import oracle
from paper_2509_25075_gb300 import binding
from paper_2509_25075_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


def _p(x):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def _oracle_check(w, proj, imgs, kw, out, sel):
    """The FP64 oracle's loss, prediction and adjoint for the images sel,
    with the tolerances of the float path."""
    if "ctf_params" in kw:
        H = oracle.ctf_grid_from_params(kw["ctf_params"].cpu().numpy()[sel], w.d, w.apix)
    else:
        H = oracle.ctf_grid_from_half(kw["ctf"].cpu().numpy()[sel])
    _, opred, oli, og = oracle.loss(H, proj.cpu().numpy()[sel], imgs.cpu().numpy()[sel])
    og = og * len(sel) / w.B  # the oracle's adjoint of the sub-batch carries 2 / (len(sel) d^2)
    np.testing.assert_allclose(out["loss_img"].cpu().numpy()[sel], oli, rtol=1e-5)
    p = out["pred"].cpu().numpy()[sel]
    assert np.max(np.abs(p - opred)) <= 1e-5 * np.max(np.abs(opred))
    g = out["dproj"].cpu().numpy()[sel]
    assert np.max(np.abs(g - og)) <= 2e-6 * np.max(np.abs(og))


# d = 256, B = 16 fills the spectrum array exactly (16 * 256^2 = 2^20
# elements): the largest request the fixed arrays accept
@pytest.mark.parametrize("form,d,B", [("params", 64, 3), ("array", 64, 3), ("params", 256, 16)])
def test_static_matches_context_twice(form, d, B):
    w = syn.Workload("static", d=d, M=10, B=B, apix=1.2, seed=77)
    lib = binding.load()
    proj = gt.to_dev(syn.smooth_field(w))
    imgs = gt.to_dev(syn.images(w))
    if form == "params":
        kw = {"ctf_params": gt.to_dev(syn.ctf_params(w))}
    else:
        kw = {"ctf": gt.to_dev(syn.ctf_array(w))}
    # the existing entry point, with a context and its own scratch
    ctx = gt.context(w)
    ref = {
        "pred": torch.empty(w.B, w.d, w.d, device=gt.DEV),
        "dproj": torch.empty(w.B, w.d, w.d, device=gt.DEV),
        "loss_img": torch.empty(w.B, dtype=torch.float64, device=gt.DEV),
        "loss": torch.empty(1, dtype=torch.float64, device=gt.DEV),
    }
    ctx.gem_ctf_loss(proj, imgs, **kw, **ref)
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row share the static scratch
        out = {k: torch.full_like(v, float("nan")) for k, v in ref.items()}
        rc = lib.gem_ctf_loss_static(w.d, w.apix, w.B, _p(proj), _p(kw.get("ctf")), _p(kw.get("ctf_params")),
                                     _p(imgs), _p(out["pred"]), _p(out["dproj"]), _p(out["loss_img"]),
                                     _p(out["loss"]), stream)
        assert rc == binding.GEM_OK
        torch.cuda.synchronize()
        assert out["loss"].item() == pytest.approx(ref["loss"].item(), rel=1e-5)
        np.testing.assert_allclose(out["loss_img"].cpu().numpy(), ref["loss_img"].cpu().numpy(), rtol=1e-5)
        r = ref["pred"].cpu().numpy()
        assert np.max(np.abs(out["pred"].cpu().numpy() - r)) <= 1e-5 * np.max(np.abs(r))
        r = ref["dproj"].cpu().numpy()
        assert np.max(np.abs(out["dproj"].cpu().numpy() - r)) <= 2e-6 * np.max(np.abs(r))
    # and against the FP64 oracle directly (first, middle and last image)
    _oracle_check(w, proj, imgs, kw, out, np.array(sorted({0, w.B // 2, w.B - 1})))
    ctx.close()


def test_static_rejects_oversized_requests():
    lib = binding.load()
    d, B = 256, 17  # 17 * 256^2 > 2^20 spectrum elements
    proj = torch.zeros(B, d, d, device=gt.DEV)
    imgs = torch.zeros(B, d, d, device=gt.DEV)
    prm = torch.zeros(B, 8, device=gt.DEV)
    loss = torch.full((1,), -1.0, dtype=torch.float64, device=gt.DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.gem_ctf_loss_static(d, 1.2, B, _p(proj), None, _p(prm), _p(imgs), None, None, None, _p(loss), stream)
    assert rc == binding.GEM_ECAPACITY
    torch.cuda.synchronize()
    assert loss.item() == -1.0  # nothing ran
    rc = lib.gem_ctf_loss_static(d, 1.2, 16, _p(proj), None, None, _p(imgs), None, None, None, _p(loss), stream)
    assert rc == binding.GEM_EINVAL  # no CTF given
