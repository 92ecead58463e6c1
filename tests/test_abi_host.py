"""Host-side checks that need no GPU: the library loads, exports every entry
point include/gem.h declares, the binding covers them, and configuration
errors are reported before any device work."""
import ctypes
import os
import re

import pytest

from paper_2509_25075_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gem_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    # the calls of the hot path's C boundary (create, set the Gaussians,
    # forward, backward, destroy, errors) and the stage calls
    for n in ["gem_create", "gem_destroy", "gem_set_gaussians", "gem_project", "gem_ctf_loss",
              "gem_project_backward", "gem_forward", "gem_backward", "gem_status", "gem_last_error"]:
        assert n in names
    src = open(os.path.join(ROOT, "include", "gem.h")).read()
    for code in ["GEM_EINVAL", "GEM_ENOMEM", "GEM_ECUDA", "GEM_ETIMEOUT", "GEM_ESTATE", "GEM_ECAPACITY"]:
        assert re.search(r"#define " + code + r" \(-\d\)", src), code
    for field in ["d", "apix", "tau", "tile", "norm_mode", "no_rotation", "isotropic", "fp64_check",
                  "max_M", "max_B"]:
        assert field in dict(binding.gem_config._fields_), field


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    for n in _declared():
        assert hasattr(lib, n), n
    assert set(_declared()) <= set(binding.SIGNATURES), set(_declared()) - set(binding.SIGNATURES)


def _create(**over):
    lib = binding.load()
    cfg = binding.gem_config()
    assert lib.gem_config_default(ctypes.byref(cfg), 64, 1.2, 4, 100) == 0
    assert (cfg.d, cfg.max_B, cfg.max_M, cfg.zsort, cfg.norm_mode) == (64, 4, 100, 1, 0)
    assert (cfg.tile, cfg.fp64_check) == (16, 0)
    for k, v in over.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    rc = lib.gem_create(ctypes.byref(h), ctypes.byref(cfg), None)
    return rc, lib.gem_create_error().decode(), h


@pytest.mark.parametrize("field,value,msg", [
    ("d", 40, "multiple of 16"),
    ("d", 80, "2^a 3^b"),
    ("d", 1024, "16..768"),
    ("apix", 0.0, "apix"),
    ("tau", -1.0, "tau"),
    ("norm_mode", 2, "norm_mode"),
    ("max_B", 0, "max_B"),
    ("max_M", 0, "max_M"),
    ("max_pairs", -5, "max_pairs"),
    ("zsort", 3, "zsort"),
    ("no_rotation", 2, "no_rotation"),
    ("isotropic", -1, "isotropic"),
    ("tile", 8, "tile"),
    ("fp64_check", 2, "fp64_check"),
])
def test_bad_config_is_rejected_before_device_work(field, value, msg):
    rc, err, h = _create(**{field: value})
    assert rc == binding.GEM_EINVAL
    assert msg in err
    assert not h.value


def test_null_arguments():
    lib = binding.load()
    assert lib.gem_create(None, None, None) == binding.GEM_EINVAL
    assert lib.gem_destroy(None) == binding.GEM_OK
    assert lib.gem_status(None) == binding.GEM_EINVAL
    assert lib.gem_project(None, None, 1, 1, None, None, None) == binding.GEM_EINVAL
    assert lib.gem_backward(None, None) == binding.GEM_EINVAL
    assert lib.gem_set_gaussians(None, None, 1) == binding.GEM_EINVAL
    assert lib.gem_last_error(None) == b""


def test_static_ctf_step_validates_before_device_work():
    """gem_ctf_loss_static checks its arguments and its fixed capacity before
    any CUDA call; the pointers here are never dereferenced."""
    lib = binding.load()
    p = ctypes.c_void_p(1 << 20)  # 16-byte aligned stand-in address
    odd = ctypes.c_void_p((1 << 20) + 4)

    def call(d=64, apix=1.2, B=2, proj=p, ctf=None, prm=p, imgs=p, pred=None, dproj=None):
        return lib.gem_ctf_loss_static(d, apix, B, proj, ctf, prm, imgs, pred, dproj, None, None, None)

    assert call(d=40) == binding.GEM_EINVAL        # not a multiple of 16
    assert call(d=80) == binding.GEM_EINVAL        # not 2^a 3^b
    assert call(d=1024) == binding.GEM_EINVAL      # above 768
    assert call(apix=0.0) == binding.GEM_EINVAL
    assert call(apix=float("nan")) == binding.GEM_EINVAL
    assert call(B=0) == binding.GEM_EINVAL
    assert call(proj=None) == binding.GEM_EINVAL
    assert call(prm=None) == binding.GEM_EINVAL    # no CTF
    assert call(ctf=p) == binding.GEM_EINVAL       # both CTF forms
    assert call(pred=odd) == binding.GEM_EINVAL    # misaligned output
    assert call(d=256, B=17) == binding.GEM_ECAPACITY  # 17 * 256^2 > 2^20 spectrum elements
    assert call(d=768, B=2) == binding.GEM_ECAPACITY
