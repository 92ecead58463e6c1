"""Thin Python binding of the C ABI in include/gem.h.

Functions carry the C names and only marshal arguments: they check shapes,
dtypes, devices and contiguity of torch tensors and pass raw pointers to
``libgem.so``.  Every step of the computation runs in the CUDA library; there
is no CPU or PyTorch fallback.  If the library has not been built the first
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

GEM_OK = 0
GEM_EINVAL = -1
GEM_ENOMEM = -2
GEM_ECUDA = -3
GEM_ESTATE = -4
GEM_ECAPACITY = -5
GEM_ETIMEOUT = -6
NPAR = 11


class GemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gem error {code}: {msg}")
        self.code = code


class gem_config(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32),
        ("apix", ctypes.c_float),
        ("tau", ctypes.c_float),
        ("norm_mode", ctypes.c_int32),
        ("max_B", ctypes.c_int32),
        ("max_M", ctypes.c_int64),
        ("max_pairs", ctypes.c_int64),
        ("zsort", ctypes.c_int32),
        ("no_rotation", ctypes.c_int32),
        ("isotropic", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("fp64_check", ctypes.c_int32),
    ]


class gem_adam_config(ctypes.Structure):
    _fields_ = [
        ("lr", ctypes.c_float * 4),
        ("beta1", ctypes.c_float),
        ("beta2", ctypes.c_float),
        ("eps", ctypes.c_float),
        ("step", ctypes.c_int32),
    ]


# name -> (restype, argtypes)
_P, _I32, _I64, _F = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
SIGNATURES = {
    "gem_config_default": (ctypes.c_int, [ctypes.POINTER(gem_config), _I32, _F, _I32, _I64]),
    "gem_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(gem_config), _P]),
    "gem_destroy": (ctypes.c_int, [_P]),
    "gem_last_error": (ctypes.c_char_p, [_P]),
    "gem_create_error": (ctypes.c_char_p, []),
    "gem_set_stream": (ctypes.c_int, [_P, _P]),
    "gem_status": (ctypes.c_int, [_P]),
    "gem_project": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P]),
    "gem_ctf_loss": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gem_project_backward": (ctypes.c_int, [_P, _P, _P]),
    "gem_set_gaussians": (ctypes.c_int, [_P, _P, _I64]),
    "gem_forward": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P, _P, _P, _P, _P]),
    "gem_backward": (ctypes.c_int, [_P, _P]),
    "gem_project_dense": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P]),
    "gem_project_backward_dense": (ctypes.c_int, [_P, _P, _P]),
    "gem_pair_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "gem_inspect_bins": (ctypes.c_int, [_P, _P, _P, _I64]),
    "gem_inspect_records": (ctypes.c_int, [_P, _P]),
    "gem_pair_stats": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "gem_raster_config_count": (ctypes.c_int, [ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "gem_raster_config_name": (ctypes.c_char_p, [_I32, _I32]),
    "gem_set_raster_config": (ctypes.c_int, [_P, _I32, _I32]),
    "gem_get_raster_config": (ctypes.c_int, [_P, _I32, _I64, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "gem_autotune": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "gem_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "gem_timing_read": (ctypes.c_int, [_P, _P, _P]),
    "gem_ctf_loss_static": (ctypes.c_int, [_I32, _F, _I32, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gem_nn_distance": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P]),
    "gem_query": (ctypes.c_int, [_P, _P, _I64, _F, _P]),
    "gem_fsc": (ctypes.c_int, [_P, _P, _P, _F, _P, _P, _P]),
    "gem_adam_step": (ctypes.c_int, [_P, _I64, ctypes.POINTER(gem_adam_config), _P, _P, _P, _P, _P, _P]),
    "gem_activate": (ctypes.c_int, [_P, _I64, _P, _P]),
    "gem_project_f64": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P]),
    "gem_ctf_loss_f64": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gem_project_backward_f64": (ctypes.c_int, [_P, _P, _P]),
}

STAGES = ["prep", "bin", "raster_fwd", "ctf", "raster_bwd", "prep_bwd"]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libgem.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError("libgem.so is missing: run __graft_entry__.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(x):
    if x is None:
        return None
    return ctypes.c_void_p(x.data_ptr())


def _check(x, name, shape, dtype=torch.float32, optional=False):
    if x is None:
        if optional:
            return
        raise ValueError(f"{name} is required")
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not x.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {tuple(shape)}")


def raster_configs():
    """-> (forward configuration names, backward configuration names)."""
    lib = load()
    nf, nb = ctypes.c_int32(), ctypes.c_int32()
    lib.gem_raster_config_count(ctypes.byref(nf), ctypes.byref(nb))
    return ([lib.gem_raster_config_name(0, i).decode() for i in range(nf.value)],
            [lib.gem_raster_config_name(1, i).decode() for i in range(nb.value)])


class Context:
    """Owns one gem_ctx.  Methods mirror the C calls of the same name."""

    def __init__(self, d: int, apix: float, max_B: int, max_M: int, tau: float = 0.0,
                 norm_mode: int = 0, zsort: int = 1, max_pairs: int = 0, no_rotation: int = 0,
                 isotropic: int = 0, stream=None, fp64_check: int = 0, tile: int = 16):
        self.lib = load()
        cfg = gem_config()
        self.lib.gem_config_default(ctypes.byref(cfg), d, apix, max_B, max_M)
        cfg.tau = tau
        cfg.norm_mode = norm_mode
        cfg.zsort = zsort
        cfg.max_pairs = max_pairs
        cfg.no_rotation = no_rotation
        cfg.isotropic = isotropic
        cfg.fp64_check = fp64_check
        cfg.tile = tile
        self.cfg = cfg
        self.d, self.apix, self.max_B, self.max_M = d, apix, max_B, max_M
        self.device = torch.cuda.current_device()
        s = torch.cuda.current_stream() if stream is None else stream
        self.stream = s
        h = ctypes.c_void_p()
        rc = self.lib.gem_create(ctypes.byref(h), ctypes.byref(cfg), ctypes.c_void_p(s.cuda_stream))
        if rc != GEM_OK:
            raise GemError(rc, self.lib.gem_create_error().decode())
        self.h = h
        self.M = None
        self.B = None
        self.M64 = None
        self.B64 = None
        self.set_M = None

    # -- plumbing ------------------------------------------------------------
    def _rc(self, rc):
        if rc != GEM_OK:
            raise GemError(rc, self.lib.gem_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def gem_set_stream(self, stream):
        self.stream = stream
        self._rc(self.lib.gem_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    def gem_status(self):
        return self.lib.gem_status(self.h)

    def _views(self, params, R, t):
        M = params.shape[0] if params.dim() == 2 else -1
        B = R.shape[0] if R.dim() >= 1 else -1
        _check(params, "params", (M, NPAR))
        _check(R, "R", (B, 3, 3))
        _check(t, "t", (B, 2))
        return M, B

    # -- steps -----------------------------------------------------------------
    def gem_project(self, params, R, t, proj):
        M, B = self._views(params, R, t)
        _check(proj, "proj", (B, self.d, self.d))
        self._rc(self.lib.gem_project(self.h, _ptr(params), M, B, _ptr(R), _ptr(t), _ptr(proj)))
        self.M, self.B = M, B

    def gem_project_dense(self, params, R, t, proj):
        M, B = self._views(params, R, t)
        _check(proj, "proj", (B, self.d, self.d))
        self._rc(self.lib.gem_project_dense(self.h, _ptr(params), M, B, _ptr(R), _ptr(t), _ptr(proj)))
        self.M, self.B = M, B

    def gem_ctf_loss(self, proj, images, ctf=None, ctf_params=None, pred=None, dproj=None,
                     loss_img=None, loss=None):
        B, d = proj.shape[0], self.d
        _check(proj, "proj", (B, d, d))
        _check(images, "images", (B, d, d))
        _check(ctf, "ctf", (B, d, d // 2 + 1), optional=True)
        _check(ctf_params, "ctf_params", (B, 8), optional=True)
        _check(pred, "pred", (B, d, d), optional=True)
        _check(dproj, "dproj", (B, d, d), optional=True)
        _check(loss_img, "loss_img", (B,), torch.float64, optional=True)
        _check(loss, "loss", (1,), torch.float64, optional=True)
        self._rc(self.lib.gem_ctf_loss(self.h, B, _ptr(proj), _ptr(ctf), _ptr(ctf_params),
                                       _ptr(images), _ptr(pred), _ptr(dproj), _ptr(loss_img),
                                       _ptr(loss)))

    def gem_project_backward(self, dproj, grad):
        _check(dproj, "dproj", (self.B, self.d, self.d))
        _check(grad, "grad", (self.M, NPAR))
        self._rc(self.lib.gem_project_backward(self.h, _ptr(dproj), _ptr(grad)))

    def gem_project_backward_dense(self, dproj, grad):
        _check(dproj, "dproj", (self.B, self.d, self.d))
        _check(grad, "grad", (self.M, NPAR))
        self._rc(self.lib.gem_project_backward_dense(self.h, _ptr(dproj), _ptr(grad)))

    def gem_set_gaussians(self, params):
        M = params.shape[0]
        _check(params, "params", (M, NPAR))
        self._rc(self.lib.gem_set_gaussians(self.h, _ptr(params), M))
        self.set_M = M

    def gem_forward(self, params, R, t, images, loss, ctf=None, ctf_params=None, pred=None):
        """params None: the Gaussians of the last gem_set_gaussians."""
        if params is None:
            if self.set_M is None:
                raise GemError(GEM_ESTATE, "params None and no gem_set_gaussians")
            M, B = self.set_M, R.shape[0]
            _check(R, "R", (B, 3, 3))
            _check(t, "t", (B, 2))
        else:
            M, B = self._views(params, R, t)
        d = self.d
        _check(images, "images", (B, d, d))
        _check(ctf, "ctf", (B, d, d // 2 + 1), optional=True)
        _check(ctf_params, "ctf_params", (B, 8), optional=True)
        _check(pred, "pred", (B, d, d), optional=True)
        _check(loss, "loss", (1,), torch.float64)
        self._rc(self.lib.gem_forward(self.h, _ptr(params), M, B, _ptr(R), _ptr(t), _ptr(ctf),
                                      _ptr(ctf_params), _ptr(images), _ptr(pred), _ptr(loss)))
        self.M, self.B = M, B

    def gem_backward(self, grad):
        _check(grad, "grad", (self.M, NPAR))
        self._rc(self.lib.gem_backward(self.h, _ptr(grad)))

    # -- inspection --------------------------------------------------------------
    def gem_pair_count(self) -> int:
        n = ctypes.c_int64()
        self._rc(self.lib.gem_pair_count(self.h, ctypes.byref(n)))
        return int(n.value)

    def gem_inspect_bins(self):
        n = self.gem_pair_count()
        T = (self.d // 16) ** 2
        ts = torch.empty(self.B * T + 1, dtype=torch.int64, device="cuda")
        lst = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        self._rc(self.lib.gem_inspect_bins(self.h, _ptr(ts), _ptr(lst), lst.numel()))
        return ts, lst[:n]

    def gem_pair_stats(self):
        """-> (kept pairs, evaluated pairs) of the last projection."""
        k, e = ctypes.c_int64(), ctypes.c_int64()
        self._rc(self.lib.gem_pair_stats(self.h, ctypes.byref(k), ctypes.byref(e)))
        return int(k.value), int(e.value)

    def gem_query(self, params, tau: float = 0.0, vol=None):
        """Density on the d^3 voxel grid (Eq. query) -> vol [d][d][d] float32."""
        M, d = params.shape[0], self.d
        _check(params, "params", (M, NPAR))
        if vol is None:
            vol = torch.empty(d, d, d, dtype=torch.float32, device=params.device)
        _check(vol, "vol", (d, d, d))
        self._rc(self.lib.gem_query(self.h, _ptr(params), M, tau, _ptr(vol)))
        self.M = self.B = None
        return vol

    def gem_fsc(self, map1, map2, threshold: float = 0.143):
        """-> (fsc [d/2+1], sums [3][d/2+1], resolution [1]) as float64 device tensors."""
        d = self.d
        _check(map1, "map1", (d, d, d))
        _check(map2, "map2", (d, d, d))
        nsh = d // 2 + 1
        fsc = torch.empty(nsh, dtype=torch.float64, device=map1.device)
        sums = torch.empty(3, nsh, dtype=torch.float64, device=map1.device)
        res = torch.empty(1, dtype=torch.float64, device=map1.device)
        self._rc(self.lib.gem_fsc(self.h, _ptr(map1), _ptr(map2), threshold, _ptr(fsc), _ptr(sums),
                                  _ptr(res)))
        return fsc, sums, res

    # -- FP64 check mode ---------------------------------------------------------
    def gem_project_f64(self, params, R, t, proj):
        M, B, d = params.shape[0], R.shape[0], self.d
        f8 = torch.float64
        _check(params, "params", (M, NPAR), f8)
        _check(R, "R", (B, 3, 3), f8)
        _check(t, "t", (B, 2), f8)
        _check(proj, "proj", (B, d, d), f8)
        self._rc(self.lib.gem_project_f64(self.h, _ptr(params), M, B, _ptr(R), _ptr(t), _ptr(proj)))
        self.M64, self.B64 = M, B

    def gem_ctf_loss_f64(self, proj, images, ctf=None, ctf_params=None, pred=None, dproj=None,
                         loss_img=None, loss=None):
        B, d, f8 = proj.shape[0], self.d, torch.float64
        _check(proj, "proj", (B, d, d), f8)
        _check(images, "images", (B, d, d), f8)
        _check(ctf, "ctf", (B, d, d // 2 + 1), f8, optional=True)
        _check(ctf_params, "ctf_params", (B, 8), f8, optional=True)
        for name, x in (("pred", pred), ("dproj", dproj)):
            _check(x, name, (B, d, d), f8, optional=True)
        _check(loss_img, "loss_img", (B,), f8, optional=True)
        _check(loss, "loss", (1,), f8, optional=True)
        self._rc(self.lib.gem_ctf_loss_f64(self.h, B, _ptr(proj), _ptr(ctf), _ptr(ctf_params),
                                           _ptr(images), _ptr(pred), _ptr(dproj), _ptr(loss_img),
                                           _ptr(loss)))

    def gem_project_backward_f64(self, dproj, grad):
        f8 = torch.float64
        _check(dproj, "dproj", (self.B64, self.d, self.d), f8)
        _check(grad, "grad", (self.M64, NPAR), f8)
        self._rc(self.lib.gem_project_backward_f64(self.h, _ptr(dproj), _ptr(grad)))

    def gem_adam_step(self, raw, m, v, grad, params, lr, step: int, beta1=0.9, beta2=0.999,
                      eps=1e-8, iso_scale=None):
        """One Adam step on the raw parameters (lr: 4 group learning rates)."""
        M = raw.shape[0]
        for name, x in (("raw", raw), ("m", m), ("v", v), ("grad", grad), ("params", params)):
            _check(x, name, (M, NPAR))
        _check(iso_scale, "iso_scale", (M,), optional=True)
        cfg = gem_adam_config()
        for k in range(4):
            cfg.lr[k] = float(lr[k])
        cfg.beta1, cfg.beta2, cfg.eps, cfg.step = beta1, beta2, eps, int(step)
        self._rc(self.lib.gem_adam_step(self.h, M, ctypes.byref(cfg), _ptr(raw), _ptr(m), _ptr(v),
                                        _ptr(grad), _ptr(params), _ptr(iso_scale)))

    def gem_activate(self, raw, params):
        M = raw.shape[0]
        _check(raw, "raw", (M, NPAR))
        _check(params, "params", (M, NPAR))
        self._rc(self.lib.gem_activate(self.h, M, _ptr(raw), _ptr(params)))

    def gem_nn_distance(self, params, k: int, dist=None, idx=None):
        """-> (dist [M][k] float32, idx [M][k] int32) of the centres' k nearest neighbours."""
        M = params.shape[0]
        _check(params, "params", (M, NPAR))
        if dist is None:
            dist = torch.empty(M, k, dtype=torch.float32, device=params.device)
        if idx is None:
            idx = torch.empty(M, k, dtype=torch.int32, device=params.device)
        _check(dist, "dist", (M, k))
        _check(idx, "idx", (M, k), torch.int32)
        self._rc(self.lib.gem_nn_distance(self.h, _ptr(params), M, k, _ptr(dist), _ptr(idx)))
        return dist, idx

    # -- rasteriser configurations and the autotuner ---------------------------
    def raster_configs(self):
        return raster_configs()

    def gem_set_raster_config(self, fwd: int = -1, bwd: int = -1):
        self._rc(self.lib.gem_set_raster_config(self.h, fwd, bwd))

    def gem_get_raster_config(self, B: int, M: int):
        f, b = ctypes.c_int32(), ctypes.c_int32()
        self._rc(self.lib.gem_get_raster_config(self.h, B, M, ctypes.byref(f), ctypes.byref(b)))
        return f.value, b.value

    def gem_autotune(self, params, R, t, reps: int = 3):
        """Time every rasteriser configuration on this shape; the fastest pair
        is recorded for the process.  -> (forward index, backward index)."""
        M, B = self._views(params, R, t)
        f, b = ctypes.c_int32(), ctypes.c_int32()
        self._rc(self.lib.gem_autotune(self.h, _ptr(params), M, B, _ptr(R), _ptr(t), reps,
                                       ctypes.byref(f), ctypes.byref(b)))
        self.M = self.B = None
        return f.value, b.value

    def gem_timing(self, enable: bool):
        self._rc(self.lib.gem_timing(self.h, 1 if enable else 0))

    def gem_timing_read(self):
        """-> (ms per stage, kernel launches per stage), dicts keyed by STAGES."""
        ms = (ctypes.c_float * len(STAGES))()
        ln = (ctypes.c_int64 * len(STAGES))()
        self._rc(self.lib.gem_timing_read(self.h, ctypes.cast(ms, ctypes.c_void_p),
                                          ctypes.cast(ln, ctypes.c_void_p)))
        return dict(zip(STAGES, list(ms))), dict(zip(STAGES, list(ln)))

    def gem_inspect_records(self):
        out = torch.empty(self.B, self.M, 8, dtype=torch.float32, device="cuda")
        self._rc(self.lib.gem_inspect_records(self.h, _ptr(out)))
        return out


class GemLoss(torch.autograd.Function):
    """loss = GemLoss.apply(params, R, t, ctf_params, images, ctx): forward a1-a4,
    backward a5-a6 through the C library (poses, CTFs and images get no
    gradient, as in Eq. recon where they are known)."""

    @staticmethod
    def forward(fctx, params, R, t, ctf_params, images, gctx):
        loss = torch.empty(1, dtype=torch.float64, device=params.device)
        gctx.gem_forward(params.detach().contiguous(), R, t, images, loss, ctf_params=ctf_params)
        fctx.gctx = gctx
        fctx.M = params.shape[0]
        return loss[0]

    @staticmethod
    def backward(fctx, gout):
        grad = torch.empty(fctx.M, NPAR, dtype=torch.float32, device=gout.device)
        fctx.gctx.gem_backward(grad)
        grad = grad * gout.to(grad.dtype)
        return grad, None, None, None, None, None
