"""FP64 CPU oracle of the GEM hot path (arXiv 2509.25075, Sec. 3.2 and the
appendix derivation of the projection).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``gem_oracle.c`` (plain C, double precision, brute
force); this module compiles it with gcc and wraps it with ctypes.  Inputs are
converted to float64 here; outputs are float64 numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgem_oracle.so")
_lock = threading.Lock()
_lib = None

NPAR = 11


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  Returns the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I, L, D = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            sig = {
                "gem_oracle_num_threads": (I, []),
                "gem_oracle_preprocess": (None, [I, L, P, I, P, P, P]),
                "gem_oracle_project": (None, [I, D, D, I, L, P, I, P, P, P]),
                "gem_oracle_project_pixels": (None, [I, D, D, I, L, P, I, P, P, L, P, P]),
                "gem_oracle_tile_hits": (None, [I, D, D, I, I, L, P, I, P, P, P]),
                "gem_oracle_ctf_value": (D, [P, D, D]),
                "gem_oracle_ctf_grid_from_params": (None, [I, D, I, P, P]),
                "gem_oracle_ctf_grid_from_half": (None, [I, I, P, P]),
                "gem_oracle_ctf_apply": (None, [I, I, P, P, P]),
                "gem_oracle_loss": (D, [I, I, P, P, P, P, P, P]),
                "gem_oracle_grad": (None, [I, D, D, I, L, P, I, P, P, P, L, P, P]),
                "gem_oracle_grad_abs": (None, [I, D, D, I, L, P, I, P, P, P, L, P, P]),
                "gem_oracle_grad_border": (None, [I, D, D, I, L, P, I, P, P, P, L, P, D, P]),
                "gem_oracle_query": (None, [I, D, D, I, L, P, P]),
                "gem_oracle_query_voxels": (None, [I, D, D, I, L, P, L, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().gem_oracle_num_threads())


def constrained(params, no_rotation: bool = False, isotropic: bool = False) -> np.ndarray:
    """Parameters under the shape constraints of the ablation study (Sec. 4,
    Design Choices of 3DGS for cryo-EM): "No Rotation" fixes R_j = I, i.e. the
    quaternion becomes (1, 0, 0, 0); "Isotropic Scaling" enforces
    S_j = s_j I, with s_j the first scale entry copied to all three."""
    th = _f64(params).copy()
    if no_rotation:
        th[:, 6:10] = (1.0, 0.0, 0.0, 0.0)
    if isotropic:
        th[:, 4] = th[:, 3]
        th[:, 5] = th[:, 3]
    return th


def fold_grad(g_eff, no_rotation: bool = False, isotropic: bool = False) -> np.ndarray:
    """Chain rule through constrained(): the gradient with respect to the
    constrained parameters, mapped back to the 11 free ones.  A fixed
    quaternion has zero gradient; the shared scale collects the three."""
    g = _f64(g_eff).copy()
    if no_rotation:
        g[:, 6:10] = 0.0
    if isotropic:
        g[:, 3] = g[:, 3] + g[:, 4] + g[:, 5]
        g[:, 4] = 0.0
        g[:, 5] = 0.0
    return g


def preprocess(params, R, t, norm_mode: int = 0, no_rotation=False, isotropic=False) -> np.ndarray:
    """Per (view, Gaussian): [mean x, mean y, cov xx, cov xy, cov yy, amp, depth, valid]."""
    params, R, t = constrained(params, no_rotation, isotropic), _f64(R), _f64(t)
    M, B = params.shape[0], R.shape[0]
    out = np.zeros((B, M, 8))
    _load().gem_oracle_preprocess(norm_mode, M, _ptr(params), B, _ptr(R), _ptr(t), _ptr(out))
    return out


def project(params, R, t, d: int, apix: float, tau: float, norm_mode: int = 0,
            no_rotation=False, isotropic=False) -> np.ndarray:
    """Eq. render with Eq. accu: [B][d][d] projections."""
    params, R, t = constrained(params, no_rotation, isotropic), _f64(R), _f64(t)
    M, B = params.shape[0], R.shape[0]
    img = np.zeros((B, d, d))
    _load().gem_oracle_project(d, apix, tau, norm_mode, M, _ptr(params), B, _ptr(R), _ptr(t), _ptr(img))
    return img


def project_pixels(params, R, t, d, apix, tau, pix, norm_mode: int = 0, no_rotation=False,
                   isotropic=False) -> np.ndarray:
    """Projection at selected flat pixel indices pix = (b*d + v)*d + u."""
    params, R, t = constrained(params, no_rotation, isotropic), _f64(R), _f64(t)
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    out = np.zeros(pix.shape[0])
    _load().gem_oracle_project_pixels(d, apix, tau, norm_mode, params.shape[0], _ptr(params), R.shape[0],
                                      _ptr(R), _ptr(t), pix.shape[0], _ptr(pix), _ptr(out))
    return out


def tile_hits(params, R, t, d, apix, tau, tile, norm_mode: int = 0) -> np.ndarray:
    """[B][M][T] uint8: some pixel centre of the tile has a value above tau."""
    params, R, t = _f64(params), _f64(R), _f64(t)
    M, B = params.shape[0], R.shape[0]
    T = (d // tile) ** 2
    out = np.zeros((B, M, T), dtype=np.uint8)
    _load().gem_oracle_tile_hits(d, apix, tau, norm_mode, tile, M, _ptr(params), B, _ptr(R), _ptr(t), _ptr(out))
    return out


def ctf_value(prm, fx: float, fy: float) -> float:
    prm = _f64(prm)
    return float(_load().gem_oracle_ctf_value(_ptr(prm), float(fx), float(fy)))


def ctf_grid_from_params(prm, d: int, apix: float) -> np.ndarray:
    """[B][d][d] symmetrised transfer function from [B][8] CTF parameters."""
    prm = _f64(prm)
    B = prm.shape[0]
    full = np.zeros((B, d, d))
    _load().gem_oracle_ctf_grid_from_params(d, apix, B, _ptr(prm), _ptr(full))
    return full


def ctf_grid_from_half(half) -> np.ndarray:
    """[B][d][d] symmetrised transfer function from a [B][d][d/2+1] array."""
    half = _f64(half)
    B, d = half.shape[0], half.shape[1]
    full = np.zeros((B, d, d))
    _load().gem_oracle_ctf_grid_from_half(d, B, _ptr(half), _ptr(full))
    return full


def ctf_apply(hfull, x) -> np.ndarray:
    hfull, x = _f64(hfull), _f64(x)
    B, d = x.shape[0], x.shape[1]
    out = np.zeros_like(x)
    _load().gem_oracle_ctf_apply(d, B, _ptr(hfull), _ptr(x), _ptr(out))
    return out


def loss(hfull, proj, images):
    """Returns (L, pred, loss_img, g) of Eq. loss and its adjoint."""
    hfull, proj, images = _f64(hfull), _f64(proj), _f64(images)
    B, d = proj.shape[0], proj.shape[1]
    pred = np.zeros_like(proj)
    g = np.zeros_like(proj)
    li = np.zeros(B)
    L = _load().gem_oracle_loss(d, B, _ptr(hfull), _ptr(proj), _ptr(images), _ptr(pred), _ptr(li), _ptr(g))
    return float(L), pred, li, g


def grad(params, R, t, d, apix, tau, g, norm_mode: int = 0, sel=None, no_rotation=False,
         isotropic=False, absolute=False) -> np.ndarray:
    """dL/dtheta [nsel][11] given g = dL/dproj [B][d][d].  absolute=True: the sum
    of the absolute values of the per-pixel terms instead, the scale that
    bounds the rounding error of a float32 sum of them (test infrastructure)."""
    if no_rotation or isotropic:
        assert not absolute
        ge = grad(constrained(params, no_rotation, isotropic), R, t, d, apix, tau, g, norm_mode, sel)
        return fold_grad(ge, no_rotation, isotropic)
    params, R, t, g = _f64(params), _f64(R), _f64(t), _f64(g)
    M, B = params.shape[0], R.shape[0]
    if sel is None:
        nsel, selp, sel_arr = M, None, None
    else:
        sel_arr = np.ascontiguousarray(np.asarray(sel, dtype=np.int64))
        nsel, selp = sel_arr.shape[0], _ptr(sel_arr)
    out = np.zeros((nsel, NPAR))
    fn = _load().gem_oracle_grad_abs if absolute else _load().gem_oracle_grad
    fn(d, apix, tau, norm_mode, M, _ptr(params), B, _ptr(R), _ptr(t), _ptr(g), nsel, selp, _ptr(out))
    return out


def grad_border(params, R, t, d, apix, tau, g, rel: float = 1e-5, norm_mode: int = 0,
                sel=None) -> np.ndarray:
    """[nsel][11]: sum of |g * dvalue/dtheta| over the (pixel, Gaussian) pairs
    whose FP64 value lies within rel * tau of tau, kept or not.  These are the
    pairs whose Eq. accu decision a float32 evaluation of the value may take
    the other way, so this bounds the gradient difference such decisions
    can make (test infrastructure; the projection's counterpart is tau per
    borderline pair)."""
    params, R, t, g = _f64(params), _f64(R), _f64(t), _f64(g)
    M, B = params.shape[0], R.shape[0]
    if sel is None:
        nsel, selp = M, None
    else:
        sel_arr = np.ascontiguousarray(np.asarray(sel, dtype=np.int64))
        nsel, selp = sel_arr.shape[0], _ptr(sel_arr)
    out = np.zeros((nsel, NPAR))
    _load().gem_oracle_grad_border(d, apix, tau, norm_mode, M, _ptr(params), B, _ptr(R), _ptr(t), _ptr(g),
                                   nsel, selp, float(rel), _ptr(out))
    return out


def forward_loss(params, R, t, hfull, images, d, apix, tau, norm_mode: int = 0, no_rotation=False,
                 isotropic=False) -> float:
    """L(theta) through the whole path; used for central differences."""
    proj = project(params, R, t, d, apix, tau, norm_mode, no_rotation, isotropic)
    return loss(hfull, proj, images)[0]


def query(params, d: int, apix: float, tau: float, norm_mode: int = 0, no_rotation=False,
          isotropic=False) -> np.ndarray:
    """Eq. query on the d^3 voxel grid, vol[z][y][x], terms above tau only."""
    params = constrained(params, no_rotation, isotropic)
    vol = np.zeros((d, d, d))
    _load().gem_oracle_query(d, apix, tau, norm_mode, params.shape[0], _ptr(params), _ptr(vol))
    return vol


def query_voxels(params, d, apix, tau, vox, norm_mode: int = 0, no_rotation=False,
                 isotropic=False) -> np.ndarray:
    """Eq. query at flat voxel indices vox = (z d + y) d + x."""
    params = constrained(params, no_rotation, isotropic)
    vox = np.ascontiguousarray(np.asarray(vox, dtype=np.int64))
    out = np.zeros(vox.shape[0])
    _load().gem_oracle_query_voxels(d, apix, tau, norm_mode, params.shape[0], _ptr(params),
                                    vox.shape[0], _ptr(vox), _ptr(out))
    return out


def nn_distance(pos, k: int):
    """k nearest neighbours of each centre, by brute force.

    pos: [M][3] centres (float32 values; Sec. 4, Design Choices: the
    isotropic scale is the distance to the nearest neighbour).  The distance
    decisions are taken in float32, in the precision the GPU kernel uses:
    d^2 = ((dx^2 + dy^2) + dz^2), every operation rounded to float32; the k
    smallest (d^2, index) pairs in lexicographic order; distance =
    sqrt(d^2) rounded to float32.  Non-finite centres are never neighbours;
    missing neighbours are (inf, -1).  Returns (dist [M][k] float32,
    idx [M][k] int64).
    """
    p = np.ascontiguousarray(np.asarray(pos, dtype=np.float32))
    M = p.shape[0]
    fin = np.all(np.isfinite(p), axis=1)
    dist = np.full((M, k), np.inf, dtype=np.float32)
    idx = np.full((M, k), -1, dtype=np.int64)
    cols = np.arange(M)
    for i0 in range(0, M, 256):
        rows = np.arange(i0, min(M, i0 + 256))
        dd = [p[rows, a][:, None] - p[None, :, a] for a in range(3)]  # float32, rounded
        d2 = (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2]
        d2[:, ~fin] = np.inf
        d2[rows - i0, rows] = np.inf  # not its own neighbour
        for r, i in enumerate(rows):
            if not fin[i]:
                continue
            order = np.lexsort((cols, d2[r]))[:k]
            ok = np.isfinite(d2[r][order])
            n = int(ok.sum())
            dist[i, :n] = np.sqrt(d2[r][order[:n]])
            idx[i, :n] = order[:n]
    return dist, idx


def fsc_shell_sums(X1, X2, nshell: int | None = None):
    """Per-shell sums of Eq. fsc: (Re sum F1 F2^*, sum |F1|^2, sum |F2|^2),
    F = the 3D DFT (numpy.fft.fftn) of each real map, shell i = frequencies
    whose signed DFT indices k have round(|k|) = i.  nshell defaults to every
    shell that holds a frequency (the cube's corners included)."""
    X1, X2 = _f64(X1), _f64(X2)
    d = X1.shape[0]
    F1, F2 = np.fft.fftn(X1), np.fft.fftn(X2)
    k = np.fft.fftfreq(d) * d
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    shell = np.floor(np.sqrt(k2) + 0.5).astype(np.int64).ravel()
    n = int(shell.max()) + 1 if nshell is None else nshell
    keep = shell < n
    num = np.bincount(shell[keep], weights=np.real(F1 * np.conj(F2)).ravel()[keep], minlength=n)
    p1 = np.bincount(shell[keep], weights=(np.abs(F1) ** 2).ravel()[keep], minlength=n)
    p2 = np.bincount(shell[keep], weights=(np.abs(F2) ** 2).ravel()[keep], minlength=n)
    return num, p1, p2


def fsc_crossing(curve, d: int, apix: float, threshold: float = 0.143) -> float:
    """Resolution (Angstrom) where the FSC curve first drops below the
    threshold (Sec. 4, GSFSC): the first shell i >= 1 with FSC(i) < threshold,
    the crossing interpolated linearly between shells i-1 and i (clamped to
    that interval), resolution d apix / k*.  A curve that never drops gives
    the last shell."""
    c = np.asarray(curve, dtype=np.float64)
    kstar = float(len(c) - 1)
    for i in range(1, len(c)):
        if c[i] < threshold:
            a, b = c[i - 1], c[i]
            frac = (a - threshold) / (a - b) if a > b else 0.0
            kstar = (i - 1) + min(max(frac, 0.0), 1.0)
            break
    return d * apix / kstar if kstar > 0 else float("inf")


def fsc(X1, X2, apix: float, threshold: float = 0.143):
    """Eq. fsc over the shells 0 .. d/2 -> (fsc, (num, p1, p2), resolution)."""
    d = np.asarray(X1).shape[0]
    num, p1, p2 = fsc_shell_sums(X1, X2, d // 2 + 1)
    den = np.sqrt(p1 * p2)
    curve = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return curve, (num, p1, p2), fsc_crossing(curve, d, apix, threshold)


# ----------------------------------------------------------------------------
# Training loop: parameter activations and the Adam step (Sec. 3.2
# "Optimizing 3D GS representations"; the paper names neither, so these are
# the 3DGS practice: scales and densities through exp, Adam).
# ----------------------------------------------------------------------------

LOG_ENTRIES = np.array([3, 4, 5, 10])
GROUP_OF = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2, 2, 3])


def activate(raw) -> np.ndarray:
    """params = (p, exp(log s), q, exp(log rho)) from raw = (p, log s, q, log rho)."""
    p = _f64(raw).copy()
    p[:, LOG_ENTRIES] = np.exp(p[:, LOG_ENTRIES])
    return p


def adam_step(raw, m, v, grad, lr, step: int, beta1=0.9, beta2=0.999, eps=1e-8, iso_scale=None):
    """One Adam step (Kingma and Ba, Algorithm 1) on raw parameters, the
    gradient given with respect to activate(raw).  Returns (raw, m, v, params)."""
    raw, m, v, grad = _f64(raw).copy(), _f64(m).copy(), _f64(v).copy(), _f64(grad)
    m0, v0 = m.copy(), v.copy()
    params = activate(raw)
    g = grad.copy()
    g[:, LOG_ENTRIES] *= params[:, LOG_ENTRIES]  # d/dlog x = x d/dx
    g[~np.isfinite(g)] = 0.0
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    lrs = np.asarray(lr, dtype=np.float64)[GROUP_OF]
    new = raw - lrs[None, :] * mhat / (np.sqrt(vhat) + eps)
    params = activate(new)
    if iso_scale is not None:
        # isotropic ablation: the scales are the given distances, not learnt
        s = _f64(iso_scale)
        new[:, 3:6] = np.log(s)[:, None]
        params[:, 3:6] = s[:, None]
        m[:, 3:6] = m0[:, 3:6]
        v[:, 3:6] = v0[:, 3:6]
    return new, m, v, params
