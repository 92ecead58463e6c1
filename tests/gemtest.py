"""Shared helpers of the GPU tests: run a case on the GPU through the C ABI
and on the oracle, and compare with the tolerances of the hot-path contract.

Tolerances (float32 path against the FP64 oracle):
  projection  max |dI| <= 1e-5 max |I| (+ tau for each pair whose value sits
              within 1e-5 relative of tau, where float32 and float64 may take
              the threshold decision differently)
  loss        relative <= 1e-5
  gradient    ||dg|| / ||g|| <= 1e-4, and per entry relative <= 1e-3 where
              |g| > 1e-3 max |g|; at full size per sampled Gaussian, plus
              the terms of the pairs within 1e-5 relative of tau
  pred, dL/dI max abs <= 1e-5 max |.|
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2509_25075_gb300 import binding
from paper_2509_25075_gb300 import synthetic as syn

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(DEV)


def inputs(w: syn.Workload, seed=None):
    return syn.batch(w, seed=seed)


def context(w: syn.Workload, **kw):
    return binding.Context(w.d, w.apix, w.B, w.M, tau=kw.pop("tau", w.tau),
                           norm_mode=kw.pop("norm_mode", w.norm_mode), **kw)


def morton_keys(params, d, apix):
    """15-bit 3D Morton key of every Gaussian's mean as the library defines
    it (gem_project): cell floor((p / (d apix) + 1/2) 32) per axis, clamped
    to 0..31 (each step rounded to float32), bits interleaved x, y, z from
    bit 0."""
    side = np.float32(np.float32(d) * np.float32(apix))
    inv = np.float32(1.0) / side
    p = np.asarray(params, dtype=np.float32)[:, :3]
    with np.errstate(invalid="ignore"):
        c = np.floor((p * inv + np.float32(0.5)) * np.float32(32.0))
    c = np.clip(np.nan_to_num(c, nan=0.0), 0, 31).astype(np.int64)
    key = np.zeros(len(p), dtype=np.int64)
    for b in range(5):
        for a in range(3):
            key |= ((c[:, a] >> b) & 1) << (3 * b + a)
    return key


def borderline_pairs(inp, w, tau, norm_mode=0, rel=1e-5):
    """Number of (pixel, Gaussian) pairs whose FP64 value lies within
    rel * tau of tau, per image (brute force, small cases only)."""
    if tau <= 0:
        return np.zeros(inp["R"].shape[0], dtype=np.int64)
    B = inp["R"].shape[0]
    M = inp["params"].shape[0]
    counts = np.zeros(B, dtype=np.int64)
    for j in range(M):
        img = oracle.project(inp["params"][j:j + 1], inp["R"], inp["t"], w.d, w.apix, 0.0, norm_mode)
        counts += np.sum(np.abs(img - tau) <= rel * tau, axis=(1, 2))
    return counts


def kept_pairs(inp, w, tau, norm_mode=0, rel=1e-5):
    """(pairs with FP64 value > tau, pairs within rel * tau of tau) over all
    images, by brute force one Gaussian at a time (small cases only)."""
    kept = border = 0
    for j in range(inp["params"].shape[0]):
        img = oracle.project(inp["params"][j:j + 1], inp["R"], inp["t"], w.d, w.apix, 0.0, norm_mode)
        kept += int(np.sum(img > tau))
        border += int(np.sum(np.abs(img - tau) <= rel * tau))
    return kept, border


def assert_proj_close(got, ref, tau=0.0, border=None, rel=1e-5):
    got = np.asarray(got, dtype=np.float64)
    scale = np.max(np.abs(ref))
    allow = rel * scale
    if border is not None:
        allow = allow + tau * float(np.max(border))
    err = np.max(np.abs(got - ref))
    assert err <= allow, f"projection max err {err:.3e} > {allow:.3e} (scale {scale:.3e})"


def assert_grad_per_gaussian(got, ref, border, norm_tol=1e-4, entry_tol=1e-3):
    """The gradient tolerance of the hot-path contract, held per Gaussian:
    ||dg_k|| <= norm_tol ||g_k|| for every compared Gaussian k, and per entry
    relative <= entry_tol where |g| > 1e-3 max |g| (over the compared set).

    border [k][11] (oracle.grad_border) is the sum of |g dvalue/dtheta| over
    the pairs whose FP64 value lies within 1e-5 relative of tau: float32 may
    keep or drop exactly those pairs differently from FP64 (Eq. accu), and a
    flipped pair moves the gradient by its own term, so border is added to
    each bound (the projection's counterpart is tau per borderline pair).
    Returns the largest ratio of error to bound, per Gaussian and per entry."""
    got = np.asarray(got, dtype=np.float64)
    worst_g = 0.0
    for k in range(ref.shape[0]):
        nrm = np.linalg.norm(ref[k])
        err = np.linalg.norm(got[k] - ref[k])
        bound = norm_tol * nrm + np.linalg.norm(border[k])
        if bound == 0:
            assert err == 0, (k, got[k], ref[k])
            continue
        worst_g = max(worst_g, err / bound)
        assert err <= bound, f"Gaussian {k}: ||dg|| {err:.3e} > {bound:.3e} (||g|| {nrm:.3e})"
    big = np.abs(ref) > 1e-3 * np.max(np.abs(ref))
    bound_e = entry_tol * np.abs(ref) + border
    ratio = np.abs(got - ref)[big] / bound_e[big]
    worst_e = float(ratio.max()) if ratio.size else 0.0
    assert worst_e <= 1.0, f"gradient per-entry error at {worst_e:.3f} of its bound"
    return worst_g, worst_e


def assert_grad_close(got, ref, norm_tol=1e-4, entry_tol=1e-3):
    got = np.asarray(got, dtype=np.float64)
    nrm = np.linalg.norm(ref)
    assert nrm > 0
    rel = np.linalg.norm(got - ref) / nrm
    assert rel <= norm_tol, f"gradient relative norm error {rel:.3e}"
    big = np.abs(ref) > 1e-3 * np.max(np.abs(ref))
    ent = np.max(np.abs(got[big] - ref[big]) / np.abs(ref[big]))
    assert ent <= entry_tol, f"gradient per-entry relative error {ent:.3e}"
    return rel, ent
