"""Benchmark of the GEM hot path on GB300: particle images per second for one
full step (projection a1-a3, CTF + loss + adjoint a4, sparse gradient a5-a6)
on the synthetic stand-in for the paper's workloads.

  python bench.py --gpus N --steps K --warmup W [--impl gem|reference] [--workload A5]

Prints one JSON line on rank 0.  The default workload is A5 (d = 384,
M = 500,000 Gaussians, 16 images per step), the largest configuration; A2 is
also timed on the device and reported under ``secondary``.  Under torchrun
every rank runs an independent replica on its own GPU (its own batch): the
method's images are independent, so the step shards with no data-path
collective ("weak" scaling); value = images of all ranks / the slowest
rank's time.

Timing: W untimed warm-up steps, the end-to-end loop, then K steps back to
back, each bracketed by CUDA events on the library's stream with an L2 flush
(a 256 MB write) between steps, outside the events; barrier + synchronize on
both sides of the timed region; max over ranks.  The per-stage times come
from a separate pass with the library's stage events on.  The ``e2e`` figure
repeats the step through the public API with the step's inputs copied from
pinned host memory and the loss and gradient copied back inside the timed
region.  After the timed region, ``parity`` states the step's error against
the FP64 oracle on sampled outputs (projected pixels, per-image losses,
sampled Gaussians' gradients), each beside its tolerance.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle images/s, forward + adjoint gradient (projection, CTF, L2 loss, sparse gradient) per GB300"
UNIT = "images/s"
# SFU (MUFU) base-2 exponentials per clock per SM on sm_103a: 32, measured on
# GB300 by a throughput probe (8 independent ex2.approx chains per thread, one
# 1024-thread block per SM, clock64 span: 31.99 per clock per SM).  One
# exponential is the irreducible SFU cost of a kept (pixel, Gaussian) pair in
# both rasterisers.
EX2_PER_CLK_PER_SM = 32
# FP32 lanes of the FMA pipe per SM per clock (nominal 128; the same probe
# with FFMA chains measured 123.6).  Packed float pairs save issue slots, not
# FMA-pipe cycles.
FP32_PER_CLK_PER_SM = 128
# FP32 operations on the FMA pipe that the definition of a kept pair needs,
# evaluated directly (the compare runs on the ALU pipe, the exponential on
# the SFU):
#   forward (Eq. render, Eq. accu): dx, dy (2); the exponent
#     log2 A - (u11 dx + u12 dy)^2 - (u22 dy)^2 (5); the accumulation (1) -> 8
#   backward (moments of g * value): dx, dy, exponent (7); w = g * value (1);
#     the six moments w {1, z1, z2, z1^2, z1 z2, z2^2} in the whitened
#     coordinates z: 3 products, 5 adds or fused adds (8)               -> 16
# The roofline's `frac` uses these counts.  Counting every FP32 operation of
# the direct evaluation instead (the compare and the exponent's scale as
# well: about 10 forward, 30 backward) raises the peak's denominator less and
# gives larger fractions; the line reports those too (`frac_all_fp32_ops`).
FP32_OPS_PER_KEPT_PAIR = {"raster_fwd": 8, "raster_bwd": 16}
ALL_FP32_OPS_PER_KEPT_PAIR = {"raster_fwd": 10, "raster_bwd": 30}

# DRAM bytes (read + write) per launch of each rasteriser configuration, per
# workload, from ncu captures of that workload's bench step
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass each), valid while
# the sources they depend on hash to the value they had then (null otherwise).
CAPTURED_TRAFFIC = {
    "source_sha256_16": "f60b6aff05b83873",
    "per_workload": {  # workload -> {configuration name: bytes per launch}
        "A5": {
            "aligned, 256-record windows, 7 CTAs/SM, persistent longest-first": 623250688.0,
            "aligned, 256-record windows, 6 CTAs/SM, persistent longest-first": 620255232.0,
            "aligned, 256-record windows, 5 CTAs/SM, persistent longest-first": 611992064.0,
            "1 lane per record, 256-record warp windows, persistent longest-first": 2406793216.0,
            "1 lane per record, 256-record warp windows, persistent longest-first, 6 CTAs/SM": 2377032704.0,
            "1 lane per record, 256-record warp windows, persistent longest-first, 5 CTAs/SM": 2201309952.0,
        },
    },
}


def _hbm_peak():
    """Measured HBM copy bandwidth of this GPU pool (GB/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "6.8 TB/s (of fallback)"


HBM_PEAK_GBS, HBM_PEAK_NOTE = _hbm_peak()


def raster_source_hash() -> str:
    """Hash of the sources the rasterisers' traffic depends on: their own
    code, the preprocess (the memory order of the records it writes), the
    binning (the order of the lists) and the shared device header."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_25075_gb300", "csrc")
    for name in ("gem_bin.cu", "gem_internal.cuh", "gem_prep.cu", "gem_raster.cu"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gem", "reference"], default="gem")
    ap.add_argument("--workload", default="A5")
    ap.add_argument("--secondary", default="A2",
                    help="comma-separated workloads also timed on the device (N=1 only; '' for none)")
    ap.add_argument("--no-parity", action="store_true", help="skip the sampled check against the oracle")
    ap.add_argument("--batch", type=int, default=None,
                    help="images per step instead of the workload's own (a smaller case of the same "
                         "workload, e.g. for a profiler capture)")
    ap.add_argument("--raster-config", default=None,
                    help="'F,B': use forward / backward rasteriser configurations F, B (indices of "
                         "binding.raster_configs()) instead of the autotuner's choice")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain dense form")
    ap.add_argument("--no-query", action="store_true",
                    help="skip timing the density query, FSC, training iteration and nearest neighbours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def physical_gpu(local: int) -> str:
    """nvidia-smi id of this rank's GPU (index or UUID)."""
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
    if cvd:
        ids = [x.strip() for x in cvd.split(",") if x.strip()]
        if local < len(ids):
            return ids[local]
    return str(local)


def reduce_max(x: float, device=None) -> float:
    """Max of x over the ranks of the default process group (x if none)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(images_per_rank: int, seconds_max: float, world: int) -> float:
    """Whole-job images per second: every rank's images over the slowest rank's time."""
    return images_per_rank * world / seconds_max


# ------------------------------------------------------------ clocks -------

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        # samples under load: the SM clock is above idle for a busy GPU
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max([num(r[3]) for r in rows if num(r[3]) is not None] or [0])}


# ------------------------------------------------------------- oracle ------

# Full images are timed when one costs the oracle at most this many
# (pixel, Gaussian) evaluations (d^2 M); larger workloads are sampled.
FULL_IMAGE_EVALS = 5e8


def oracle_full(w, n_images: int, seed: int = 0):
    """Time the FP64 oracle on n_images whole images of workload w (full M
    and d).  Returns (seconds per image, threads, description)."""
    import oracle
    from paper_2509_25075_gb300 import synthetic as syn

    sub = syn.Workload(w.name, d=w.d, M=w.M, B=n_images, apix=w.apix, s_lo=w.s_lo, s_hi=w.s_hi,
                       n_clusters=w.n_clusters, seed=w.seed)
    inp = syn.batch(sub, seed=seed)
    inp["params"] = syn.gaussians(w)  # the workload's own Gaussian set
    t0 = time.perf_counter()
    proj = oracle.project(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, w.norm_mode)
    H = oracle.ctf_grid_from_params(inp["ctf_params"], w.d, w.apix)
    _, _, _, g = oracle.loss(H, proj, inp["images"])
    oracle.grad(inp["params"], inp["R"], inp["t"], w.d, w.apix, w.tau, g, w.norm_mode)
    dt = time.perf_counter() - t0
    return dt / n_images, dt, oracle.num_threads(), (
        f"{n_images} whole image(s) of workload {w.name} (d={w.d}, M={w.M}) through projection, "
        f"CTF + loss + adjoint and the full gradient, FP64 brute force")


def oracle_sampled(w, seed: int = 0, n_pix: int = 256, n_sel: int = 256):
    """Time the FP64 oracle on a bounded sample of one image of workload w and
    extrapolate to the whole image: the projection at n_pix pixels (each
    against all M Gaussians), the CTF + loss + adjoint of one d x d image,
    the gradient of n_sel Gaussians (each over all d^2 pixels).  Seconds per
    image = t_pix d^2 / n_pix + t_ctf + t_grad M / n_sel."""
    import numpy as np

    import oracle
    from paper_2509_25075_gb300 import synthetic as syn

    sub = syn.Workload(w.name, d=w.d, M=w.M, B=1, apix=w.apix, s_lo=w.s_lo, s_hi=w.s_hi,
                       n_clusters=w.n_clusters, seed=w.seed)
    inp = syn.batch(sub, seed=seed)
    params = syn.gaussians(w)
    rng = np.random.default_rng(seed)
    pix = rng.choice(w.d * w.d, size=n_pix, replace=False)
    sel = rng.choice(w.M, size=n_sel, replace=False)
    t0 = time.perf_counter()
    oracle.project_pixels(params, inp["R"], inp["t"], w.d, w.apix, w.tau, pix, w.norm_mode)
    t1 = time.perf_counter()
    # the CTF step's cost does not depend on the image's content: a stand-in
    # projection of the right size
    H = oracle.ctf_grid_from_params(inp["ctf_params"], w.d, w.apix)
    _, _, _, g = oracle.loss(H, syn.smooth_field(sub, seed=seed), inp["images"])
    t2 = time.perf_counter()
    oracle.grad(params, inp["R"], inp["t"], w.d, w.apix, w.tau, g, w.norm_mode, sel=sel)
    t3 = time.perf_counter()
    per_image = (t1 - t0) * w.d * w.d / n_pix + (t2 - t1) + (t3 - t2) * w.M / n_sel
    return per_image, t3 - t0, oracle.num_threads(), (
        f"workload {w.name} (d={w.d}, M={w.M}), one image sampled and extrapolated: projection at "
        f"{n_pix} pixels x {w.M} Gaussians, CTF + loss + adjoint of one {w.d}x{w.d} image, gradient of "
        f"{n_sel} Gaussians over all pixels; FP64 brute force")


def oracle_per_image(w, seed: int = 0):
    """(seconds per image, wall seconds spent, threads, description)."""
    if w.d * w.d * w.M <= FULL_IMAGE_EVALS:
        return oracle_full(w, 1, seed)
    return oracle_sampled(w, seed)


def cpu_baseline(w, budget_s: float = 15.0):
    """The oracle on the host cores: whole images while they fit the budget,
    else repeated samples of one image, extrapolated."""
    if w.d * w.d * w.M <= FULL_IMAGE_EVALS:
        dt1, _, thr, desc = oracle_full(w, 1, seed=0)
        n = max(1, min(16, int(budget_s / max(dt1, 1e-3))))
        secs = dt1
        if n > 1:
            secs, _, thr, desc = oracle_full(w, n, seed=1)
    else:
        reps, wall = [], 0.0
        while len(reps) < 8 and wall < budget_s:
            d, dw, thr, desc = oracle_sampled(w, seed=len(reps))
            reps.append(d)
            wall += dw
        secs = sum(reps) / len(reps)
        desc = f"{len(reps)} samples ({wall:.1f} s of host time), each " + desc + " (value extrapolated)"
    return {"value": 1.0 / secs, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": desc + f"; {secs:.3g} s per image on {thr} host threads"}


def run_reference(args):
    """--impl reference: the oracle on the host cores, K steps, each a bounded
    sample of the workload (one whole image, or one image sampled and
    extrapolated when whole images are too costly).  ms_per_step is the
    steps' own wall time; value is images per second of oracle work (for a
    sampled step, the image's extrapolated cost)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2509_25075_gb300 import synthetic as syn

    w = syn.WORKLOADS[args.workload]
    for i in range(args.warmup):
        oracle_per_image(w, seed=100 + i)
    per_image, wall, thr, desc = 0.0, 0.0, 1, ""
    for i in range(args.steps):
        dt, dw, thr, desc = oracle_per_image(w, seed=200 + i)
        per_image += dt
        wall += dw
    value = args.steps / per_image
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(w),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": "per step: " + desc + (
                             "" if w.d * w.d * w.M <= FULL_IMAGE_EVALS else
                             f" (value extrapolated: {per_image / args.steps:.3g} s per image)")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(w):
    return {"workload": f"{w.name}: GEM step on d={w.d} px images, M={w.M} Gaussians, B={w.B} images "
                        f"per step, apix={w.apix} A, tau={w.tau:.4g}, scales {w.s_lo}-{w.s_hi} px, "
                        f"{w.n_clusters} clusters, CTF from parameters",
            "d": w.d, "M": w.M, "global_batch": w.B, "tau": w.tau, "norm_mode": w.norm_mode,
            "zsort": 1, "l2": "flushed between timed steps (256 MB write)"}


# ------------------------------------------------------- parity -------------

def parity_check(ctx, w, D, host, dev, n_pix: int = 96, n_img: int = 2, n_sel: int = 12):
    """Error of this workload's step against the FP64 oracle, on outputs the
    oracle can compute one by one at full size (run after the timed region):
      projection   n_pix sampled pixels (half near the particle) against
                   oracle.project_pixels; tolerance 1e-5 of the image maximum
                   plus tau for each pair float32 may decide differently
                   (at most a few per pixel here: 8 tau);
      ctf_loss     per-image losses of n_img images: the oracle's Eq. loss on
                   this step's projection of those images (an oracle
                   projection of a whole image at this size takes minutes on
                   the host); relative tolerance 1e-5;
      gradient     n_sel sampled Gaussians, upstream gradient = this step's
                   dL/dI^, against oracle.grad: per Gaussian ||dg|| <= 1e-4
                   ||g|| plus the terms of its pairs within 1e-5 relative of
                   tau (oracle.grad_border)."""
    import numpy as np
    import torch

    import oracle

    B, d = w.B, w.d
    proj = torch.empty(B, d, d, device=dev)
    ctx.gem_project(D["params"], D["R"], D["t"], proj)
    li = torch.empty(B, dtype=torch.float64, device=dev)
    dproj = torch.empty(B, d, d, device=dev)
    ctx.gem_ctf_loss(proj, D["images"], ctf_params=D["ctf_params"], dproj=dproj, loss_img=li)
    grad = torch.empty(w.M, 11, device=dev)
    ctx.gem_project_backward(dproj, grad)
    if ctx.gem_status() != 0:
        raise RuntimeError("device status in the parity check: " + ctx.lib.gem_last_error(ctx.h).decode())
    P = proj.cpu().numpy()
    rng = np.random.default_rng(2024)
    b = rng.integers(0, B, n_pix)
    c, r = d // 2, int(0.3 * d)
    near = np.arange(n_pix) < n_pix // 2
    v = np.where(near, rng.integers(c - r, c + r, n_pix), rng.integers(0, d, n_pix))
    u = np.where(near, rng.integers(c - r, c + r, n_pix), rng.integers(0, d, n_pix))
    pix = (b * d + v) * d + u
    ref = oracle.project_pixels(host["params"], host["R"], host["t"], d, w.apix, w.tau, pix, w.norm_mode)
    perr = float(np.max(np.abs(P.reshape(-1)[pix] - ref)))
    scale = float(np.abs(P).max())
    ptol = 1e-5 * scale + 8 * w.tau
    imgs = np.unique(np.linspace(0, B - 1, n_img).astype(int))
    H = oracle.ctf_grid_from_params(host["ctf_params"][imgs], d, w.apix)
    _, _, oli, _ = oracle.loss(H, P[imgs], host["images"][imgs])
    lerr = float(np.max(np.abs(li.cpu().numpy()[imgs] - oli) / np.abs(oli)))
    sel = rng.choice(w.M, size=n_sel, replace=False)
    g = dproj.cpu().numpy().astype(np.float64)
    gref = oracle.grad(host["params"], host["R"], host["t"], d, w.apix, w.tau, g, w.norm_mode, sel=sel)
    gb = oracle.grad_border(host["params"], host["R"], host["t"], d, w.apix, w.tau, g, 1e-5, w.norm_mode, sel=sel)
    got = grad.cpu().numpy().astype(np.float64)[sel]
    ratio, rel = 0.0, 0.0
    for k in range(n_sel):
        nrm = np.linalg.norm(gref[k])
        err = np.linalg.norm(got[k] - gref[k])
        if nrm > 0:
            rel = max(rel, err / nrm)
        bound = 1e-4 * nrm + np.linalg.norm(gb[k])
        ratio = max(ratio, err / bound if bound > 0 else (0.0 if err == 0 else float("inf")))
    return {
        "oracle": "FP64 brute force on the host (every pixel against every Gaussian)",
        "projection": {"pixels": int(n_pix), "max_abs_err": perr, "image_max": scale, "tol": ptol,
                       "ok": bool(perr <= ptol)},
        "ctf_loss": {"images": int(len(imgs)), "max_rel_err": lerr, "tol": 1e-5, "ok": bool(lerr <= 1e-5),
                     "input": "this step's projection of those images"},
        "gradient": {"gaussians": int(n_sel), "max_rel_err": float(rel), "tol": 1e-4,
                     "max_err_over_bound": float(ratio), "ok": bool(ratio <= 1.0),
                     "bound": "1e-4 ||g_k|| + the terms of its pairs within 1e-5 relative of tau",
                     "upstream": "this step's dL/dI^"},
    }


def time_secondary(w, dev, stream, flush, steps: int, warm: int):
    """Device time of the step on another workload (same protocol as the
    main timed region, one GPU)."""
    import torch

    from paper_2509_25075_gb300 import binding
    from paper_2509_25075_gb300 import synthetic as syn

    host = syn.batch(w, seed=w.seed + 1000)
    host["params"] = syn.gaussians(w)
    D = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    ctx = binding.Context(w.d, w.apix, w.B, w.M, tau=w.tau, norm_mode=w.norm_mode, zsort=1, stream=stream)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.empty(w.M, 11, device=dev)

    def step():
        ctx.gem_forward(D["params"], D["R"], D["t"], D["images"], loss, ctf_params=D["ctf_params"])
        ctx.gem_backward(grad)

    tuned = ctx.gem_autotune(D["params"], D["R"], D["t"], reps=3)
    for _ in range(warm):
        flush.zero_()
        step()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step()
    for _ in range(2):
        flush.zero_()
        graph.replay()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if ctx.gem_status() != 0:
        raise RuntimeError("device status (secondary): " + ctx.lib.gem_last_error(ctx.h).decode())
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    ctx.gem_timing(True)
    stage = {k: 0.0 for k in binding.STAGES}
    n = max(1, min(steps, 10))
    for _ in range(n):
        flush.zero_()
        step()
        m, _ = ctx.gem_timing_read()
        for k in stage:
            stage[k] += m[k] / n
    ctx.close()
    fn, bn = binding.raster_configs()
    return {"value": w.B / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "config": workload_config(w), "stages_ms": stage,
            "timing": "device (CUDA events), L2 flushed, each step one CUDA-graph replay",
            "raster_configs": {"forward": fn[tuned[0]], "backward": bn[tuned[1]]}}


# --------------------------------------------------------------- main ------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2509_25075_gb300 import binding
    from paper_2509_25075_gb300 import synthetic as syn

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = syn.WORKLOADS[args.workload]
    if args.batch:
        w = dataclasses.replace(w, B=args.batch)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    host = syn.batch(w, seed=w.seed + 1000 * rank)
    # the Gaussians are the model: the same on every rank
    host["params"] = syn.gaussians(w)
    D = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    ctx = binding.Context(w.d, w.apix, w.B, w.M, tau=w.tau, norm_mode=w.norm_mode, zsort=1, stream=stream)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.empty(w.M, 11, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(X=None):
        X = D if X is None else X
        ctx.gem_forward(X["params"], X["R"], X["t"], X["images"], loss, ctf_params=X["ctf_params"])
        ctx.gem_backward(grad)

    # the rasterisers' kernel configurations for this shape (the library's
    # autotuner, once, outside every timed region)
    fwd_names, bwd_names = binding.raster_configs()
    if args.raster_config:
        tuned = tuple(int(x) for x in args.raster_config.split(","))
        ctx.gem_set_raster_config(*tuned)
        chosen = "--raster-config"
    else:
        tuned = ctx.gem_autotune(D["params"], D["R"], D["t"], reps=3)
        chosen = "gem_autotune (every configuration timed 3x on this shape)"
    raster_cfg = {"forward": fwd_names[tuned[0]], "backward": bwd_names[tuned[1]], "chosen_by": chosen}

    warm = max(args.warmup, 3)
    for _ in range(warm):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if ctx.gem_status() != 0:
        raise RuntimeError("device status after warm-up: " + ctx.lib.gem_last_error(ctx.h).decode())

    # The step as a CUDA graph: gem_forward and gem_backward only enqueue
    # kernels and copies on the context's stream, with no host
    # synchronisation and no allocation, so a captured step replays the same
    # work on the same buffers without the launch gaps.  The timed steps and
    # the end-to-end loop replay graphs; the per-stage pass runs eagerly.
    step_graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(step_graph, stream=stream):
        step()
    for _ in range(2):
        flush.zero_()
        step_graph.replay()
    torch.cuda.synchronize()
    if ctx.gem_status() != 0:
        raise RuntimeError("device status after the graph warm-up: " + ctx.lib.gem_last_error(ctx.h).decode())

    # the clock sampler runs from here to the end of the device-timed region
    clocks = ClockSampler(physical_gpu(local))
    clocks.start()
    time.sleep(0.3)

    # ---- plain dense form (timed before the tiled path; its load also
    # brings the GPU to its clocks) ----------------------------------------------
    plain = None
    if not args.no_plain:
        pd = torch.empty(w.B, w.d, w.d, device=dev)
        dp = torch.empty(w.B, w.d, w.d, device=dev)
        g2 = torch.empty(w.M, 11, device=dev)

        def pstep():
            ctx.gem_project_dense(D["params"], D["R"], D["t"], pd)
            ctx.gem_ctf_loss(pd, D["images"], ctf_params=D["ctf_params"], dproj=dp, loss=loss)
            ctx.gem_project_backward_dense(dp, g2)

        pstep()
        torch.cuda.synchronize()
        n_plain = 2
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n_plain):
            pstep()
        b.record(stream)
        torch.cuda.synchronize()
        pv = w.B * n_plain / (a.elapsed_time(b) / 1e3)
        plain = {"value": pv, "unit": UNIT,
                 "form": "one thread per pixel over all M Gaussians; one thread per (image, Gaussian) over all pixels"}

    # ---- end to end through the public API, host buffers (run before the
    # device-timed region, whose steps follow it directly).  Every step copies
    # its inputs from pinned host memory and reads its loss and gradient back;
    # the inputs of step i + 1 are copied on a second stream into the other
    # of two device buffers while step i runs, as a data loader would, and
    # the loss and gradient of step i are read back on a third stream from
    # the other of two output buffers while step i + 1 runs.  The timed
    # region runs from the first copy to the last read, L2 flushes between
    # steps included. ------------------------------------------------------------
    pinned = {k: torch.from_numpy(host[k]).pin_memory() for k in ("images", "R", "t", "ctf_params")}
    out_grads = [torch.empty(w.M, 11).pin_memory() for _ in range(2)]
    out_losses = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    dev_grads = [grad, torch.empty_like(grad)]
    dev_losses = [loss, torch.zeros_like(loss)]
    h2d = sum(v.numel() * v.element_size() for v in pinned.values())
    d2h = out_grads[0].numel() * 4 + 8
    e2e_steps = max(1, min(args.steps, 50))
    bufs = [dict(D, **{k: torch.empty_like(D[k]) for k in pinned}) for _ in range(2)]
    copy_stream = torch.cuda.Stream(device=dev)
    read_stream = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event() for _ in range(2)]  # inputs of buffer i copied
    done = [torch.cuda.Event() for _ in range(2)]   # the step reading buffer i finished
    readback = [torch.cuda.Event() for _ in range(2)]  # outputs of buffer i read back
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # one graph of the step per input / output buffer pair
    e2e_graphs = []
    for p in range(2):
        gph = torch.cuda.CUDAGraph()
        X = bufs[p]
        with torch.cuda.graph(gph, stream=stream):
            ctx.gem_forward(X["params"], X["R"], X["t"], X["images"], dev_losses[p],
                            ctf_params=X["ctf_params"])
            ctx.gem_backward(dev_grads[p])
        e2e_graphs.append(gph)

    def copy_inputs(i):
        with torch.cuda.stream(copy_stream):
            if i >= 2:
                copy_stream.wait_event(done[i % 2])
            for k, v in pinned.items():
                bufs[i % 2][k].copy_(v, non_blocking=True)
            ready[i % 2].record(copy_stream)

    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e_start.record(copy_stream)
    copy_inputs(0)
    for i in range(e2e_steps):
        if i + 1 < e2e_steps:
            copy_inputs(i + 1)
        stream.wait_event(ready[i % 2])
        if i >= 2:
            stream.wait_event(readback[i % 2])  # step i - 2's outputs are read
        flush.zero_()
        e2e_graphs[i % 2].replay()
        done[i % 2].record(stream)
        with torch.cuda.stream(read_stream):
            read_stream.wait_event(done[i % 2])
            out_grads[i % 2].copy_(dev_grads[i % 2], non_blocking=True)
            out_losses[i % 2].copy_(dev_losses[i % 2], non_blocking=True)
            readback[i % 2].record(read_stream)
    stream.wait_event(readback[(e2e_steps - 1) % 2])
    e_end.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e2e_s = reduce_max(e_start.elapsed_time(e_end) / 1e3, dev)
    e2e = {"value": throughput(w.B * e2e_steps, e2e_s, ws), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "steps": e2e_steps,
           "overlap": "inputs of the next step copied, outputs of the last one read back, on two "
                      "more streams (two buffers each)",
           "l2": "flushed between steps, inside the timed region"}

    # ---- device-timed region: K steps back to back ----------------------------
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ctx.gem_status() != 0:
        raise RuntimeError("device status after the end-to-end loop: " + ctx.lib.gem_last_error(ctx.h).decode())
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step_graph.replay()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(step_ms) / 1e3
    status = ctx.gem_status()
    if status != 0:
        raise RuntimeError("device status after timed region: " + ctx.lib.gem_last_error(ctx.h).decode())
    total_max = reduce_max(total_s, dev)
    value = throughput(w.B * args.steps, total_max, ws)
    step_loss = float(loss.item())
    if plain is not None:
        plain["speedup_of_tiled"] = value / ws / plain["value"]

    # ---- per-stage device times and launch counts: a separate pass with the
    # library's stage events on (reading them synchronises after every step)
    ctx.gem_timing(True)
    n_stage = max(1, min(args.steps, 20))
    stage_ms = {k: 0.0 for k in binding.STAGES}
    launches_per_step = 0
    for i in range(n_stage):
        flush.zero_()
        step()
        ms, ln = ctx.gem_timing_read()
        for k in stage_ms:
            stage_ms[k] += ms[k]
        launches_per_step = sum(ln.values())
    ctx.gem_timing(False)
    launches = launches_per_step * args.steps

    # ---- roofline of the dominant kernel ----------------------------------------
    kept, evaluated = ctx.gem_pair_stats()
    pairs = ctx.gem_pair_count()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    per_stage = {k: v / n_stage for k, v in stage_ms.items()}
    dom = max(("raster_fwd", "raster_bwd"), key=lambda k: per_stage[k])
    mhz = clk.get("sm_mhz") or 1455.0
    ops = FP32_OPS_PER_KEPT_PAIR[dom]
    per_clk = min(FP32_PER_CLK_PER_SM / ops, EX2_PER_CLK_PER_SM)  # kept pairs per clock per SM
    peak = sms * per_clk * mhz * 1e6 / 1e9  # Gpair/s
    peak_sfu = sms * EX2_PER_CLK_PER_SM * mhz * 1e6 / 1e9
    achieved = kept / (per_stage[dom] / 1e3) / 1e9
    cap = CAPTURED_TRAFFIC["per_workload"].get(w.name, {}) \
        if raster_source_hash() == CAPTURED_TRAFFIC["source_sha256_16"] and not args.batch else {}
    cfg_name = {"raster_fwd": raster_cfg["forward"], "raster_bwd": raster_cfg["backward"]}
    traffic = cap.get(cfg_name[dom])
    other = "raster_bwd" if dom == "raster_fwd" else "raster_fwd"
    o_peak = sms * min(FP32_PER_CLK_PER_SM / FP32_OPS_PER_KEPT_PAIR[other], EX2_PER_CLK_PER_SM) * mhz * 1e6 / 1e9
    o_ach = kept / (per_stage[other] / 1e3) / 1e9

    def all_ops_peak(k):
        return sms * min(FP32_PER_CLK_PER_SM / ALL_FP32_OPS_PER_KEPT_PAIR[k], EX2_PER_CLK_PER_SM) * mhz * 1e6 / 1e9

    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "Gpair/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
            "ops_per_kept_pair": FP32_OPS_PER_KEPT_PAIR[dom],
            "frac_all_fp32_ops": achieved / all_ops_peak(dom),
            "other_rasteriser": {"kernel": other, "achieved": o_ach, "peak": o_peak, "frac": o_ach / o_peak,
                                 "ops_per_kept_pair": FP32_OPS_PER_KEPT_PAIR[other],
                                 "frac_all_fp32_ops": o_ach / all_ops_peak(other),
                                 "traffic": cap.get(cfg_name[other])},
            "peak_note": f"{sms} SMs x min({FP32_PER_CLK_PER_SM} FP32 lanes / {ops} FMA-pipe ops per kept "
                         f"pair, {EX2_PER_CLK_PER_SM} ex2) per clock x {mhz:.0f} MHz median SM clock under load",
            "sfu_only": {"peak": peak_sfu, "frac": achieved / peak_sfu,
                         "note": "one SFU exponential per kept pair, no other work counted"},
            "kept_pairs_per_launch": kept, "evaluated_pairs_per_launch": evaluated,
            "listed_pairs_per_launch": pairs}

    # ---- density query on the d^3 grid (Eq. query) -----------------------------
    query = None
    if not args.no_query:
        vol = torch.empty(w.d, w.d, w.d, device=dev)
        tq = w.tau_query
        for _ in range(3):
            ctx.gem_query(D["params"], tq, vol)
        torch.cuda.synchronize()
        nq = 10
        qe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nq)]
        for i in range(nq):
            flush.zero_()
            qe[i][0].record(stream)
            ctx.gem_query(D["params"], tq, vol)
            qe[i][1].record(stream)
        torch.cuda.synchronize()
        if ctx.gem_status() != 0:
            raise RuntimeError("device status after the query: " + ctx.lib.gem_last_error(ctx.h).decode())
        q_ms = sum(a.elapsed_time(b) for a, b in qe) / nq
        nbatch = -(-w.d // w.B)
        query = {"ms": q_ms, "voxels_per_s": w.d ** 3 / (q_ms / 1e3), "grid": w.d, "M": w.M, "tau": tq,
                 "slice_batches": nbatch, "gpu_launches_per_call": 1 + 6 * nbatch,
                 "l2": "flushed before each call (256 MB write)"}
        # Fourier shell correlation of the map against the map of perturbed
        # Gaussians (the two half-maps of Eq. fsc)
        vol2 = torch.empty_like(vol)
        p2 = D["params"].clone()
        p2[:, 0:3] += 0.3 * w.apix * torch.randn(w.M, 3, device=dev, generator=torch.Generator(dev).manual_seed(5))
        ctx.gem_query(p2, tq, vol2)
        fsc_out = None
        for _ in range(3):
            fsc_out = ctx.gem_fsc(vol, vol2)
        torch.cuda.synchronize()
        fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nq)]
        for i in range(nq):
            flush.zero_()
            fe[i][0].record(stream)
            ctx.gem_fsc(vol, vol2)
            fe[i][1].record(stream)
        torch.cuda.synchronize()
        f_ms = sum(a.elapsed_time(b) for a, b in fe) / nq
        f_bytes = 64 * w.d ** 3  # 3 FFT passes (read + write d^3 complex) and the shell pass (2 reads)
        f_gbs = f_bytes / (f_ms / 1e3) / 1e9
        query["fsc"] = {"ms": f_ms, "resolution_A": float(fsc_out[2].item()), "gpu_launches_per_call": 5,
                        "roofline": {"bound": "hbm", "achieved": f_gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                     "frac": f_gbs / HBM_PEAK_GBS, "algorithmic_bytes": f_bytes,
                                     "peak_note": HBM_PEAK_NOTE}}
        if nbatch == 1:
            qk, qv = ctx.gem_pair_stats()
            qa = qk / (q_ms / 1e3) / 1e9
            qpeak = sms * min(FP32_PER_CLK_PER_SM / FP32_OPS_PER_KEPT_PAIR["raster_fwd"],
                              EX2_PER_CLK_PER_SM) * mhz * 1e6 / 1e9
            query.update({"kept_pairs": qk, "evaluated_pairs": qv,
                          "roofline": {"bound": "alu", "kernel": "whole query", "achieved": qa, "peak": qpeak,
                                       "unit": "Gpair/s", "frac": qa / qpeak}})

    # ---- training iteration (step + Adam on raw parameters), nearest neighbours
    train = None
    if not args.no_query:
        raw = D["params"].clone()
        raw[:, 3:6] = torch.log(raw[:, 3:6].abs())
        raw[:, 10] = torch.log(raw[:, 10])
        m_a, v_a, p_a = torch.zeros_like(raw), torch.zeros_like(raw), torch.empty_like(raw)
        ctx.gem_activate(raw, p_a)
        lr = (1e-3, 1e-3, 1e-3, 1e-3)
        nn_d = torch.empty(w.M, 1, device=dev)
        nn_i = torch.empty(w.M, 1, dtype=torch.int32, device=dev)

        def tstep(i):
            ctx.gem_forward(p_a, D["R"], D["t"], D["images"], loss, ctf_params=D["ctf_params"])
            ctx.gem_backward(grad)
            ctx.gem_adam_step(raw, m_a, v_a, grad, p_a, lr, i + 1)

        for i in range(3):
            tstep(i)
        torch.cuda.synchronize()
        nt = 10
        te = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nt)]
        ae = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nt)]
        ke = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nt)]
        for i in range(nt):
            flush.zero_()
            te[i][0].record(stream)
            tstep(3 + i)
            te[i][1].record(stream)
            flush.zero_()
            ae[i][0].record(stream)
            ctx.gem_adam_step(raw, m_a, v_a, grad, p_a, lr, 4 + nt + i)
            ae[i][1].record(stream)
            flush.zero_()
            ke[i][0].record(stream)
            ctx.gem_nn_distance(p_a, 1, nn_d, nn_i)
            ke[i][1].record(stream)
        torch.cuda.synchronize()
        if ctx.gem_status() != 0:
            raise RuntimeError("device status after the training loop: " + ctx.lib.gem_last_error(ctx.h).decode())
        t_ms = sum(a.elapsed_time(b) for a, b in te) / nt
        a_ms = sum(a.elapsed_time(b) for a, b in ae) / nt
        k_ms = sum(a.elapsed_time(b) for a, b in ke) / nt
        a_bytes = 8 * 4 * w.M * 11  # raw, m, v, grad read; raw, m, v, params written
        a_gbs = a_bytes / (a_ms / 1e3) / 1e9
        train = {"images_per_s": w.B / (t_ms / 1e3), "ms_per_iteration": t_ms,
                 "iteration": "projection, CTF + loss + adjoint, sparse gradient, Adam on raw parameters",
                 "adam_ms": a_ms,
                 "adam_roofline": {"bound": "hbm", "achieved": a_gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                   "frac": a_gbs / HBM_PEAK_GBS, "algorithmic_bytes": a_bytes,
                                   "peak_note": HBM_PEAK_NOTE},
                 "nearest_neighbour_ms": k_ms, "nearest_neighbour_k": 1,
                 "l2": "flushed before each timed call (256 MB write)"}

    # ---- error against the FP64 oracle, on sampled outputs of this step's inputs
    parity = None
    if rank == 0 and not args.no_parity:
        parity = parity_check(ctx, w, D, host, dev)

    # ---- other workloads, device-timed (one GPU only)
    secondary = None
    if ws == 1 and args.secondary:
        secondary = {}
        for name in [x for x in args.secondary.split(",") if x and x != w.name]:
            secondary[name] = time_secondary(syn.WORKLOADS[name], dev, stream, flush, args.steps, warm)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(w)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": warm, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(w), "clocks": clk, "e2e": e2e,
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "plain": plain,
            "stages_ms": per_stage, "raster_configs": raster_cfg, "loss": step_loss, "parity": parity,
            "timing": "device (CUDA events); each step one replay of a CUDA graph of gem_forward + "
                      "gem_backward (e2e: one graph per input/output buffer pair); stages_ms from a "
                      "separate eager pass",
            "secondary": secondary,
            "query": query, "train": train,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
