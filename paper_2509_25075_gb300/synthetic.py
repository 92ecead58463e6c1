"""Seeded synthetic inputs shaped like single-particle cryo-EM workloads.

This module draws random numbers only.  It holds none of the method's
arithmetic (no projection, no quaternion-to-rotation, no CTF formula), so both
the CUDA path and the CPU oracle can consume its arrays without sharing code.

Recipe (the paper's EMPIAR stacks are not available; these stand in for them):
  * Gaussian centres: ``n_clusters`` cluster centres uniform in a ball of
    radius 0.3 * d * apix, members N(0, (0.04 * d * apix)^2) per axis.
  * Scales s (3 per Gaussian): log-uniform over [s_lo, s_hi] pixels, times apix.
  * Quaternions: N(0, I_4), left unnormalised (the method normalises).
  * rho ~ U(0.5, 1.5).
  * Views: Haar-random rotations (QR of a Gaussian 3x3, sign-fixed, det +1);
    in-plane shifts t ~ N(0, (2 px * apix)^2).
  * CTF parameters per image: 300 kV, Cs 2.7 mm, amplitude contrast 0.1,
    defocus U(1.0, 2.5) um with astigmatism up to 0.05 um at a uniform angle,
    no phase shift, no B-factor.
  * Images: N(0, sigma^2) noise, sigma = nominal signal / sqrt(0.1), where the
    nominal signal is the mean mass per square Angstrom over the particle's
    projected disc (SNR 0.1).  The content of the images does not change the
    cost of any step.
  * apix = 1.2 A (close to the 1.215-1.31 A implied by the paper's Nyquist
    limits).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

NPAR = 11


@dataclass(frozen=True)
class Workload:
    name: str
    d: int
    M: int
    B: int
    apix: float = 1.2
    s_lo: float = 0.5          # smallest scale, pixels
    s_hi: float = 3.0          # largest scale, pixels
    n_clusters: int = 64
    cluster_sigma: float = 0.04  # fraction of d * apix
    forward_only: bool = False
    norm_mode: int = 0
    seed: int = 0

    def __post_init__(self):
        # the library takes apix as float32: hold the float32 value so that
        # every consumer sees the same number
        object.__setattr__(self, "apix", float(np.float32(self.apix)))

    @property
    def tau(self) -> float:
        """Threshold of Eq. accu: 1e-4 of the largest possible 2D peak
        (rho_max / (2 pi s_min^2)) of this recipe, rounded to float32."""
        s_min = self.s_lo * self.apix
        return float(np.float32(1e-4 * 1.5 / (2.0 * math.pi * s_min * s_min)))

    @property
    def tau_query(self) -> float:
        """Threshold of the density query (Eq. query with Eq. accu applied to
        the 3D value): 1e-4 of the largest possible mode-0 peak density
        rho_max / ((2 pi)^3/2 s_min^3), rounded to float32."""
        s_min = self.s_lo * self.apix
        return float(np.float32(1e-4 * 1.5 / ((2.0 * math.pi) ** 1.5 * s_min ** 3)))

    def as_config(self) -> dict:
        c = asdict(self)
        c["tau"] = self.tau
        return c


# The five workloads of the hot-path contract.  A5 is the benchmark workload.
WORKLOADS = {
    "A1": Workload("A1", d=64, M=2000, B=32, forward_only=True),
    "A2": Workload("A2", d=128, M=20000, B=256),
    "A3": Workload("A3", d=256, M=100000, B=64),
    "A4": Workload("A4", d=128, M=50000, B=512, s_lo=0.3, s_hi=12.0, n_clusters=8),
    "A5": Workload("A5", d=384, M=500000, B=16),
}


def gaussians(w: Workload, M: int | None = None, seed: int | None = None) -> np.ndarray:
    """[M][11] float32: p (3, A), s (3, A), q (4, w x y z), rho (1)."""
    M = w.M if M is None else M
    rng = np.random.default_rng(w.seed if seed is None else seed)
    box = w.d * w.apix
    nc = w.n_clusters
    # cluster centres uniform in a ball of radius 0.3 * box
    dirs = rng.normal(size=(nc, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    radii = 0.3 * box * rng.random(nc) ** (1.0 / 3.0)
    centres = dirs * radii[:, None]
    member = rng.integers(0, nc, size=M)
    p = centres[member] + rng.normal(scale=w.cluster_sigma * box, size=(M, 3))
    s = np.exp(rng.uniform(math.log(w.s_lo), math.log(w.s_hi), size=(M, 3))) * w.apix
    q = rng.normal(size=(M, 4))
    rho = rng.uniform(0.5, 1.5, size=(M, 1))
    return np.concatenate([p, s, q, rho], axis=1).astype(np.float32)


def rotations(n: int, rng: np.random.Generator) -> np.ndarray:
    """n Haar-random 3x3 rotation matrices (QR of Gaussian matrices)."""
    out = np.empty((n, 3, 3))
    for i in range(n):
        a = rng.normal(size=(3, 3))
        qm, r = np.linalg.qr(a)
        qm = qm * np.sign(np.diag(r))[None, :]
        if np.linalg.det(qm) < 0:
            qm[:, 0] = -qm[:, 0]
        out[i] = qm
    return out


def views(w: Workload, B: int | None = None, seed: int | None = None):
    """(R [B][3][3] float32 row-major, t [B][2] float32 in Angstrom)."""
    B = w.B if B is None else B
    rng = np.random.default_rng((w.seed if seed is None else seed) + 1)
    R = rotations(B, rng)
    t = rng.normal(scale=2.0 * w.apix, size=(B, 2))
    return R.astype(np.float32), t.astype(np.float32)


def ctf_params(w: Workload, B: int | None = None, seed: int | None = None) -> np.ndarray:
    """[B][8] float32: defocus U (A), defocus V (A), astigmatism angle (rad),
    voltage (kV), Cs (mm), amplitude contrast, phase shift (rad), B-factor (A^2)."""
    B = w.B if B is None else B
    rng = np.random.default_rng((w.seed if seed is None else seed) + 2)
    df = rng.uniform(1.0e4, 2.5e4, size=B)
    astig = rng.uniform(0.0, 500.0, size=B)
    ang = rng.uniform(0.0, math.pi, size=B)
    out = np.zeros((B, 8))
    out[:, 0] = df + 0.5 * astig
    out[:, 1] = df - 0.5 * astig
    out[:, 2] = ang
    out[:, 3] = 300.0
    out[:, 4] = 2.7
    out[:, 5] = 0.1
    return out.astype(np.float32)


def ctf_array(w: Workload, B: int | None = None, seed: int | None = None) -> np.ndarray:
    """[B][d][d/2+1] float32 arbitrary real transfer arrays U(-1, 1) for the
    array form of the CTF input (not a physical CTF)."""
    B = w.B if B is None else B
    rng = np.random.default_rng((w.seed if seed is None else seed) + 3)
    return rng.uniform(-1.0, 1.0, size=(B, w.d, w.d // 2 + 1)).astype(np.float32)


def images(w: Workload, B: int | None = None, seed: int | None = None) -> np.ndarray:
    """[B][d][d] float32 noise images at SNR 0.1 against the nominal signal."""
    B = w.B if B is None else B
    rng = np.random.default_rng((w.seed if seed is None else seed) + 4)
    disc = math.pi * (0.3 * w.d * w.apix) ** 2
    signal = w.M * 1.0 / disc
    sigma = signal / math.sqrt(0.1)
    return rng.normal(scale=sigma, size=(B, w.d, w.d)).astype(np.float32)


def smooth_field(w: Workload, B: int | None = None, seed: int | None = None) -> np.ndarray:
    """[B][d][d] float32 random field used where a test needs an arbitrary
    dense input (a projection or an upstream gradient): noise plus a coarse
    piecewise-constant pattern, so that it has both high and low frequencies."""
    B = w.B if B is None else B
    rng = np.random.default_rng((w.seed if seed is None else seed) + 5)
    coarse = rng.normal(size=(B, w.d // 8, w.d // 8))
    coarse = np.repeat(np.repeat(coarse, 8, axis=1), 8, axis=2)
    return (coarse + 0.25 * rng.normal(size=(B, w.d, w.d))).astype(np.float32)


def batch(w: Workload, seed: int | None = None) -> dict:
    """Every input of one step of workload ``w``."""
    R, t = views(w, seed=seed)
    return {
        "params": gaussians(w, seed=seed),
        "R": R,
        "t": t,
        "ctf_params": ctf_params(w, seed=seed),
        "images": images(w, seed=seed),
    }
