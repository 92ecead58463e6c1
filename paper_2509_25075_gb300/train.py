"""Training loop of GEM (Sec. 3.2, Fig. pipeline): fit the Gaussians to a
stack of particle images with known poses and CTFs by minimising Eq. loss,
one batch of images per step, with Adam on unconstrained parameters.

Every step runs in the library's kernels: gem_forward (projection, CTF,
loss), gem_backward (gradient), gem_adam_step (optimiser), and for the
strict isotropic ablation gem_nn_distance.  This module only holds the
device tensors, draws the batch indices (a seeded host generator, so a
resumed run draws the same batches), and saves / restores checkpoints.
"""
from __future__ import annotations

import dataclasses
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import binding

NPAR = binding.NPAR


@dataclass
class TrainConfig:
    batch: int = 64
    lr: tuple = (0.05, 0.01, 0.002, 0.02)  # centre (A), log scale, quaternion, log density
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    seed: int = 0
    iso_nn: bool = False  # isotropic ablation: s_j = nearest-neighbour distance, every step
    checkpoint_every: int = 0
    checkpoint_path: str = ""


@dataclass
class ModelConfig:
    d: int
    apix: float
    M: int
    tau: float = 0.0
    norm_mode: int = 0
    no_rotation: int = 0
    isotropic: int = 0
    zsort: int = 1


def raw_from_params(params: np.ndarray) -> np.ndarray:
    """Inverse of the activation: (p, log s, q, log rho)."""
    raw = np.array(params, dtype=np.float32, copy=True)
    raw[:, 3:6] = np.log(np.abs(raw[:, 3:6]))
    raw[:, 10] = np.log(raw[:, 10])
    return raw


class Trainer:
    """Owns a context, the parameters and optimiser state, and the dataset
    (images [N][d][d], R [N][3][3], t [N][2], ctf_params [N][8]) on the GPU."""

    def __init__(self, model: ModelConfig, cfg: TrainConfig, params0: np.ndarray, data: dict,
                 device=None):
        self.model, self.cfg = model, cfg
        self.dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        self.ctx = binding.Context(model.d, model.apix, cfg.batch, model.M, tau=model.tau,
                                   norm_mode=model.norm_mode, zsort=model.zsort,
                                   no_rotation=model.no_rotation, isotropic=model.isotropic)
        self.data = {k: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float32).to(self.dev)
                     for k, v in data.items()}
        self.N = self.data["images"].shape[0]
        if self.N < cfg.batch:
            raise ValueError("fewer images than one batch")
        self.raw = torch.as_tensor(raw_from_params(params0)).to(self.dev)
        self.m = torch.zeros_like(self.raw)
        self.v = torch.zeros_like(self.raw)
        self.params = torch.empty_like(self.raw)
        self.grad = torch.empty_like(self.raw)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
        self.nn = torch.empty(model.M, 1, device=self.dev) if cfg.iso_nn else None
        self.nn_idx = torch.empty(model.M, 1, dtype=torch.int32, device=self.dev) if cfg.iso_nn else None
        self.ctx.gem_activate(self.raw, self.params)
        self.step_count = 0
        self.rng = np.random.default_rng(cfg.seed)
        self.history: list[float] = []

    # -- one optimisation step ------------------------------------------------
    def _batch(self):
        idx = self.rng.choice(self.N, size=self.cfg.batch, replace=False)
        ix = torch.as_tensor(np.sort(idx), device=self.dev)
        return {k: v.index_select(0, ix).contiguous() for k, v in self.data.items()}

    def step(self) -> torch.Tensor:
        b = self._batch()
        self.ctx.gem_forward(self.params, b["R"], b["t"], b["images"], self.loss,
                             ctf_params=b["ctf_params"])
        self.ctx.gem_backward(self.grad)
        iso = None
        if self.nn is not None:
            self.ctx.gem_nn_distance(self.params, 1, dist=self.nn, idx=self.nn_idx)
            iso = self.nn.view(-1)
        self.step_count += 1
        self.ctx.gem_adam_step(self.raw, self.m, self.v, self.grad, self.params, self.cfg.lr,
                               self.step_count, self.cfg.beta1, self.cfg.beta2, self.cfg.eps,
                               iso_scale=iso)
        if self.cfg.checkpoint_every and self.step_count % self.cfg.checkpoint_every == 0:
            self.save(self.cfg.checkpoint_path)
        return self.loss

    def run(self, steps: int, record_every: int = 1) -> list[float]:
        for _ in range(steps):
            loss = self.step()
            if record_every and self.step_count % record_every == 0:
                self.history.append(float(loss.item()))
        status = self.ctx.gem_status()
        if status != binding.GEM_OK:
            raise binding.GemError(status, self.ctx.lib.gem_last_error(self.ctx.h).decode())
        return self.history

    # -- checkpoints ----------------------------------------------------------
    def state_dict(self) -> dict:
        return {
            "raw": self.raw.cpu(), "m": self.m.cpu(), "v": self.v.cpu(),
            "step": self.step_count, "rng": self.rng.bit_generator.state,
            "train": dataclasses.asdict(self.cfg), "model": dataclasses.asdict(self.model),
            "history": list(self.history),
        }

    def load_state_dict(self, st: dict):
        if st["model"] != dataclasses.asdict(self.model):
            raise ValueError("checkpoint was written for another model configuration")
        self.raw.copy_(st["raw"])
        self.m.copy_(st["m"])
        self.v.copy_(st["v"])
        self.step_count = int(st["step"])
        self.rng.bit_generator.state = st["rng"]
        self.history = list(st["history"])
        self.ctx.gem_activate(self.raw, self.params)

    def save(self, path: str):
        """Write atomically: a crash mid-write leaves the previous checkpoint."""
        tmp = path + ".tmp"
        torch.save(self.state_dict(), tmp)
        os.replace(tmp, path)

    def load(self, path: str):
        self.load_state_dict(torch.load(path, weights_only=True))

    def close(self):
        self.ctx.close()
