"""Training loop of Sec. 4.4 on the library's kernels.

One iteration renders a view (gs3_render), evaluates L = 0.8 L1 + 0.2 D-SSIM
and its image gradient (gs3_loss_l1_dssim), runs the hand-written backward
(gs3_render_backward) and applies one fused Adam step per parameter group
(gs3_adam_step).  This module only sequences those calls and holds the
optimiser state tensors.

Schedule (Sec. 4.4): a first stage with the Lambertian term only (the lobes
switched off with GS3_ABLATE_SPECULAR), then the full appearance; Adam with
momentum 0.9; learning rate 0.01 for the albedos, and 0.01 for the angular
Gaussians until `decay_start`, decaying exponentially to 1e-4 at `decay_end`
and fixed afterwards.  The paper gives the other groups' rates only by
reference to the base splatting method; the defaults below are of that
order.  Iteration counts default to the paper's (15K first stage, decay
40K -> 90K) and are parameters, so short synthetic runs can scale them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import torch

from . import _native as N
from .render import Renderer, opts_struct

LOBES = ("lobe_rot", "lobe_sigma", "lobe_amp")


def default_rates() -> dict:
    return {"mean_op": 1.6e-4, "scale": 5e-4, "rot": 1e-3, "shade_rot": 1e-3, "albedo_d": 1e-2,
            "albedo_s": 1e-2, "latent": 1e-3, "lobe_rot": 1e-2, "lobe_sigma": 1e-2, "lobe_amp": 1e-2,
            "phi_w": 1e-3, "phi_b": 1e-3, "psi_w": 1e-3, "psi_b": 1e-3}


# parameters that must stay positive
LOWER_BOUND = {"scale": 1e-4, "lobe_sigma": 1e-3}


@dataclass
class Schedule:
    stage1: int = 15_000
    decay_start: int = 40_000
    decay_end: int = 90_000
    lobe_final: float = 1e-4
    rates: dict = field(default_factory=default_rates)

    def lr(self, name: str, it: int) -> float:
        base = self.rates[name]
        if name not in LOBES or it < self.decay_start:
            return base
        if it >= self.decay_end:
            return self.lobe_final
        f = (it - self.decay_start) / (self.decay_end - self.decay_start)
        return base * math.exp(f * math.log(self.lobe_final / base))

    def ablate(self, it: int) -> int:
        return N.GS3_ABLATE_SPECULAR if it < self.stage1 else 0


class Trainer:
    """Optimises the tensors of a DeviceScene (FP32 MLPs) in place."""

    def __init__(self, dscene, width: int, height: int, key_capacity: int, schedule: Schedule | None = None,
                 lam: float = 0.2, betas=(0.9, 0.999), eps: float = 1e-15, device="cuda"):
        self.scene = dscene
        self.rd = Renderer(dscene, width, height, key_capacity, device=device)
        self.schedule = schedule or Schedule()
        self.lam, self.betas, self.eps = lam, betas, eps
        self.m = {f: torch.zeros_like(dscene.t[f]) for f in N.GRAD_FIELDS}
        self.v = {f: torch.zeros_like(dscene.t[f]) for f in N.GRAD_FIELDS}
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.dimg = torch.empty((height, width, 3), dtype=torch.float32, device=device)
        self.scratch = torch.empty(N.gs3_loss_scratch_size(width, height), dtype=torch.uint8, device=device)
        self.width, self.height = width, height
        self.it = 0

    def step(self, cam, light, target: torch.Tensor) -> torch.Tensor:
        """One iteration on one view; returns the loss (device scalar) of the
        parameters before the update."""
        s = torch.cuda.current_stream()
        opts = opts_struct(ablate=self.schedule.ablate(self.it))
        img = self.rd.render(cam, light, opts)
        N.gs3_loss_l1_dssim(img, target, self.lam, self.loss, self.dimg, self.scratch, s.cuda_stream)
        grads = self.rd.backward(cam, light, self.dimg, opts)
        t = self.it + 1
        for f in N.GRAD_FIELDS:
            N.gs3_adam_step(self.scene.t[f], grads[f], self.m[f], self.v[f], self.schedule.lr(f, self.it),
                            self.betas[0], self.betas[1], self.eps, t, LOWER_BOUND.get(f, -math.inf),
                            s.cuda_stream)
        self.it += 1
        return self.loss.clone()
