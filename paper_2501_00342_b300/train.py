"""Training loop of the rasterizer: render -> L1 loss -> backward -> fused Adam step, all in
the library's kernels (four calls per step after the forward's three), on one GPU or
view-sharded over several (ShardedTrainer: one all-reduce of the gradients per step).

The optimiser owns raw planes (log-scale, logit-opacity, the rest as is) and the activated
planes the renderer reads; identity planes are shared.  Learning rates follow the 3D-GS
conventions the paper keeps (Sec. "Implementation"): position 1.6e-4 x scene extent decaying
exponentially to 1.6e-6 x extent over the run, scale 5e-3, rotation 1e-3, opacity 5e-2, SH
band 0 2.5e-3 and higher bands 2.5e-3 / 20; the SG lobes join after `sg_start` iterations
(2,000 in the paper) with learning rate 2.5e-3 and their own Adam step count.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import binding as B
from .render import PLANES, GaussianModel, Rasterizer, RenderSettings, l1_loss


@dataclasses.dataclass
class TrainConfig:
    iterations: int = 30_000
    sg_start: int = 2_000
    extent: float = 1.0          # scene extent scaling the position learning rate
    lr_mean: float = 1.6e-4
    lr_mean_final: float = 1.6e-6
    lr_scale: float = 5e-3
    lr_rot: float = 1e-3
    lr_opacity: float = 5e-2
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 2.5e-3 / 20.0
    lr_sg: float = 2.5e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15


def _grads_struct(planes: Dict[str, Optional[torch.Tensor]]) -> B.Grads:
    return B.Grads(*[B.ptr(planes[p]) for p in PLANES])


class Trainer:
    """Fits a GaussianModel to target images of fixed cameras.  `model` holds the activated
    starting parameters (scale > 0, opacity in (0, 1)); its planes are updated in place."""

    def __init__(self, model: GaussianModel, cams: Sequence, targets: torch.Tensor,
                 settings: RenderSettings = RenderSettings(), config: TrainConfig = TrainConfig()):
        self.model, self.cams, self.config = model, list(cams), config
        self.target = targets.contiguous()
        self.act = model.planes
        self.raw = dict(self.act)
        self.raw["scale"] = torch.log(self.act["scale"])
        o = self.act["opacity"].clamp(1e-6, 1.0 - 1e-6)
        self.raw["opacity"] = torch.log(o / (1.0 - o))
        zero = {p: (None if t is None else torch.zeros_like(t)) for p, t in self.act.items()}
        self.m = zero
        self.v = {p: (None if t is None else torch.zeros_like(t)) for p, t in self.act.items()}
        self.grads = model.empty_grads()
        self.rast = Rasterizer(model, self.cams, settings)
        self.img = torch.empty(3 * self.rast.num_pixels, device=self.target.device)
        self.iteration = 0
        self._structs = [_grads_struct(d) for d in (self.raw, self.act, self.grads, self.m, self.v)]

    def learning_rates(self, it: int):
        c = self.config
        frac = min(1.0, it / max(1, c.iterations))
        lr_mean = math.exp((1 - frac) * math.log(c.lr_mean) + frac * math.log(c.lr_mean_final)) * c.extent
        lrs = [lr_mean, c.lr_scale, c.lr_rot, c.lr_opacity, c.lr_sh_dc, c.lr_sh_rest,
               c.lr_sg if it >= c.sg_start else 0.0]
        steps = [it + 1] * 6 + [max(1, it - c.sg_start + 1)]
        return lrs, steps

    def adam_config(self, it: int) -> B.AdamConfig:
        lrs, steps = self.learning_rates(it)
        cfg = B.AdamConfig()
        for k in range(len(B.GROUPS)):
            cfg.lr[k], cfg.step[k] = lrs[k], steps[k]
        cfg.beta1, cfg.beta2, cfg.eps = self.config.beta1, self.config.beta2, self.config.eps
        return cfg

    def step(self, sync: bool = False) -> torch.Tensor:
        """One iteration; returns the loss (a device scalar)."""
        stream = torch.cuda.current_stream().cuda_stream
        self.rast.forward(self.model, out_rgb=self.img, sync=sync)
        loss, dimg = l1_loss(self.img, self.target)
        self.rast.backward(self.model, dimg, grads=self.grads)
        B.adam_step(self.model.struct(), *self._structs, self.adam_config(self.iteration), stream)
        self.iteration += 1
        return loss


def numpy_planes(model: GaussianModel) -> Dict[str, Optional[np.ndarray]]:
    return {p: (None if t is None else t.detach().cpu().numpy().astype(np.float64)) for p, t in model.planes.items()}


# ------------------------------------------------------------------ view-sharded training
def shard_views(num_views: int, world: int, rank: int) -> range:
    """The views of rank ``rank`` when ``num_views`` views are split over ``world`` ranks:
    a contiguous block, the first ``num_views % world`` ranks one view more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    base, extra = divmod(num_views, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


class GradientBucket:
    """Every gradient plane of a model as a view into one flat buffer, so that the
    exchange of a view-sharded step is a single all-reduce.  ``planes`` has the layout of
    ``GaussianModel.empty_grads`` (padding entries zero)."""

    def __init__(self, model: GaussianModel, dtype=torch.float32, device=None):
        device = device if device is not None else model.planes["mean"].device
        shapes = {p: (None if t is None else tuple(t.shape)) for p, t in model.planes.items()}
        total = sum(int(np.prod(sh)) for sh in shapes.values() if sh is not None)
        # planes start on 16-byte boundaries: every plane's length is a multiple of the
        # stride, itself a multiple of 4 floats
        self.flat = torch.zeros(total, dtype=dtype, device=device)
        self.planes: Dict[str, Optional[torch.Tensor]] = {}
        off = 0
        for p in PLANES:
            sh = shapes[p]
            if sh is None:
                self.planes[p] = None
                continue
            k = int(np.prod(sh))
            self.planes[p] = self.flat[off:off + k].view(sh)
            off += k

    def allreduce(self, group=None) -> None:
        """Sums the buffer over the ranks of ``group`` in place (every rank gets the sum)."""
        import torch.distributed as dist
        dist.all_reduce(self.flat, op=dist.ReduceOp.SUM, group=group)


class ShardedTrainer(Trainer):
    """Data-parallel training over views: each rank renders only its own cameras (its
    shard of the batch) against a full replica of the Gaussians, the loss of every rank is
    normalised by the pixel values of all ranks' views, the gradient planes (one flat
    bucket) are summed over the ranks by one all-reduce, and every rank then runs the same
    Adam step on its replica -- so the replicas stay identical and the step equals one-GPU
    training on all the views at once (up to the order of the float additions).  The paper
    trains on one GPU (Sec. "Experiment Settings"); this is the split its per-view
    independence allows.  ``cams``/``targets`` are this rank's shard; ``total_values`` the
    3 x pixels of every rank's views together."""

    def __init__(self, model: GaussianModel, cams: Sequence, targets: torch.Tensor, total_values: int,
                 settings: RenderSettings = RenderSettings(), config: TrainConfig = TrainConfig(), group=None):
        super().__init__(model, cams, targets, settings, config)
        self.group, self.total_values = group, int(total_values)
        self.bucket = GradientBucket(model)
        self.grads = self.bucket.planes
        self._structs = [_grads_struct(d) for d in (self.raw, self.act, self.grads, self.m, self.v)]

    def step(self, sync: bool = False) -> torch.Tensor:
        """One iteration; returns this rank's share of the loss (the all-reduced sum of the
        shares is the mean absolute error over every view)."""
        stream = torch.cuda.current_stream().cuda_stream
        self.rast.forward(self.model, out_rgb=self.img, sync=sync)
        loss, dimg = l1_loss(self.img, self.target, norm=self.total_values)
        self.rast.backward(self.model, dimg, grads=self.grads)
        self.bucket.allreduce(self.group)
        B.adam_step(self.model.struct(), *self._structs, self.adam_config(self.iteration), stream)
        self.iteration += 1
        return loss
