"""Autotuner for the rasterizer's launch settings: tile size, Gaussians per shared-memory
batch, radix-sort digit width and the blend kernels' pixels per thread.

The image does not depend on any of them (the support is the 3-sigma ellipse, not the
tile), so they can be chosen for speed alone.  The tuner times one forward + backward
step per candidate on the caller's own Gaussians and cameras (coordinate descent: tile
size first, then batch depth, digit width, pixels per thread and persistent or one-CTA-per-tile
blend kernels) and caches the winner per workload signature in a JSON file.
"""
from __future__ import annotations

import dataclasses
import gc
import hashlib
import json
import os
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import binding as B
from .render import GaussianModel, Rasterizer, RenderSettings

TILES: Tuple[Tuple[int, int], ...] = ((16, 16), (32, 16), (16, 32), (32, 32), (64, 16), (32, 8), (16, 8), (64, 8), (8, 8))
BATCHES: Tuple[int, ...] = (128, 256, 512, 1024)
DIGITS: Tuple[int, ...] = (8, 9, 10)
FWD_PIXELS: Tuple[int, ...] = (1, 2)
BWD_PIXELS: Tuple[int, ...] = (2, 4)
PERSISTENT: Tuple[int, ...] = (0, 1)


def signature(model: GaussianModel, cams) -> str:
    """Workload key: Gaussian count and colour layout, camera resolutions, GPU name."""
    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    desc = [model.n, model.sh_degree, model.num_lobes, model.axis_mode, dev] + \
        [(c.width, c.height) for c in cams]
    return hashlib.sha1(json.dumps(desc).encode()).hexdigest()[:16]


def time_step(model: GaussianModel, cams, settings: RenderSettings, steps: int = 3,
              grad: Optional[torch.Tensor] = None) -> float:
    """Milliseconds of one forward + backward step (after one sizing step and one warm-up)."""
    rast = Rasterizer(model, cams, settings)
    rast.forward(model, sync=True)
    rast = Rasterizer(model, cams, settings, capacity=int(rast.num_instances * 1.02) + 4096)
    img = torch.empty(3 * rast.num_pixels, device="cuda")
    if grad is None or grad.numel() != img.numel():
        grad = torch.full_like(img, 1.0 / img.numel())
    grads = model.empty_grads()

    def step():
        rast.forward(model, out_rgb=img, sync=False)
        rast.backward(model, grad, grads=grads)

    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    return ms


def _measure(model, cams, settings, steps) -> float:
    """time_step, then release the trial's workspace at once (workspaces are tens of GB; a
    reference cycle anywhere would otherwise keep several alive until the next collection)."""
    try:
        return time_step(model, cams, settings, steps)
    finally:
        gc.collect()
        torch.cuda.empty_cache()


def autotune(model: GaussianModel, cams, base: RenderSettings = RenderSettings(),
             cache_path: Optional[str] = None, steps: int = 3,
             tiles: Sequence[Tuple[int, int]] = TILES, batches: Sequence[int] = BATCHES,
             digits: Sequence[int] = DIGITS, fwd_pixels: Sequence[int] = FWD_PIXELS,
             bwd_pixels: Sequence[int] = BWD_PIXELS, persistent: Sequence[int] = PERSISTENT,
             log: Optional[List[Dict]] = None) -> RenderSettings:
    """Best settings for this workload (from the cache when present)."""
    key = signature(model, cams)
    cache: Dict[str, Dict] = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if key in cache:
            return RenderSettings(**{**dataclasses.asdict(base), **cache[key]["settings"],
                                     "bg": base.bg})
    best = base
    best_ms = _measure(model, cams, best, steps)
    trials = [dict(settings=dataclasses.asdict(best), ms=best_ms)]
    for field, values in (("tile", tiles), ("batch_depth", batches), ("digit_bits", digits),
                          ("fwd_pixels", fwd_pixels), ("bwd_pixels", bwd_pixels), ("persistent", persistent)):
        for v in values:
            if field == "tile":
                cand = dataclasses.replace(best, tile_w=v[0], tile_h=v[1])
            else:
                cand = dataclasses.replace(best, **{field: v})
            if cand == best:
                continue
            try:
                ms = _measure(model, cams, cand, steps)
            except B.SgsError:  # a combination the library rejects (e.g. 4 rows of 8-high tiles)
                continue
            trials.append(dict(settings=dataclasses.asdict(cand), ms=ms))
            if ms < best_ms:
                best, best_ms = cand, ms
    if log is not None:
        log.extend(trials)
    if cache_path:
        cache[key] = dict(settings={k: v for k, v in dataclasses.asdict(best).items() if k != "bg"},
                          ms=best_ms, trials=len(trials))
        d = os.path.dirname(os.path.abspath(cache_path))
        os.makedirs(d, exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best
