"""PyTorch-facing renderer: device parameter planes, a Rasterizer that owns one workspace,
and the autograd Function.  PyTorch provides device memory and streams only; every stage
runs in the CUDA kernels behind the C ABI (binding.py)."""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
from typing import Dict, List, Optional

import torch

from . import binding as B

PLANES = ("mean", "scale", "rot", "opacity", "sh", "sg_amp", "sg_axis", "sg_sharp")


@dataclasses.dataclass
class RenderSettings:
    tile_w: int = 16
    tile_h: int = 16
    batch_depth: int = 256
    digit_bits: int = 9
    bg: tuple = (0.0, 0.0, 0.0)
    fwd_pixels: int = 0  # pixels per thread of the blend kernels (0: the library's choice)
    bwd_pixels: int = 0
    persistent: int = 0  # 1: persistent two-pixel blend kernels (tiles claimed from a counter)

    def struct(self) -> B.Settings:
        s = B.Settings()
        s.tile_w, s.tile_h = self.tile_w, self.tile_h
        s.batch_depth, s.digit_bits, s.memory_mode = self.batch_depth, self.digit_bits, 0
        s.fwd_pixels, s.bwd_pixels = self.fwd_pixels, self.bwd_pixels
        s.persistent = self.persistent
        for k in range(3):
            s.bg[k] = float(self.bg[k])
        return s


class GaussianModel:
    """Gaussian parameter planes on the device, in the layout of ``sgs_gaussians``."""

    def __init__(self, n, sh_degree, num_lobes, axis_mode, sh_adaptive=0, sh_radius=(0.0, 0.0), **planes):
        self.n, self.sh_degree, self.num_lobes, self.axis_mode = n, sh_degree, num_lobes, axis_mode
        # adaptive SH degree: bands up to 0 / 1 / 2 for records of pixel radius below
        # sh_radius[0] / below sh_radius[1] / above (see sgs_gaussians)
        self.sh_adaptive, self.sh_radius = int(sh_adaptive), (float(sh_radius[0]), float(sh_radius[1]))
        self.planes: Dict[str, Optional[torch.Tensor]] = {p: planes.get(p) for p in PLANES}
        self.stride = self.planes["mean"].shape[-1]
        for p, t in self.planes.items():
            if t is not None:
                assert t.dtype == torch.float32 and t.is_contiguous() and t.shape[-1] == self.stride, p

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        planes = {p: (None if getattr(scene, p) is None else
                      torch.from_numpy(getattr(scene, p)).to(device).contiguous()) for p in PLANES}
        return cls(scene.n, scene.sh_degree, scene.num_lobes, scene.axis_mode,
                   getattr(scene, "sh_adaptive", 0), getattr(scene, "sh_radius", (0.0, 0.0)), **planes)

    def with_planes(self, **planes) -> "GaussianModel":
        d = dict(self.planes)
        d.update(planes)
        return GaussianModel(self.n, self.sh_degree, self.num_lobes, self.axis_mode, self.sh_adaptive,
                             self.sh_radius, **d)

    def struct(self) -> B.Gaussians:
        g = B.Gaussians()
        g.n, g.stride = self.n, self.stride
        g.sh_degree, g.num_lobes, g.axis_mode = self.sh_degree, self.num_lobes, self.axis_mode
        for p in PLANES:
            setattr(g, p, B.ptr(self.planes[p]))
        g.sh_adaptive = self.sh_adaptive
        g.sh_radius[0], g.sh_radius[1] = self.sh_radius
        return g

    def empty_grads(self) -> Dict[str, Optional[torch.Tensor]]:
        """Gradient planes; the kernels write entries [0, n), the padding is zeroed here."""
        out = {}
        for p, t in self.planes.items():
            if t is None:
                out[p] = None
                continue
            g = torch.empty_like(t)
            if self.stride > self.n:
                g[..., self.n:] = 0.0
            out[p] = g
        return out


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class Rasterizer:
    """One workspace for B cameras and one Gaussian layout.

    ``forward`` runs preprocess -> bin/sort -> blend; ``backward`` runs the reverse pass of
    the most recent ``forward``.  With ``sync=False`` no call synchronises the host, so the
    sequence can be captured in a CUDA graph (the instance capacity must then suffice).
    """

    def __init__(self, model: GaussianModel, cams, settings: RenderSettings = RenderSettings(),
                 capacity: Optional[int] = None, device="cuda"):
        self.cams = list(cams)
        self.settings = settings
        self.device = torch.device(device)
        self.layout = (model.n, model.stride, model.sh_degree, model.num_lobes, model.axis_mode)
        self._plan_for(model, capacity if capacity is not None else max(1024, 4 * model.n * len(self.cams)))
        self.num_instances = None

    def _plan_for(self, model, capacity):
        self.plan, self.nbytes = B.workspace_size(model.struct(), self.cams, self.settings.struct(), capacity)
        self.capacity = capacity
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        self.num_pixels = self.plan.num_pixels

    @property
    def pixel_base(self) -> List[int]:
        return [self.plan.pixel_base[v] for v in range(len(self.cams) + 1)]

    def images(self, flat: torch.Tensor) -> List[torch.Tensor]:
        """Splits a packed planar image buffer into [3, H, W] views."""
        out = []
        for v, c in enumerate(self.cams):
            b = self.plan.pixel_base[v]
            out.append(flat[3 * b:3 * b + 3 * c.height * c.width].view(3, c.height, c.width))
        return out

    def region(self, name: str, dtype=torch.uint8) -> torch.Tensor:
        off, nb = B.region_info(self.plan, name)
        return self.workspace[off:off + nb].view(dtype)

    def forward(self, model: GaussianModel, out_rgb: Optional[torch.Tensor] = None,
                out_T: Optional[torch.Tensor] = None, sync: bool = True) -> torch.Tensor:
        assert (model.n, model.stride, model.sh_degree, model.num_lobes, model.axis_mode) == self.layout
        if out_rgb is None:
            out_rgb = torch.empty(3 * self.num_pixels, dtype=torch.float32, device=self.device)
        g = model.struct()
        s = _stream()
        while True:
            B.preprocess(self.plan, g, self.workspace.data_ptr(), self.nbytes, s)
            try:
                self.num_instances = B.bin_sort(self.plan, s, sync)
                break
            except B.SgsError as e:
                if e.code != B.SGS_ERR_CAPACITY:
                    raise
                self._plan_for(model, int(math.ceil(e.instances * 1.15)) + 1024)
        B.render(self.plan, out_rgb.data_ptr(), B.ptr(out_T), s)
        return out_rgb

    def backward(self, model: GaussianModel, dL_drgb: torch.Tensor,
                 grads: Optional[Dict[str, Optional[torch.Tensor]]] = None):
        assert dL_drgb.is_contiguous() and dL_drgb.numel() == 3 * self.num_pixels
        grads = grads if grads is not None else model.empty_grads()
        gs = B.Grads(*[B.ptr(grads[p]) for p in PLANES])
        B.render_backward(self.plan, model.struct(), dL_drgb.data_ptr(), gs, _stream())
        return grads

    def device_status(self) -> int:
        return B.read_device_status(self.plan, _stream())


class _RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast: Rasterizer, model: GaussianModel, *tensors):
        planes = {p: t for p, t in zip(PLANES, tensors)}
        m = model.with_planes(**{p: (None if t is None else t.detach()) for p, t in planes.items()})
        ctx.rast, ctx.model = rast, m
        ctx.present = [t is not None for t in tensors]
        return rast.forward(m)

    @staticmethod
    def backward(ctx, grad_rgb):
        grads = ctx.rast.backward(ctx.model, grad_rgb.contiguous())
        return (None, None) + tuple(grads[p] if present else None
                                    for p, present in zip(PLANES, ctx.present))


def render(rast: Rasterizer, model: GaussianModel) -> torch.Tensor:
    """Differentiable render of all of ``rast``'s views; returns the packed planar image.
    Gradients flow to every parameter plane of ``model`` that requires grad."""
    return _RenderFunction.apply(rast, model, *[model.planes[p] for p in PLANES])


def l1_loss(img: torch.Tensor, target: torch.Tensor, norm: Optional[int] = None):
    """Mean absolute error and its gradient, computed by the library's kernel.  With
    ``norm`` the sum is divided by ``norm`` instead of the element count (view-sharded
    training: the element count of every rank's views)."""
    loss = torch.empty(1, dtype=torch.float32, device=img.device)
    grad = torch.empty_like(img)
    if norm is None:
        B.l1_loss(img.data_ptr(), target.data_ptr(), img.numel(), loss.data_ptr(), grad.data_ptr(), _stream())
    else:
        B.l1_loss_scaled(img.data_ptr(), target.data_ptr(), img.numel(), 1.0 / norm, loss.data_ptr(),
                         grad.data_ptr(), _stream())
    return loss, grad
