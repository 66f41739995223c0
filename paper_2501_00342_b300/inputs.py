"""Seeded synthetic scenes and cameras.

This module only draws inputs: Gaussian parameter planes and pinhole cameras
shaped like the scenes the SG-Splatting paper renders (1-8 M Gaussians,
720p-4K views; Sec. "Experiment Settings").  It holds none of the rendering
arithmetic, so both the CUDA path and the CPU oracle consume exactly the same
float32 arrays.

Layout (structure of arrays, each plane padded to ``stride`` floats, ``stride``
a multiple of 32 so every plane starts 128-byte aligned):

* ``mean``     [3][stride]            world position X (Eq. 2)
* ``scale``    [3][stride]            activated scale s > 0 (Eq. 3)
* ``rot``      [4][stride]            quaternion q = (w, x, y, z), any norm (Eq. 3)
* ``opacity``  [stride]               activated opacity in (0, 1)
* ``sh``       [(L+1)^2][3][stride]   SH coefficients c_lm per RGB channel (Eq. 4)
* ``sg_amp``   [K][3][stride]         SG amplitudes alpha_k per channel (Eq. 5, 7)
* ``sg_axis``  [K][3][stride]         SG axes mu_k, any norm (free-axis mode only)
* ``sg_sharp`` [K][stride]            SG sharpness lambda_k (Eq. 5)

Random streams: ``numpy.random.Generator(PCG64(1000 * config + stream))``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

AXIS_FREE = 0
AXIS_ORTHO_FIXED = 1
AXIS_ORTHO_FRAME = 2  # lobe axes = columns of the rotation of 3 per-Gaussian parameters

CAM_FLOATS = 22  # viewmat[12], campos[3], fx, fy, cx, cy, width, height, near


def _rng(config: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * config + stream))


def padded_stride(n: int) -> int:
    return max(32, (n + 31) // 32 * 32)


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV axes (+x right, +y down, +z forward).

    ``viewmat`` is the 3x4 world-to-camera matrix [R | t] in row-major order.
    """
    viewmat: np.ndarray  # (12,) float32
    campos: np.ndarray   # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2

    def as_array(self) -> np.ndarray:
        a = np.zeros(CAM_FLOATS, np.float32)
        a[0:12] = self.viewmat
        a[12:15] = self.campos
        a[15:19] = (self.fx, self.fy, self.cx, self.cy)
        a[19:21] = (self.width, self.height)
        a[21] = self.near
        return a


def look_at(eye, target, width: int, height: int, fov_x_deg: float,
            up=(0.0, 1.0, 0.0), near: float = 0.2) -> Camera:
    """Camera at ``eye`` looking at ``target``; horizontal field of view, square pixels,
    principal point at the image centre."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    rot = np.stack([r, d, f])
    t = -rot @ eye
    vm = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32).reshape(12)
    fx = (0.5 * width) / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(vm, eye.astype(np.float32), float(np.float32(fx)), float(np.float32(fx)),
                  0.5 * width, 0.5 * height, int(width), int(height), near)


def orbit_cameras(num: int, width, height, fov_x_deg: float = 50.0, radius: float = 6.0,
                  elevation_deg: float = 20.0) -> List[Camera]:
    """``num`` cameras on a circle of ``radius`` at ``elevation_deg``, even azimuths,
    all looking at the origin.  ``width``/``height`` may be per-camera sequences."""
    cams = []
    el = math.radians(elevation_deg)
    for k in range(num):
        az = 2.0 * math.pi * k / num
        eye = (radius * math.cos(el) * math.sin(az), radius * math.sin(el),
               radius * math.cos(el) * math.cos(az))
        w = width[k] if hasattr(width, "__len__") else width
        h = height[k] if hasattr(height, "__len__") else height
        cams.append(look_at(eye, (0.0, 0.0, 0.0), int(w), int(h), fov_x_deg))
    return cams


def cameras_array(cams: List[Camera]) -> np.ndarray:
    return np.stack([c.as_array() for c in cams]).astype(np.float32)


@dataclasses.dataclass
class Scene:
    n: int
    stride: int
    sh_degree: int
    num_lobes: int
    axis_mode: int
    mean: np.ndarray
    scale: np.ndarray
    rot: np.ndarray
    opacity: np.ndarray
    sh: np.ndarray
    sg_amp: np.ndarray
    sg_axis: Optional[np.ndarray]
    sg_sharp: np.ndarray
    # adaptive SH degree: 0 off; 1: bands up to 0 / 1 / 2 as a record's pixel radius is
    # below sh_radius[0] / below sh_radius[1] / not
    sh_adaptive: int = 0
    sh_radius: Tuple[float, float] = (0.0, 0.0)

    PLANES = ("mean", "scale", "rot", "opacity", "sh", "sg_amp", "sg_axis", "sg_sharp")

    @property
    def num_sh(self) -> int:
        return (self.sh_degree + 1) ** 2

    def floats_per_gaussian(self) -> int:
        """Parameter floats read per Gaussian: geometry 11, SH 3(L+1)^2,
        SG 7K (free axes), 4K (world axes, no axis stored) or 4K + 3 (a frame)."""
        sg = (7 if self.axis_mode == AXIS_FREE else 4) * self.num_lobes
        if self.axis_mode == AXIS_ORTHO_FRAME and self.num_lobes:
            sg += 3  # the frame's 3 parameters
        return 11 + 3 * self.num_sh + sg

    def subset(self, idx) -> "Scene":
        """A new scene holding the Gaussians ``idx`` (in that order)."""
        idx = np.asarray(idx, np.int64)
        n = len(idx)
        s = padded_stride(n)

        def take(a):
            if a is None:
                return None
            out = np.zeros(a.shape[:-1] + (s,), np.float32)
            out[..., :n] = a[..., idx]
            return out

        return Scene(n, s, self.sh_degree, self.num_lobes, self.axis_mode,
                     *(take(getattr(self, p)) for p in self.PLANES),
                     sh_adaptive=self.sh_adaptive, sh_radius=self.sh_radius)


def _unit_rows(g: np.ndarray) -> np.ndarray:
    return g / np.linalg.norm(g, axis=-1, keepdims=True)


def _colour_planes(rng, n, s, sh_degree, num_lobes, axis_mode, dc=(0.5, 0.2), rest_sd=0.1):
    nsh = (sh_degree + 1) ** 2
    sh = np.zeros((nsh, 3, s), np.float32)
    sh[0, :, :n] = rng.normal(dc[0], dc[1], (3, n))
    if nsh > 1:
        sh[1:, :, :n] = rng.normal(0.0, rest_sd, (nsh - 1, 3, n))
    amp = np.zeros((num_lobes, 3, s), np.float32)
    sharp = np.zeros((num_lobes, s), np.float32)
    axis = None
    if num_lobes:
        amp[:, :, :n] = rng.normal(0.0, 0.2, (num_lobes, 3, n))
        sharp[:, :n] = np.exp(rng.uniform(0.0, math.log(50.0), (num_lobes, n)))
        if axis_mode == AXIS_FREE:
            axis = np.zeros((num_lobes, 3, s), np.float32)
            ax = _unit_rows(rng.normal(size=(num_lobes, n, 3)))
            axis[:, :, :n] = np.transpose(ax, (0, 2, 1))
        elif axis_mode == AXIS_ORTHO_FRAME:
            # frame parameters f: uniform random unit quaternions q, f = q_xyz / q_w
            axis = np.zeros((3, s), np.float32)
            q = _unit_rows(rng.normal(size=(n, 4)))
            q *= np.sign(q[:, :1] + 1e-30)
            axis[:, :n] = (q[:, 1:] / np.maximum(q[:, :1], 0.05)).T
    return sh, amp, axis, sharp


def _geometry_planes(rng, n, s, means_xyz, log_scale=(-3.5, 0.5), opacity_sd=1.5):
    mean = np.zeros((3, s), np.float32)
    mean[:, :n] = means_xyz.T
    scale = np.zeros((3, s), np.float32)
    scale[:, :n] = np.exp(rng.normal(log_scale[0], log_scale[1], (3, n)))
    rot = np.zeros((4, s), np.float32)
    rot[:, :n] = _unit_rows(rng.normal(size=(n, 4))).T
    opa = np.zeros((s,), np.float32)
    opa[:n] = 1.0 / (1.0 + np.exp(-rng.normal(0.0, opacity_sd, n)))
    return mean, scale, rot, opa


def uniform_cube_scene(n: int = 2000, sh_degree: int = 0, num_lobes: int = 3,
                       axis_mode: int = AXIS_FREE, config: int = 0, stream: int = 0,
                       log_scale=(-3.5, 0.5)) -> Scene:
    """Means uniform in [-1,1]^3; log-scales N(-3.5, 0.5); uniform unit quaternions;
    opacity sigmoid(N(0,1.5)); SH DC ~ N(0.5, 0.2); K lobes with axes uniform on
    S^2, sharpness log-uniform [1, 50], RGB amplitudes N(0, 0.2)."""
    rng = _rng(config, stream)
    s = padded_stride(n)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    geo = _geometry_planes(rng, n, s, means, log_scale)
    col = _colour_planes(rng, n, s, sh_degree, num_lobes, axis_mode)
    return Scene(n, s, sh_degree, num_lobes, axis_mode, *geo, *col)


def cluster_scene(n: int, sh_degree: int = 1, num_lobes: int = 3, axis_mode: int = AXIS_FREE,
                  config: int = 1, stream: int = 0, num_clusters: int = 64,
                  shell_fraction: float = 0.1, shell_radius: float = 20.0) -> Scene:
    """Means from ``num_clusters`` anisotropic Gaussian clusters (centres U[-2,2]^3,
    per-axis sigma log-uniform [0.05, 0.5], random orientation) plus ``shell_fraction``
    of the points uniform on a far sphere of ``shell_radius``.  Other parameters as in
    :func:`uniform_cube_scene`."""
    rng = _rng(config, stream)
    s = padded_stride(n)
    centres = rng.uniform(-2.0, 2.0, (num_clusters, 3))
    sig = np.exp(rng.uniform(math.log(0.05), math.log(0.5), (num_clusters, 3)))
    # cluster orientations: Q factor of a Gaussian matrix (a random orthogonal matrix)
    rots = np.linalg.qr(rng.normal(size=(num_clusters, 3, 3)))[0]
    n_shell = int(round(shell_fraction * n))
    n_cl = n - n_shell
    which = rng.integers(0, num_clusters, n_cl)
    local = rng.normal(size=(n_cl, 3)) * sig[which]
    pts = centres[which] + np.einsum("nij,nj->ni", rots[which], local)
    shell = _unit_rows(rng.normal(size=(n_shell, 3))) * shell_radius
    means = np.concatenate([pts, shell], 0)
    means = means[rng.permutation(n)]
    geo = _geometry_planes(rng, n, s, means)
    col = _colour_planes(rng, n, s, sh_degree, num_lobes, axis_mode)
    return Scene(n, s, sh_degree, num_lobes, axis_mode, *geo, *col)


# ----------------------------------------------------------------------------------------
# The five workloads (sizes and distributions of the paper-shaped synthetic scenes).
# ----------------------------------------------------------------------------------------

MIXED_RESOLUTIONS = ((640, 360), (1280, 720), (1600, 900), (1920, 1080))


def workload(config: int, n: Optional[int] = None, sh_degree: Optional[int] = None,
             num_lobes: Optional[int] = None, axis_mode: int = AXIS_FREE):
    """Returns (scene, cameras) for one of the five workloads:

    0. 2,000 Gaussians in [-1,1]^3, SH-0 + 3 SG lobes, one 128x128 camera (fov 60) at
       distance 4 looking at the origin.
    1. 1 M Gaussians in 64 clusters + far shell, SH-1 + 3 SG lobes, 32 orbit cameras at
       1280x720 (fov 50).  (``sh_degree=3, num_lobes=0`` gives the 48-coefficient variant.)
    2. 2.5 M clustered Gaussians, SH-1 + 4 SG lobes, one 1264x832 view.
    3. 3 M clustered Gaussians, SH-1 + 4 SG lobes, 16 orbit views whose resolutions are
       drawn from {640x360, 1280x720, 1600x900, 1920x1080}.
    4. 8 M clustered Gaussians, SH-1 + 4 SG lobes, 8 orbit views at 3840x2160.
    """
    if config == 0:
        sc = uniform_cube_scene(n or 2000, 0 if sh_degree is None else sh_degree,
                                3 if num_lobes is None else num_lobes, axis_mode, config=0)
        cams = [look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 128, 128, 60.0)]
        return sc, cams
    defaults = {1: (1_000_000, 1, 3), 2: (2_500_000, 1, 4), 3: (3_000_000, 1, 4),
                4: (8_000_000, 1, 4)}
    dn, dl, dk = defaults[config]
    sc = cluster_scene(n or dn, dl if sh_degree is None else sh_degree,
                       dk if num_lobes is None else num_lobes, axis_mode, config=config)
    if config == 1:
        cams = orbit_cameras(32, 1280, 720, 50.0)
    elif config == 2:
        cams = orbit_cameras(1, 1264, 832, 50.0)
    elif config == 3:
        rng = _rng(3, 7)
        pick = rng.integers(0, len(MIXED_RESOLUTIONS), 16)
        ws = [MIXED_RESOLUTIONS[p][0] for p in pick]
        hs = [MIXED_RESOLUTIONS[p][1] for p in pick]
        cams = orbit_cameras(16, ws, hs, 50.0)
    else:
        cams = orbit_cameras(8, 3840, 2160, 50.0)
    return sc, cams


def target_images(cams: List[Camera], config: int = 2, stream: int = 11) -> List[np.ndarray]:
    """Seeded U(0,1) target images, planar [3][H][W] float32, one per camera."""
    rng = _rng(config, stream)
    return [rng.uniform(0.0, 1.0, (3, c.height, c.width)).astype(np.float32) for c in cams]


def sample_pixels(cams: List[Camera], patches_per_view: int = 64, patch: int = 16,
                  config: int = 9, stream: int = 0) -> np.ndarray:
    """Seeded pixel sample: ``patches_per_view`` square patches of side ``patch`` per view.
    Returns int32 [P][3] rows of (view, x, y)."""
    rng = _rng(config, stream)
    rows = []
    for v, c in enumerate(cams):
        for _ in range(patches_per_view):
            x0 = int(rng.integers(0, max(1, c.width - patch + 1)))
            y0 = int(rng.integers(0, max(1, c.height - patch + 1)))
            ys, xs = np.mgrid[y0:min(y0 + patch, c.height), x0:min(x0 + patch, c.width)]
            rows.append(np.stack([np.full(xs.size, v), xs.ravel(), ys.ravel()], 1))
    return np.concatenate(rows, 0).astype(np.int32)
