"""CPU oracle of the SG-Splatting rasterizer -- TEST INFRASTRUCTURE.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline / reference leg may
import this package.  The product path (paper_2501_00342_b300) never imports it, and it
never imports the product path: the two share only the seeded input generator
``paper_2501_00342_b300.inputs``, which holds no rendering arithmetic.

* FP32 binning mirror: cull, depth bits, screen mean, conic, radius, tile rectangle,
  tile|depth keys, stable sort, per-tile ranges, support membership -- the integer
  decisions, in single precision with a written-out operation order.
* FP64 forward: brute force per pixel over all Gaussians, no tiles (Eq. 2-9 and the EWA
  projection cited in Sec. "Preliminaries").
* FP64 adjoint: hand-written reverse mode of the forward.

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("stride", C.c_int64), ("sh_degree", C.c_int32),
                ("num_lobes", C.c_int32), ("axis_mode", C.c_int32)] + \
               [(f, C.c_void_p) for f in ("mean", "scale", "rot", "opacity", "sh", "sg_amp",
                                          "sg_axis", "sg_sharp")] + \
               [("sh_adaptive", C.c_int32), ("sh_radius", C.c_float * 2)]


class _Grads(C.Structure):
    _fields_ = [(f, C.c_void_p) for f in ("mean", "scale", "rot", "opacity", "sh", "sg_amp",
                                          "sg_axis", "sg_sharp")]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.orc_mirror_preprocess.argtypes = [vp, vp, i32, i32, i32] + [vp] * 7
        L.orc_num_tiles.argtypes = [vp, i32, i32, i32]
        L.orc_num_tiles.restype = i64
        L.orc_mirror_count.argtypes = [vp, vp, i32, i32, i32]
        L.orc_mirror_count.restype = i64
        L.orc_mirror_bin.argtypes = [vp, vp, i32, i32, i32] + [vp] * 5
        L.orc_stable_sort_pairs.argtypes = [i64, vp, vp]
        L.orc_preprocess64.argtypes = [vp, vp, i32] + [vp] * 5
        L.orc_render_pixels.argtypes = [vp, vp, i32, vp, vp, i64] + [vp] * 5 + [i32]
        L.orc_adjoint_pixels.argtypes = [vp, vp, i32, vp, vp, i64, vp, vp, i32]
        L.orc_sh_basis.argtypes = [i32, i32, vp]
        L.orc_sh_basis.restype = C.c_double
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, np.float32)


def _scene_struct(sc):
    keep = [_f32(getattr(sc, f)) for f in ("mean", "scale", "rot", "opacity", "sh", "sg_amp",
                                           "sg_axis", "sg_sharp")]
    st = _Scene(sc.n, sc.stride, sc.sh_degree, sc.num_lobes, sc.axis_mode, *[_ptr(a) for a in keep])
    st.sh_adaptive = int(getattr(sc, "sh_adaptive", 0))
    r = getattr(sc, "sh_radius", (0.0, 0.0))
    st.sh_radius[0], st.sh_radius[1] = float(r[0]), float(r[1])
    return st, keep


def _cams(cams):
    from paper_2501_00342_b300.inputs import cameras_array
    a = cams if isinstance(cams, np.ndarray) else cameras_array(cams)
    return np.ascontiguousarray(a, np.float32).reshape(-1, 22)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ------------------------------------------------------------------ FP32 mirror
def mirror_preprocess(sc, cams, tile_w=16, tile_h=16):
    st, keep = _scene_struct(sc)
    ca = _cams(cams)
    R = ca.shape[0] * sc.n
    out = dict(visible=np.zeros(R, np.uint8), depth_bits=np.zeros(R, np.uint32),
               mean2d=np.zeros((R, 2), np.float32), conic=np.zeros((R, 3), np.float32),
               radius=np.zeros(R, np.float32), rect=np.zeros((R, 4), np.int32),
               tiles_touched=np.zeros(R, np.uint32))
    lib().orc_mirror_preprocess(C.byref(st), _ptr(ca), ca.shape[0], tile_w, tile_h,
                                *[_ptr(out[k]) for k in ("visible", "depth_bits", "mean2d", "conic",
                                                         "radius", "rect", "tiles_touched")])
    out["visible"] = out["visible"].astype(bool)
    return out


def num_tiles(cams, tile_w=16, tile_h=16) -> int:
    ca = _cams(cams)
    return int(lib().orc_num_tiles(_ptr(ca), ca.shape[0], tile_w, tile_h))


def mirror_bin(sc, cams, tile_w=16, tile_h=16):
    """Instances (record order, tiles row-major), their stable sort by key, and the
    per-tile [start, end) table."""
    st, keep = _scene_struct(sc)
    ca = _cams(cams)
    m = int(lib().orc_mirror_count(C.byref(st), _ptr(ca), ca.shape[0], tile_w, tile_h))
    nt = num_tiles(ca, tile_w, tile_h)
    out = dict(keys_in=np.zeros(m, np.uint64), vals_in=np.zeros(m, np.uint32),
               keys=np.zeros(m, np.uint64), vals=np.zeros(m, np.uint32),
               ranges=np.zeros((nt, 2), np.uint32))
    lib().orc_mirror_bin(C.byref(st), _ptr(ca), ca.shape[0], tile_w, tile_h,
                         *[_ptr(out[k]) for k in ("keys_in", "vals_in", "keys", "vals", "ranges")])
    return out


def stable_sort_pairs(keys, vals):
    k = np.ascontiguousarray(keys, np.uint64).copy()
    v = np.ascontiguousarray(vals, np.uint32).copy()
    lib().orc_stable_sort_pairs(len(k), _ptr(k), _ptr(v))
    return k, v


# ------------------------------------------------------------------ FP64 forward
def preprocess64(sc, cams):
    st, keep = _scene_struct(sc)
    ca = _cams(cams)
    R = ca.shape[0] * sc.n
    out = dict(visible=np.zeros(R, np.uint8), mean2d=np.zeros((R, 2)), conic=np.zeros((R, 3)),
               rgb=np.zeros((R, 3)), depth=np.zeros(R))
    lib().orc_preprocess64(C.byref(st), _ptr(ca), ca.shape[0],
                           *[_ptr(out[k]) for k in ("visible", "mean2d", "conic", "rgb", "depth")])
    out["visible"] = out["visible"].astype(bool)
    return out


def render_pixels(sc, cams, pix, bg=(0.0, 0.0, 0.0), threads=None):
    """Renders the pixels ``pix`` (int32 rows of view, x, y).  Returns rgb [P,3], T [P],
    margin [P,2] (image decisions, image+clamp decisions), ncontrib [P], sig [P]."""
    st, keep = _scene_struct(sc)
    ca = _cams(cams)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    P = pix.shape[0]
    bgv = np.asarray(bg, np.float64)
    out = dict(rgb=np.zeros((P, 3)), T=np.zeros(P), margin=np.zeros((P, 2)),
               ncontrib=np.zeros(P, np.int32), sig=np.zeros(P, np.uint64))
    lib().orc_render_pixels(C.byref(st), _ptr(ca), ca.shape[0], _ptr(bgv), _ptr(pix), P,
                            *[_ptr(out[k]) for k in ("rgb", "T", "margin", "ncontrib", "sig")],
                            threads or default_threads())
    return out


def all_pixels(cam, view=0):
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    return np.stack([np.full(xs.size, view), xs.ravel(), ys.ravel()], 1).astype(np.int32)


def render_image(sc, cams, view=0, bg=(0.0, 0.0, 0.0), threads=None):
    """Full planar image [3][H][W] of one view plus T [H][W], margins [H][W][2], ncontrib."""
    from paper_2501_00342_b300.inputs import Camera  # noqa: F401  (type only)
    cam = cams[view]
    pix = all_pixels(cam, view)
    r = render_pixels(sc, cams, pix, bg, threads)
    H, W = cam.height, cam.width
    return dict(rgb=r["rgb"].reshape(H, W, 3).transpose(2, 0, 1).copy(), T=r["T"].reshape(H, W),
                margin=r["margin"].reshape(H, W, 2), ncontrib=r["ncontrib"].reshape(H, W),
                sig=r["sig"].reshape(H, W))


# ------------------------------------------------------------------ FP64 adjoint
def grad_buffers(sc):
    S = sc.stride
    g = dict(mean=np.zeros((3, S)), scale=np.zeros((3, S)), rot=np.zeros((4, S)),
             opacity=np.zeros(S), sh=np.zeros((sc.num_sh, 3, S)),
             sg_amp=np.zeros((max(sc.num_lobes, 0), 3, S)),
             sg_axis=(None if sc.sg_axis is None else np.zeros(sc.sg_axis.shape[:-1] + (S,))),
             sg_sharp=np.zeros((sc.num_lobes, S)))
    return g


def adjoint_pixels(sc, cams, pix, dL_drgb, bg=(0.0, 0.0, 0.0), threads=None):
    """Gradients of sum_p dL_drgb[p] . rgb[p] w.r.t. every parameter plane (FP64)."""
    st, keep = _scene_struct(sc)
    ca = _cams(cams)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    gin = np.ascontiguousarray(dL_drgb, np.float64).reshape(-1, 3)
    assert gin.shape[0] == pix.shape[0]
    g = grad_buffers(sc)
    gs = _Grads(*[_ptr(g[f]) for f in ("mean", "scale", "rot", "opacity", "sh", "sg_amp",
                                       "sg_axis", "sg_sharp")])
    bgv = np.asarray(bg, np.float64)
    lib().orc_adjoint_pixels(C.byref(st), _ptr(ca), ca.shape[0], _ptr(bgv), _ptr(pix),
                             pix.shape[0], _ptr(gin), C.byref(gs), threads or default_threads())
    return g


def adjoint_image(sc, cams, dL_dimg, view=0, bg=(0.0, 0.0, 0.0), threads=None):
    """``dL_dimg`` planar [3][H][W] for view ``view``."""
    cam = cams[view]
    pix = all_pixels(cam, view)
    gin = np.asarray(dL_dimg, np.float64).reshape(3, -1).T
    return adjoint_pixels(sc, cams, pix, gin, bg, threads)


def sh_basis(l, m, d):
    d = np.ascontiguousarray(d, np.float64)
    return float(lib().orc_sh_basis(l, m, _ptr(d)))
