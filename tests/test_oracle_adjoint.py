"""Pins for the oracle's hand-written FP64 adjoint: central finite differences of the FP64
forward, for every parameter entry of small scenes, including active clamps (frustum,
colour at 0, alpha at 0.99), both SG axis modes, SH degrees 0-3 and a background."""
import copy

import numpy as np
import pytest

import oracle as O
from paper_2501_00342_b300 import inputs as I
from tests.helpers import axis_camera, make_scene, random_small_scene

PLANES = ("mean", "scale", "rot", "opacity", "sh", "sg_amp", "sg_axis", "sg_sharp")


def _with_extras(sc):
    """Append a frustum-clamped Gaussian, one with a clamped (negative) colour and one whose
    alpha clamps at 0.99 near its centre."""
    n = sc.n
    means = np.vstack([sc.mean[:, :n].T, [[2.75, 0.3, 0.0], [0.1, 0.1, 0.5], [-0.2, 0.3, 0.9]]])
    scales = np.vstack([sc.scale[:, :n].T, [[0.7, 0.4, 0.5], [0.3, 0.2, 0.25], [0.15, 0.2, 0.1]]])
    quats = np.vstack([sc.rot[:, :n].T, [[0.9, 0.1, 0.3, 0.2], [0.8, -0.3, 0.1, 0.4], [1, 0, 0.2, 0]]])
    opa = np.concatenate([sc.opacity[:n], [0.8, 0.6, 0.9995]])
    sh_extra = np.zeros((3, sc.num_sh, 3))
    sh_extra[:, 0, :] = [[0.4, 0.6, 0.2], [-3.0, 0.5, -2.5], [0.3, 0.2, 0.9]]
    sh = np.concatenate([np.transpose(sc.sh[:, :, :n], (2, 0, 1)), sh_extra])
    K = sc.num_lobes
    amp = axis = sharp = None
    if K:
        amp = np.concatenate([np.transpose(sc.sg_amp[:, :, :n], (2, 0, 1)), np.full((3, K, 3), 0.1)])
        sharp = np.concatenate([sc.sg_sharp[:, :n].T, np.full((3, K), 4.0)])
        if sc.sg_axis is not None:
            axis = np.concatenate([np.transpose(sc.sg_axis[:, :, :n], (2, 0, 1)),
                                   np.tile(np.eye(3)[:K][None] + 0.3, (3, 1, 1))])
    return make_scene(means, scales, quats, opa, sh, amp, axis, sharp, sc.axis_mode)


def _loss_and_sig(sc, cam, w, bg):
    img = O.render_image(sc, [cam], bg=bg, threads=1)
    return float((img["rgb"] * w).sum()), img["sig"]


def _fd_check(sc, cam, seed, bg=(0.0, 0.0, 0.0), min_checked=200):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(3, cam.height, cam.width))
    g = O.adjoint_image(sc, [cam], w, bg=bg, threads=1)
    _, sig0 = _loss_and_sig(sc, cam, w, bg)
    checked = skipped = 0
    worst = 0.0
    for name in PLANES:
        arr = getattr(sc, name)
        if arr is None or arr.size == 0:
            continue
        gmax = np.abs(g[name]).max()
        for idx in np.ndindex(arr.shape[:-1]):
            for i in range(sc.n):
                x = float(arr[idx + (i,)])
                h = 1e-4 * max(abs(x), 0.1)
                vals = []
                ok = True
                for sgn in (+1, -1):
                    s2 = copy.copy(sc)
                    a2 = arr.copy()
                    a2[idx + (i,)] = np.float32(x + sgn * h)
                    setattr(s2, name, a2)
                    L, sig = _loss_and_sig(s2, cam, w, bg)
                    ok &= bool((sig == sig0).all())
                    vals.append((L, float(a2[idx + (i,)])))
                if not ok:
                    skipped += 1
                    continue
                fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
                ad = g[name][idx + (i,)]
                err = abs(fd - ad) / (abs(ad) + 1e-4 * gmax + 1e-12)
                worst = max(worst, err)
                assert err < 2e-4, (name, idx, i, fd, ad)
                checked += 1
    assert checked >= min_checked and skipped < 0.05 * checked
    return worst


def test_adjoint_fd_sh1_free_axes_with_clamps():
    sc = _with_extras(random_small_scene(10, seed=21, sh_degree=1, K=2))
    cam = axis_camera(24, 24, 60.0, 3.5)
    _fd_check(sc, cam, seed=1)


def test_adjoint_fd_world_axes_and_background():
    sc = _with_extras(random_small_scene(8, seed=22, sh_degree=0, K=3, axis_mode=I.AXIS_ORTHO_FIXED))
    cam = I.look_at((0.6, -0.4, 3.4), (0.0, 0.0, 0.0), 20, 24, 60.0)
    _fd_check(sc, cam, seed=2, bg=(0.3, 0.1, 0.7), min_checked=150)


def test_adjoint_fd_sh3_no_lobes():
    sc = random_small_scene(6, seed=23, sh_degree=3, K=0)
    cam = I.look_at((-0.5, 0.8, 3.3), (0.1, 0.0, 0.0), 20, 20, 60.0)
    _fd_check(sc, cam, seed=3, min_checked=150)


def test_adjoint_fd_sh2():
    sc = random_small_scene(5, seed=24, sh_degree=2, K=1)
    cam = axis_camera(18, 22, 55.0, 3.2)
    _fd_check(sc, cam, seed=4, min_checked=120)


def test_adjoint_pixel_subset_is_restriction():
    """The gradient of a loss on a pixel subset equals the full-image gradient with the
    weights outside the subset set to zero."""
    sc = random_small_scene(12, seed=25)
    cam = axis_camera(20, 20, 60.0, 3.5)
    rng = np.random.default_rng(5)
    w = rng.normal(size=(3, 20, 20))
    mask = rng.uniform(size=(20, 20)) < 0.3
    w_masked = w * mask
    g_full = O.adjoint_image(sc, [cam], w_masked)
    ys, xs = np.nonzero(mask)
    pix = np.stack([np.zeros_like(xs), xs, ys], 1).astype(np.int32)
    g_sub = O.adjoint_pixels(sc, [cam], pix, w[:, ys, xs].T)
    for name in PLANES:
        if g_full[name] is not None:
            assert np.abs(g_full[name] - g_sub[name]).max() <= 1e-12 * (1 + np.abs(g_full[name]).max())


def test_adjoint_multi_view_sums_views():
    sc = random_small_scene(10, seed=26)
    cams = [axis_camera(16, 16, 60.0, 3.5), I.look_at((2.0, 1.0, 2.5), (0, 0, 0), 16, 16, 60.0)]
    rng = np.random.default_rng(6)
    ws = [rng.normal(size=(3, 16, 16)) for _ in cams]
    pix = np.concatenate([O.all_pixels(c, v) for v, c in enumerate(cams)])
    gin = np.concatenate([w.reshape(3, -1).T for w in ws])
    g = O.adjoint_pixels(sc, cams, pix, gin)
    g0 = O.adjoint_image(sc, cams, ws[0], view=0)
    g1 = O.adjoint_image(sc, cams, ws[1], view=1)
    for name in PLANES:
        if g[name] is not None:
            assert np.abs(g[name] - g0[name] - g1[name]).max() <= 1e-12 * (1 + np.abs(g[name]).max())
