"""Pins for the oracle's front-to-back blending: closed forms for one and two Gaussians,
the alpha clamp / skip / stop conventions, the 3-sigma support, invariants."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2501_00342_b300 import inputs as I
from tests.helpers import axis_camera, make_scene, random_small_scene

Y00 = 0.5 / math.sqrt(math.pi)


def _f32(v):
    return np.asarray(np.asarray(v, np.float32), np.float64)


def _rgb_of(dc):
    return np.maximum(0.0, _f32(dc) * Y00 + 0.5)


def _centred_cam():
    # principal point on a pixel centre: pixel (64, 64) sees the optical axis
    return axis_camera(128, 128, 60.0, 4.0, cx=64.5, cy=64.5)


def _px(sc, cam, x, y, bg=(0, 0, 0)):
    r = O.render_pixels(sc, [cam], np.array([[0, x, y]], np.int32), bg)
    return r["rgb"][0], r["T"][0], r["ncontrib"][0]


def test_single_gaussian_at_its_mean():
    cam = _centred_cam()
    for o in (0.3, 0.9, 0.995):
        sc = make_scene([[0, 0, 0.5]], [[0.1, 0.05, 0.08]], [[1, 0.3, 0.1, 0]], [o],
                        [[[0.7, -0.3, 1.2]]])
        rgb, T, n = _px(sc, cam, 64, 64)
        a = min(0.99, _f32(o))
        assert rgb == pytest.approx(a * _rgb_of([0.7, -0.3, 1.2]), abs=1e-12)
        assert T == pytest.approx(1.0 - a, abs=1e-12) and n == 1


def test_single_gaussian_with_background():
    cam = _centred_cam()
    sc = make_scene([[0, 0, 0]], [[0.1, 0.1, 0.1]], [[1, 0, 0, 0]], [0.6], [[[0.2, 0.4, 0.6]]])
    bg = (0.25, 0.5, 1.0)
    rgb, T, _ = _px(sc, cam, 64, 64, bg)
    a = _f32(0.6)
    assert rgb == pytest.approx(a * _rgb_of([0.2, 0.4, 0.6]) + (1 - a) * np.array(bg), abs=1e-12)


def test_two_coincident_gaussians_front_to_back():
    cam = _centred_cam()
    # both on the optical axis; index 0 is the FAR one, so order must come from depth
    sc = make_scene([[0, 0, -1.0], [0, 0, 1.0]], [[0.1] * 3, [0.1] * 3], [[1, 0, 0, 0]] * 2,
                    [0.5, 0.7], [[[1.0, 0.0, 0.0]], [[0.0, 1.0, 0.0]]])
    rgb, T, n = _px(sc, cam, 64, 64)
    a_near, a_far = _f32(0.7), _f32(0.5)
    c_near, c_far = _rgb_of([0.0, 1.0, 0.0]), _rgb_of([1.0, 0.0, 0.0])
    assert rgb == pytest.approx(a_near * c_near + (1 - a_near) * a_far * c_far, abs=1e-12)
    assert T == pytest.approx((1 - a_near) * (1 - a_far), abs=1e-12) and n == 2


def test_low_alpha_is_skipped():
    cam = _centred_cam()
    sc = make_scene([[0, 0, 0]], [[0.1] * 3], [[1, 0, 0, 0]], [0.003], [[[1.0, 1.0, 1.0]]])
    rgb, T, n = _px(sc, cam, 64, 64)
    assert n == 0 and T == 1.0 and (rgb == 0).all()


def test_stop_before_transmittance_drops_below_1e4():
    cam = _centred_cam()
    # alphas 0.99, 0.98, 0.9 front to back: T 1 -> 0.01 -> 2e-4 -> (2e-5 < 1e-4: stop)
    zs = [1.0, 0.5, 0.0]
    ops = [0.995, 0.98, 0.9]
    cols = [[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]
    sc = make_scene([[0, 0, z] for z in zs], [[0.1] * 3] * 3, [[1, 0, 0, 0]] * 3, ops,
                    [[c] for c in cols])
    rgb, T, n = _px(sc, cam, 64, 64)
    a1, a2 = 0.99, _f32(0.98)
    expect = a1 * _rgb_of(cols[0]) + (1 - a1) * a2 * _rgb_of(cols[1])
    assert n == 2 and rgb == pytest.approx(expect, abs=1e-12)
    assert T == pytest.approx((1 - a1) * (1 - a2), abs=1e-15)


def test_support_is_three_sigma_ellipse():
    cam = _centred_cam()
    sc = make_scene([[0.1, -0.05, 0]], [[0.3, 0.12, 0.05]], [[0.9, 0.1, 0.2, 0.3]], [0.9],
                    [[[1.0, 1.0, 1.0]]])
    img = O.render_image(sc, [cam])
    p = O.preprocess64(sc, [cam])
    A, B, Cc = p["conic"][0]
    mx, my = p["mean2d"][0]
    ys, xs = np.mgrid[0:128, 0:128]
    dx, dy = mx - (xs + 0.5), my - (ys + 0.5)
    power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy
    alpha = np.minimum(0.99, _f32(0.9) * np.exp(power))
    inside = (power >= -4.5) & (alpha >= 1 / 255)
    sure = np.abs(power + 4.5) > 1e-4
    got = img["ncontrib"] > 0
    assert inside.sum() > 200
    assert (got[sure] == inside[sure]).all()
    # the support is the ellipse, not its bounding box: far corners of the box are empty
    assert (~got & (np.abs(dx) < 3 * np.sqrt(Cc / (A * Cc - B * B))) &
            (np.abs(dy) < 3 * np.sqrt(A / (A * Cc - B * B)))).sum() > 0


def test_permutation_invariance():
    sc, cams = I.workload(0)
    small = sc.subset(np.arange(600))
    perm = np.random.default_rng(3).permutation(600)
    a = O.render_image(small, cams)
    b = O.render_image(small.subset(perm), cams)
    assert np.abs(a["rgb"] - b["rgb"]).max() < 1e-13
    assert (a["ncontrib"] == b["ncontrib"]).all()


def test_transmittance_is_product_and_bounded():
    sc = random_small_scene(30, seed=2, sh_degree=0, K=0)
    cam = axis_camera(24, 24, 60.0, 4.0)
    img = O.render_image(sc, [cam])
    assert (img["T"] <= 1.0).all() and (img["T"] >= 1e-4).all()
    # adding a Gaussian in front never raises T anywhere
    front = make_scene(np.vstack([sc.mean[:, :sc.n].T, [[0.0, 0.0, 2.0]]]),
                       np.vstack([sc.scale[:, :sc.n].T, [[0.4, 0.4, 0.1]]]),
                       np.vstack([sc.rot[:, :sc.n].T, [[1, 0, 0, 0]]]),
                       np.concatenate([sc.opacity[:sc.n], [0.5]]),
                       np.concatenate([np.transpose(sc.sh[:, :, :sc.n], (2, 0, 1)), [[[0.1, 0.1, 0.1]]]]))
    img2 = O.render_image(front, [cam])
    assert (img2["T"] <= img["T"] + 1e-15).all() and (img2["T"] < img["T"]).any()


def test_config0_image_is_sane():
    sc, cams = I.workload(0)
    img = O.render_image(sc, cams)
    assert img["rgb"].shape == (3, 128, 128)
    assert 0.05 < img["rgb"].mean() < 0.5 and img["ncontrib"].max() > 10
    # ambiguous pixels (a discrete FP64 decision within 1e-5 relative of its threshold)
    assert (img["margin"][..., 0] < 1e-5).mean() < 1e-3
