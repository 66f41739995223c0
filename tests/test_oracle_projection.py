"""Pins for the oracle's geometry: Eq. 3 covariance, the EWA projection to a 2D conic, the
3-sigma radius, and agreement of the FP32 mirror with the FP64 forward."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2501_00342_b300 import inputs as I
from tests.helpers import axis_camera, make_scene, random_small_scene


def _f64(a):
    return np.asarray(a, np.float64)


def _project(cam, X):
    V = _f64(cam.viewmat).reshape(3, 4)
    t = V[:, :3] @ X + V[:, 3]
    return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])


def _num_jacobian(cam, X, h=1e-5):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3); e[k] = h
        J[:, k] = (_project(cam, X + e) - _project(cam, X - e)) / (2 * h)
    return J


def _cov3d_scipy(scale, quat_wxyz):
    w, x, y, z = quat_wxyz
    R = Rotation.from_quat([x, y, z, w]).as_matrix()  # normalises; scalar-last order
    return R @ np.diag(np.asarray(scale) ** 2) @ R.T


def test_isotropic_on_axis_closed_form():
    cam = axis_camera(128, 128, 60.0, 4.0)
    for s, z0 in [(0.05, 0.0), (0.2, 1.0), (0.01, -2.0)]:
        sc = make_scene([[0.0, 0.0, z0]], [[s, s, s]], [[0.3, -0.5, 0.2, 0.7]], [0.5],
                        np.zeros((1, 1, 3)))
        pre = O.preprocess64(sc, [cam])
        ss, zz, fx = _f64(np.float32(s)), 4.0 - _f64(np.float32(z0)), _f64(np.float32(cam.fx))
        v = (fx * ss / zz) ** 2 + 0.3
        assert pre["conic"][0] == pytest.approx([1.0 / v, 0.0, 1.0 / v], rel=1e-12, abs=1e-12)
        assert pre["mean2d"][0] == pytest.approx([cam.cx, cam.cy], abs=1e-9)
        m = O.mirror_preprocess(sc, [cam])
        r_expect = math.ceil(3.0 * math.sqrt(v + math.sqrt(0.1)))
        assert m["radius"][0] == r_expect


def test_isotropic_covariance_ignores_rotation():
    cam = I.look_at((1.0, 2.0, 3.5), (0.1, 0.0, 0.0), 96, 64, 55.0)
    qs = np.random.default_rng(1).normal(size=(6, 4))
    sc = make_scene(np.tile([[0.2, -0.1, 0.3]], (6, 1)), np.full((6, 3), 0.07), qs, np.full(6, 0.5),
                    np.zeros((6, 1, 3)))
    con = O.preprocess64(sc, [cam])["conic"]
    assert np.abs(con - con[0]).max() < 1e-12 * np.abs(con).max()


def test_ewa_against_numerical_jacobian_and_scipy_rotation():
    """Sigma2D - 0.3 I = Jn Sigma Jn^T with Jn the finite-difference Jacobian of the pinhole
    projection and Sigma from scipy's quaternion -> matrix (pins J, W, R and Eq. 3)."""
    sc = random_small_scene(40, seed=11, log_scale=(-2.0, 0.5))
    cam = I.look_at((0.7, -1.2, 3.2), (0.0, 0.1, 0.0), 80, 60, 50.0)
    pre = O.preprocess64(sc, [cam])
    checked = 0
    for i in range(sc.n):
        X = _f64(sc.mean[:, i])
        V = _f64(cam.viewmat).reshape(3, 4)
        t = V[:, :3] @ X + V[:, 3]
        limx = 1.3 * 0.5 * cam.width / _f64(np.float32(cam.fx))
        limy = 1.3 * 0.5 * cam.height / _f64(np.float32(cam.fy))
        if t[2] <= 0.2:
            continue
        # the frustum clamp evaluates J at the clamped point t'
        tc = np.array([np.clip(t[0] / t[2], -limx, limx) * t[2], np.clip(t[1] / t[2], -limy, limy) * t[2], t[2]])
        Xc = V[:, :3].T @ (tc - V[:, 3])
        Jn = _num_jacobian(cam, Xc)
        S = _cov3d_scipy(_f64(sc.scale[:, i]), _f64(sc.rot[:, i]))
        S2 = Jn @ S @ Jn.T + 0.3 * np.eye(2)
        A, B, Cc = pre["conic"][i]
        S2_oracle = np.linalg.inv(np.array([[A, B], [B, Cc]]))
        assert np.abs(S2_oracle - S2).max() <= 1e-6 * np.abs(S2).max()
        assert pre["mean2d"][i] == pytest.approx(_project(cam, X), rel=1e-12, abs=1e-9)
        checked += 1
    assert checked > 30


def test_frustum_clamp_changes_conic_off_screen():
    cam = axis_camera(64, 64, 60.0, 4.0)
    # x/z = 1.2 is beyond 1.3 * tan(30 deg) = 0.75 -> clamped
    sc = make_scene([[-4.8, 0.0, 0.0]], [[0.3, 0.1, 0.2]], [[1, 0.2, 0, 0]], [0.5], np.zeros((1, 1, 3)))
    pre = O.preprocess64(sc, [cam])
    V = _f64(cam.viewmat).reshape(3, 4)
    t = V[:, :3] @ _f64(sc.mean[:, 0]) + V[:, 3]
    lim = 1.3 * 32.0 / _f64(np.float32(cam.fx))
    assert abs(t[0] / t[2]) > lim
    unclamped = _num_jacobian(cam, _f64(sc.mean[:, 0]))
    S = _cov3d_scipy(_f64(sc.scale[:, 0]), _f64(sc.rot[:, 0]))
    S2_unclamped = unclamped @ S @ unclamped.T + 0.3 * np.eye(2)
    A, B, Cc = pre["conic"][0]
    S2 = np.linalg.inv(np.array([[A, B], [B, Cc]]))
    assert np.abs(S2 - S2_unclamped).max() > 1e-3 * np.abs(S2).max()


def test_mirror32_agrees_with_fp64():
    sc, cams = I.workload(0)
    m = O.mirror_preprocess(sc, cams)
    p = O.preprocess64(sc, cams)
    vis = m["visible"]
    assert vis.sum() > 1900 and (p["visible"] == vis).all()
    assert np.abs(m["mean2d"][vis] - p["mean2d"][vis]).max() < 1e-4
    rel = np.abs(m["conic"][vis] - p["conic"][vis]) / np.abs(p["conic"][vis]).max(1, keepdims=True)
    assert rel.max() < 2e-5
    # radius: ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det)) of Sigma2D
    A, B, Cc = p["conic"][vis].T
    det = A * Cc - B * B
    a, b, c = Cc / det, -B / det, A / det
    mid = 0.5 * (a + c)
    lam = mid + np.sqrt(np.maximum(0.1, mid * mid - (a * c - b * b)))
    r64 = 3.0 * np.sqrt(lam)
    safe = np.abs(r64 - np.round(r64)) > 1e-4
    assert (m["radius"][vis][safe] == np.ceil(r64[safe])).all()
    # depth bits are the float32 view depth
    z32 = m["depth_bits"][vis].view(np.float32).astype(np.float64)
    assert np.abs(z32 - p["depth"][vis]).max() < 1e-5


def test_cull_near_plane_and_behind():
    cam = axis_camera(64, 64, 60.0, 4.0)
    # depths 4 - z: 8 (ok), 0.1 (< near 0.2), -1 (behind)
    sc = make_scene([[0, 0, -4.0], [0, 0, 3.9], [0, 0, 5.0]], np.full((3, 3), 0.1),
                    np.tile([[1, 0, 0, 0]], (3, 1)), [0.5] * 3, np.zeros((3, 1, 3)))
    m = O.mirror_preprocess(sc, [cam])
    assert m["visible"].tolist() == [True, False, False]
    assert (m["tiles_touched"][1:] == 0).all()


def test_rect_and_tiles_touched():
    sc, cams = I.workload(0)
    for tw, th in [(16, 16), (8, 8), (32, 16), (8, 32)]:
        m = O.mirror_preprocess(sc, cams, tw, th)
        vis = m["visible"]
        px, py = m["mean2d"][vis].T.astype(np.float64)
        r = m["radius"][vis].astype(np.float64)
        TW, TH = -(-cams[0].width // tw), -(-cams[0].height // th)
        x0 = np.maximum(np.floor((px - r) / tw), 0)
        x1 = np.minimum(np.floor((px + r) / tw), TW - 1)
        y0 = np.maximum(np.floor((py - r) / th), 0)
        y1 = np.minimum(np.floor((py + r) / th), TH - 1)
        rect = m["rect"][vis]
        assert (rect[:, 0] == x0).all() and (rect[:, 2] == x1).all()
        assert (rect[:, 1] == y0).all() and (rect[:, 3] == y1).all()
        # the ellipse reaches at least one and at most all tiles of the rectangle
        tt = m["tiles_touched"][vis]
        assert (tt >= 1).all() and (tt <= (x1 - x0 + 1) * (y1 - y0 + 1)).all()
