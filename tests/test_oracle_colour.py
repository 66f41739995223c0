"""Pins for the oracle's colour model: real SH basis (Eq. 4), SG lobes (Eq. 5-8), the SH+SG
mix (Eq. 9) and the parameter counts the paper states."""
import math
import os

import numpy as np
import pytest
from scipy.special import sph_harm_y

import oracle as O
from paper_2501_00342_b300 import inputs as I
from tests.helpers import make_scene

Y00 = 0.5 / math.sqrt(math.pi)


def _real_sh_scipy(l, m, d):
    """Real SH from scipy's complex Y_l^m (Condon-Shortley phase included):
    sqrt(2) Re Y_l^m (m > 0), sqrt(2) Im Y_l^|m| (m < 0), Y_l^0 (m = 0)."""
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    y = complex(sph_harm_y(l, abs(m), theta, phi))
    if m > 0:
        return math.sqrt(2.0) * y.real
    if m < 0:
        return math.sqrt(2.0) * y.imag
    return y.real


def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def _f32(v):
    """Values as the float32 planes store them."""
    return np.asarray(np.asarray(v, np.float32), np.float64)


def _dirs(k, seed=0):
    g = np.random.default_rng(seed).normal(size=(k, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def test_sh_basis_matches_scipy_real_sh():
    for d in _dirs(25, 1):
        for l in range(0, 5):
            for m in range(-l, l + 1):
                assert O.sh_basis(l, m, d) == pytest.approx(_real_sh_scipy(l, m, d), abs=1e-12)


def test_sh_degree1_closed_form_signs():
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    for d in _dirs(10, 2):
        x, y, z = d
        assert O.sh_basis(0, 0, d) == pytest.approx(Y00, abs=1e-15)
        assert O.sh_basis(1, -1, d) == pytest.approx(-c1 * y, abs=1e-14)
        assert O.sh_basis(1, 0, d) == pytest.approx(c1 * z, abs=1e-14)
        assert O.sh_basis(1, 1, d) == pytest.approx(-c1 * x, abs=1e-14)


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi integrates products of degree <= 8 exactly
    nt, nphi = 12, 24
    ct, wt = np.polynomial.legendre.leggauss(nt)
    idx = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    G = np.zeros((len(idx), len(idx)))
    for c, w in zip(ct, wt):
        st = math.sqrt(1.0 - c * c)
        for k in range(nphi):
            ph = 2.0 * math.pi * k / nphi
            d = np.array([st * math.cos(ph), st * math.sin(ph), c])
            y = np.array([O.sh_basis(l, m, d) for l, m in idx])
            G += np.outer(y, y) * w * (2.0 * math.pi / nphi)
    assert np.abs(G - np.eye(len(idx))).max() < 1e-12


# ---------------------------------------------------------------- colour via preprocess64
def _colour_at(scene, dirs, return_dirs=False):
    """Colour of Gaussian 0 (at the origin) seen along each unit direction d (camera at -4d).
    With ``return_dirs`` also the exact directions, from the float32 camera centres."""
    cams = []
    for d in dirs:
        up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.9 else (1.0, 0.0, 0.0)
        cams.append(I.look_at(-4.0 * np.asarray(d), (0.0, 0.0, 0.0), 64, 64, 60.0, up=up))
    pre = O.preprocess64(scene, cams)
    rgb = pre["rgb"].reshape(len(cams), scene.n, 3)[:, 0, :]
    if return_dirs:
        exact = np.array([-_f32(c.campos) / np.linalg.norm(_f32(c.campos)) for c in cams])
        return rgb, exact
    return rgb


def _one(sh, amp=None, axis=None, sharp=None, axis_mode=I.AXIS_FREE):
    return make_scene([[0.0, 0.0, 0.0]], [[0.05, 0.05, 0.05]], [[1, 0, 0, 0]], [0.5],
                      np.asarray(sh)[None], None if amp is None else np.asarray(amp)[None],
                      None if axis is None else np.asarray(axis)[None],
                      None if sharp is None else np.asarray(sharp)[None], axis_mode)


def test_dc_colour_offset_and_clamp():
    sc = _one([[1.0, -0.2, -4.0]])
    rgb = _colour_at(sc, _dirs(3, 3))
    expect = np.maximum(0.0, _f32([1.0, -0.2, -4.0]) * Y00 + 0.5)
    assert np.abs(rgb - expect).max() < 1e-14
    assert (rgb[:, 2] == 0.0).all()


def test_sh3_colour_against_scipy_basis():
    rng = np.random.default_rng(4)
    coef = _f32(rng.normal(0.0, 0.3, (16, 3)))
    sc = _one(coef)
    rgb, dirs = _colour_at(sc, _dirs(12, 5), return_dirs=True)
    idx = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    for d, got in zip(dirs, rgb):
        pre = 0.5 + sum(coef[k] * _real_sh_scipy(l, m, d) for k, (l, m) in enumerate(idx))
        assert np.abs(got - np.maximum(pre, 0.0)).max() < 1e-12


def test_sg_lobe_peak_and_angular_falloff():
    mu = np.array([0.3, -1.2, 0.8])  # unnormalised on purpose
    lam, a = 7.5, _f32([0.4, -0.1, 0.25])
    sc = _one([[0.0, 0.0, 0.0]], [a], [mu], [lam])
    muh = _unit(_f32(mu))
    # at d = mu the lobe equals its amplitude (up to the float32 camera position)
    rgb = _colour_at(sc, [muh])[0]
    assert np.abs(rgb - np.maximum(0.0, 0.5 + a)).max() < 1e-6
    # at angle theta it equals a exp(-lambda (1 - cos theta))
    perp = _unit(np.cross(muh, [1.0, 0.0, 0.0]))
    for th in (0.1, 0.5, 1.0, 2.0, 3.0):
        d = math.cos(th) * muh + math.sin(th) * perp
        rgb, ex = _colour_at(sc, [d], return_dirs=True)
        cos_th = float(ex[0] @ muh)
        expect = 0.5 + a * math.exp(-lam * (1.0 - cos_th))
        assert np.abs(rgb[0] - np.maximum(0.0, expect)).max() < 1e-13


def test_sg_sphere_integral():
    # integral over S^2 of a exp(lambda (mu.d - 1)) = 2 pi a (1 - exp(-2 lambda)) / lambda
    lam, a = 3.0, _f32([0.3, 0.2, 0.1])
    mu = np.array([0.2, 0.5, -1.0])
    sc = _one([[0.0, 0.0, 0.0]], [a], [mu], [lam])
    nt, nphi = 48, 16
    ct, wt = np.polynomial.legendre.leggauss(nt)
    dirs, wts = [], []
    for c, w in zip(ct, wt):
        st = math.sqrt(1.0 - c * c)
        for k in range(nphi):
            ph = 2.0 * math.pi * (k + 0.5) / nphi
            dirs.append([st * math.cos(ph), st * math.sin(ph), c])
            wts.append(w * 2.0 * math.pi / nphi)
    rgb = _colour_at(sc, np.array(dirs))
    integral = (np.asarray(wts)[:, None] * (rgb - 0.5)).sum(0)
    expect = 2.0 * math.pi * a * (1.0 - math.exp(-2.0 * lam)) / lam
    assert np.abs(integral - expect).max() < 1e-6


def test_ortho_fixed_axes_are_world_axes():
    amps = _f32([[0.2, 0.0, 0.0], [0.0, 0.3, 0.0], [0.0, 0.0, 0.4]])
    lams = np.array([2.0, 5.0, 9.0])
    sc = _one([[0.0, 0.0, 0.0]], amps, None, lams, axis_mode=I.AXIS_ORTHO_FIXED)
    assert sc.sg_axis is None
    for k in range(3):
        d = np.eye(3)[k]
        rgb = _colour_at(sc, [d])[0]
        expect = 0.5 + sum(amps[j] * math.exp(lams[j] * (float(j == k) - 1.0)) for j in range(3))
        assert np.abs(rgb - expect).max() < 1e-14


def test_sh_plus_sg_mix_is_additive():
    # Eq. 9: colour = SH + SG; with both present the result is the sum of the parts
    rng = np.random.default_rng(6)
    coef = rng.normal(0.0, 0.3, (4, 3)); coef[0] += 1.5
    amp = rng.normal(0.0, 0.3, (2, 3)); axis = rng.normal(size=(2, 3)); lam = np.array([3.0, 11.0])
    both = _one(coef, amp, axis, lam)
    sh_only = _one(coef)
    sg_only = _one(np.zeros((4, 3)), amp, axis, lam)
    dirs = _dirs(6, 7)
    got = _colour_at(both, dirs)
    parts = _colour_at(sh_only, dirs) + _colour_at(sg_only, dirs) - 0.5
    assert (got > 0).all() and np.abs(got - parts).max() < 1e-13


def test_parameter_counts_against_paper():
    path = os.path.join(os.path.dirname(__file__), "golden", "param_counts.txt")
    counts = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            counts[name] = int(value)

    def fl(L, K, mode):
        sc = make_scene([[0, 0, 0]], [[1, 1, 1]], [[1, 0, 0, 0]], [0.5], np.zeros((1, (L + 1) ** 2, 3)),
                        np.zeros((1, K, 3)) if K else None, np.ones((1, K, 3)) if K else None,
                        np.ones((1, K)) if K else None, mode)
        return sc.floats_per_gaussian()

    geometry = 11
    assert fl(3, 0, I.AXIS_FREE) == counts["3dgs_total"]
    assert fl(3, 0, I.AXIS_FREE) - geometry == counts["3dgs_sh_coefficients"]
    assert fl(0, 1, I.AXIS_FREE) - fl(0, 0, I.AXIS_FREE) == counts["single_sg_view_dependent"]
    assert fl(3, 0, I.AXIS_FREE) - fl(0, 0, I.AXIS_FREE) == counts["sh3_view_dependent"]
    assert fl(0, 1, I.AXIS_FREE) - geometry == counts["diffuse_plus_sg_colour"]
    # world-axis lobes store no frame: the paper's 15 minus its 3 frame parameters
    assert fl(0, 3, I.AXIS_ORTHO_FIXED) - fl(0, 0, I.AXIS_FREE) == counts["three_ortho_sg"] - 3
