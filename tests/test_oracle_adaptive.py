"""Pins for the adaptive SH degree of the oracle (Sec. "Mixing Spherical Harmonics and
Spherical Gaussians": the SH degree, 0-2, follows the Gaussian's projected size).  A record
whose FP32 pixel radius r is below sh_radius[0] sums band 0 only, below sh_radius[1] bands
0-1, otherwise bands 0-2.  Each pin compares against the fixed-degree oracle on a scene
whose unused bands are zeroed, so a wrong threshold, band count or comparison fails."""
import copy

import numpy as np

import oracle as O
from paper_2501_00342_b300 import inputs as I
from tests.helpers import axis_camera, random_small_scene


def _scene(n=60, seed=31):
    # degree-2 storage, two lobes, sizes spread so that all three degrees occur
    return random_small_scene(n, seed=seed, sh_degree=2, K=2, log_scale=(-2.2, 0.6))


def _adaptive(sc, t0, t1):
    a = copy.copy(sc)
    a.sh_adaptive, a.sh_radius = 1, (float(t0), float(t1))
    return a


def _bands_zeroed(sc, top):
    """The same scene, fixed degree, with every SH band above `top` set to zero."""
    z = copy.copy(sc)
    sh = sc.sh.copy()
    sh[(top + 1) ** 2:] = 0.0
    z.sh = sh
    return z


def test_zero_thresholds_use_every_band():
    sc = _scene()
    cam = axis_camera(40, 40, 60.0, 3.0)
    a = O.render_image(_adaptive(sc, 0, 0), [cam])
    b = O.render_image(sc, [cam])
    assert np.array_equal(a["rgb"], b["rgb"]) and np.array_equal(a["T"], b["T"])


def test_huge_thresholds_use_band_zero_only():
    sc = _scene()
    cam = axis_camera(40, 40, 60.0, 3.0)
    a = O.render_image(_adaptive(sc, 1e9, 1e9), [cam])
    b = O.render_image(_bands_zeroed(sc, 0), [cam])
    assert np.array_equal(a["rgb"], b["rgb"])


def test_each_record_takes_the_degree_of_its_radius():
    sc = _scene()
    cams = [axis_camera(48, 40, 60.0, 3.0), I.look_at((1.2, -0.8, 2.6), (0, 0, 0), 40, 48, 55.0)]
    radius = O.mirror_preprocess(sc, cams)["radius"]
    vis = O.mirror_preprocess(sc, cams)["visible"]
    r = radius[vis]
    u = np.unique(r)
    t0, t1 = u[len(u) // 3], u[2 * len(u) // 3]  # radii that occur: r == t0 takes degree 1
    assert len(u) >= 3 and (r == t0).any() and (r == t1).any()
    got = O.preprocess64(_adaptive(sc, t0, t1), cams)["rgb"]
    want = {top: O.preprocess64(_bands_zeroed(sc, top), cams)["rgb"] for top in (0, 1, 2)}
    top = np.where(radius < t0, 0, np.where(radius < t1, 1, 2))
    for D in (0, 1, 2):
        sel = vis & (top == D)
        assert sel.any()
        assert np.array_equal(got[sel], want[D][sel]), D
    # degree-2 storage capped: with stored degree 1 a "degree 2" record sums bands 0-1
    sc1 = random_small_scene(30, seed=32, sh_degree=1, K=1, log_scale=(-2.2, 0.6))
    a = O.preprocess64(_adaptive(sc1, 0, 0), cams[:1])["rgb"]
    b = O.preprocess64(sc1, cams[:1])["rgb"]
    assert np.array_equal(a, b)


def test_adjoint_follows_the_chosen_degree():
    """Bands above a record's degree receive no gradient from it; the rest match central
    differences of the adaptive forward."""
    sc = _adaptive(_scene(14, seed=33), 0, 0)
    cam = axis_camera(22, 22, 60.0, 3.0)
    r = O.mirror_preprocess(sc, [cam])["radius"]
    vis = O.mirror_preprocess(sc, [cam])["visible"]
    t0, t1 = np.quantile(r[vis], [0.34, 0.67])
    sc.sh_radius = (float(t0), float(t1))
    rng = np.random.default_rng(3)
    w = rng.normal(size=(3, 22, 22))
    g = O.adjoint_image(sc, [cam], w, threads=1)
    top = np.where(r < t0, 0, np.where(r < t1, 1, 2))
    for i in range(sc.n):
        assert np.all(g["sh"][(top[i] + 1) ** 2:, :, i] == 0.0), i
    # central differences on every SH coefficient of the records in view
    img0 = O.render_image(sc, [cam], threads=1)
    checked = 0
    gmax = np.abs(g["sh"]).max()
    for k in range(9):
        for c in range(3):
            for i in np.nonzero(vis)[0]:
                x = float(sc.sh[k, c, i])
                h = 1e-4 * max(abs(x), 0.1)
                vals = []
                for sgn in (1, -1):
                    s2 = copy.copy(sc)
                    a2 = sc.sh.copy()
                    a2[k, c, i] = np.float32(x + sgn * h)
                    s2.sh = a2
                    img = O.render_image(s2, [cam], threads=1)
                    assert (img["sig"] == img0["sig"]).all()
                    vals.append(((img["rgb"] * w).sum(), float(a2[k, c, i])))
                fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
                ad = g["sh"][k, c, i]
                assert abs(fd - ad) <= 2e-4 * (abs(ad) + 1e-4 * gmax + 1e-12), (k, c, i, fd, ad)
                checked += 1
    assert checked >= 200
