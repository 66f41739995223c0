"""Pins for the orthogonal-frame lobe axes of the oracle (Sec. "Multi-Axis Orthogonal
Gaussians": 3 orthogonal lobes, 4 parameters each plus 3 that fix the directions, 15 in
all).  The frame of parameters f is the rotation of the unit quaternion (1, f)/|(1, f)|;
lobe k's axis is its column k."""
import copy

import numpy as np
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2501_00342_b300 import inputs as I
from tests.helpers import axis_camera, random_small_scene


def _frame_scene(n=30, seed=51, K=3, L=1):
    return random_small_scene(n, seed=seed, sh_degree=L, K=K, axis_mode=I.AXIS_ORTHO_FRAME)


def _as_free(sc):
    """The same scene with every lobe's axis written out explicitly (free-axis mode), the
    axes being the columns of scipy's rotation for the frame quaternion."""
    f = sc.sg_axis[:, :sc.n].T.astype(np.float64)
    R = Rotation.from_quat(np.concatenate([f, np.ones((sc.n, 1))], 1)).as_matrix()  # (x, y, z, w)
    free = copy.copy(sc)
    free.axis_mode = I.AXIS_FREE
    ax = np.zeros((sc.num_lobes, 3, sc.stride), np.float32)
    for k in range(sc.num_lobes):
        ax[k, :, :sc.n] = R[:, :, k].T
    free.sg_axis = ax
    return free, R


def test_parameter_count_is_fifteen_for_three_lobes():
    sc = _frame_scene(K=3, L=0)
    # geometry 11 + SH DC 3 + lobes: 3 x (3 amplitudes + sharpness) + 3 frame parameters
    assert sc.floats_per_gaussian() - 11 - 3 == 15


def test_frame_axes_are_orthonormal_and_match_a_rotation_library():
    sc = _frame_scene()
    free, R = _as_free(sc)
    for i in range(sc.n):
        assert np.allclose(R[i].T @ R[i], np.eye(3), atol=1e-12)
        assert np.isclose(np.linalg.det(R[i]), 1.0)
    cams = [axis_camera(40, 36, 60.0, 3.0), I.look_at((1.0, 0.7, 2.8), (0, 0, 0), 36, 40, 55.0)]
    a = O.preprocess64(sc, cams)["rgb"]
    b = O.preprocess64(free, cams)["rgb"]
    vis = O.mirror_preprocess(sc, cams)["visible"]
    # the free-axis path renormalises float32 columns: agreement to float32 rounding
    assert np.abs(a[vis] - b[vis]).max() < 1e-5
    ia = O.render_image(sc, cams, view=1)
    ib = O.render_image(free, cams, view=1)
    assert np.abs(ia["rgb"] - ib["rgb"]).max() < 1e-5


def test_zero_frame_is_the_world_frame():
    sc = _frame_scene()
    sc.sg_axis = np.zeros_like(sc.sg_axis)
    world = copy.copy(sc)
    world.axis_mode, world.sg_axis = I.AXIS_ORTHO_FIXED, None
    cams = [axis_camera(40, 36, 60.0, 3.0)]
    assert np.array_equal(O.preprocess64(sc, cams)["rgb"], O.preprocess64(world, cams)["rgb"])


def test_frame_adjoint_matches_central_differences():
    sc = _frame_scene(12, seed=52, K=3, L=0)
    cam = axis_camera(22, 22, 60.0, 3.0)
    rng = np.random.default_rng(4)
    w = rng.normal(size=(3, 22, 22))
    g = O.adjoint_image(sc, [cam], w, threads=1)
    img0 = O.render_image(sc, [cam], threads=1)
    gmax = np.abs(g["sg_axis"]).max()
    assert gmax > 0
    checked = 0
    for j in range(3):
        for i in range(sc.n):
            x = float(sc.sg_axis[j, i])
            h = 1e-4 * max(abs(x), 0.1)
            vals = []
            for sgn in (1, -1):
                s2 = copy.copy(sc)
                a2 = sc.sg_axis.copy()
                a2[j, i] = np.float32(x + sgn * h)
                s2.sg_axis = a2
                img = O.render_image(s2, [cam], threads=1)
                assert (img["sig"] == img0["sig"]).all()
                vals.append(((img["rgb"] * w).sum(), float(a2[j, i])))
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            ad = g["sg_axis"][j, i]
            assert abs(fd - ad) <= 2e-4 * (abs(ad) + 1e-4 * gmax + 1e-12), (j, i, fd, ad)
            checked += 1
    assert checked == 36
