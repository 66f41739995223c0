"""Small hand-built scenes and cameras for the pins and parity tests."""
import numpy as np

from paper_2501_00342_b300 import inputs as I


def make_scene(means, scales, quats, opacity, sh, sg_amp=None, sg_axis=None, sg_sharp=None,
               axis_mode=I.AXIS_FREE):
    """means [n,3], scales [n,3], quats [n,4] (w,x,y,z), opacity [n], sh [n,(L+1)^2,3],
    sg_amp [n,K,3], sg_axis [n,K,3], sg_sharp [n,K]."""
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = means.shape[0]
    s = I.padded_stride(n)
    sh = np.asarray(sh, np.float64).reshape(n, -1, 3)
    nsh = sh.shape[1]
    L = int(round(np.sqrt(nsh))) - 1
    K = 0 if sg_amp is None else np.asarray(sg_amp).reshape(n, -1, 3).shape[1]

    def plane(shape):
        return np.zeros(shape + (s,), np.float32)

    mean = plane((3,)); mean[:, :n] = means.T
    scale = plane((3,)); scale[:, :n] = np.asarray(scales, np.float64).reshape(n, 3).T
    rot = plane((4,)); rot[:, :n] = np.asarray(quats, np.float64).reshape(n, 4).T
    opa = plane(()); opa[:n] = np.asarray(opacity, np.float64).reshape(n)
    shp = plane((nsh, 3)); shp[:, :, :n] = np.transpose(sh, (1, 2, 0))
    amp = plane((K, 3)); sharp = plane((K,)); axis = None
    if K:
        amp[:, :, :n] = np.transpose(np.asarray(sg_amp, np.float64).reshape(n, K, 3), (1, 2, 0))
        sharp[:, :n] = np.asarray(sg_sharp, np.float64).reshape(n, K).T
        if axis_mode == I.AXIS_FREE:
            axis = plane((K, 3))
            axis[:, :, :n] = np.transpose(np.asarray(sg_axis, np.float64).reshape(n, K, 3), (1, 2, 0))
        elif axis_mode == I.AXIS_ORTHO_FRAME:  # sg_axis: [n][3] frame parameters
            axis = plane((3,))
            axis[:, :n] = np.asarray(sg_axis, np.float64).reshape(n, 3).T
    return I.Scene(n, s, L, K, axis_mode, mean, scale, rot, opa, shp, amp, axis, sharp)


def axis_camera(width=128, height=128, fov=60.0, dist=4.0, cx=None, cy=None):
    """Camera on +z at ``dist`` looking at the origin; optional principal point."""
    cam = I.look_at((0.0, 0.0, dist), (0.0, 0.0, 0.0), width, height, fov)
    if cx is not None:
        cam.cx = cx
    if cy is not None:
        cam.cy = cy
    return cam


def random_small_scene(n, seed, sh_degree=1, K=2, axis_mode=I.AXIS_FREE, log_scale=(-1.6, 0.3),
                       extent=0.8):
    """Bigger Gaussians than the workloads, so that each covers many pixels of a small
    image (useful for finite differences)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, (n, 3))
    scales = np.exp(rng.normal(log_scale[0], log_scale[1], (n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    q *= rng.uniform(0.5, 2.0, (n, 1))  # unnormalised on purpose
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.5, n)))
    nsh = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, nsh, 3))
    sh[:, 0, :] = rng.normal(0.5, 0.3, (n, 3))
    amp = rng.normal(0.0, 0.3, (n, K, 3))
    axis = rng.normal(size=(n, K, 3)) * rng.uniform(0.5, 2.0, (n, K, 1))
    if axis_mode == I.AXIS_ORTHO_FRAME:
        axis = rng.normal(0.0, 0.8, (n, 3))  # frame parameters
    sharp = np.exp(rng.uniform(0.0, np.log(20.0), (n, K)))
    return make_scene(means, scales, q, opacity, sh, amp if K else None,
                      axis if K else None, sharp if K else None, axis_mode)


def grad_violation(g, ref, rel=1e-3):
    """Worst ratio |g - g*| / (rel * max(|g*|, rel * max|g*|)) over one parameter tensor:
    element-wise relative error with a floor at rel of the tensor's largest entry."""
    import numpy as np
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    big = np.abs(ref).max()
    if big == 0:
        return 0.0 if np.abs(g).max() == 0 else np.inf
    return float((np.abs(g - ref) / (rel * np.maximum(np.abs(ref), rel * big))).max())


COND_REL = 1e-4  # error bound of a cancelling gradient entry, relative to its term magnitudes


def check_gradients(scene, cams, pix, dL, grads, ref, planes, bg=(0.0, 0.0, 0.0), rel=1e-3):
    """Per element: |g - g*| <= rel * max(|g*|, rel * max|g*|).  An entry that misses this
    bound is a sum over pixels whose terms cancel; single-precision evaluation of each term
    bounds its error by a small multiple of A = sum_p |term_p|, not of |g*|.  For such an
    entry A is taken from the FP64 oracle, one pixel at a time over the pixels the
    Gaussian's 3-sigma disc can reach, and |g - g*| <= COND_REL * A is required instead.
    Returns the number of entries that needed the second bound (at most 1e-3 of them)."""
    import numpy as np

    import oracle as O
    pix = np.asarray(pix, np.int32).reshape(-1, 3)
    dL = np.asarray(dL, np.float64).reshape(-1, 3)
    m = O.mirror_preprocess(scene, cams)
    n = scene.n
    cancelling = total = 0
    for p in planes:
        if ref.get(p) is None or grads.get(p) is None or ref[p].size == 0:
            continue
        a = np.asarray(grads[p], np.float64)[..., :n]
        b = np.asarray(ref[p], np.float64)[..., :n]
        big = np.abs(b).max()
        total += b.size
        if big == 0:
            assert np.abs(a).max() == 0, p
            continue
        err = np.abs(a - b)
        bad = np.argwhere(err > rel * np.maximum(np.abs(b), rel * big))
        for idx in bad:
            idx = tuple(idx)
            gi = idx[-1]
            A = 0.0
            for v in range(len(cams)):
                r = v * n + gi
                if not m["visible"][r]:
                    continue
                cx, cy = m["mean2d"][r]
                rad = m["radius"][r] + 1.0
                near = np.nonzero((pix[:, 0] == v) & (np.abs(pix[:, 1] + 0.5 - cx) <= rad)
                                  & (np.abs(pix[:, 2] + 0.5 - cy) <= rad))[0]
                vis = m["visible"][v * n:(v + 1) * n]
                mx, my = m["mean2d"][v * n:(v + 1) * n, 0], m["mean2d"][v * n:(v + 1) * n, 1]
                rr = m["radius"][v * n:(v + 1) * n] + 1.0
                for j in near:
                    # the pixel's value depends only on the Gaussians whose disc reaches it;
                    # the subset keeps their relative order, so its terms are the same
                    x, y = pix[j, 1] + 0.5, pix[j, 2] + 0.5
                    keep = np.nonzero(vis & (np.abs(x - mx) <= rr) & (np.abs(y - my) <= rr))[0]
                    sub = scene.subset(keep)
                    local = int(np.searchsorted(keep, gi))
                    row = np.array([[0, pix[j, 1], pix[j, 2]]], np.int32)
                    term = O.adjoint_pixels(sub, [cams[v]], row, dL[j:j + 1], bg, threads=1)[p]
                    A += abs(float(np.asarray(term)[idx[:-1] + (local,)]))
            assert err[idx] <= COND_REL * A, (p, idx, a[idx], b[idx], A)
            cancelling += 1
    assert cancelling <= max(3, 1e-3 * total), cancelling
    return cancelling
