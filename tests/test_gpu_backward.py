"""GPU parity of the hand-written backward pass against the FP64 oracle adjoint (itself
pinned by finite differences in test_oracle_adjoint.py), finite differences of the oracle
on a 200-Gaussian 32x32 slice, and the autograd Function + L1 loss."""
import copy

import numpy as np
import pytest
import torch

import oracle as O
from paper_2501_00342_b300 import inputs as I
from paper_2501_00342_b300.render import (PLANES, GaussianModel, Rasterizer, RenderSettings, l1_loss,
                                          render)
from tests.helpers import axis_camera, check_gradients, random_small_scene

pytestmark = pytest.mark.gpu

GRAD_REL = 1e-3     # |g - g*| <= GRAD_REL * max(|g*|, GRAD_REL * max|g*|) per element (see check_gradients)
AMBIGUOUS = 1e-5


def _weights(scene, cams, seed, bg=(0.0, 0.0, 0.0)):
    """Random dL/dpixel, zero on pixels where a discrete decision (or a clamp) of the FP64
    forward is within AMBIGUOUS of its threshold."""
    rng = np.random.default_rng(seed)
    ws = []
    for v, c in enumerate(cams):
        ref = O.render_image(scene, cams, view=v, bg=bg)
        keep = ref["margin"][..., 1] >= AMBIGUOUS
        ws.append((rng.normal(size=(3, c.height, c.width)) * keep).astype(np.float32))
    return ws


def _gpu_grads(scene, cams, ws, settings=RenderSettings()):
    model = GaussianModel.from_scene(scene)
    rast = Rasterizer(model, cams, settings)
    rast.forward(model)
    flat = torch.from_numpy(np.concatenate([w.reshape(-1) for w in ws])).cuda()
    g = rast.backward(model, flat)
    torch.cuda.synchronize()
    assert rast.device_status() == 0
    return {p: (None if t is None else t.cpu().numpy().astype(np.float64)) for p, t in g.items()}


def _oracle_grads(scene, cams, ws, bg=(0.0, 0.0, 0.0)):
    pix = np.concatenate([O.all_pixels(c, v) for v, c in enumerate(cams)])
    gin = np.concatenate([w.reshape(3, -1).T for w in ws]).astype(np.float64)
    return O.adjoint_pixels(scene, cams, pix, gin, bg)


def _compare(scene, cams, ws, g, ref, bg=(0.0, 0.0, 0.0)):
    pix = np.concatenate([O.all_pixels(c, v) for v, c in enumerate(cams)])
    dL = np.concatenate([w.reshape(3, -1).T for w in ws])
    return check_gradients(scene, cams, pix, dL, g, ref, PLANES, bg, GRAD_REL)


def test_gradients_config0_vs_adjoint():
    sc, cams = I.workload(0)
    ws = _weights(sc, cams, 1)
    _compare(sc, cams, ws, _gpu_grads(sc, cams, ws), _oracle_grads(sc, cams, ws))


@pytest.mark.parametrize("L,K,mode", [(1, 4, I.AXIS_FREE), (3, 0, I.AXIS_FREE), (0, 3, I.AXIS_ORTHO_FIXED),
                                      (2, 2, I.AXIS_FREE), (1, 3, I.AXIS_ORTHO_FRAME), (0, 2, I.AXIS_ORTHO_FRAME)])
def test_gradients_colour_variants_vs_adjoint(L, K, mode):
    sc = random_small_scene(60, seed=40 + L * 5 + K, sh_degree=L, K=K, axis_mode=mode)
    cams = [axis_camera(48, 40, 60.0, 3.5), I.look_at((1.5, -1.0, 3.0), (0, 0, 0), 40, 48, 55.0)]
    bg = (0.3, 0.1, 0.6)
    ws = _weights(sc, cams, 2, bg)
    _compare(sc, cams, ws, _gpu_grads(sc, cams, ws, RenderSettings(bg=bg)), _oracle_grads(sc, cams, ws, bg), bg)


def test_gradients_adaptive_sh_vs_adjoint():
    sc = random_small_scene(60, seed=42, sh_degree=2, K=2, log_scale=(-2.0, 0.5))
    cams = [axis_camera(48, 40, 60.0, 3.2), I.look_at((1.0, 0.8, 3.0), (0, 0, 0), 40, 48, 55.0)]
    m = O.mirror_preprocess(sc, cams)
    u = np.unique(m["radius"][m["visible"]])
    sc.sh_adaptive, sc.sh_radius = 1, (float(u[len(u) // 3]), float(u[2 * len(u) // 3]))
    ws = _weights(sc, cams, 6)
    g = _gpu_grads(sc, cams, ws)
    _compare(sc, cams, ws, g, _oracle_grads(sc, cams, ws))
    # bands above every record's degree get no gradient at all
    top = np.where(m["radius"] < sc.sh_radius[0], 0, np.where(m["radius"] < sc.sh_radius[1], 1, 2))
    top = np.where(m["visible"], top, -1).reshape(len(cams), sc.n).max(0)
    for i in range(sc.n):
        assert np.all(g["sh"][(top[i] + 1) ** 2:, :, i] == 0.0)


@pytest.mark.parametrize("tile,bwd,fwd", [((16, 16), 4, 0), ((16, 32), 4, 0), ((16, 32), 1, 0), ((8, 8), 2, 0),
                                          ((32, 32), 2, 0), ((64, 16), 4, 0), ((16, 32), 2, 1)])
def test_backward_pixels_per_thread(tile, bwd, fwd):
    # fwd = 1 with bwd = 2: the backward computes its warp-block masks instead of reading
    # the ones a two-pixel forward stores
    sc, cams = I.workload(0)
    ws = _weights(sc, cams, 8)
    g = _gpu_grads(sc, cams, ws, RenderSettings(tile_w=tile[0], tile_h=tile[1], bwd_pixels=bwd, fwd_pixels=fwd))
    _compare(sc, cams, ws, g, _oracle_grads(sc, cams, ws))
    ref = _gpu_grads(sc, cams, ws)
    for p in PLANES:
        if ref[p] is not None:  # the same sums, added in another order
            assert np.abs(g[p] - ref[p]).max() <= 1e-5 * np.abs(ref[p]).max(), p


@pytest.mark.parametrize("batch", [32, 96, 100, 1024])
def test_backward_batch_depth(batch):
    # the reverse walk over batches of other depths, including one that is not a whole
    # number of 32-entry groups
    sc, cams = I.workload(0)
    ws = _weights(sc, cams, 8)
    g = _gpu_grads(sc, cams, ws, RenderSettings(tile_w=32, tile_h=32, batch_depth=batch))
    _compare(sc, cams, ws, g, _oracle_grads(sc, cams, ws))
    ref = _gpu_grads(sc, cams, ws)
    for p in PLANES:
        if ref[p] is not None:  # the same sums, added in another order
            assert np.abs(g[p] - ref[p]).max() <= 1e-5 * np.abs(ref[p]).max(), p


def _slice_200():
    """200 clustered Gaussians (the training-step distribution), one 32x32 view."""
    sc = I.cluster_scene(200, 1, 4, config=2, num_clusters=8)
    cam = I.look_at((0.0, 1.0, 4.5), (0.0, 0.0, 0.0), 32, 32, 50.0)
    return sc, [cam]


def test_fd_slice_200_gaussians_32x32():
    sc, cams = _slice_200()
    ws = _weights(sc, cams, 3)
    g = _gpu_grads(sc, cams, ws)
    ref = _oracle_grads(sc, cams, ws)
    _compare(sc, cams, ws, g, ref)
    # central differences of the FP64 oracle on a sample of parameters
    w = ws[0].astype(np.float64)

    def loss(s2):
        img = O.render_image(s2, cams, threads=4)
        return float((img["rgb"] * w).sum()), img["sig"]

    _, sig0 = loss(sc)
    rng = np.random.default_rng(7)
    checked = 0
    for p in PLANES:
        arr = getattr(sc, p)
        if arr is None:
            continue
        scale = np.abs(ref[p][..., :sc.n]).max()
        hit = np.argwhere(np.abs(ref[p][..., :sc.n]) > 0.05 * scale)
        for idx in hit[rng.permutation(len(hit))[:6]]:
            idx = tuple(idx)
            x = float(arr[idx])
            h = 1e-4 * max(abs(x), 0.1)
            vals, ok = [], True
            for sgn in (1, -1):
                s2 = copy.copy(sc)
                a2 = arr.copy()
                a2[idx] = np.float32(x + sgn * h)
                setattr(s2, p, a2)
                L, sig = loss(s2)
                ok &= bool((sig == sig0).all())
                vals.append((L, float(a2[idx])))
            if not ok:
                continue
            fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
            assert abs(g[p][idx] - fd) <= GRAD_REL * scale + 1e-3 * abs(fd), (p, idx, g[p][idx], fd)
            checked += 1
    assert checked >= 30


def test_autograd_function_and_l1_loss():
    sc, cams = _slice_200()
    model = GaussianModel.from_scene(sc)
    leaves = {p: (t.clone().requires_grad_(True) if t is not None else None) for p, t in model.planes.items()}
    m = model.with_planes(**leaves)
    rast = Rasterizer(m, cams, RenderSettings())
    img = render(rast, m)
    target = torch.from_numpy(I.target_images(cams)[0].reshape(-1)).cuda()
    loss, dimg = l1_loss(img.detach(), target)
    ref_loss = (img.detach() - target).abs().mean()
    assert abs(loss.item() - ref_loss.item()) <= 1e-6 * max(1.0, ref_loss.item())
    assert torch.equal(dimg, torch.sign(img.detach() - target) / img.numel())
    img.backward(dimg)
    direct = rast.backward(model, dimg)
    for p in PLANES:
        if leaves[p] is not None:  # float atomics: equal up to summation order
            scale = direct[p].abs().max()
            assert (leaves[p].grad - direct[p]).abs().max() <= 1e-5 * scale, p


def test_backward_is_repeatable():
    sc, cams = I.workload(0)
    ws = _weights(sc, cams, 4)
    a = _gpu_grads(sc, cams, ws)
    b = _gpu_grads(sc, cams, ws)
    for p in PLANES:
        if a[p] is not None:
            scale = np.abs(a[p]).max()
            assert np.abs(a[p] - b[p]).max() <= 1e-5 * scale  # only atomic-order rounding differs


def test_persistent_backward_equals_one_cta_per_tile():
    """The persistent two-pixel backward gives the gradients of one CTA per tile (the same
    sums, the float atomics adding in another order), on more tiles than resident CTAs."""
    sc = I.cluster_scene(30000, 1, 4, config=3)
    cams = I.orbit_cameras(2, 1280, 720, 50.0)
    rng = np.random.default_rng(3)
    ws = [rng.normal(size=(3, c.height, c.width)).astype(np.float32) for c in cams]
    base = RenderSettings(tile_w=16, tile_h=16, fwd_pixels=2, bwd_pixels=2)
    a = _gpu_grads(sc, cams, ws, base)
    b = _gpu_grads(sc, cams, ws, RenderSettings(**{**base.__dict__, "persistent": 1}))
    for p in PLANES:
        if a[p] is not None:
            assert np.abs(a[p]).max() > 0, p
            assert np.abs(a[p] - b[p]).max() <= 1e-5 * np.abs(a[p]).max(), p


def test_backwards_on_one_workspace_leave_the_2d_gradients_zero():
    """The reverse blend adds into per-record 2D gradients that the preprocess backward
    clears as it reads them: after every backward the region is zero, and backwards in a
    row (other weights, another forward in between) on one workspace give the gradients of
    a fresh workspace."""
    sc, cams = I.workload(0)
    w1, w2 = _weights(sc, cams, 21), _weights(sc, cams, 22)
    model = GaussianModel.from_scene(sc)
    rast = Rasterizer(model, cams, RenderSettings())
    flat = [torch.from_numpy(np.concatenate([w.reshape(-1) for w in ws])).cuda() for ws in (w1, w2, w1)]
    got = []
    for k, dl in enumerate(flat):
        if k != 1:
            rast.forward(model)
        g = rast.backward(model, dl)
        torch.cuda.synchronize()
        assert rast.device_status() == 0
        R = sc.n * len(cams)  # float4[2][R] then float[R]; the region's tail is alignment padding
        assert not bool(rast.region("GRAD2D", torch.float32)[:9 * R].any().item())
        got.append({p: (None if t is None else t.cpu().numpy().astype(np.float64)) for p, t in g.items()})
    for ws, g in ((w1, got[0]), (w2, got[1]), (w1, got[2])):
        ref = _gpu_grads(sc, cams, ws)
        for p in PLANES:
            if ref[p] is not None:
                assert np.abs(ref[p]).max() > 0, p
                assert np.abs(g[p] - ref[p]).max() <= 1e-5 * np.abs(ref[p]).max(), p
