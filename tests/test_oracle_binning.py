"""Pins for the oracle's FP32 binning mirror: tile|depth keys, stable sort, tile ranges."""
import numpy as np

import oracle as O
from paper_2501_00342_b300 import inputs as I


def row_spans_np(px, py, A, B, C, tw, th, TW, TH):
    """The row-span rule restated with numpy float32 scalars (each op rounded on its own):
    the tiles of each row whose pixel-centre columns meet the x-extent of the band's slice
    of the ellipse Q <= 9.01 (padded by 1/64 px).  Returns [(ty, tx0, tx1), ...]."""
    f = np.float32
    k, pad = f(9.01), f(0.015625)
    px, py, A, B, C = (f(v) for v in (px, py, A, B, C))
    det = f(f(A * C) - f(B * B))
    if not det > 0:
        return []
    ex = f(np.sqrt(f(f(k * C) / det)))
    ey = f(np.sqrt(f(f(k * A) / det)))
    dyr = -f(B * f(np.sqrt(f(k / f(det * C)))))
    invA = f(f(1) / A)
    Ak = f(A * k)
    t0 = f(f(f(py - ey) - pad) - f(0.5))
    t1 = f(f(f(py + ey) + pad) - f(0.5))
    out = []
    y0, y1 = np.ceil(t0), np.floor(t1)
    if not y0 <= y1:
        return out
    r0 = max(np.floor(f(y0 / f(th))), f(0))
    r1 = min(np.floor(f(y1 / f(th))), f(TH - 1))
    if not r0 <= r1:
        return out
    eyp = f(ey + pad)
    for ty in range(int(r0), int(r1) + 1):
        ly, hy = f(f(ty * th) + f(0.5)), f(f(ty * th + th) - f(0.5))
        u0, u1 = max(f(ly - py), -eyp), min(f(hy - py), eyp)
        if not u0 <= u1:
            continue
        s0 = f(np.sqrt(max(f(0), f(Ak - f(f(det * u0) * u0)))))
        s1 = f(np.sqrt(max(f(0), f(Ak - f(f(det * u1) * u1)))))
        b0, b1 = f(B * u0), f(B * u1)
        hi0, hi1 = f(f(s0 - b0) * invA), f(f(s1 - b1) * invA)
        lo0, lo1 = f(-f(b0 + s0) * invA), f(-f(b1 + s1) * invA)
        xmax = ex if (u0 <= dyr and dyr <= u1) else max(hi0, hi1)
        xmin = -ex if (u0 <= -dyr and -dyr <= u1) else min(lo0, lo1)
        xs0, xs1 = f(f(px + xmin) - pad), f(f(px + xmax) + pad)
        x0, x1 = np.ceil(f(xs0 - f(0.5))), np.floor(f(xs1 - f(0.5)))
        if not x0 <= x1:
            continue
        c0 = max(np.floor(f(x0 / f(tw))), f(0))
        c1 = min(np.floor(f(x1 / f(tw))), f(TW - 1))
        if c0 <= c1:
            out.append((ty, int(c0), int(c1)))
    return out


def _box_min_q(a, b, c, mx, my, x0, x1, y0, y1):
    """Exact (FP64) minimum of a dx^2 + 2b dx dy + c dy^2 over the box of points p,
    d = p - mean."""
    if x0 <= mx <= x1 and y0 <= my <= y1:
        return 0.0
    best = np.inf
    for e in (x0, x1):
        dx = e - mx
        dy = np.clip(my - b * dx / c, y0, y1) - my
        best = min(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
    for e in (y0, y1):
        dy = e - my
        dx = np.clip(mx - b * dy / a, x0, x1) - mx
        best = min(best, a * dx * dx + 2 * b * dx * dy + c * dy * dy)
    return best


def _enumerate(sc, cams, tw, th):
    """Brute-force instance list from the mirror's per-record rects and depth bits, keeping
    the rectangle's tiles that pass the (numpy) tile test."""
    m = O.mirror_preprocess(sc, cams, tw, th)
    keys, vals = [], []
    base = 0
    for v, cam in enumerate(cams):
        TW, TH = -(-cam.width // tw), -(-cam.height // th)
        for i in range(sc.n):
            r = v * sc.n + i
            if not m["visible"][r]:
                continue
            A, B, C = m["conic"][r]
            spans = row_spans_np(m["mean2d"][r, 0], m["mean2d"][r, 1], A, B, C, tw, th, TW, TH)
            assert sum(c1 - c0 + 1 for _, c0, c1 in spans) == m["tiles_touched"][r]
            for tyy, c0, c1 in spans:
                for txx in range(c0, c1 + 1):
                    keys.append(((base + tyy * TW + txx) << 32) | int(m["depth_bits"][r]))
                    vals.append(r)
        base += TW * TH
    return np.array(keys, np.uint64), np.array(vals, np.uint32), base


def test_keys_sort_ranges_single_view():
    sc, cams = I.workload(0)
    for tw, th in [(16, 16), (8, 16)]:
        keys, vals, ntiles = _enumerate(sc, cams, tw, th)
        b = O.mirror_bin(sc, cams, tw, th)
        assert (b["keys_in"] == keys).all() and (b["vals_in"] == vals).all()
        order = np.argsort(keys, kind="stable")
        assert (b["keys"] == keys[order]).all() and (b["vals"] == vals[order]).all()
        tiles = (b["keys"] >> np.uint64(32)).astype(np.int64)
        start = np.searchsorted(tiles, np.arange(ntiles), "left")
        end = np.searchsorted(tiles, np.arange(ntiles), "right")
        empty = start == end
        start[empty] = 0
        end[empty] = 0
        assert (b["ranges"][:, 0] == start).all() and (b["ranges"][:, 1] == end).all()


def test_keys_multi_view_tile_bases():
    sc = I.cluster_scene(3000, 1, 2, config=1)
    cams = I.orbit_cameras(3, [96, 64, 80], [48, 64, 40], 50.0)
    keys, vals, ntiles = _enumerate(sc, cams, 16, 16)
    b = O.mirror_bin(sc, cams, 16, 16)
    assert ntiles == O.num_tiles(cams, 16, 16)
    assert (b["keys_in"] == keys).all() and (b["vals_in"] == vals).all()
    order = np.argsort(keys, kind="stable")
    assert (b["keys"] == keys[order]).all() and (b["vals"] == vals[order]).all()
    # every tile's entries belong to one view: value // n == view of the tile
    tiles = (b["keys"] >> np.uint64(32)).astype(np.int64)
    bases = np.cumsum([0] + [(-(-c.width // 16)) * (-(-c.height // 16)) for c in cams])
    view_of_tile = np.searchsorted(bases, tiles, "right") - 1
    assert (view_of_tile == b["vals"] // sc.n).all()


def test_stable_sort_adversarial():
    rng = np.random.default_rng(0)
    cases = {
        "all_equal": np.full(5000, 0x123456789, np.uint64),
        "all_distinct": rng.permutation(5000).astype(np.uint64) * np.uint64(0x10001),
        "one_digit": rng.integers(0, 256, 5000).astype(np.uint64) << np.uint64(40),
        "random64": rng.integers(0, 2**63, 5000, dtype=np.uint64),
        "empty": np.zeros(0, np.uint64),
        "one": np.array([7], np.uint64),
    }
    for name, k in cases.items():
        v = np.arange(len(k), dtype=np.uint32)
        ks, vs = O.stable_sort_pairs(k, v)
        order = np.argsort(k, kind="stable")
        assert (ks == k[order]).all() and (vs == v[order]).all(), name


def test_instance_count_depends_on_tile_size_only_through_rects():
    sc, cams = I.workload(0)
    for tw, th in [(16, 16), (8, 8), (32, 32)]:
        m = O.mirror_preprocess(sc, cams, tw, th)
        b = O.mirror_bin(sc, cams, tw, th)
        assert len(b["keys"]) == int(m["tiles_touched"].sum())


def test_row_spans_keep_every_support_tile_and_little_else():
    """Superset: every pixel centre inside the FP64 3-sigma ellipse (with 1e-6 slack) lies in
    a kept tile.  Tightness: every kept tile's box of pixel centres comes within the padded
    Q <= 9.01 ellipse (exact FP64 box minimum)."""
    sc, cams = I.workload(0)
    cam = cams[0]
    for tw, th in [(16, 16), (8, 8), (32, 16)]:
        m = O.mirror_preprocess(sc, cams, tw, th)
        p = O.preprocess64(sc, cams)
        TW, TH = -(-cam.width // tw), -(-cam.height // th)
        kept_total = rect_total = 0
        ys, xs = np.mgrid[0:cam.height, 0:cam.width]
        for r in np.nonzero(m["visible"])[0]:
            x0, y0, x1, y1 = m["rect"][r]
            rect_total += (x1 - x0 + 1) * (y1 - y0 + 1)
            A, B, C = m["conic"][r]
            spans = row_spans_np(m["mean2d"][r, 0], m["mean2d"][r, 1], A, B, C, tw, th, TW, TH)
            kept = {(ty, tx) for ty, c0, c1 in spans for tx in range(c0, c1 + 1)}
            kept_total += len(kept)
            a, b, c = p["conic"][r]
            mx, my = p["mean2d"][r]
            dx, dy = mx - (xs + 0.5), my - (ys + 0.5)
            sup = a * dx * dx + 2 * b * dx * dy + c * dy * dy <= 9.0 * (1 + 1e-6)
            need = set(zip((ys[sup] // th).tolist(), (xs[sup] // tw).tolist()))
            assert need <= kept, (r, need - kept)
            slack = (np.sqrt(9.01) + 0.02 * np.sqrt(a + c + 2 * abs(b))) ** 2 * (1 + 1e-5)
            for ty, tx in kept:
                q = _box_min_q(a, b, c, mx, my, tx * tw + 0.5, tx * tw + tw - 0.5, ty * th + 0.5, ty * th + th - 0.5)
                assert q <= slack, (r, ty, tx, q)
        assert kept_total < rect_total
