"""Pins for the oracle's FP32 binning mirror: tile|depth keys, stable sort, tile ranges."""
import numpy as np

import oracle as O
from paper_2501_00342_b300 import inputs as I


def _enumerate(sc, cams, tw, th):
    """Brute-force instance list from the mirror's per-record rects and depth bits."""
    m = O.mirror_preprocess(sc, cams, tw, th)
    keys, vals = [], []
    base = 0
    for v, cam in enumerate(cams):
        TW, TH = -(-cam.width // tw), -(-cam.height // th)
        for i in range(sc.n):
            r = v * sc.n + i
            if not m["visible"][r]:
                continue
            x0, y0, x1, y1 = m["rect"][r]
            for ty in range(y0, y1 + 1):
                for tx in range(x0, x1 + 1):
                    keys.append(((base + ty * TW + tx) << 32) | int(m["depth_bits"][r]))
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
