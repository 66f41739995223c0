"""CPU checks of the C ABI: the library loads without a GPU, exports every function
include/sgs.h declares, its struct layouts match the binding, and the host-only planning
call validates its arguments.  No compute call is made."""
import ctypes as C
import os
import re

import pytest

from paper_2501_00342_b300 import binding as B
from paper_2501_00342_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "sgs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgs_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    lib = B.lib()
    declared = _declared_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(B.EXPORTS)


def test_struct_layouts_match():
    sizes = (C.c_size_t * 6)()
    B.lib().sgs_abi_sizes(sizes)
    assert tuple(sizes) == (C.sizeof(B.Plan), C.sizeof(B.Camera), C.sizeof(B.Gaussians), C.sizeof(B.Settings),
                            C.sizeof(B.AdamConfig), C.sizeof(B.Grads))
    assert C.sizeof(B.Camera) == 88


def _g(n=100, L=1, K=3, mode=0):
    g = B.Gaussians()
    g.n, g.stride, g.sh_degree, g.num_lobes, g.axis_mode = n, I.padded_stride(n), L, K, mode
    return g


def _s(tw=16, th=16, batch=256, digit=8, fwd=0, bwd=0, count=0):
    s = B.Settings()
    s.tile_w, s.tile_h, s.batch_depth, s.digit_bits, s.memory_mode = tw, th, batch, digit, 0
    s.fwd_pixels, s.bwd_pixels, s.count_pairs = fwd, bwd, count
    return s


def test_plan_sizes_and_key_bits():
    cams = I.orbit_cameras(3, [1280, 640, 1920], [720, 360, 1080])
    plan, nbytes = B.workspace_size(_g(1000), cams, _s(), 50_000)
    tiles = 80 * 45 + 40 * 23 + 120 * 68
    assert plan.num_tiles == tiles and plan.B == 3
    assert plan.key_bits == 32 + (tiles - 1).bit_length()
    # the record sort orders the depth half; the instance sort takes the tile bits only
    assert plan.sort_passes == -(-(plan.key_bits - 32) // 8)
    plan9, _ = B.workspace_size(_g(1000), cams, _s(digit=9), 50_000)
    assert plan9.sort_passes == -(-(plan9.key_bits - 32) // 9)
    assert [plan.pixel_base[v] for v in range(4)] == [0, 1280 * 720, 1280 * 720 + 640 * 360,
                                                      1280 * 720 + 640 * 360 + 1920 * 1080]
    assert nbytes % 256 == 0 and nbytes == plan.workspace_bytes
    _, bigger = B.workspace_size(_g(1000), cams, _s(), 500_000)
    assert bigger > nbytes
    off, nb = B.region_info(plan, "REC0")
    assert off % 256 == 0 and nb >= 16 * 3000


@pytest.mark.parametrize("bad", [
    dict(tw=16, th=12), dict(tw=0, th=16), dict(tw=4, th=32), dict(tw=2, th=32), dict(tw=64, th=4),
    dict(tw=64, th=32), dict(tw=32, th=32, fwd=1), dict(tw=64, th=16, bwd=1), dict(batch=16), dict(batch=4096), dict(digit=3), dict(digit=11),
    dict(fwd=3), dict(fwd=-1), dict(bwd=3), dict(bwd=8), dict(tw=32, th=8, bwd=4), dict(count=2),
])
def test_invalid_settings_rejected(bad):
    cams = [I.look_at((0, 0, 4), (0, 0, 0), 64, 64, 60)]
    kw = dict(tw=16, th=16, batch=256, digit=8)
    kw.update(bad)
    with pytest.raises(B.SgsError) as e:
        B.workspace_size(_g(), cams, _s(**kw), 1000)
    assert e.value.code == B.SGS_ERR_INVALID


@pytest.mark.parametrize("ok", [dict(tw=32, th=32), dict(tw=64, th=16, fwd=2, bwd=4), dict(tw=8, th=64),
                                dict(tw=32, th=16, fwd=1, bwd=1)])
def test_tile_shapes_accepted(ok):
    cams = [I.look_at((0, 0, 4), (0, 0, 0), 64, 64, 60)]
    kw = dict(tw=16, th=16, batch=256, digit=8)
    kw.update(ok)
    plan, _ = B.workspace_size(_g(), cams, _s(**kw), 1000)
    assert plan.num_tiles == -(-64 // kw["tw"]) * -(-64 // kw["th"])


def _adaptive(flag, r0, r1):
    g = _g(L=2)
    g.sh_adaptive, g.sh_radius[0], g.sh_radius[1] = flag, r0, r1
    return g


@pytest.mark.parametrize("g", [_g(L=4), _g(K=5), _g(K=4, mode=1), _g(K=4, mode=2), _g(mode=3),
                               _adaptive(2, 1.0, 2.0), _adaptive(1, 3.0, 2.0), _adaptive(1, -1.0, 2.0),
                               _adaptive(1, float("nan"), 2.0)])
def test_invalid_gaussians_rejected(g):
    cams = [I.look_at((0, 0, 4), (0, 0, 0), 64, 64, 60)]
    with pytest.raises(B.SgsError):
        B.workspace_size(g, cams, _s(), 1000)


def test_invalid_views_and_capacity_rejected():
    cam = I.look_at((0, 0, 4), (0, 0, 0), 64, 64, 60)
    with pytest.raises(B.SgsError):
        B.workspace_size(_g(), [cam] * 65, _s(), 1000)
    with pytest.raises(B.SgsError):
        B.workspace_size(_g(), [cam], _s(), 1 << 33)
    bad = I.look_at((0, 0, 4), (0, 0, 0), 64, 64, 60)
    bad.width = 0
    with pytest.raises(B.SgsError):
        B.workspace_size(_g(), [bad], _s(), 1000)


def test_sort_temp_bytes_validation():
    assert B.sort_temp_bytes(1000, 44, 8) > 12 * 1000
    with pytest.raises(B.SgsError):
        B.sort_temp_bytes(1000, 65, 8)
    with pytest.raises(B.SgsError):
        B.sort_temp_bytes(1000, 64, 3)
    with pytest.raises(B.SgsError):
        B.sort_temp_bytes(1000, 64, 11)


def test_status_strings():
    for code in (B.SGS_OK, B.SGS_ERR_INVALID, B.SGS_ERR_CAPACITY, B.SGS_ERR_TIMEOUT, B.SGS_ERR_CUDA):
        assert len(B.status_string(code)) > 1


def test_selftest_lookback_rejects_bad_arguments_on_host():
    with pytest.raises(B.SgsError) as e:
        B.selftest_lookback(None, -1, 8, 8, None)
    assert e.value.code == B.SGS_ERR_INVALID
    with pytest.raises(B.SgsError):
        B.selftest_lookback(None, 4, 8, 8, None)  # slots missing
    with pytest.raises(B.SgsError):
        B.selftest_lookback(8, 4, None, 8, None)  # sum missing


def test_valid_colour_layouts_accepted():
    cams = [I.look_at((0, 0, 4), (0, 0, 0), 64, 64, 60)]
    for g in (_g(K=3, mode=2), _g(K=0, mode=2), _adaptive(1, 0.0, 0.0), _adaptive(1, 4.0, 16.0)):
        B.workspace_size(g, cams, _s(), 1000)
