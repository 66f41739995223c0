"""The launch-settings autotuner: cache keys and cache reuse (CPU), and on the GPU that a
tuned configuration renders the same image as the default one."""
import dataclasses
import json
import types

import pytest

from paper_2501_00342_b300 import inputs as I
from paper_2501_00342_b300.autotune import autotune, signature
from paper_2501_00342_b300.render import RenderSettings


def _fake_model(n=1000, L=1, K=4, mode=0):
    return types.SimpleNamespace(n=n, sh_degree=L, num_lobes=K, axis_mode=mode)


def test_signature_separates_workloads():
    cams = I.orbit_cameras(2, [640, 1280], [360, 720])
    base = signature(_fake_model(), cams)
    assert base == signature(_fake_model(), I.orbit_cameras(2, [640, 1280], [360, 720], radius=9.0))
    assert base != signature(_fake_model(n=1001), cams)
    assert base != signature(_fake_model(K=3), cams)
    assert base != signature(_fake_model(), cams[:1])
    assert base != signature(_fake_model(), I.orbit_cameras(2, [1280, 640], [720, 360]))


def test_cache_hit_skips_timing(tmp_path, monkeypatch):
    cams = I.orbit_cameras(1, 320, 200)
    model = _fake_model()
    path = tmp_path / "tune.json"
    chosen = dict(tile_w=32, tile_h=8, batch_depth=512, digit_bits=10)
    path.write_text(json.dumps({signature(model, cams): {"settings": chosen, "ms": 1.0}}))

    def no_timing(*a, **k):
        raise AssertionError("timed despite a cache hit")

    monkeypatch.setattr("paper_2501_00342_b300.autotune.time_step", no_timing)
    bg = (0.1, 0.2, 0.3)
    got = autotune(model, cams, base=RenderSettings(bg=bg), cache_path=str(path))
    assert (got.tile_w, got.tile_h, got.batch_depth, got.digit_bits) == (32, 8, 512, 10)
    assert got.bg == bg


def test_coordinate_descent_keeps_the_fastest(tmp_path, monkeypatch):
    """With a synthetic cost the tuner visits each axis once and keeps the minimum."""
    cost = {(16, 16): 5.0, (16, 8): 4.0, (32, 8): 6.0, (8, 8): 7.0, (32, 16): 4.5, (16, 32): 4.6, (64, 8): 6.5,
            (32, 32): 4.2, (64, 16): 4.8}
    seen = []

    def fake_time(model, cams, st, steps=3, grad=None):
        seen.append(st)
        return cost[(st.tile_w, st.tile_h)] + {128: 0.5, 256: 0.0, 512: 0.2, 1024: 0.3}[st.batch_depth] + \
            {8: 0.3, 9: 0.0, 10: 0.1}[st.digit_bits] + {0: 0.05, 1: 0.0, 2: 0.1}[st.fwd_pixels] + \
            {0: 0.05, 2: 0.0, 4: 0.2}[st.bwd_pixels] + {0: 0.02, 1: 0.0}[st.persistent]

    monkeypatch.setattr("paper_2501_00342_b300.autotune.time_step", fake_time)
    log = []
    path = tmp_path / "t.json"
    got = autotune(_fake_model(), I.orbit_cameras(1, 64, 64), cache_path=str(path), log=log)
    assert (got.tile_w, got.tile_h, got.batch_depth, got.digit_bits) == (16, 8, 256, 9)
    assert (got.fwd_pixels, got.bwd_pixels, got.persistent) == (1, 2, 1)
    assert len(seen) == len(log) == 1 + 8 + 3 + 2 + 2 + 2 + 1
    stored = json.loads(path.read_text())
    assert list(stored.values())[0]["settings"] == {k: v for k, v in dataclasses.asdict(got).items() if k != "bg"}


@pytest.mark.gpu
def test_tuned_settings_render_identical_image(tmp_path):
    import torch

    from paper_2501_00342_b300.render import GaussianModel, Rasterizer

    sc, cams = I.workload(0)
    model = GaussianModel.from_scene(sc)
    path = str(tmp_path / "tune.json")
    log = []
    st = autotune(model, cams, cache_path=path, steps=1, log=log)
    assert len(log) >= 2 and all(t["ms"] > 0 for t in log)
    assert autotune(model, cams, cache_path=path) == st
    a = Rasterizer(model, cams, st).forward(model)
    b = Rasterizer(model, cams, RenderSettings()).forward(model)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
