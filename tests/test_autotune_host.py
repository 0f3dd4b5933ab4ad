"""The batched form's autotuner: selection, capacity handling and caching (host logic; the timed
launches are replaced by fakes, so no GPU is needed)."""
import math

import pytest
import torch

from paper_2606_11529_gb300 import batched
from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import scenes


def _fakes(monkeypatch, times, fail=None):
    """render_views raises `fail` for 8x8 tiles; the timer returns times[(tw, th, batch)]."""
    calls = []

    def fake_render(*args):
        c = args[6]
        calls.append((c.tile_w, c.tile_h, c.batch_depth))
        if fail is not None and c.tile_w == 8:
            raise fail
        return torch.ones(3, requires_grad=True) * 2.0  # a differentiable stand-in for the images

    def fake_time(fn, reps):
        fn()
        return times[calls[-1]]

    monkeypatch.setattr(batched, "render_views", fake_render)
    monkeypatch.setattr(batched, "_time_ms", fake_time)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "fake")
    monkeypatch.setattr(batched, "_CACHE", {})
    return calls


def _inputs():
    cams = [scenes.pinhole(64, 48, 64.0, scenes.yaw_view(3.0, (0.0, 0.0, 0.0)))] * 2
    params = [torch.zeros(4, 3) for _ in range(5)]  # mu, scale, quat, opacity, sh
    return params, cams, scenes.RenderConfig()


def test_picks_the_fastest_candidate_and_caches(monkeypatch):
    cands = [(t, b) for t in batched.TILE_CANDIDATES for b in batched.BATCH_CANDIDATES]
    times = {(t[0], t[1], b): 10.0 + i for i, (t, b) in enumerate(cands)}
    best_key = (16, 16, 64)
    times[best_key] = 1.0
    calls = _fakes(monkeypatch, times)
    params, cams, cfg = _inputs()
    best, table = batched.autotune(params, cams, cfg, scene_id="s")
    assert (best.tile_w, best.tile_h, best.batch_depth) == best_key
    assert table == times
    n = len(calls)
    again = batched.autotune(params, cams, cfg, scene_id="s")
    assert again[0] is best and len(calls) == n  # served from the cache: nothing re-run
    batched.autotune(params, cams, cfg, scene_id="other")
    assert len(calls) > n  # another scene is tuned afresh


def test_capacity_error_marks_the_candidate_infeasible(monkeypatch):
    times = {(16, 16, b): float(b) for b in batched.BATCH_CANDIDATES}
    _fakes(monkeypatch, times, fail=B.XprError(B.XPR_ERR_CAPACITY, "xpr_tile_bin_views", "too many pairs"))
    params, cams, cfg = _inputs()
    best, table = batched.autotune(params, cams, cfg, scene_id="s")
    assert all(math.isinf(table[(8, 8, b)]) for b in batched.BATCH_CANDIDATES)
    assert (best.tile_w, best.batch_depth) == (16, min(batched.BATCH_CANDIDATES))


def test_other_errors_propagate(monkeypatch):
    times = {(16, 16, b): 1.0 for b in batched.BATCH_CANDIDATES}
    _fakes(monkeypatch, times, fail=B.XprError(B.XPR_ERR_INVALID, "xpr_render_fwd_views", "bad argument"))
    params, cams, cfg = _inputs()
    with pytest.raises(B.XprError):
        batched.autotune(params, cams, cfg, scene_id="s")
