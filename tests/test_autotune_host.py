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


def test_view_chunks_partition():
    cams = list(range(8))
    assert batched.view_chunks(cams, 1) == [cams]
    assert batched.view_chunks(cams, 3) == [[0, 1, 2], [3, 4, 5], [6, 7]]
    assert batched.view_chunks(cams, 20) == [[c] for c in cams]
    assert sum(batched.view_chunks(cams, 5), []) == cams


def _fake_splat(monkeypatch, max_views, calls):
    """MultiViewSplat stand-in: a batch of more than ``max_views`` views is over the pair limit."""

    class Fake:
        @staticmethod
        def apply(mu, scale, quat, opacity, sh, part, cfg, ws, persistent):
            calls.append(list(part))
            if len(part) > max_views:
                raise B.XprError(B.XPR_ERR_CAPACITY, "xpr_tile_bin_views", "more than 2^31 - 1 pairs")
            return torch.stack([torch.full((3, 2, 2), float(c)) for c in part])

    monkeypatch.setattr(batched, "MultiViewSplat", Fake)


def test_render_views_splits_views_over_the_pair_limit(monkeypatch):
    calls = []
    _fake_splat(monkeypatch, 3, calls)
    ws = batched.ViewsWorkspace()
    params = [torch.zeros(1) for _ in range(5)]
    img = batched.render_views(*params, list(range(8)), None, ws)
    # 8 views fail, 2 x 4 fail on the first chunk, 4 x 2 fit; images in view order
    assert ws.chunks == 4
    assert img[:, 0, 0, 0].tolist() == [float(c) for c in range(8)]
    n = len(calls)
    batched.render_views(*params, list(range(8)), None, ws)
    assert calls[n:] == [[0, 1], [2, 3], [4, 5], [6, 7]]  # the chunk count is kept


def test_render_views_raises_when_one_view_is_over_the_limit(monkeypatch):
    _fake_splat(monkeypatch, 0, [])
    with pytest.raises(B.XprError):
        batched.render_views(*[torch.zeros(1) for _ in range(5)], list(range(4)), None, batched.ViewsWorkspace())
