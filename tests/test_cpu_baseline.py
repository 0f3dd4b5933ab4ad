"""The CPU-baseline estimator's sampling (host logic, no GPU)."""
import numpy as np

from oracle import baseline
from oracle import oracle as O
from paper_2606_11529_gb300 import scenes


def _small():
    sc = scenes.uniform_scene(3000, seed=2, sh_degree=1)
    cam = scenes.pinhole(128, 96, 128.0, scenes.yaw_view(3.0, (0.0, 0.0, 0.0)))
    cfg = scenes.RenderConfig(tile_w=16, tile_h=16, sh_degree=1)
    return sc, cam, cfg


def test_estimate_runs_on_a_small_scene():
    sc, cam, cfg = _small()
    est, measured, desc = baseline.estimate_fwd_bwd_seconds(sc, cam, cfg, prim_frac=0.5, n_tiles=10, seed=0)
    assert est > 0 and measured > 0
    assert "1500 of 3000 primitives" in desc and "10 of 48 tiles" in desc


def test_sampled_tiles_walk_the_full_scene_lists():
    """The timed compositing walks every primitive of a sampled tile (lists of the whole scene, not
    of the primitive sample), and the lists are built once per scene and camera."""
    sc, cam, cfg = _small()
    baseline.estimate_fwd_bwd_seconds(sc, cam, cfg, prim_frac=0.1, n_tiles=5, seed=1)
    rec, vals, ranges = baseline._full_lists(sc, cam, cfg, 48)
    pr = O.project_scene(sc, cam, cfg)
    _, k, v = O.bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False)
    _, v, r = O.sort_pairs(k, v, 48)
    assert np.array_equal(ranges, r) and np.array_equal(vals, v) and np.array_equal(rec, pr["rec"])
    assert ranges[:, 1].max() > 300  # several hundred entries: more than a 10% sample would hold
    baseline.estimate_fwd_bwd_seconds(sc, cam, cfg, prim_frac=0.1, n_tiles=5, seed=2)
    assert baseline._full_lists(sc, cam, cfg, 48)[1] is vals
