"""The CPU-baseline estimator's sampling (host logic, no GPU)."""
import numpy as np

from oracle import baseline
from paper_2606_11529_gb300 import scenes


def test_covering_equals_per_tile_box_test():
    """The summed-area-table selection keeps exactly the primitives whose box holds a sampled tile."""
    rng = np.random.default_rng(11)
    Wt, Ht, n = 37, 23, 20000
    x0 = rng.integers(-3, Wt + 2, n)
    y0 = rng.integers(-3, Ht + 2, n)
    bb = np.stack([x0, y0, x0 + rng.integers(0, 6, n), y0 + rng.integers(0, 6, n)], 1).astype(np.int32)
    bb[::97] = 0  # culled primitives carry an empty box
    tiles = rng.choice(Wt * Ht, 40, replace=False)
    tx, ty = tiles % Wt, tiles // Wt
    want = np.zeros(n, bool)
    for x, y in zip(tx, ty):
        want |= (bb[:, 0] <= x) & (x < bb[:, 2]) & (bb[:, 1] <= y) & (y < bb[:, 3])
    assert want.any() and not want.all()
    assert np.array_equal(baseline.covering(bb, tx, ty, Wt, Ht), want)


def test_estimate_runs_on_a_small_scene():
    sc = scenes.uniform_scene(3000, seed=2, sh_degree=1)
    cam = scenes.pinhole(128, 96, 128.0, scenes.yaw_view(3.0, (0.0, 0.0, 0.0)))
    cfg = scenes.RenderConfig(tile_w=16, tile_h=16, sh_degree=1)
    est, measured, desc = baseline.estimate_fwd_bwd_seconds(sc, cam, cfg, prim_frac=0.5, n_tiles=10, seed=0)
    assert est > 0 and measured > 0
    assert "1500 of 3000 primitives" in desc and "10 of 48 tiles" in desc
