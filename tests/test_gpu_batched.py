"""The batched (multi-view, persistent) form computes exactly the single-view
path for every view: images bit-identical, gradients equal to the sum of the
per-view gradients; plus its work list, batch-depth invariance, oracle parity
of one view and the autotuner."""
import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import batched as BT
from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import BAND, GRAD_TOL, IMG_TOL, dev, rel_err

pytestmark = pytest.mark.gpu

NAMES = ["mu", "scale", "quat", "opacity", "sh"]


def _views(n_views=3, W=200, H=136, f=200.0):
    return scenes.multiview_cameras(n_views, W, H, f, seed=1)


@pytest.mark.parametrize("persistent,tile,deg,method", [(True, 16, 1, 0), (False, 16, 0, 0), (True, 8, 3, 0),
                                                        (True, 16, 1, 1), (False, 8, 0, 1), (True, 8, 3, 1)])
def test_views_equal_single_view_path(persistent, tile, deg, method):
    # method 1: 3DGUT, whose single-view path is checked against the oracle in test_gpu_ut.py
    sc = scenes.uniform_scene(8000, seed=2, sh_degree=deg)
    cams = _views()
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=deg, bg=(0.1, 0.2, 0.3), method=method)
    P = [t.requires_grad_(True) for t in R.scene_to_device(sc)]
    imgs = BT.render_views(*P, cams, cfg, persistent=persistent)
    w = torch.from_numpy(np.random.default_rng(3).normal(size=tuple(imgs.shape)).astype(np.float32)).cuda()
    (imgs * w).sum().backward()
    g_multi = [p.grad.clone() for p in P]
    g_sum = [torch.zeros_like(p) for p in P]
    for v, cam in enumerate(cams):
        for p in P:
            p.grad = None
        img = R.render(*P, cam, cfg)
        assert torch.equal(img, imgs[v].detach()), f"view {v} differs"
        (img * w[v]).sum().backward()
        for a, p in zip(g_sum, P):
            a += p.grad
    for name, gm, gs in zip(NAMES, g_multi, g_sum):
        assert rel_err(gm.cpu().numpy(), gs.cpu().numpy()) < 1e-5, name


def test_one_view_against_oracle(oracle):
    sc = scenes.uniform_scene(6000, seed=4, sh_degree=3)
    cams = _views(2)
    cfg = scenes.RenderConfig(sh_degree=3)
    imgs = BT.forward_views(*R.scene_to_device(sc), cams, cfg).image
    ref = oracle.pipeline_tiled(sc, cams[1], cfg, delta=BAND)
    ok = ~ref["band"]
    assert ok.mean() > 0.99
    assert np.abs(imgs[1].cpu().numpy()[:, ok] - ref["image"][:, ok]).max() <= IMG_TOL


def test_worklist_is_descending_permutation():
    sc = scenes.uniform_scene(5000, seed=5)
    fr = BT.forward_views(*R.scene_to_device(sc), _views(2), scenes.RenderConfig())
    wl = fr.worklist.cpu().numpy()
    lengths = (fr.ranges[:, 1] - fr.ranges[:, 0]).cpu().numpy()
    assert sorted(wl.tolist()) == list(range(len(lengths)))
    assert np.all(np.diff(lengths[wl]) <= 0)


def test_batch_depth_does_not_change_the_image():
    sc = scenes.uniform_scene(6000, seed=6)
    cams = _views(2)
    ref = None
    for bd in (16, 64, 256):
        img = BT.forward_views(*R.scene_to_device(sc), cams, scenes.RenderConfig(batch_depth=bd)).image
        if ref is None:
            ref = img
        assert torch.equal(img, ref), bd


def test_ut_autotuner_and_worklist():
    sc = scenes.uniform_scene(20_000, seed=7, sh_degree=1)
    cams = _views(4)
    cfg = scenes.RenderConfig(sh_degree=1, method=1)
    P = list(R.scene_to_device(sc))
    best, table = BT.autotune(P, cams, cfg, scene_id="ut-test", reps=2, batches=(32, 256))
    assert best.method == 1 and len(table) == 4 and all(np.isfinite(v) for v in table.values())
    fr = BT.forward_views(*P, cams, best)
    ranges = fr.ranges.cpu().numpy()
    lens = ranges[:, 1] - ranges[:, 0]
    wl = fr.worklist.cpu().numpy()
    assert sorted(wl.tolist()) == list(range(len(lens))) and np.all(np.diff(lens[wl]) <= 0)


def test_autotuner_picks_a_candidate():
    sc = scenes.uniform_scene(3000, seed=7)
    cams = _views(2, 128, 96, 128.0)
    best, table = BT.autotune(R.scene_to_device(sc), cams, scenes.RenderConfig(), scene_id="t", reps=2,
                              batches=(32, 128))
    assert len(table) == 4 and all(v > 0 for v in table.values())
    assert (best.tile_w, best.tile_h, best.batch_depth) == min(table, key=table.get)
    assert BT.autotune(R.scene_to_device(sc), cams, scenes.RenderConfig(), scene_id="t", reps=2,
                       batches=(32, 128))[0] is best  # cached


def test_views_reject_mixed_sizes():
    sc = scenes.uniform_scene(100, seed=8)
    cams = [scenes.pinhole(64, 64, 64.0), scenes.pinhole(80, 64, 64.0)]
    with pytest.raises(ValueError):
        BT.forward_views(*R.scene_to_device(sc), cams, scenes.RenderConfig())
