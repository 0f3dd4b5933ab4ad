"""The multi-scene batched form: K (scene, camera) items with scenes of uneven size and cameras of
different image sizes, one launch per stage.  Per item it computes exactly the single-view path
(records, sorted lists, image, t_final, n_contrib bit for bit; gradients equal to the sum over
the items of each scene's single-view gradients), and one item matches the oracle."""
import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import batched as BT
from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import BAND_E2E, check_band, dev, rel_err

pytestmark = pytest.mark.gpu

NAMES = ["mu", "scale", "quat", "opacity", "sh"]


def _batch(deg=3):
    scs = [scenes.clustered_scene(n, seed=s, n_centers=20, width=W, height=H, focal=float(W), sh_degree=deg)
           for s, (n, W, H) in enumerate([(5003, 320, 180), (20_000, 256, 256), (1201, 200, 150)])]
    cams = [scenes.pinhole(320, 180, 320.0, scenes.yaw_view(2.0, (0.01, 0.0, 0.02))),
            scenes.pinhole(256, 256, 256.0),
            scenes.pinhole(200, 150, 200.0),
            scenes.pinhole(250, 170, 256.0, scenes.yaw_view(-4.0, (0.0, 0.02, 0.0))),  # scene 1 again, ragged
            scenes.pinhole(64, 48, 64.0)]
    scene_of_item = [0, 1, 2, 1, 0]
    return scs, cams, scene_of_item


@pytest.mark.parametrize("persistent,tile", [(True, 16), (False, 16), (True, 8)])
def test_items_equal_single_view_path(persistent, tile):
    scs, cams, soi = _batch()
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=3, bg=(0.1, 0.2, 0.3))
    dev_scenes = [R.scene_to_device(s) for s in scs]
    ss = BT.SceneSet(dev_scenes)
    layout = ss.layout(soi, cams, cfg)
    fr = BT.forward_items(*ss.params, layout, cfg, persistent=persistent)
    imgs = fr.images()
    tf, nc = layout.planes(fr.t_final), layout.planes(fr.n_contrib)
    for k, (s, cam) in enumerate(zip(soi, cams)):
        ref = R.forward_frame(*dev_scenes[s], cam, cfg)
        assert torch.equal(imgs[k], ref.image), k
        assert torch.equal(tf[k], ref.t_final), k
        assert torch.equal(nc[k], ref.n_contrib), k
        r0 = layout.rec_offsets[k]
        assert torch.equal(fr.rec[r0:r0 + ss.counts[s]], ref.rec), k
        t0, T = layout.tile_offsets[k], ref.ranges.shape[0]
        rg = fr.ranges[t0:t0 + T].to(torch.int64)
        for t in range(0, T, 7):  # each tile's list is the single-view list, renumbered
            a, b = int(rg[t, 0]), int(rg[t, 1])
            ra, rb = int(ref.ranges[t, 0]), int(ref.ranges[t, 1])
            assert b - a == rb - ra
            if b > a:
                assert torch.equal(fr.vals_sorted[a:b] - r0, ref.vals_sorted[ra:rb]), (k, t)


def test_items_gradients_are_the_sum_over_items():
    scs, cams, soi = _batch()
    cfg = scenes.RenderConfig(sh_degree=3, bg=(0.1, 0.2, 0.3))
    dev_scenes = [R.scene_to_device(s) for s in scs]
    ss = BT.SceneSet(dev_scenes)
    layout = ss.layout(soi, cams, cfg)
    P = [p.clone().requires_grad_(True) for p in ss.params]
    imgs = BT.render_items(*P, layout, cfg)
    rng = np.random.default_rng(3)
    ws = [dev(rng.normal(size=tuple(im.shape))) for im in imgs]
    sum(((im * w).sum() for im, w in zip(imgs, ws))).backward()
    ref = [torch.zeros_like(p) for p in ss.params]
    for k, (s, cam) in enumerate(zip(soi, cams)):
        Q = [t.clone().requires_grad_(True) for t in dev_scenes[s]]
        (R.render(*Q, cam, cfg) * ws[k]).sum().backward()
        o, n = ss.offsets[s], ss.counts[s]
        for a, q in zip(ref, Q):
            a[o:o + n] += q.grad
    for name, p, r in zip(NAMES, P, ref):
        assert rel_err(p.grad.cpu().numpy(), r.cpu().numpy()) < 1e-5, name


def test_items_against_oracle(oracle):
    scs, cams, soi = _batch()
    cfg = scenes.RenderConfig(sh_degree=3)
    dev_scenes = [R.scene_to_device(s) for s in scs]
    ss = BT.SceneSet(dev_scenes)
    layout = ss.layout(soi, cams, cfg)
    imgs = BT.forward_items(*ss.params, layout, cfg).images()
    for k in (1, 3):
        ref = oracle.pipeline_tiled(scs[soi[k]], cams[k], cfg, band=BAND_E2E)
        check_band(imgs[k].cpu().numpy(), ref, max_frac=1e-2, what=f"item {k}")


def test_items_at_serving_sizes():
    # the serving workload's smallest and largest scenes, requests of 512x512, 1920x1080 and 1280x720
    scs = scenes.serving_scenes(16, seed=0)
    sizes = [s.n for s in scs]
    small, large = int(np.argmin(sizes)), int(np.argmax(sizes))
    cfg = scenes.RenderConfig(sh_degree=3)
    dev_scenes = [R.scene_to_device(scs[i]) for i in (small, large)]
    ss = BT.SceneSet(dev_scenes)
    cams = [scenes.pinhole(1920, 1080, 1920.0, scenes.yaw_view(3.0)), scenes.pinhole(512, 512, 512.0),
            scenes.pinhole(1280, 720, 1280.0, scenes.yaw_view(-2.0, (0.02, 0.0, 0.0)))]
    soi = [1, 0, 1]
    layout = ss.layout(soi, cams, cfg)
    imgs = BT.forward_items(*ss.params, layout, cfg).images()
    for k, (s, cam) in enumerate(zip(soi, cams)):
        assert torch.equal(imgs[k], R.forward_frame(*dev_scenes[s], cam, cfg).image), k


def test_items_reject_inconsistent_offsets():
    scs, cams, soi = _batch()
    cfg = scenes.RenderConfig(sh_degree=3)
    ss = BT.SceneSet([R.scene_to_device(s) for s in scs])
    layout = ss.layout(soi, cams, cfg)
    layout.arr[2].tile_offset += 1
    with pytest.raises(B.XprError) as e:
        B.xpr_project_items(*ss.params, layout, B.make_config(cfg))
    assert e.value.status == B.XPR_ERR_INVALID


def test_native_forward_equals_staged_calls():
    # xpr_forward_items (one call, every intermediate in one workspace) gives the staged path's
    # outputs bit for bit, including after a capacity retry
    scs, cams, soi = _batch()
    cfg = scenes.RenderConfig(sh_degree=3, bg=(0.3, 0.2, 0.1))
    ss = BT.SceneSet([R.scene_to_device(s) for s in scs])
    layout = ss.layout(soi, cams, cfg)
    ref = BT.forward_items(*ss.params, layout, cfg)
    for cap in (ref.n_isect + 7, 16):
        img, tf, nc, I, ws = B.xpr_forward_items(*ss.params, layout, B.make_config(cfg), cap)
        assert I == ref.n_isect
        assert torch.equal(img, ref.image) and torch.equal(tf, ref.t_final) and torch.equal(nc, ref.n_contrib)
