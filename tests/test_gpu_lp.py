"""Parity of the LinPrim CUDA path (octahedron projection, chord-bound binning, slab-intersection
compositing and the adjoints) with the FP64 oracle, through the C ABI.  The compositing stages get
the GPU's own tile lists on both sides (the oracle checks those lists bit for bit with its mirror of
the FP32 cull on the GPU's shader data).  Images and loss weights exclude, besides the gate
ambiguity band, the pixels the oracle finds ill-conditioned at float32 scale
(oracle.condition_band_lp: silhouettes of faces seen almost edge-on)."""
import math

import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import BAND, GRAD_TOL, IMG_TOL, dev, near_integer_bbox, rel_err

pytestmark = pytest.mark.gpu

A_T = float(np.float32(1 / 255))
SIGNS = ((1, 1), (1, -1), (-1, 1), (-1, -1))


def _lp_case(deg=0, tile=16, view=False, n=6000, W=256, H=256, seed=0, big_every=0):
    sc = scenes.uniform_scene(n, seed=seed, sh_degree=deg)
    if big_every:
        sc.scale[::big_every] *= 6.0
    vm = scenes.yaw_view(4.0, (0.05, -0.02, 0.1)) if view else None
    cam = scenes.pinhole(W, H, float(W), vm)
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=deg, method=2)
    return sc, cam, cfg


def _oracle_lists(oracle, fr, cam, cfg):
    rec32 = fr.rec.cpu().numpy()
    sd32 = fr.sd.cpu().numpy()
    Wt, Ht = oracle.tiles_of(cam, cfg)
    counts, keys, vals = oracle.bin_pairs_lp(rec32, sd32, fr.bbox.cpu().numpy(), cam, cfg, exact32=True)
    sk, sv, ranges = oracle.sort_pairs(keys, vals, Wt * Ht)
    return counts, sv, ranges


@pytest.mark.parametrize("deg,tile,view", [(0, 16, False), (3, 8, True), (1, 16, True)])
def test_lp_project_matches_oracle(oracle, deg, tile, view):
    sc, cam, cfg = _lp_case(deg, tile, view, big_every=37)
    pr = oracle.project_lp(*sc.arrays(), cam, cfg)
    rec, sd, bbox, tc, cnt = B.xpr_project_lp(*R.scene_to_device(sc), cam, cfg)
    torch.cuda.synchronize()
    rec, sd, bbox, tc, cnt = (x.cpu().numpy() for x in (rec, sd, bbox, tc, cnt))
    ref = pr["rec"]
    amb = near_integer_bbox(pr["pre"])
    vis_o, vis_g = ref[:, 11] > 0, rec[:, 11] > 0
    assert np.all((vis_o == vis_g) | amb)
    both = vis_o & vis_g
    assert both.sum() > 1000
    np.testing.assert_allclose(rec[both, 0:2], ref[both, 0:2], rtol=1e-5, atol=2e-3)
    np.testing.assert_allclose(rec[both, 6:9], ref[both, 6:9], atol=2e-5)
    np.testing.assert_allclose(rec[:, 9], ref[:, 9], rtol=2e-6, atol=1e-6)
    exact = both & ~amb
    np.testing.assert_array_equal(bbox[exact], pr["bbox"][exact])
    np.testing.assert_array_equal(tc[exact], pr["tc"][exact])
    assert np.all(tc[~vis_g] == 0) and np.all(sd[~vis_g] == 0)
    # shader data: the oracle's slabs in the kernels' (p, q, h) form
    S = pr["sd"][both]
    np.testing.assert_allclose(sd[both, 0:2], S[:, 0:2], rtol=1e-5, atol=2e-3)
    np.testing.assert_allclose(sd[both, 2], S[:, 11], rtol=2e-5)
    assert np.all(sd[:, 3][both] == np.float32(sd[both, 3][0]))
    assert sd[both, 3][0] == pytest.approx(-math.log1p(-A_T), rel=1e-6)
    for i, (a, b) in enumerate(SIGNS):
        nv = S[:, 2:5] + a * S[:, 5:8] + b * S[:, 8:11]
        want = np.stack([nv[:, 0] / nv[:, 2], nv[:, 1] / nv[:, 2], 1 / np.abs(nv[:, 2])], 1)
        got = sd[both, 4 + 3 * i:7 + 3 * i]
        scale = np.abs(want).max(1)
        # n = c0 +- c1 +- c2 cancels for a face seen nearly edge-on; the float32 slab data then carry
        # the cancellation factor kappa in their relative error (and such a slab does not bind)
        kappa = (np.abs(S[:, 4]) + np.abs(S[:, 7]) + np.abs(S[:, 10])) / np.abs(nv[:, 2])
        assert np.all(np.abs(got - want).max(1) / scale < 2e-4 + 4e-6 * kappa), i
    np.testing.assert_allclose(sd[both, 16:19], S[:, 12:15], atol=2e-5)
    # kept-tile counts: the oracle's mirror of the FP32 cull on the GPU's shader data
    counts, _, _ = oracle.bin_pairs_lp(rec, sd, bbox, cam, cfg, exact32=True)
    np.testing.assert_array_equal(cnt, counts)


@pytest.mark.parametrize("tile,W,H", [(16, 250, 170), (8, 250, 170), (16, 256, 256)])
def test_lp_tile_lists_bit_exact(oracle, tile, W, H):
    sc, cam, cfg = _lp_case(0, tile, n=12_345, W=W, H=H, big_every=53)
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    torch.cuda.synchronize()
    _, sv, ranges = _oracle_lists(oracle, fr, cam, cfg)
    assert fr.n_isect == len(sv) and len(sv) > 5_000
    np.testing.assert_array_equal(fr.vals_sorted.cpu().numpy().view(np.uint32), sv)
    np.testing.assert_array_equal(fr.ranges.cpu().numpy(), ranges)
    # the cull removes pairs from the boxes
    assert len(sv) < fr.tile_count.sum().item()


def _gpu_frame(sc, cam, cfg):
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    torch.cuda.synchronize()
    return fr, fr.vals_sorted.cpu().numpy().view(np.uint32), fr.ranges.cpu().numpy()


@pytest.mark.parametrize("tile,W,H,bg,deg", [(16, 256, 256, (0, 0, 0), 0), (8, 250, 170, (0.2, 0.5, 1.0), 3),
                                             (16, 200, 120, (1, 1, 1), 1)])
def test_lp_render_fwd_matches_oracle(oracle, tile, W, H, bg, deg):
    sc, cam, cfg = _lp_case(deg, tile, W=W, H=H, view=deg > 0, n=8000)
    sc.scale *= 2.0
    cfg.bg = bg
    fr, sv, ranges = _gpu_frame(sc, cam, cfg)
    pr = oracle.project_lp(*sc.arrays(), cam, cfg)
    ref = oracle.render_tiles_lp(pr["sd"], sv, ranges, cam, cfg, delta=BAND)
    cond = oracle.condition_band_lp(pr["sd"], sv, ranges, cam, cfg)
    img, tf, nc = fr.image.cpu().numpy(), fr.t_final.cpu().numpy(), fr.n_contrib.cpu().numpy()
    ok = ~ref["gband"] & ~cond
    assert ok.mean() > 0.95
    assert np.abs(img[:, ok] - ref["image"][:, ok]).max() <= IMG_TOL
    assert np.abs(tf[ok] - ref["t_final"][ok]).max() <= IMG_TOL
    assert (nc[ok] != ref["n_contrib"][ok]).mean() <= 1e-3
    assert (ref["t_final"] < 0.05).mean() > 0.01


@pytest.mark.parametrize("deg,view,tile", [(0, False, 16), (3, True, 8)])
def test_lp_gradients_match_oracle(oracle, deg, view, tile):
    sc, cam, cfg = _lp_case(deg, tile, view, n=5000)
    sc.scale *= 2.0
    cfg.bg = (0.3, 0.1, 0.6)
    fr, sv, ranges = _gpu_frame(sc, cam, cfg)
    pr = oracle.project_lp(*sc.arrays(), cam, cfg)
    ref = oracle.render_tiles_lp(pr["sd"], sv, ranges, cam, cfg, delta=BAND)
    ok = ~ref["gband"] & ~oracle.condition_band_lp(pr["sd"], sv, ranges, cam, cfg)
    assert ok.mean() > 0.95
    w = np.random.default_rng(5).normal(size=(3, cam.height, cam.width)) * ok[None]
    d_sd_ref = oracle.render_bwd_tiles_lp(pr["sd"], sv, ranges, cam, cfg, w)
    g_ref = oracle.project_lp_bwd(*sc.arrays(), cam, cfg, d_sd_ref)
    d_sd = B.xpr_render_lp_bwd(fr.sd, fr.vals_sorted, fr.ranges, cam, cfg, fr.t_final, fr.n_contrib, dev(w))
    got = B.xpr_project_lp_bwd(*R.scene_to_device(sc), cam, cfg, d_sd)
    for name, g in zip(["mu", "scale", "quat", "opacity", "sh"], got):
        assert rel_err(g.cpu().numpy(), g_ref[name]) < GRAD_TOL, name
    d = d_sd.cpu().numpy()
    assert np.all(d[:, 3] == 0) and np.all(d[:, 19] == 0)


def test_lp_autograd_matches_direct_calls():
    sc = scenes.uniform_scene(3000, seed=2, sh_degree=1)
    sc.scale *= 2.0
    cam = scenes.pinhole(128, 96, 128.0)
    cfg = scenes.RenderConfig(sh_degree=1, method=2)
    params = [t.clone().requires_grad_(True) for t in R.scene_to_device(sc)]
    img = R.render(*params, cam, cfg)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    assert torch.equal(fr.image, img.detach())
    d_sd = B.xpr_render_lp_bwd(fr.sd, fr.vals_sorted, fr.ranges, cam, cfg, fr.t_final, fr.n_contrib, w)
    direct = B.xpr_project_lp_bwd(*R.scene_to_device(sc), cam, cfg, d_sd)
    for p, g in zip(params, direct):
        assert torch.isfinite(p.grad).all()
        assert rel_err(p.grad.cpu().numpy(), g.cpu().numpy()) < 1e-5


def test_lp_method_is_checked():
    sc = scenes.uniform_scene(100, seed=1)
    cam = scenes.pinhole(64, 64, 64.0)
    t = R.scene_to_device(sc)
    with pytest.raises(B.XprError):
        B.xpr_project_lp(*t, cam, scenes.RenderConfig(method=0))
    rec, sd, bbox, tc, cnt = B.xpr_project_lp(*t, cam, scenes.RenderConfig(method=2))
    with pytest.raises(B.XprError):  # LinPrim records cannot be binned without their shader data
        B.xpr_tile_bin(rec, bbox, tc, cam, scenes.RenderConfig(method=2))


def test_lp_empty_and_all_invisible():
    cam = scenes.pinhole(64, 48, 64.0)
    cfg = scenes.RenderConfig(method=2, bg=(0.25, 0.5, 0.75))
    sc = scenes.uniform_scene(50, seed=3)
    sc.mu[:, 2] = -3.0
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    img = fr.image.cpu().numpy()
    assert fr.n_isect == 0
    np.testing.assert_array_equal(img, np.broadcast_to(np.array([0.25, 0.5, 0.75], np.float32)[:, None, None],
                                                       img.shape))
    empty = [torch.empty((0,) + tuple(x.shape[1:]), device="cuda") for x in R.scene_to_device(sc)]
    fr = R.forward_frame(*empty, cam, cfg)
    assert fr.n_isect == 0 and torch.all(fr.t_final == 1)


def test_lp_full_size_sampled_tiles(oracle):
    """500k octahedra (log half-extents N(-3, 0.5)), 1280x720 pinhole f=1280, 16x16 tiles (the
    benchmarked LinPrim configuration): sampled tiles' pixels and the gradients of a loss on them."""
    sc, cam, cfg = scenes.linprim_case()
    P = [t.clone().requires_grad_(True) for t in R.scene_to_device(sc)]
    fr = R.forward_frame(*[p.detach() for p in P], cam, cfg)
    img = R.render(*P, cam, cfg)
    torch.cuda.synchronize()
    assert torch.equal(img.detach(), fr.image)
    ranges = fr.ranges.cpu().numpy()
    sv = fr.vals_sorted.cpu().numpy().view(np.uint32)
    lengths = ranges[:, 1] - ranges[:, 0]
    rng = np.random.default_rng(0)
    busy = np.nonzero(lengths > np.percentile(lengths, 50))[0]
    tiles = np.concatenate([rng.choice(busy, 20, replace=False), rng.choice(len(lengths), 4, replace=False)])
    sub = np.zeros_like(ranges)
    sub[tiles] = ranges[tiles]
    pr = oracle.project_lp(*sc.arrays(), cam, cfg)
    ref = oracle.render_tiles_lp(pr["sd"], sv, sub, cam, cfg, delta=BAND)
    cond = oracle.condition_band_lp(pr["sd"], sv, sub, cam, cfg)
    Wt = (cam.width + 15) // 16
    mask = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        ty, tx = divmod(int(t), Wt)
        mask[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    ok = mask & ~ref["gband"] & ~cond
    assert ok.sum() > 0.9 * mask.sum()
    got = fr.image.cpu().numpy()
    assert np.abs(got[:, ok] - ref["image"][:, ok]).max() <= IMG_TOL
    assert (ref["t_final"][ok] < 0.5).mean() > 0.2
    w = rng.normal(size=(3, cam.height, cam.width)) * ok[None]
    (img * dev(w)).sum().backward()
    d_sd = oracle.render_bwd_tiles_lp(pr["sd"], sv, sub, cam, cfg, w)
    g = oracle.project_lp_bwd(*sc.arrays(), cam, cfg, d_sd)
    for name, p in zip(["mu", "scale", "quat", "opacity", "sh"], P):
        assert rel_err(p.grad.cpu().numpy(), g[name]) < GRAD_TOL, name
