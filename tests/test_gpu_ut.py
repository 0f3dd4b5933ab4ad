"""Parity of the 3DGUT CUDA path (unscented projection, ray-offset binning, ray-evaluated
compositing and the adjoints) with the FP64 oracle, through the C ABI.

Both sides get the same inputs: the scene, and for the compositing stages the GPU's own tile lists
(the ray-offset cull decides them in FP32; the oracle checks those decisions bit for bit on the
GPU's float32 records).  Primitives whose visibility is decided within a relative 1e-3 of the
opacity threshold are removed from the scenes (there both answers are right)."""
import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import (BAND, GRAD_TOL, IMG_TOL, assert_same_tile_lists, check_band, dev, dev_i32, near_integer_bbox,
                      oracle_lists, rel_err)

pytestmark = pytest.mark.gpu

A_T = float(np.float32(1 / 255))


def _ut_case(oracle, deg=0, tile=16, view=False, n=8000, W=256, H=256, seed=0, big_every=0, fish=False):
    sc = scenes.uniform_scene(n, seed=seed, sh_degree=deg)
    if big_every:
        sc.scale[::big_every] *= 12.0
    vm = scenes.yaw_view(4.0, (0.05, -0.02, 0.1)) if view else None
    # the fisheye sees the same scene with a wider field (focal W/2, radial terms of the workload)
    cam = scenes.fisheye(W, H, W / 2.0, viewmat=vm) if fish else scenes.pinhole(W, H, float(W), vm)
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=deg, method=1)
    pr = oracle.project_ut(*sc.arrays(), cam, cfg)
    o = pr["sd"][:, 12]
    keep = ~((np.abs(o / A_T - 1.0) < 1e-3) & (o > 0))
    if not keep.all():
        sc = sc.subset(np.nonzero(keep)[0])
        pr = oracle.project_ut(*sc.arrays(), cam, cfg)
    return sc, cam, cfg, pr


def _oracle_sd_in_kernel_form(pr, sc, cam):
    """The kernels' shader-data layout computed from the oracle's FP64 quantities."""
    V = np.asarray(cam.viewmat, np.float64)
    W3, t = V[:, :3], V[:, 3]
    mc = sc.mu.astype(np.float64) @ W3.T + t
    M = pr["sd"][:, 3:12].reshape(-1, 3, 3)
    Mc = M @ W3.T
    z = mc[:, 2]
    out = np.zeros((sc.n, 16))
    if getattr(cam, "model", 0) == 1:  # fisheye: normalised image coordinates
        fx = fy = 1.0
        cx = cy = 0.0
    else:
        fx, fy, cx, cy = cam.fx, cam.fy, cam.cx, cam.cy
    out[:, 0] = fx * mc[:, 0] / z + cx
    out[:, 1] = fy * mc[:, 1] / z + cy
    out[:, 2:5] = (z / fx)[:, None] * Mc[:, :, 0]
    out[:, 5:8] = (z / fy)[:, None] * Mc[:, :, 1]
    out[:, 8:11] = pr["sd"][:, 0:3]
    out[:, 11] = pr["sd"][:, 12]
    out[:, 12:15] = pr["sd"][:, 13:16]
    out[:, 15] = np.sum(pr["sd"][:, 0:3] ** 2, 1)
    return out


@pytest.mark.parametrize("deg,tile,view,fish", [(0, 16, False, False), (3, 8, True, False), (1, 16, True, False),
                                                (0, 16, False, True), (3, 8, True, True)])
def test_ut_project_matches_oracle(oracle, deg, tile, view, fish):
    sc, cam, cfg, pr = _ut_case(oracle, deg, tile, view, fish=fish)
    rec, sd, bbox, tc, cnt = B.xpr_project_ut(*R.scene_to_device(sc), cam, cfg)
    torch.cuda.synchronize()
    rec, sd, bbox, tc, cnt = (x.cpu().numpy() for x in (rec, sd, bbox, tc, cnt))
    ref = pr["rec"]
    amb = near_integer_bbox(pr["pre"])
    vis_o, vis_g = ref[:, 11] > 0, rec[:, 11] > 0
    assert np.all((vis_o == vis_g) | amb)
    both = vis_o & vis_g
    assert both.sum() > 1000
    np.testing.assert_allclose(rec[both, 0:2], ref[both, 0:2], rtol=1e-5, atol=2e-3)
    scale = np.maximum(np.abs(ref[both, 2]), np.abs(ref[both, 4]))[:, None]
    assert np.max(np.abs(rec[both, 2:5] - ref[both, 2:5]) / scale) < 2e-4
    np.testing.assert_allclose(rec[both, 5], ref[both, 5], rtol=2e-5)
    np.testing.assert_allclose(rec[both, 6:9], ref[both, 6:9], atol=2e-5)
    np.testing.assert_allclose(rec[:, 9], ref[:, 9], rtol=2e-6, atol=1e-6)
    np.testing.assert_allclose(rec[both, 10], ref[both, 10], atol=5e-5)
    exact = both & ~amb
    np.testing.assert_array_equal(bbox[exact], pr["bbox"][exact])
    np.testing.assert_array_equal(tc[exact], pr["tc"][exact])
    assert np.all(rec[~vis_g][:, [0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 11]] == 0) and np.all(tc[~vis_g] == 0)
    # shader data against the oracle's quantities in the kernels' form
    want = _oracle_sd_in_kernel_form(pr, sc, cam)
    np.testing.assert_allclose(sd[both, 0:2], want[both, 0:2], rtol=1e-5, atol=2e-3 if not fish else 2e-6)
    for lo, hi in [(2, 5), (5, 8), (8, 11)]:
        err = np.linalg.norm(sd[both, lo:hi] - want[both, lo:hi], axis=1) / np.linalg.norm(want[both, lo:hi], axis=1)
        assert err.max() < 1e-4, (lo, err.max())
    np.testing.assert_allclose(sd[both, 11], want[both, 11], rtol=2e-5)
    np.testing.assert_allclose(sd[both, 12:15], want[both, 12:15], atol=2e-5)
    np.testing.assert_allclose(sd[both, 15], want[both, 15], rtol=1e-4)
    # kept-tile counts: the oracle's ray-offset cull in exact FP32 on the GPU's own records
    counts, *_ = oracle_lists(oracle, rec.astype(np.float32), bbox, cam, cfg)
    np.testing.assert_array_equal(cnt, counts)


@pytest.mark.parametrize("tile,W,H,fish", [(16, 250, 170, False), (8, 250, 170, False), (16, 256, 256, False),
                                           (16, 250, 170, True)])
def test_ut_tile_lists_bit_exact(oracle, tile, W, H, fish):
    sc, cam, cfg, pr = _ut_case(oracle, 0, tile, n=12_345, W=W, H=H, big_every=97, fish=fish)
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    torch.cuda.synchronize()
    rec32 = fr.rec.cpu().numpy()
    _, _, _, sk, sv, ranges = oracle_lists(oracle, rec32, fr.bbox.cpu().numpy(), cam, cfg)
    assert fr.n_isect == len(sv) and len(sv) > 10_000
    assert_same_tile_lists(fr.vals_sorted, fr.ranges, sv.astype(np.int64), ranges)
    # the offset matters: the 3DGS cull keeps a different set on the same records
    cfg0 = scenes.RenderConfig(tile_w=tile, tile_h=tile, method=0)
    c0, *_ = oracle_lists(oracle, rec32, fr.bbox.cpu().numpy(), cam, cfg0)
    assert c0.sum() != len(sv)


def _gpu_frame(sc, cam, cfg):
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    torch.cuda.synchronize()
    return fr, fr.vals_sorted.cpu().numpy().view(np.uint32), fr.ranges.cpu().numpy()


@pytest.mark.parametrize("tile,W,H,bg,deg,fish", [(16, 256, 256, (0, 0, 0), 0, False),
                                                  (8, 250, 170, (0.2, 0.5, 1.0), 3, False),
                                                  (16, 200, 120, (1, 1, 1), 1, False),
                                                  (16, 256, 256, (0, 0, 0), 0, True),
                                                  (8, 250, 170, (0.2, 0.5, 1.0), 3, True)])
def test_ut_render_fwd_matches_oracle(oracle, tile, W, H, bg, deg, fish):
    sc, cam, cfg, pr = _ut_case(oracle, deg, tile, W=W, H=H, view=deg > 0, fish=fish)
    cfg.bg = bg
    fr, sv, ranges = _gpu_frame(sc, cam, cfg)
    ref = oracle.render_tiles_ut(pr["rec"], pr["sd"], sv, ranges, cam, cfg, delta=BAND)
    img, tf, nc = fr.image.cpu().numpy(), fr.t_final.cpu().numpy(), fr.n_contrib.cpu().numpy()
    ok = check_band(img, ref, max_frac=1e-2, what=f"3DGUT fwd {W}x{H}")
    assert np.abs(tf[ok] - ref["t_final"][ok]).max() <= IMG_TOL
    assert (nc[ok] != ref["n_contrib"][ok]).mean() <= 1e-3
    assert (ref["t_final"] < 0.01).mean() > 0.02  # saturated pixels: early termination exercised


@pytest.mark.parametrize("deg,view,tile,fish", [(0, False, 16, False), (3, True, 8, False), (1, True, 16, True)])
def test_ut_gradients_match_oracle(oracle, deg, view, tile, fish):
    sc, cam, cfg, pr = _ut_case(oracle, deg, tile, view, n=6000, fish=fish)
    cfg.bg = (0.3, 0.1, 0.6)
    fr, sv, ranges = _gpu_frame(sc, cam, cfg)
    ref = oracle.render_tiles_ut(pr["rec"], pr["sd"], sv, ranges, cam, cfg, delta=BAND)
    w = np.random.default_rng(5).normal(size=(3, cam.height, cam.width)) * ~ref["gband"][None]
    d_sd_ref = oracle.render_bwd_tiles_ut(pr["sd"], sv, ranges, cam, cfg, w)
    g_ref = oracle.project_ut_bwd(*sc.arrays(), cam, cfg, d_sd_ref)
    d_sd = B.xpr_render_ut_bwd(fr.sd, fr.vals_sorted, fr.ranges, cam, cfg, fr.t_final, fr.n_contrib, dev(w))
    got = B.xpr_project_ut_bwd(*R.scene_to_device(sc), cam, cfg, d_sd)
    for name, g in zip(["mu", "scale", "quat", "opacity", "sh"], got):
        assert rel_err(g.cpu().numpy(), g_ref[name]) < GRAD_TOL, name
    assert np.all(d_sd.cpu().numpy()[:, 15] == 0)


def test_ut_autograd_matches_direct_calls():
    sc = scenes.uniform_scene(3000, seed=2, sh_degree=1)
    cam = scenes.pinhole(128, 96, 128.0)
    cfg = scenes.RenderConfig(sh_degree=1, method=1)
    params = [t.clone().requires_grad_(True) for t in R.scene_to_device(sc)]
    img = R.render(*params, cam, cfg)
    w = torch.randn_like(img)
    (img * w).sum().backward()
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    assert torch.equal(fr.image, img.detach())
    d_sd = B.xpr_render_ut_bwd(fr.sd, fr.vals_sorted, fr.ranges, cam, cfg, fr.t_final, fr.n_contrib, w)
    direct = B.xpr_project_ut_bwd(*R.scene_to_device(sc), cam, cfg, d_sd)
    for p, g in zip(params, direct):
        assert torch.isfinite(p.grad).all()
        assert rel_err(p.grad.cpu().numpy(), g.cpu().numpy()) < 1e-5


def test_fisheye_needs_3dgut():
    sc = scenes.uniform_scene(100, seed=1)
    t = R.scene_to_device(sc)
    cam = scenes.fisheye(64, 64, 32.0)
    with pytest.raises(B.XprError):  # the EWA projection linearises a pinhole
        B.xpr_project(*t, cam, scenes.RenderConfig(method=0))
    B.xpr_project_ut(*t, cam, scenes.RenderConfig(method=1))


def test_ut_method_is_checked():
    sc = scenes.uniform_scene(100, seed=1)
    cam = scenes.pinhole(64, 64, 64.0)
    ut = scenes.RenderConfig(method=1)
    gs = scenes.RenderConfig(method=0)
    t = R.scene_to_device(sc)
    with pytest.raises(B.XprError):
        B.xpr_project(*t, cam, ut)
    with pytest.raises(B.XprError):
        B.xpr_project_ut(*t, cam, gs)
    bad = scenes.RenderConfig(method=2)
    with pytest.raises(B.XprError):
        B.xpr_project_ut(*t, cam, bad)


def test_ut_empty_and_all_invisible():
    cam = scenes.pinhole(64, 48, 64.0)
    cfg = scenes.RenderConfig(method=1, bg=(0.25, 0.5, 0.75))
    sc = scenes.uniform_scene(50, seed=3)
    sc.mu[:, 2] = -3.0  # behind the camera
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    img = fr.image.cpu().numpy()
    assert fr.n_isect == 0
    np.testing.assert_array_equal(img, np.broadcast_to(np.array([0.25, 0.5, 0.75], np.float32)[:, None, None],
                                                       img.shape))
    empty = [torch.empty((0,) + tuple(x.shape[1:]), device="cuda") for x in R.scene_to_device(sc)]
    fr = R.forward_frame(*empty, cam, cfg)
    assert fr.n_isect == 0 and torch.all(fr.t_final == 1)


def test_ut_headline_workload_sampled_tiles(oracle):
    """1M SH-3 Gaussians, 1920x1080, 16x16 tiles with the 3DGUT path (the benchmarked launch
    configuration): the pixels of sampled tiles against the oracle walking the GPU's lists for those
    tiles, and the gradients of a loss on those pixels."""
    import dataclasses
    sc, cam, cfg = scenes.headline_case()
    cfg = dataclasses.replace(cfg, method=1)
    pr = oracle.project_ut(*sc.arrays(), cam, cfg)
    o = pr["sd"][:, 12]
    keep = ~((np.abs(o / A_T - 1.0) < 1e-3) & (o > 0))
    sc = sc.subset(np.nonzero(keep)[0])
    pr = oracle.project_ut(*sc.arrays(), cam, cfg)
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
    ref = oracle.render_tiles_ut(pr["rec"], pr["sd"], sv, sub, cam, cfg, delta=BAND)
    Wt = (cam.width + 15) // 16
    mask = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        ty, tx = divmod(int(t), Wt)
        mask[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    got = fr.image.cpu().numpy()
    ok = check_band(got, ref, mask=mask, max_frac=3e-2, what="3DGUT 1M / 1080p sampled tiles")
    ok &= ~ref["gband"]
    assert (ref["t_final"][ok] < 0.5).mean() > 0.2  # sampled tiles are not mostly empty
    w = rng.normal(size=(3, cam.height, cam.width)) * ok[None]
    (img * dev(w)).sum().backward()
    d_sd = oracle.render_bwd_tiles_ut(pr["sd"], sv, sub, cam, cfg, w)
    g = oracle.project_ut_bwd(*sc.arrays(), cam, cfg, d_sd)
    for name, p in zip(["mu", "scale", "quat", "opacity", "sh"], P):
        assert rel_err(p.grad.cpu().numpy(), g[name]) < GRAD_TOL, name
