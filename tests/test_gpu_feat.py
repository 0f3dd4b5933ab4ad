"""Rendered features on the GPU (3DGS compositing with extra channels: semantics rows and expected
depth) against the FP64 oracle, through the C ABI and the autograd function."""
import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import BAND_E2E, BAND_STAGE, GRAD_TOL, IMG_TOL, dev, dev_i32, oracle_lists, rel_err

pytestmark = pytest.mark.gpu


def _case(tile=16, n=8000, W=256, H=256, deg=1, seed=0):
    sc = scenes.uniform_scene(n, seed=seed, sh_degree=deg)
    cam = scenes.pinhole(W, H, float(W), scenes.yaw_view(3.0, (0.02, 0.0, 0.05)))
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=deg, bg=(0.2, 0.3, 0.4))
    return sc, cam, cfg


@pytest.mark.parametrize("nfeat,depth,tile", [(0, True, 16), (3, True, 8), (8, False, 16), (15, True, 16),
                                              (2, False, 8), (10, True, 8), (12, False, 16)])
def test_features_match_oracle(oracle, nfeat, depth, tile):
    sc, cam, cfg = _case(tile, W=250, H=170)
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    *_, sv, ranges = oracle_lists(oracle, rec32, pr["bbox"], cam, cfg)
    feat = np.random.default_rng(nfeat).normal(size=(sc.n, nfeat)).astype(np.float32) if nfeat else None
    ref = oracle.render_tiles_feat(rec32, feat, sv, ranges, cam, cfg, with_depth=depth)
    band = oracle.render_tiles(rec32.astype(np.float64), sv, ranges, cam, cfg, band=BAND_STAGE)["gband"]
    rec_d, sv_d, rg_d = dev(rec32), dev_i32(sv), dev_i32(ranges)
    img, feats, tf, nc = B.xpr_render_fwd_feat(rec_d, None if feat is None else dev(feat), sv_d, rg_d, cam, cfg,
                                               with_depth=depth)
    img0, _, _ = B.xpr_render_fwd(rec_d, sv_d, rg_d, cam, cfg)
    assert torch.equal(img, img0)  # the colour is the plain compositing, bit for bit
    ok = ~band
    assert band.mean() <= 3e-3  # decisions within the float32 precision of the walk itself
    got = feats.cpu().numpy()
    assert got.shape[0] == nfeat + int(depth)
    for c in range(got.shape[0]):
        scale = max(1.0, np.abs(ref["features"][c]).max())
        assert np.abs(got[c][ok] - ref["features"][c][ok]).max() <= IMG_TOL * scale, c
    # gradients of an image + feature loss
    wi = np.random.default_rng(1).normal(size=(3, cam.height, cam.width)) * ok[None]
    wf = np.random.default_rng(2).normal(size=got.shape) * ok[None]
    d_rec_ref, d_feat_ref = oracle.render_bwd_tiles_feat(rec32, feat, sv, ranges, cam, cfg, wi, wf, with_depth=depth)
    d_rec, d_feat = B.xpr_render_bwd_feat(rec_d, None if feat is None else dev(feat), sv_d, rg_d, cam, cfg, tf, nc,
                                          dev(wi), dev(wf), with_depth=depth)
    d_rec = d_rec.cpu().numpy()
    for j, name in enumerate(["dmx", "dmy", "dc00", "dc01", "dc11", "do", "dr", "dg", "db", "ddepth"]):
        if name == "ddepth" and not depth:
            assert np.all(d_rec[:, 9] == 0)
            continue
        assert rel_err(d_rec[:, j], d_rec_ref[:, j]) < GRAD_TOL, name
    if nfeat:
        assert rel_err(d_feat.cpu().numpy(), d_feat_ref) < GRAD_TOL


def test_feature_autograd_against_oracle(oracle):
    sc, cam, cfg = _case(16, n=5000, W=200, H=136, deg=3)
    feat = np.random.default_rng(3).normal(size=(sc.n, 4)).astype(np.float32)
    P = [t.clone().requires_grad_(True) for t in R.scene_to_device(sc)]
    f = dev(feat).requires_grad_(True)
    img, feats = R.render_features(*P, f, cam, cfg, with_depth=True)
    pr = oracle.project_scene(sc, cam, cfg)
    ref_img = oracle.render_tiles(pr["rec"], *oracle_lists(oracle, pr["rec"].astype(np.float32), pr["bbox"], cam,
                                                           cfg)[4:], cam, cfg, band=BAND_E2E, unc=pr["unc"])
    ok = ~ref_img["gband"]
    wi = np.random.default_rng(4).normal(size=(3, cam.height, cam.width)) * ok[None]
    wf = np.random.default_rng(5).normal(size=(5, cam.height, cam.width)) * ok[None]
    ((img * dev(wi)).sum() + (feats * dev(wf)).sum()).backward()
    g = oracle.grads_tiled_feat(sc.arrays(), feat, cam, cfg, wi, wf, with_depth=True)
    for name, p in zip(["mu", "scale", "quat", "opacity", "sh"], P):
        assert rel_err(p.grad.cpu().numpy(), g[name]) < GRAD_TOL, name
    assert rel_err(f.grad.cpu().numpy(), g["feat"]) < GRAD_TOL
    # the depth channel reaches the means: its gradient alone is non-zero on mu
    for p in P:
        p.grad = None
    img, feats = R.render_features(*P, None, cam, cfg, with_depth=True)
    feats.sum().backward()
    assert P[0].grad.abs().max() > 0 and torch.isfinite(P[0].grad).all()


def test_features_checked():
    sc, cam, cfg = _case(16, n=100, W=64, H=64)
    rec, bbox, tc = B.xpr_project(*R.scene_to_device(sc), cam, cfg)
    with pytest.raises(B.XprError):  # no channel at all
        B.xpr_render_fwd_feat(rec, None, torch.zeros(1, dtype=torch.int32, device="cuda"),
                              torch.zeros((16, 2), dtype=torch.int32, device="cuda"), cam, cfg, with_depth=False)
    big = torch.zeros((sc.n, 17), dtype=torch.float32, device="cuda")
    with pytest.raises(B.XprError):  # more than 16 channels
        B.xpr_render_fwd_feat(rec, big, torch.zeros(1, dtype=torch.int32, device="cuda"),
                              torch.zeros((16, 2), dtype=torch.int32, device="cuda"), cam, cfg)


def test_features_headline_sampled_tiles(oracle):
    """1M SH-3 Gaussians, 1920x1080, 16x16 tiles, 8 semantic channels and depth: sampled tiles."""
    sc, cam, cfg = scenes.headline_case()
    feat = np.random.default_rng(7).normal(size=(sc.n, 8)).astype(np.float32)
    P = R.scene_to_device(sc)
    fr = R.forward_frame(*P, cam, cfg, render=False)
    img, feats, tf, nc = B.xpr_render_fwd_feat(fr.rec, dev(feat), fr.vals_sorted, fr.ranges, cam, cfg,
                                               with_depth=True)
    torch.cuda.synchronize()
    ranges = fr.ranges.cpu().numpy()
    sv = fr.vals_sorted.cpu().numpy().view(np.uint32)
    lengths = ranges[:, 1] - ranges[:, 0]
    rng = np.random.default_rng(0)
    busy = np.nonzero(lengths > np.percentile(lengths, 50))[0]
    tiles = rng.choice(busy, 16, replace=False)
    sub = np.zeros_like(ranges)
    sub[tiles] = ranges[tiles]
    rec32 = fr.rec.cpu().numpy()
    ref = oracle.render_tiles_feat(rec32, feat, sv, sub, cam, cfg, with_depth=True)
    band = oracle.render_tiles(rec32.astype(np.float64), sv, sub, cam, cfg, band=BAND_STAGE)["gband"]
    Wt = (cam.width + 15) // 16
    mask = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        ty, tx = divmod(int(t), Wt)
        mask[ty * 16:(ty + 1) * 16, tx * 16:(tx + 1) * 16] = True
    ok = mask & ~band
    assert band[mask].mean() <= 1e-2
    got = feats.cpu().numpy()
    for c in range(9):
        scale = max(1.0, np.abs(ref["features"][c][ok]).max())
        assert np.abs(got[c][ok] - ref["features"][c][ok]).max() <= IMG_TOL * scale, c
