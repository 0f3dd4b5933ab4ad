"""xpr_bin_sorted (fused bin + sort) is bit-exact: its sorted record indices and
tile ranges equal the oracle's exact-FP32 binning followed by the oracle's sort
by (tile, depth, index), and equal the key path (xpr_tile_bin + xpr_sort_tiles)
for single and multi-view launches, across chunk sizes, band splits, ragged
grids and the capacity protocol."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import batched as BT
from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import dev, dev_i32, host_u32

pytestmark = pytest.mark.gpu


def _oracle_sorted(oracle, sc, cam, cfg):
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    order = oracle.depth_order(rec32, pr["tc"]).astype(np.int32)
    _, keys, vals = oracle.bin_pairs(rec32, pr["bbox"], cam, cfg, exact32=True, order=order)
    Wt, Ht = oracle.tiles_of(cam, cfg)
    _, sv, ranges = oracle.sort_pairs(keys, vals, Wt * Ht)
    return pr, rec32, order, sv, ranges


@pytest.mark.parametrize("n,W,H,tile,big", [
    (12_345, 250, 170, 16, True),     # ragged grid, big boxes, one band split
    (12_345, 250, 170, 8, True),      # 8x8 tiles: 32 x 22 grid
    (700, 64, 48, 16, False),         # one chunk, one band
    (300_001, 320, 200, 16, False),   # several chunk sizes' worth of positions (P > 256)
    (40_000, 17000, 64, 16, False),   # wide grid (1063 tile columns): one tile row per band
    (20_000, 12000, 100, 16, False),  # 750 tile columns: two tile rows per band
])
def test_bin_sorted_matches_oracle(oracle, n, W, H, tile, big):
    sc = scenes.uniform_scene(n, seed=n % 97)
    if big:
        sc.scale[::97] *= 12.0
    cam = scenes.pinhole(W, H, float(W))
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile)
    pr, rec32, order, sv, ranges = _oracle_sorted(oracle, sc, cam, cfg)
    rg, v, I = B.xpr_bin_sorted(dev(rec32), dev_i32(pr["bbox"]), dev_i32(pr["tc"]), dev_i32(order), n, cam, cfg)
    assert I == sv.size > 0
    np.testing.assert_array_equal(host_u32(v), sv)
    np.testing.assert_array_equal(rg.cpu().numpy(), ranges)


@pytest.mark.parametrize("tile", [8, 16])
def test_bin_sorted_equals_key_path_on_gpu_records(tile):
    sc = scenes.clustered_scene(60_000, seed=3, n_centers=30, width=480, height=270, focal=480.0, sh_degree=1)
    cam = scenes.pinhole(480, 270, 480.0)
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=1)
    P = R.scene_to_device(sc)
    a = R.forward_frame(*P, cam, cfg, fused=True)
    b = R.forward_frame(*P, cam, cfg, R.Workspace(rows=False), fused=False)
    assert a.n_isect == b.n_isect > 100_000
    assert torch.equal(a.vals_sorted, b.vals_sorted) and torch.equal(a.ranges, b.ranges)
    assert torch.equal(a.image, b.image)


def test_bin_sorted_views_equal_key_path():
    sc = scenes.uniform_scene(30_000, seed=4)
    cams = scenes.multiview_cameras(5, 300, 200, 300.0, seed=2)
    cfg = scenes.RenderConfig()
    P = R.scene_to_device(sc)
    a = BT.forward_views(*P, cams, cfg, fused=True)
    b = BT.forward_views(*P, cams, cfg, fused=False)
    assert a.n_isect == b.n_isect > 0
    assert torch.equal(a.vals_sorted, b.vals_sorted) and torch.equal(a.ranges, b.ranges)
    assert torch.equal(a.image, b.image)


def test_bin_sorted_capacity_protocol(oracle):
    sc = scenes.uniform_scene(3000, seed=5)
    cam = scenes.pinhole(256, 256, 256.0)
    cfg = scenes.RenderConfig()
    pr, rec32, order, sv, ranges = _oracle_sorted(oracle, sc, cam, cfg)
    n = rec32.shape[0]
    L = B.load()
    c, g = B.make_camera(cam), B.make_config(cfg)
    rec, bbox, tc, od = dev(rec32), dev_i32(pr["bbox"]), dev_i32(pr["tc"]), dev_i32(order)
    rg = torch.empty((256, 2), dtype=torch.int32, device="cuda")
    vbuf = torch.full((8,), -7, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.bin_sorted_workspace_bytes(n, 1, c, g), dtype=torch.uint8, device="cuda")
    got = ctypes.c_int64(0)
    s = L.xpr_bin_sorted(rec.data_ptr(), bbox.data_ptr(), tc.data_ptr(), od.data_ptr(), n, 1, ctypes.byref(c),
                         ctypes.byref(g), rg.data_ptr(), vbuf.data_ptr(), 8, ctypes.byref(got), ws.data_ptr(),
                         ws.numel(), None)
    torch.cuda.synchronize()
    assert s == B.XPR_ERR_CAPACITY and got.value == sv.size
    assert torch.all(vbuf == -7)
    np.testing.assert_array_equal(rg.cpu().numpy(), ranges)  # ranges are final already
    _, v, I = B.xpr_bin_sorted(rec, bbox, tc, od, n, cam, cfg, capacity=8)
    np.testing.assert_array_equal(host_u32(v), sv)


def test_bin_sorted_nothing_visible():
    sc = scenes.uniform_scene(5000, seed=6)
    sc.mu[:, 2] = -3.0  # behind the camera
    cam = scenes.pinhole(128, 96, 128.0)
    cfg = scenes.RenderConfig()
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    assert fr.n_isect == 0 and int(fr.ranges.abs().sum()) == 0
    assert torch.all(fr.t_final == 1.0)
