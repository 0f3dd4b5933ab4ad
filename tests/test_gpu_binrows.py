"""xpr_bin_rows (binning and tile sort by rows) is bit-exact: every tile's list of
record indices equals the oracle's exact-FP32 binning followed by the oracle's
sort by (tile, depth, index), and equals the key path (xpr_tile_bin +
xpr_sort_tiles) on the GPU's own records, for 3DGS and 3DGUT, ragged grids, 8x8
tiles, the headline workload, with and without the kept counts, and across the
capacity and workspace protocol.  The batch forms (xpr_bin_rows_views over the
views of one camera, xpr_bin_rows_items over multi-scene items, and the one-call
xpr_forward_items that bins by rows) give every view's and item's lists of the
key path and of the fused counting sort.  (Their tiles' segments lie in
column-major tile order, the key path's in row-major order; the ranges locate
them.)"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import batched as BT
from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import assert_same_tile_lists, dev, dev_i32

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
    (12_345, 250, 170, 16, True),    # ragged grid (16 x 11 tiles), big boxes
    (12_345, 250, 170, 8, True),     # 8x8 tiles: 32 x 22 grid
    (700, 64, 48, 16, False),        # a handful of spans
    (300_001, 320, 200, 16, False),  # several warps of spans per row, many positions
    (40_000, 2040, 2040, 16, False), # the largest grid taken: 128 x 128 tiles
])
def test_bin_rows_matches_oracle(oracle, n, W, H, tile, big):
    sc = scenes.uniform_scene(n, seed=n % 89)
    if big:
        sc.scale[::97] *= 12.0
    cam = scenes.pinhole(W, H, float(W))
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile)
    pr, rec32, order, sv, ranges = _oracle_sorted(oracle, sc, cam, cfg)
    rg, v, I, S, _ = B.xpr_bin_rows(dev(rec32), dev_i32(pr["bbox"]), dev_i32(pr["tc"]), dev_i32(order), n, cam, cfg)
    assert I == sv.size > 0
    assert S >= np.count_nonzero(np.diff(ranges, axis=1))  # at least one span slot per non-empty tile row
    assert_same_tile_lists(v, rg, sv.astype(np.int64), ranges)


@pytest.mark.parametrize("method,tile", [(0, 16), (0, 8), (1, 16)])
def test_bin_rows_equals_key_path_on_gpu_records(method, tile):
    sc = scenes.clustered_scene(60_000, seed=3, n_centers=30, width=480, height=270, focal=480.0, sh_degree=1)
    cam = scenes.pinhole(480, 270, 480.0)
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=1, method=method)
    P = R.scene_to_device(sc)
    a = R.forward_frame(*P, cam, cfg, R.Workspace())
    b = R.forward_frame(*P, cam, cfg, R.Workspace(rows=False))
    assert a.tiles is None and b.tiles is not None  # the two paths ran
    assert a.n_isect == b.n_isect > 100_000
    assert_same_tile_lists(a.vals_sorted, a.ranges, b.vals_sorted, b.ranges)
    assert torch.equal(a.image, b.image)


def test_bin_rows_equals_key_path_at_the_headline_size():
    sc, cam, cfg = scenes.headline_case()
    P = R.scene_to_device(sc)
    a = R.forward_frame(*P, cam, cfg, R.Workspace())
    b = R.forward_frame(*P, cam, cfg, R.Workspace(rows=False))
    assert a.n_isect == b.n_isect > 40_000_000
    assert_same_tile_lists(a.vals_sorted, a.ranges, b.vals_sorted, b.ranges)
    assert torch.equal(a.image, b.image) and torch.equal(a.n_contrib, b.n_contrib)


def _raw_call(rec, bbox, tc, cnt, order, n, cam, cfg, ranges, vals, ws):
    L = B.load()
    c, g = B.make_camera(cam), B.make_config(cfg)
    gi, gs = ctypes.c_int64(0), ctypes.c_int64(0)
    s = L.xpr_bin_rows(B._ptr(rec), B._ptr(bbox), B._ptr(tc), B._ptr(cnt), B._ptr(order), n, ctypes.byref(c),
                       ctypes.byref(g), B._ptr(ranges), B._ptr(vals), vals.numel(), ctypes.byref(gi),
                       ctypes.byref(gs), B._ptr(ws), ws.numel(), B._stream())
    return s, gi.value, gs.value


@pytest.mark.parametrize("with_counts", [True, False])
def test_bin_rows_capacity_and_workspace_protocol(with_counts):
    sc = scenes.uniform_scene(20_000, seed=7)
    cam = scenes.pinhole(300, 200, 300.0)
    cfg = scenes.RenderConfig()
    P = R.scene_to_device(sc)
    ref = R.forward_frame(*P, cam, cfg, R.Workspace(rows=False), render=False)
    rec, bbox, tc, order = ref.rec, ref.bbox, ref.tile_count, ref.order
    cnt = ref.isect_count if with_counts else None
    n = sc.n
    Wt, Ht = B.tiles_of(cam, cfg)
    ranges = torch.full((Wt * Ht, 2), -7, dtype=torch.int32, device="cuda")
    small = torch.zeros(16, dtype=torch.int32, device="cuda")
    ws0 = torch.empty(B.bin_rows_workspace_bytes(n, 0, 0, cam, cfg), dtype=torch.uint8, device="cuda")
    # too little of both: the counts come back (without the kept counts the pairs are counted only
    # once the spans exist, so the first call reports the span slots alone), ranges and vals untouched
    s, I, S = _raw_call(rec, bbox, tc, cnt, order, n, cam, cfg, ranges, small, ws0)
    assert s == B.XPR_ERR_CAPACITY and S > 0
    if not with_counts:
        assert I == 0
        ws1 = torch.empty(B.bin_rows_workspace_bytes(n, S, 0, cam, cfg), dtype=torch.uint8, device="cuda")
        s, I, S1 = _raw_call(rec, bbox, tc, cnt, order, n, cam, cfg, ranges, small, ws1)
        assert s == B.XPR_ERR_CAPACITY and S1 == S
    assert I == ref.n_isect
    assert torch.all(ranges == -7) and torch.all(small == 0)
    vals = torch.empty(I, dtype=torch.int32, device="cuda")
    ws = torch.empty(B.bin_rows_workspace_bytes(n, S, I, cam, cfg), dtype=torch.uint8, device="cuda")
    s, I2, S2 = _raw_call(rec, bbox, tc, cnt, order, n, cam, cfg, ranges, vals, ws)
    assert s == B.XPR_OK and (I2, S2) == (I, S)
    assert_same_tile_lists(vals, ranges, ref.vals_sorted, ref.ranges)
    # below the least workspace the call is rejected before any launch
    s, _, _ = _raw_call(rec, bbox, tc, cnt, order, n, cam, cfg, ranges, vals, ws0[:128])
    assert s == B.XPR_ERR_INVALID


def test_bin_rows_rejects_wide_grids_and_takes_empty_input():
    cam = scenes.pinhole(2064, 64, 2064.0)  # 129 tile columns
    cfg = scenes.RenderConfig()
    assert not B.bin_rows_ok(cam, cfg)
    assert B.bin_rows_workspace_bytes(10, 0, 0, cam, cfg) == 0
    buf = torch.zeros(4096, dtype=torch.int32, device="cuda")
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    s, _, _ = _raw_call(buf, buf, buf, buf, buf, 10, cam, cfg, buf, buf, ws)
    assert s == B.XPR_ERR_INVALID
    # no primitives: every range empty, no pairs
    cam = scenes.pinhole(100, 60, 100.0)
    rg, v, I, S, _ = B.xpr_bin_rows(buf.view(torch.float32), buf, buf, buf, 0, cam, cfg)
    assert (I, S) == (0, 0) and v.numel() == 0 and torch.all(rg == 0)


@pytest.mark.parametrize("method,tile", [(0, 16), (0, 8), (1, 16)])
def test_bin_rows_views_equal_key_path(method, tile):
    sc = scenes.uniform_scene(30_000, seed=11, sh_degree=1)
    sc.scale[::89] *= 8.0
    cams = scenes.multiview_cameras(5, 330, 200, 330.0, seed=1)  # ragged: 21 x 13 tiles of 16
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=1, method=method)
    P = R.scene_to_device(sc)
    a = BT.forward_views(*P, cams, cfg)             # by rows
    b = BT.forward_views(*P, cams, cfg, rows=False)  # tile ids, then the tile sort
    assert a.n_isect == b.n_isect > 100_000
    assert_same_tile_lists(a.vals_sorted, a.ranges, b.vals_sorted, b.ranges)
    assert torch.equal(a.image, b.image) and torch.equal(a.n_contrib, b.n_contrib)


def test_bin_rows_views_capacity_protocol():
    sc = scenes.uniform_scene(20_000, seed=12)
    cams = scenes.multiview_cameras(3, 300, 200, 300.0, seed=2)
    cfg = scenes.RenderConfig()
    P = R.scene_to_device(sc)
    ref = BT.forward_views(*P, cams, cfg, rows=False)
    n, V = sc.n, len(cams)
    rec, bbox, tc, cnt = B.xpr_project_views(*P, cams, B.make_config(cfg), with_isect_count=True)
    order = B.xpr_depth_order_views(rec, tc, n, V)
    # started with room for 16 pairs and no workspace: grown from the reported counts
    rg, v, I, S, ws = B.xpr_bin_rows_views(rec, bbox, tc, order, n, V, cams[0], B.make_config(cfg), capacity=16)
    assert I == ref.n_isect and S > 0 and ws.numel() >= B.bin_rows_views_workspace_bytes(n, V, S, I, cams[0], cfg)
    assert_same_tile_lists(v, rg, ref.vals_sorted, ref.ranges)
    rg2, v2, I2, S2, _ = B.xpr_bin_rows_views(rec, bbox, tc, order, n, V, cams[0], B.make_config(cfg),
                                              isect_count=cnt, capacity=16)
    assert (I2, S2) == (I, S) and torch.equal(rg2, rg) and torch.equal(v2, v)


def _items(tile=16):
    scs = [scenes.clustered_scene(n, seed=s, n_centers=20, width=W, height=H, focal=float(W), sh_degree=1)
           for s, (n, W, H) in enumerate([(9003, 320, 180), (40_000, 256, 256), (1201, 200, 150)])]
    cams = [scenes.pinhole(320, 180, 320.0, scenes.yaw_view(2.0, (0.01, 0.0, 0.02))),
            scenes.pinhole(256, 256, 256.0),
            scenes.pinhole(200, 150, 200.0),
            scenes.pinhole(250, 170, 256.0, scenes.yaw_view(-4.0, (0.0, 0.02, 0.0))),
            scenes.pinhole(64, 48, 64.0)]
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=1)
    ss = BT.SceneSet([R.scene_to_device(s) for s in scs])
    return ss, ss.layout([0, 1, 2, 1, 0], cams, cfg), cfg


@pytest.mark.parametrize("tile", [16, 8])
def test_bin_rows_items_equal_the_fused_sort_and_the_one_call_forward(tile):
    ss, layout, cfg = _items(tile)
    a = BT.forward_items(*ss.params, layout, cfg)             # by rows
    b = BT.forward_items(*ss.params, layout, cfg, rows=False)  # the fused counting sort
    assert a.n_isect == b.n_isect > 50_000
    assert_same_tile_lists(a.vals_sorted, a.ranges, b.vals_sorted, b.ranges)
    assert torch.equal(a.image, b.image) and torch.equal(a.n_contrib, b.n_contrib)
    image, tfin, ncon, I, _ = B.xpr_forward_items(*ss.params, layout, B.make_config(cfg), capacity=a.n_isect)
    assert I == a.n_isect
    assert torch.equal(image, a.image) and torch.equal(tfin, a.t_final) and torch.equal(ncon, a.n_contrib)


def test_forward_items_bins_tall_boxes_by_the_key_path_when_the_spans_outgrow_their_room():
    # needles one tile wide and many rows tall: about one pair per span, so at a capacity of exactly
    # the pair count the cap / 2 + R span slots the one-call forward reserves are too few for the
    # rows binning, and it bins by tile ids and the tile sort instead (the same lists and image)
    sc = scenes.uniform_scene(3000, seed=13, sh_degree=0)
    sc.scale[:, 0] = 0.002
    sc.scale[:, 1] = 0.4
    sc.scale[:, 2] = 0.002
    sc.quat[:] = np.array([1.0, 0.0, 0.0, 0.0], np.float32)
    cam = scenes.pinhole(480, 480, 480.0)
    cfg = scenes.RenderConfig(sh_degree=0)
    ss = BT.SceneSet([R.scene_to_device(sc)])
    layout = ss.layout([0], [cam], cfg)
    ref = BT.forward_items(*ss.params, layout, cfg, rows=False)
    rec, bbox, tc = B.xpr_project_items(*ss.params, layout, B.make_config(cfg))
    order = B.xpr_depth_order_items(rec, tc, layout)
    _, _, I, S, _ = B.xpr_bin_rows_items(rec, bbox, tc, order, layout, B.make_config(cfg))
    assert I == ref.n_isect and S > I // 2 + layout.R  # the fallback's condition holds
    image, tfin, ncon, I2, _ = B.xpr_forward_items(*ss.params, layout, B.make_config(cfg), capacity=I)
    assert I2 == I
    assert torch.equal(image, ref.image) and torch.equal(ncon, ref.n_contrib)
