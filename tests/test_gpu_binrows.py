"""xpr_bin_rows (binning and tile sort by rows) is bit-exact: every tile's list of
record indices equals the oracle's exact-FP32 binning followed by the oracle's
sort by (tile, depth, index), and equals the key path (xpr_tile_bin +
xpr_sort_tiles) on the GPU's own records, for 3DGS and 3DGUT, ragged grids, 8x8
tiles, the headline workload, with and without the kept counts, and across the
capacity and workspace protocol.  (Its tiles' segments lie in column-major tile
order, the key path's in row-major order; the ranges locate them.)"""
import ctypes

import numpy as np
import pytest
import torch

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
