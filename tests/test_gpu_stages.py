"""Stage-wise parity of the CUDA path (through the C ABI) with the FP64 oracle.

Each stage gets the same float32 inputs on both sides (oracle projections
rounded to float32, oracle lists); integer and index outputs must match bit for
bit, floating-point outputs within the stated tolerances."""
import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import (BAND_STAGE, GRAD_TOL, IMG_TOL, check_band, dev, dev_i32, dev_i64, host_u32, host_u64,
                      near_integer_bbox, oracle_lists, rel_err)

pytestmark = pytest.mark.gpu


def _case(deg=0, tile=16, view=False, n=10_000, W=256, H=256, seed=0):
    sc = scenes.uniform_scene(n, seed=seed, sh_degree=deg)
    vm = scenes.yaw_view(4.0, (0.05, -0.02, 0.1)) if view else None
    cam = scenes.pinhole(W, H, float(W), vm)
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=deg)
    return sc, cam, cfg


@pytest.mark.parametrize("deg,tile,view", [(0, 16, False), (3, 8, True), (1, 16, True), (2, 8, False)])
def test_project_matches_oracle(oracle, deg, tile, view):
    sc, cam, cfg = _case(deg, tile, view)
    pr = oracle.project_scene(sc, cam, cfg)
    rec, bbox, tc = B.xpr_project(*R.scene_to_device(sc), cam, cfg)
    torch.cuda.synchronize()
    rec, bbox, tc = rec.cpu().numpy(), bbox.cpu().numpy(), tc.cpu().numpy()
    ref = pr["rec"]
    amb = near_integer_bbox(pr["pre"])
    vis_o, vis_g = ref[:, 11] > 0, rec[:, 11] > 0
    assert np.all((vis_o == vis_g) | amb)
    both = vis_o & vis_g
    assert both.sum() > 1000
    np.testing.assert_allclose(rec[both, 0:2], ref[both, 0:2], rtol=1e-5, atol=2e-3)
    scale = np.maximum(np.abs(ref[both, 2]), np.abs(ref[both, 4]))[:, None]
    assert np.max(np.abs(rec[both, 2:5] - ref[both, 2:5]) / scale) < 2e-4
    np.testing.assert_array_equal(rec[both, 5], sc.opacity[both])
    np.testing.assert_allclose(rec[both, 6:9], ref[both, 6:9], atol=2e-5)
    np.testing.assert_allclose(rec[:, 9], ref[:, 9], rtol=2e-6, atol=1e-6)
    np.testing.assert_allclose(rec[both, 10], ref[both, 10], atol=2e-5)
    exact = both & ~amb
    np.testing.assert_array_equal(bbox[exact], pr["bbox"][exact])
    np.testing.assert_array_equal(tc[exact], pr["tc"][exact])
    assert np.all(rec[~vis_g][:, [0, 1, 2, 3, 4, 5, 6, 7, 8, 10, 11]] == 0)
    assert np.all(tc[~vis_g] == 0)


@pytest.mark.parametrize("tile,ordered", [(8, False), (16, False), (16, True), (8, True)])
def test_tile_bin_bit_exact(oracle, tile, ordered):
    sc, cam, cfg = _case(0, tile, n=12_345, W=250, H=170)  # ragged image: partial edge tiles
    sc.scale[::97] *= 12.0  # some large footprints: boxes of many tiles take the warp-cooperative path
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    order = oracle.depth_order(rec32, pr["tc"]) if ordered else None
    counts, keys, vals = oracle.bin_pairs(rec32, pr["bbox"], cam, cfg, exact32=True, order=order)
    off, k, v, I = B.xpr_tile_bin(dev(rec32), dev_i32(pr["bbox"]), dev_i32(pr["tc"]), cam, cfg,
                                  order=None if order is None else dev_i32(order.astype(np.int32)))
    assert I == keys.size > 10_000
    assert (pr["tc"] > 16).sum() > 50
    np.testing.assert_array_equal(off.cpu().numpy(), np.concatenate([[0], np.cumsum(counts)]).astype(np.int32))
    np.testing.assert_array_equal(host_u64(k), keys)
    np.testing.assert_array_equal(host_u32(v), vals)


def test_tile_bin_capacity_protocol(oracle):
    sc, cam, cfg = _case(0, 16, n=3000)
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    _, keys, vals = oracle.bin_pairs(rec32, pr["bbox"], cam, cfg, exact32=True)
    args = (dev(rec32), dev_i32(pr["bbox"]), dev_i32(pr["tc"]))
    # raw call with a too-small buffer: status 2, required count reported, buffer untouched
    L = B.load()
    import ctypes
    n = rec32.shape[0]
    kbuf = torch.full((8,), -7, dtype=torch.int64, device="cuda")
    vbuf = torch.full((8,), -7, dtype=torch.int32, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    ws = torch.empty(L.xpr_tile_bin_workspace(n), dtype=torch.uint8, device="cuda")
    got = ctypes.c_int64(0)
    c, g = B.make_camera(cam), B.make_config(cfg)
    s = L.xpr_tile_bin(args[0].data_ptr(), args[1].data_ptr(), args[2].data_ptr(), None, None, n, ctypes.byref(c),
                       ctypes.byref(g), off.data_ptr(), kbuf.data_ptr(), None, vbuf.data_ptr(), 8,
                       ctypes.byref(got), ws.data_ptr(), ws.numel(), None)
    torch.cuda.synchronize()
    assert s == B.XPR_ERR_CAPACITY and got.value == keys.size
    assert torch.all(kbuf == -7) and torch.all(vbuf == -7)
    # the binding re-sizes and retries
    _, k, v, I = B.xpr_tile_bin(*args, cam, cfg, capacity=8)
    np.testing.assert_array_equal(host_u64(k), keys)


def test_sort_bit_exact_on_binned_pairs(oracle):
    sc, cam, cfg = _case(0, 16)
    pr = oracle.project_scene(sc, cam, cfg)
    _, keys, vals, sk, sv, ranges = oracle_lists(oracle, pr["rec"].astype(np.float32), pr["bbox"], cam, cfg)
    ks, vs, rg = B.xpr_sort(dev_i64(keys), dev_i32(vals), ranges.shape[0])
    np.testing.assert_array_equal(host_u64(ks), sk)
    np.testing.assert_array_equal(host_u32(vs), sv)
    np.testing.assert_array_equal(rg.cpu().numpy(), ranges)


@pytest.mark.parametrize("tile", [8, 16])
def test_projection_counts_equal_binning_counts(oracle, tile):
    # xpr_project's per-primitive kept-tile counts drive the emit directly; they must equal what the
    # binning's own counting pass finds, and the emitted pairs must not change
    sc, cam, cfg = _case(0, tile, n=30_000, W=250, H=170)
    sc.scale[::53] *= 15.0
    rec, bbox, tc, cnt = B.xpr_project(*R.scene_to_device(sc), cam, cfg, with_isect_count=True)
    order = B.xpr_depth_order(rec, tc)
    off0, k0, v0, I0 = B.xpr_tile_bin(rec, bbox, tc, cam, cfg, order=order)
    off1, k1, v1, I1 = B.xpr_tile_bin(rec, bbox, tc, cam, cfg, order=order, isect_count=cnt)
    assert I0 == I1 > 10_000
    assert torch.equal(off0, off1) and torch.equal(k0, k1) and torch.equal(v0, v1)
    assert torch.equal(cnt[order.long()], (off0[1:] - off0[:-1]))
    # and against the oracle's own projection + exact-FP32 cull (equal except near ties)
    pr = oracle.project_scene(sc, cam, cfg)
    c_o, _, _ = oracle.bin_pairs(pr["rec"].astype(np.float32), pr["bbox"], cam, cfg, exact32=True)
    assert (cnt.cpu().numpy() == c_o).mean() > 0.998
    # u32 tile ids carry the same pairs as the u64 keys
    _, t2, v2, I2 = B.xpr_tile_bin(rec, bbox, tc, cam, cfg, order=order, isect_count=cnt, tile_ids=True)
    assert torch.equal(v2, v0) and torch.equal(t2.long() & 0xffffffff, (k0 >> 32) & 0xffffffff)


@pytest.mark.parametrize("tile", [8, 16])
def test_sort_tiles_of_depth_ordered_pairs_bit_exact(oracle, tile):
    sc, cam, cfg = _case(0, tile, n=20_000, W=250, H=170)
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    order = oracle.depth_order(rec32, pr["tc"])
    _, keys, vals = oracle.bin_pairs(rec32, pr["bbox"], cam, cfg, exact32=True, order=order)
    Wt, Ht = oracle.tiles_of(cam, cfg)
    sk, sv, ranges = oracle.sort_pairs(keys, vals, Wt * Ht)
    tiles = (keys >> np.uint64(32)).astype(np.uint32)
    ts, vs, rg = B.xpr_sort_tiles(dev_i32(tiles), dev_i32(vals), Wt * Ht)
    np.testing.assert_array_equal(host_u32(ts), (sk >> np.uint64(32)).astype(np.uint32))
    np.testing.assert_array_equal(host_u32(vs), sv)
    np.testing.assert_array_equal(rg.cpu().numpy(), ranges)


@pytest.mark.parametrize("n,n_tiles", [(1, 1), (2047, 256), (2049, 8160), (100_003, 5000), (300_000, 65536),
                                       (5000, 2), (9000, 5), (20_000, 16), (70_000, 31), (70_000, 64),
                                       (70_000, 100), (50_000, 3000), (10_000, (1 << 20) + 3)])
def test_sort_tiles_random_stable(oracle, n, n_tiles):
    # every digit width of a pass (1 .. 8 bits) and one to three passes
    rng = np.random.default_rng(n + 1)
    tiles = rng.integers(0, n_tiles, size=n).astype(np.uint32)
    vals = rng.permutation(n).astype(np.uint32)
    order = np.argsort(tiles, kind="stable")
    ts, vs, rg = B.xpr_sort_tiles(dev_i32(tiles), dev_i32(vals), n_tiles)
    np.testing.assert_array_equal(host_u32(ts), tiles[order])
    np.testing.assert_array_equal(host_u32(vs), vals[order])
    _, _, ranges = oracle.sort_pairs(tiles.astype(np.uint64) << np.uint64(32), np.arange(n, dtype=np.uint32), n_tiles)
    np.testing.assert_array_equal(rg.cpu().numpy(), ranges)


def test_depth_order_matches_lexsort(oracle):
    sc, cam, cfg = _case(0, 16, n=50_000)
    sc.mu[::50, 2] = -1.0  # some invisible primitives go last, in index order
    sc.mu[1::1000, 2] = sc.mu[0::1000, 2][: len(sc.mu[1::1000])]  # exact depth ties keep index order
    rec, bbox, tc = B.xpr_project(*R.scene_to_device(sc), cam, cfg)
    order = B.xpr_depth_order(rec, tc).cpu().numpy()
    ref = oracle.depth_order(rec.cpu().numpy(), tc.cpu().numpy())
    np.testing.assert_array_equal(order, ref.astype(np.int32))


@pytest.mark.parametrize("tile", [8, 16])
def test_tile_only_sort_of_depth_ordered_pairs_equals_full_sort(oracle, tile):
    sc, cam, cfg = _case(0, tile, n=20_000)
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    order = oracle.depth_order(rec32, pr["tc"])
    _, keys, vals = oracle.bin_pairs(rec32, pr["bbox"], cam, cfg, exact32=True, order=order)
    Wt, Ht = oracle.tiles_of(cam, cfg)
    sk, sv, ranges = oracle.sort_pairs(keys, vals, Wt * Ht)
    ks, vs, rg = B.xpr_sort(dev_i64(keys), dev_i32(vals), Wt * Ht, begin_bit=32)
    np.testing.assert_array_equal(host_u64(ks), sk)
    np.testing.assert_array_equal(host_u32(vs), sv)
    np.testing.assert_array_equal(rg.cpu().numpy(), ranges)


@pytest.mark.parametrize("n,n_tiles", [(1, 1), (4095, 256), (4097, 8160), (100_003, 5000), (262_144, 65536)])
def test_sort_random_keys_stable(oracle, n, n_tiles):
    rng = np.random.default_rng(n)
    tiles = rng.integers(0, n_tiles, size=n).astype(np.uint64)
    depth = rng.choice(np.array([0x40000000, 0x40000001, 0x3f800000, 0x41200000, 0x40490fdb], np.uint64), size=n)
    keys = (tiles << np.uint64(32)) | depth
    vals = rng.permutation(n).astype(np.uint32)
    order = np.lexsort((np.arange(n), keys))  # stable by key
    ks, vs, rg = B.xpr_sort(dev_i64(keys), dev_i32(vals), n_tiles)
    np.testing.assert_array_equal(host_u64(ks), keys[order])
    np.testing.assert_array_equal(host_u32(vs), vals[order])
    _, _, ranges = oracle.sort_pairs(keys, np.arange(n, dtype=np.uint32), n_tiles)
    np.testing.assert_array_equal(rg.cpu().numpy(), ranges)


@pytest.mark.parametrize("n", [2_500_003, 9_000_001])
@pytest.mark.parametrize("skew", ["one_tile", "two_tiles", "runs"])
def test_sort_tiles_many_blocks_skewed(skew, n):
    # 2.5M keys (over 600 blocks of the chained scan) and 9M keys (past the chained scan's limit:
    # the reduce-then-scan offsets): one tile only (every block's count of all but one digit is
    # zero), two interleaved tiles, and long runs of equal tiles with a ragged tail
    n_tiles = 8160
    rng = np.random.default_rng(11)
    if skew == "one_tile":
        tiles = np.full(n, 4097, np.uint32)
    elif skew == "two_tiles":
        tiles = np.where(rng.random(n) < 0.5, 3, 8159).astype(np.uint32)
    else:
        tiles = np.repeat(rng.integers(0, n_tiles, size=n // 1000 + 1), 1000)[:n].astype(np.uint32)
    vals = np.arange(n, dtype=np.uint32)
    order = np.argsort(tiles, kind="stable")
    ts, vs, rg = B.xpr_sort_tiles(dev_i32(tiles), dev_i32(vals), n_tiles)
    np.testing.assert_array_equal(host_u32(ts), tiles[order])
    np.testing.assert_array_equal(host_u32(vs), vals[order])
    counts = np.bincount(tiles, minlength=n_tiles)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]])
    r = rg.cpu().numpy()
    nz = counts > 0
    np.testing.assert_array_equal(r[nz, 0], starts[nz])
    np.testing.assert_array_equal(r[nz, 1], starts[nz] + counts[nz])
    assert np.all(r[~nz] == 0)
    B.xpr_device_check()


def test_sort_empty():
    ks, vs, rg = B.xpr_sort(torch.empty(0, dtype=torch.int64, device="cuda"),
                            torch.empty(0, dtype=torch.int32, device="cuda"), 77)
    assert ks.numel() == 0 and torch.all(rg == 0)


def _stage_inputs(oracle, sc, cam, cfg):
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    *_, sk, sv, ranges = oracle_lists(oracle, rec32, pr["bbox"], cam, cfg)
    return rec32, sv, ranges


@pytest.mark.parametrize("tile,W,H,bg", [(16, 256, 256, (0, 0, 0)), (8, 250, 170, (0.2, 0.5, 1.0)),
                                         (16, 200, 120, (1, 1, 1))])
def test_render_fwd_matches_oracle(oracle, tile, W, H, bg):
    sc, cam, cfg = _case(0, tile, W=W, H=H)
    cfg.bg = bg
    rec32, sv, ranges = _stage_inputs(oracle, sc, cam, cfg)
    ref = oracle.render_tiles(rec32.astype(np.float64), sv, ranges, cam, cfg, band=BAND_STAGE)
    img, tf, nc = B.xpr_render_fwd(dev(rec32), dev_i32(sv), dev_i32(ranges), cam, cfg)
    img, tf, nc = img.cpu().numpy(), tf.cpu().numpy(), nc.cpu().numpy()
    # both sides composite the same float32 records: the band holds only the decisions within the
    # float32 precision of the walk itself (about 1e-3 of the pixels of this dense scene)
    ok = check_band(img, ref, max_frac=3e-3, what=f"render fwd {W}x{H}")
    assert np.abs(tf[ok] - ref["t_final"][ok]).max() <= IMG_TOL
    assert (nc[ok] != ref["n_contrib"][ok]).mean() <= 1e-4
    assert (ref["t_final"] < 0.01).mean() > 0.05  # some pixels saturate (early termination exercised)


def test_render_bwd_matches_oracle(oracle):
    sc, cam, cfg = _case(0, 16)
    cfg.bg = (0.3, 0.1, 0.6)
    rec32, sv, ranges = _stage_inputs(oracle, sc, cam, cfg)
    rec64 = rec32.astype(np.float64)
    ref = oracle.render_tiles(rec64, sv, ranges, cam, cfg, band=BAND_STAGE)
    w = np.random.default_rng(5).normal(size=(3, cam.height, cam.width)) * ~ref["gband"][None]
    d_ref = oracle.render_bwd_tiles(rec64, sv, ranges, cam, cfg, w)
    rec_d, sv_d, rg_d = dev(rec32), dev_i32(sv), dev_i32(ranges)
    _, tf, nc = B.xpr_render_fwd(rec_d, sv_d, rg_d, cam, cfg)
    d_rec = B.xpr_render_bwd(rec_d, sv_d, rg_d, cam, cfg, tf, nc, dev(w)).cpu().numpy()
    for j, name in enumerate(["dmx", "dmy", "dc00", "dc01", "dc11", "do", "dr", "dg", "db"]):
        assert rel_err(d_rec[:, j], d_ref[:, j]) < GRAD_TOL, name
    assert np.all(d_rec[:, 9:] == 0)


def test_project_bwd_matches_oracle(oracle):
    for deg, view in [(3, True), (0, False)]:
        sc, cam, cfg = _case(deg, 16, view, n=4000)
        pr = oracle.project_scene(sc, cam, cfg)
        vis = (pr["rec"][:, 11] > 0) & ~near_integer_bbox(pr["pre"])
        rng = np.random.default_rng(deg)
        d_rec = np.zeros((sc.n, 12))
        d_rec[:, :9] = rng.normal(size=(sc.n, 9)) * np.array([1, 1, 50, 50, 50, 1, 1, 1, 1])
        d_rec[~vis] = 0
        ref = oracle.project_bwd(*sc.arrays(), cam, cfg, d_rec)
        got = B.xpr_project_bwd(*R.scene_to_device(sc), cam, cfg, dev(d_rec))
        for name, g in zip(["mu", "scale", "quat", "opacity", "sh"], got):
            assert rel_err(g.cpu().numpy(), ref[name]) < GRAD_TOL, (deg, name)


def test_sort_wait_timeout_is_reported_and_the_device_stays_usable():
    # the chained scan's look-back wait, run against words that nothing publishes, gives up after
    # its poll limit and records a timeout that xpr_device_check reports (once); a sort right after
    # is still exact
    B.xpr_device_check()
    counts = B.xpr_selftest_wait(polls=2000)
    torch.cuda.synchronize()
    with pytest.raises(B.XprError) as e:
        B.xpr_device_check()
    assert e.value.status == B.XPR_ERR_TIMEOUT
    assert torch.all(counts == 0)
    B.xpr_device_check()  # the flag was cleared by the first check
    rng = np.random.default_rng(5)
    tiles = rng.integers(0, 300, size=50_000).astype(np.uint32)
    vals = np.arange(50_000, dtype=np.uint32)
    order = np.argsort(tiles, kind="stable")
    _, vs, _ = B.xpr_sort_tiles(dev_i32(tiles), dev_i32(vals), 300)
    np.testing.assert_array_equal(host_u32(vs), vals[order])
