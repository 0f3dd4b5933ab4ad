"""Pins of the oracle's replicate / tile-ID / cull / sort (Sec. 4.2) against
the paper's worked example, an independent optimiser and brute force."""
import json
import os

import numpy as np
import pytest

from paper_2606_11529_gb300 import scenes

GOLD = os.path.join(os.path.dirname(__file__), "golden")
A_T = float(np.float32(1 / 255))


def _rec(mx, my, conic, o=0.9, depth=3.0):
    r = np.zeros(12)
    r[0], r[1] = mx, my
    r[2:5] = conic
    r[5] = o
    r[6:9] = 1.0
    r[9] = depth
    r[10] = np.log(o / A_T)
    r[11] = 1.0
    return r


def test_tile_enumeration_matches_paper_example(oracle):
    g = json.load(open(os.path.join(GOLD, "tile_enumeration.json")))
    tw = 16
    cam = scenes.pinhole(g["grid_tiles_x"] * tw, g["grid_tiles_y"] * tw, 64.0)
    cfg = scenes.RenderConfig()
    # a wide, opaque Gaussian centred on the shared corner of tiles 0,1,3,4: nothing is culled
    rec = _rec(16.0, 16.0, [1 / 100.0, 0.0, 1 / 100.0])[None]
    bbox = np.array([g["bbox"]], np.int32)
    counts, keys, vals = oracle.bin_pairs(rec, bbox, cam, cfg, exact32=False)
    assert list((keys >> np.uint64(32)).astype(int)) == g["tiles"]
    assert list(vals) == [0] * len(g["tiles"]) and counts[0] == len(g["tiles"])


def _conic(rng):
    A = rng.normal(size=(2, 2))
    S = A @ A.T * rng.uniform(1, 40) + 0.3 * np.eye(2)
    C = np.linalg.inv(S)
    return [C[0, 0], C[0, 1], C[1, 1]]


def test_cull_matches_box_constrained_minimum(oracle):
    # keep <=> min over the tile rectangle of d^T conic d / 2 <= ln(o/alpha_t); the minimum from scipy
    from scipy.optimize import minimize
    rng = np.random.default_rng(0)
    cam = scenes.pinhole(128, 128, 128.0)
    cfg = scenes.RenderConfig()
    checked = 0
    for _ in range(300):
        c = _conic(rng)
        mx, my = rng.uniform(-20, 148, size=2)
        o = rng.uniform(0.01, 1.0)
        rec = _rec(mx, my, c, o)
        tx, ty = rng.integers(0, 8, size=2)
        x0, y0 = tx * 16, ty * 16
        x1, y1 = x0 + 15, y0 + 15
        Q = np.array([[c[0], c[1]], [c[1], c[2]]])
        f = lambda p: 0.5 * (np.array([mx, my]) - p) @ Q @ (np.array([mx, my]) - p)
        best = min(minimize(f, np.array(s0, float), bounds=[(x0, x1), (y0, y1)], method="L-BFGS-B",
                            options=dict(ftol=1e-15, gtol=1e-12)).fun
                   for s0 in [(x0, y0), (x1, y1), (x0, y1), (x1, y0), ((x0 + x1) / 2, (y0 + y1) / 2)])
        lt = rec[10]
        if abs(best - lt) < 1e-6 * max(1.0, lt):
            continue
        assert oracle.cull_one(rec, int(tx), int(ty), cam, cfg) == (best <= lt)
        checked += 1
    assert checked > 250


def test_row_form_equals_per_tile_minimum(oracle):
    # the row form (x-extent of ellipse ∩ tile-row strip) keeps exactly the tiles whose rectangle
    # minimum passes, on random conics, means in and around a ragged image (partial edge tiles),
    # both tile sizes; the FP32 row form on float-rounded records agrees away from near-ties
    rng = np.random.default_rng(11)
    flips32 = 0
    total = 0
    for W, H, tile in [(250, 170, 16), (250, 170, 8), (64, 48, 16)]:
        cam = scenes.pinhole(W, H, float(W))
        cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile)
        Wt, Ht = (W + tile - 1) // tile, (H + tile - 1) // tile
        for _ in range(120):
            c = _conic(rng)
            mx, my = rng.uniform(-30, W + 30), rng.uniform(-30, H + 30)
            rec = _rec(mx, my, c, rng.uniform(0.01, 1.0))
            for ty in range(Ht):
                for tx in range(Wt):
                    a = oracle.cull_one(rec, tx, ty, cam, cfg, form=0)
                    assert oracle.cull_one(rec, tx, ty, cam, cfg, form=1) == a, (W, tile, tx, ty, rec)
                    flips32 += oracle.cull_one(rec, tx, ty, cam, cfg, form=2) != a
                    total += 1
    assert total > 50_000 and flips32 <= total * 1e-4


def test_cull_is_conservative_at_pixels(oracle):
    # every (primitive, tile) pair with alpha >= alpha_t at some pixel of the tile is kept
    cam = scenes.pinhole(128, 128, 128.0)
    cfg = scenes.RenderConfig()
    sc = scenes.uniform_scene(150, seed=2, xy_range=0.7)
    pr = oracle.project_scene(sc, cam, cfg)
    _, keys, vals = oracle.bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False)
    kept = set(zip((keys >> np.uint64(32)).astype(int).tolist(), vals.tolist()))
    ys, xs = np.mgrid[0:128, 0:128]
    for i in range(sc.n):
        R = pr["rec"][i]
        if R[11] == 0:
            continue
        dx, dy = xs - R[0], ys - R[1]
        power = -0.5 * (R[2] * dx * dx + 2 * R[3] * dx * dy + R[4] * dy * dy)
        hit = np.minimum(float(np.float32(0.99)), R[5] * np.exp(power)) >= A_T
        for t in set(((ys[hit] // 16) * 8 + xs[hit] // 16).tolist()):
            assert (t, i) in kept


def test_exact32_agrees_with_fp64_away_from_ties(oracle):
    cam = scenes.pinhole(256, 256, 256.0)
    cfg = scenes.RenderConfig()
    sc = scenes.uniform_scene(2000, seed=3)
    pr = oracle.project_scene(sc, cam, cfg)
    c64, k64, v64 = oracle.bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False)
    c32, k32, v32 = oracle.bin_pairs(pr["rec"].astype(np.float32), pr["bbox"], cam, cfg, exact32=True)
    diff = np.nonzero(c64 != c32)[0]
    assert len(diff) <= 2  # only near-ties may flip
    assert k32.size > 1000


def test_sort_and_ranges_partition(oracle):
    cam = scenes.pinhole(256, 256, 256.0)
    cfg = scenes.RenderConfig(tile_w=8, tile_h=8)
    sc = scenes.uniform_scene(3000, seed=4)
    pr = oracle.project_scene(sc, cam, cfg)
    counts, keys, vals = oracle.bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False)
    Wt, Ht = oracle.tiles_of(cam, cfg)
    sk, sv, ranges = oracle.sort_pairs(keys, vals, Wt * Ht)
    assert np.all(sk[1:] >= sk[:-1])
    # the multiset of pairs is unchanged and equal keys are ordered by primitive index
    assert sorted(zip(keys.tolist(), vals.tolist())) == list(zip(sk.tolist(), sv.tolist()))
    tiles = (sk >> np.uint64(32)).astype(np.int64)
    pos = 0
    for t in range(Wt * Ht):
        s, e = ranges[t]
        n_t = int((tiles == t).sum())
        assert e - s == n_t
        if n_t:
            assert s == pos
            assert np.all(tiles[s:e] == t)
            pos = e
    assert pos == sk.size
    # per-tile count equals brute-force count of (bbox tile, cull) pairs
    brute = np.zeros(Wt * Ht, int)
    for i in range(sc.n):
        b = pr["bbox"][i]
        for ty in range(b[1], b[3]):
            for tx in range(b[0], b[2]):
                if oracle.cull_one(pr["rec"][i], tx, ty, cam, cfg):
                    brute[ty * Wt + tx] += 1
    np.testing.assert_array_equal(ranges[:, 1] - ranges[:, 0], brute)
    assert counts.sum() == sk.size


def test_emission_order_does_not_change_sorted_lists(oracle):
    # emitting in (depth, index) order and sorting by tile only == emitting in index order and
    # sorting by the full (tile, depth) key with index tie-break
    cam = scenes.pinhole(128, 96, 128.0)
    cfg = scenes.RenderConfig(tile_w=8, tile_h=8)
    sc = scenes.uniform_scene(1500, seed=9)
    pr = oracle.project_scene(sc, cam, cfg)
    rec32 = pr["rec"].astype(np.float32)
    Wt, Ht = oracle.tiles_of(cam, cfg)
    _, k0, v0 = oracle.bin_pairs(rec32, pr["bbox"], cam, cfg, exact32=True)
    sk0, sv0, r0 = oracle.sort_pairs(k0, v0, Wt * Ht)
    order = oracle.depth_order(rec32, pr["tc"])
    c1, k1, v1 = oracle.bin_pairs(rec32, pr["bbox"], cam, cfg, exact32=True, order=order)
    tiles = (k1 >> np.uint64(32)).astype(np.int64)
    st = np.argsort(tiles, kind="stable")  # tile-only stable sort
    np.testing.assert_array_equal(k1[st], sk0)
    np.testing.assert_array_equal(v1[st], sv0)
    assert c1.sum() == k0.size


def test_empty_input(oracle):
    cam = scenes.pinhole(64, 64, 64.0)
    cfg = scenes.RenderConfig()
    counts, keys, vals = oracle.bin_pairs(np.zeros((0, 12)), np.zeros((0, 4), np.int32), cam, cfg, exact32=False)
    assert keys.size == 0
    _, _, ranges = oracle.sort_pairs(keys, vals, 16)
    assert np.all(ranges == 0)
