"""Pins of the oracle's compositing (Sec. 2 Shader, Algorithm 1) against
closed forms, invariants and brute force."""
import math

import numpy as np
import pytest

from paper_2606_11529_gb300 import scenes

A_T = float(np.float32(1 / 255))
A_MAX = float(np.float32(0.99))
T_EPS = float(np.float32(1e-4))


def _rec(mx, my, conic, o, rgb, depth):
    r = np.zeros(12)
    r[0], r[1] = mx, my
    r[2:5] = conic
    r[5] = o
    r[6:9] = rgb
    r[9] = depth
    r[10] = math.log(o / A_T)
    r[11] = 1.0
    return r


def test_single_isotropic_gaussian_closed_form(oracle):
    # C(px) = rgb * min(0.99, o exp(-|px - mu|^2 / (2 s^2))) when >= 1/255, else 0; T = 1 - alpha
    cam = scenes.pinhole(48, 40, 48.0)
    cfg = scenes.RenderConfig()
    s, o, rgb = 4.5, 0.7, np.array([0.2, 0.5, 0.9])
    rec = _rec(20.3, 17.6, [1 / s ** 2, 0.0, 1 / s ** 2], o, rgb, 3.0)[None]
    r = oracle.render_brute(rec, cam, cfg)
    ys, xs = np.mgrid[0:40, 0:48]
    a = np.minimum(A_MAX, o * np.exp(-((xs - 20.3) ** 2 + (ys - 17.6) ** 2) / (2 * s * s)))
    a = np.where(a >= A_T, a, 0.0)
    np.testing.assert_allclose(r["image"], rgb[:, None, None] * a[None], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(r["t_final"], 1 - a, rtol=1e-13)


def test_clamp_at_alpha_max(oracle):
    cam = scenes.pinhole(16, 16, 16.0)
    cfg = scenes.RenderConfig()
    rec = _rec(8.0, 8.0, [0.01, 0, 0.01], 0.9999, [1, 1, 1], 2.0)[None]
    r = oracle.render_brute(rec, cam, cfg)
    assert r["image"][0, 8, 8] == pytest.approx(A_MAX, rel=1e-15)


def test_two_gaussians_hand_case(oracle):
    # front (depth 2) and back (depth 5) both cover pixel (10, 10):
    # C = c1 a1 + c2 a2 (1 - a1),  T = (1 - a1)(1 - a2), independent of input order
    cam = scenes.pinhole(20, 20, 20.0)
    cfg = scenes.RenderConfig()
    f = _rec(10.0, 10.0, [0.05, 0, 0.05], 0.6, [1.0, 0.0, 0.0], 2.0)
    b = _rec(11.0, 9.0, [0.02, 0.004, 0.03], 0.8, [0.0, 1.0, 0.5], 5.0)
    for recs in (np.stack([f, b]), np.stack([b, f])):
        r = oracle.render_pixels(recs, np.array([[10, 10]]), cfg)
        a1 = 0.6
        dx, dy = -1.0, 1.0
        a2 = 0.8 * math.exp(-0.5 * (0.02 * dx * dx + 2 * 0.004 * dx * dy + 0.03 * dy * dy))
        np.testing.assert_allclose(r["color"][0], [a1, a2 * (1 - a1), 0.5 * a2 * (1 - a1)], rtol=1e-14)
        assert r["t_final"][0] == pytest.approx((1 - a1) * (1 - a2), rel=1e-14)


def test_telescoping_white(oracle):
    # with every colour 1 and black background: sum a_i T_i = 1 - T_final exactly
    cam = scenes.pinhole(64, 64, 64.0)
    cfg = scenes.RenderConfig()
    sc = scenes.uniform_scene(400, seed=1, xy_range=0.8)
    pr = oracle.project_scene(sc, cam, cfg)
    rec = pr["rec"].copy()
    rec[:, 6:9] = 1.0
    r = oracle.render_brute(rec, cam, cfg)
    np.testing.assert_allclose(r["image"], np.broadcast_to(1 - r["t_final"], (3, 64, 64)), atol=1e-13)
    # white background makes the image 1 everywhere
    cfg.bg = (1.0, 1.0, 1.0)
    r = oracle.render_brute(rec, cam, cfg)
    np.testing.assert_allclose(r["image"], 1.0, atol=1e-13)


def test_transmittance_monotone_and_termination(oracle):
    # T never drops below T_eps: the primitive that would push it under is not blended (reading 3)
    cam = scenes.pinhole(64, 64, 64.0)
    cfg = scenes.RenderConfig()
    sc = scenes.uniform_scene(3000, seed=2, xy_range=0.5)
    sc.opacity[:] = 0.98
    pr = oracle.project_scene(sc, cam, cfg)
    r = oracle.render_brute(pr["rec"], cam, cfg)
    assert r["t_final"].min() >= T_EPS
    assert (r["t_final"] < 1e-3).mean() > 0.15  # the covered centre really saturates
    # prefix transmittances along the depth order are non-increasing: the image with fewer
    # (front) primitives never has smaller T than with more
    order = np.argsort(pr["rec"][:, 9])
    front = pr["rec"].copy()
    front[order[len(order) // 2:], 11] = 0
    rf = oracle.render_brute(front, cam, cfg)
    assert np.all(rf["t_final"] >= r["t_final"] - 1e-15)


def test_input_permutation_invariance(oracle):
    cam = scenes.pinhole(64, 48, 64.0)
    cfg = scenes.RenderConfig()
    sc = scenes.uniform_scene(500, seed=3, xy_range=0.6)
    pr = oracle.project_scene(sc, cam, cfg)
    r0 = oracle.render_brute(pr["rec"], cam, cfg)
    perm = np.random.default_rng(0).permutation(sc.n)
    r1 = oracle.render_brute(pr["rec"][perm], cam, cfg)
    np.testing.assert_array_equal(r0["image"], r1["image"])
    np.testing.assert_array_equal(r0["t_final"], r1["t_final"])


@pytest.mark.parametrize("tile", [8, 16])
def test_tiled_equals_brute_force(oracle, tile):
    # culling is conservative (Sec. 4.2, LinPrim appendix argument): the tiled image is the brute-force one
    cam = scenes.pinhole(96, 80, 96.0)
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile)
    sc = scenes.uniform_scene(1500, seed=4, xy_range=0.7)
    pr = oracle.project_scene(sc, cam, cfg)
    # both walk every pixel's primitives in the same order (float32 depth keys, then index) and a
    # culled pair is gated at every pixel of its tile, so the two images agree bit for bit
    rb = oracle.render_brute(pr["rec"], cam, cfg, key=pr["key"])
    rt = oracle.pipeline_tiled(sc, cam, cfg)
    np.testing.assert_array_equal(rt["image"], rb["image"])
    np.testing.assert_array_equal(rt["t_final"], rb["t_final"])


def test_tile_size_invariance(oracle):
    cam = scenes.pinhole(80, 64, 80.0)
    sc = scenes.uniform_scene(800, seed=5, xy_range=0.7)
    r8 = oracle.pipeline_tiled(sc, cam, scenes.RenderConfig(tile_w=8, tile_h=8))
    r16 = oracle.pipeline_tiled(sc, cam, scenes.RenderConfig(tile_w=16, tile_h=16))
    np.testing.assert_allclose(r8["image"], r16["image"], atol=1e-12)


def test_empty_and_invisible_scene(oracle):
    cam = scenes.pinhole(32, 32, 32.0)
    cfg = scenes.RenderConfig(bg=(0.25, 0.5, 0.75))
    sc = scenes.uniform_scene(10, seed=6)
    sc.mu[:, 2] = -1.0  # everything behind the camera
    r = oracle.pipeline_tiled(sc, cam, cfg)
    assert r["keys"].size == 0
    np.testing.assert_allclose(r["image"], np.array([0.25, 0.5, 0.75])[:, None, None] * np.ones((3, 32, 32)))
    assert np.all(r["t_final"] == 1.0) and np.all(r["n_contrib"] == 0)


def test_depth_keys_identity_view_are_the_means_depth(oracle):
    sc = scenes.uniform_scene(2000, seed=12)
    key = oracle.depth_keys(sc.mu, scenes.pinhole(64, 64, 64.0))
    np.testing.assert_array_equal(key, sc.mu[:, 2])


@pytest.mark.parametrize("euclid", [False, True])
def test_depth_keys_within_rounding_of_the_exact_depth(oracle, euclid):
    # four float32 roundings of terms bounded by s = sum |V_2j mu_j| + |t_2| (and for the Euclidean
    # distance three more of the squares and one of the root): the key lies within a few units of
    # roundoff of the exact value, and it is exactly what float32 arithmetic in that order gives
    sc = scenes.uniform_scene(5000, seed=13)
    vm = scenes.yaw_view(-11.0, (0.07, -0.03, 0.4))
    key = oracle.depth_keys(sc.mu, scenes.pinhole(64, 64, 64.0, vm), euclid=euclid).astype(np.float64)
    V = np.asarray(vm, np.float64).reshape(3, 4)
    m = sc.mu.astype(np.float64)
    mc = m @ V[:, :3].T + V[:, 3]
    exact = np.linalg.norm(mc, axis=1) if euclid else mc[:, 2]
    s = (np.abs(m) @ np.abs(V[:, :3]).T + np.abs(V[:, 3])).max(1)
    e = 2.0 ** -24
    assert np.all(np.abs(key - exact) <= e * (4 * s + (8 * np.abs(exact) if euclid else 0)) + 1e-30)
    assert np.mean(key != exact.astype(np.float32)) > 0.01  # not simply the rounded exact value


def test_brute_force_order_breaks_equal_keys_by_index(oracle):
    # two Gaussians with the same depth key over the same pixel: the lower index is in front
    cam = scenes.pinhole(32, 32, 32.0)
    cfg = scenes.RenderConfig()
    rec = np.zeros((2, 12))
    for i, col in enumerate([(1.0, 0.0, 0.0), (0.0, 0.0, 1.0)]):
        rec[i] = [16.0, 16.0, 0.1, 0.0, 0.1, 0.8, *col, 3.0, math.log(0.8 * 255), 1.0]
    pix = np.array([[16, 16]])
    front = oracle.render_pixels(rec, pix, cfg)["color"][0]
    assert front[0] > front[2]  # red (index 0) in front
    key = np.array([3.0, 3.0], np.float32)
    np.testing.assert_array_equal(oracle.render_pixels(rec, pix, cfg, key=key)["color"][0], front)
    key = np.array([3.0, np.nextafter(np.float32(3.0), np.float32(0))], np.float32)
    back = oracle.render_pixels(rec, pix, cfg, key=key)["color"][0]
    assert back[2] > back[0]  # one unit of roundoff closer: blue in front


@pytest.mark.parametrize("seed", [0, 1])
def test_band_holds_every_decision_a_perturbation_within_the_model_can_flip(oracle, seed):
    # Move every projected centre by up to 0.9 of its modelled uncertainty (here 2e-3 px for all)
    # and re-render in FP64: every pixel where a decision flipped (its decision hash changed) lies
    # in the unperturbed render's band (gate cascades included) and moves by at most its jump bound
    # plus the smooth change of the shift.
    sc = scenes.uniform_scene(3000, seed=20 + seed, xy_range=0.8)
    cam = scenes.pinhole(96, 80, 96.0)
    cfg = scenes.RenderConfig(bg=(0.2, 0.3, 0.1))
    pr = oracle.project_scene(sc, cam, cfg)
    unc = np.zeros((sc.n, 5))
    unc[:, 0] = 2e-3
    band = oracle.Band(1e-9, 1.0, 0.0)
    ys, xs = np.mgrid[0:80, 0:96]
    pix = np.stack([xs.ravel(), ys.ravel()], 1)
    ref = oracle.render_pixels(pr["rec"], pix, cfg, band=band, key=pr["key"], unc=unc)
    assert 0.002 < ref["gband"].mean() < 0.2
    rng = np.random.default_rng(seed)
    for _ in range(3):
        rec = pr["rec"].copy()
        rec[:, 0:2] += 0.9 * 2e-3 * rng.uniform(-1, 1, (sc.n, 2))
        got = oracle.render_pixels(rec, pix, cfg, key=pr["key"])
        d = np.abs(got["color"] - ref["color"]).max(1)
        flip = got["pixel_sig"] != ref["pixel_sig"]
        assert flip.any()
        assert np.all(ref["band"][flip]), np.nonzero(flip & ~ref["band"])[0][:5]
        smooth = d[~flip].max()
        assert np.all(d[flip] <= ref["jump"][flip] + smooth)
