"""Pins of the oracle's analytic adjoint: central finite differences of its own
FP64 forward (checked to make no gate decision flip), closed-form derivatives
of a single Gaussian, and tiled-vs-brute agreement."""
import math

import numpy as np
import pytest

from paper_2606_11529_gb300 import scenes

A_T = float(np.float32(1 / 255))


def _tiny_scene(seed, n=6, deg=3):
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2.5, 4.0, n)], 1)
    s = np.exp(rng.normal(-1.6, 0.3, (n, 3)))
    q = rng.normal(size=(n, 4))
    o = 1 / (1 + np.exp(-rng.normal(0.5, 0.8, n)))
    K = (deg + 1) ** 2
    sh = rng.normal(0, 0.3, (n, K, 3))
    sh[:, 0, :] = rng.uniform(0.5, 1.5, (n, 3))  # keep colours positive (away from the max(0,.) kink)
    return [mu, s, q, o, sh]


def _view(seed):
    from scipy.spatial.transform import Rotation
    R = Rotation.from_euler("xyz", np.random.default_rng(seed).normal(0, 0.1, 3)).as_matrix()
    t = np.array([0.05, -0.03, 0.1])
    return np.hstack([R, t[:, None]])


@pytest.mark.parametrize("seed,deg,view", [(0, 3, False), (1, 3, True), (2, 0, True), (3, 1, False)])
def test_adjoint_matches_central_differences(oracle, seed, deg, view):
    cam = scenes.pinhole(32, 32, 32.0)
    if view:
        cam.viewmat = _view(seed).astype(np.float32)
    cfg = scenes.RenderConfig(sh_degree=deg, bg=(0.1, 0.2, 0.3))
    P = _tiny_scene(seed, deg=deg)
    w = np.random.default_rng(100 + seed).normal(size=(3, 32, 32))
    g = oracle.grads_brute(P, cam, cfg, w)
    names = ["mu", "scale", "quat", "opacity", "sh"]
    skipped = 0
    total = 0
    for a, name in enumerate(names):
        fd = np.zeros_like(P[a], dtype=float)
        it = np.nditer(P[a], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            x0 = P[a][idx]
            h = 1e-6 * max(abs(x0), 1e-2)
            Pp = [p.copy() for p in P]
            Pm = [p.copy() for p in P]
            Pp[a][idx] = x0 + h
            Pm[a][idx] = x0 - h
            lp, sp = oracle.loss_brute(Pp, cam, cfg, w)
            lm, sm = oracle.loss_brute(Pm, cam, cfg, w)
            total += 1
            if sp != sm:
                skipped += 1
                fd[idx] = g[name][idx]
                continue
            fd[idx] = (lp - lm) / (2 * h)
        an = g[name]
        err = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-5, (name, err)
    assert skipped <= 0.02 * total
    assert np.abs(g["mu"]).max() > 0 and np.abs(g["quat"]).max() > 0


def test_single_gaussian_closed_form_derivatives(oracle):
    # C = rgb * o * G for an unclamped, ungated pixel:  dC/drgb = o G,  dC/do = rgb G,
    # dC/dmu_2D = rgb o G conic (px - mu)
    cam = scenes.pinhole(24, 24, 24.0)
    cfg = scenes.RenderConfig()
    c = [0.08, 0.01, 0.05]
    o, rgb = 0.6, np.array([0.3, 0.6, 0.9])
    rec = np.zeros((1, 12))
    rec[0, :11] = [12.2, 11.7, *c, o, *rgb, 3.0, math.log(o / A_T)]
    rec[0, 11] = 1
    d_image = np.zeros((3, 24, 24))
    px, py = 14, 10
    d_image[:, py, px] = [1.0, 2.0, -1.0]
    d = oracle.render_bwd_brute(rec, cam, cfg, d_image)[0]
    dx, dy = px - 12.2, py - 11.7
    G = math.exp(-0.5 * (c[0] * dx * dx + 2 * c[1] * dx * dy + c[2] * dy * dy))
    gsum = (np.array([1.0, 2.0, -1.0]) * rgb).sum()
    np.testing.assert_allclose(d[6:9], o * G * np.array([1.0, 2.0, -1.0]), rtol=1e-13)
    assert d[5] == pytest.approx(gsum * G, rel=1e-13)
    np.testing.assert_allclose(d[0:2], gsum * o * G * np.array([c[0] * dx + c[1] * dy, c[1] * dx + c[2] * dy]),
                               rtol=1e-12)
    np.testing.assert_allclose(d[2:5], gsum * o * G * np.array([-0.5 * dx * dx, -dx * dy, -0.5 * dy * dy]),
                               rtol=1e-12)


def test_clamped_alpha_has_no_opacity_gradient(oracle):
    cam = scenes.pinhole(16, 16, 16.0)
    cfg = scenes.RenderConfig()
    rec = np.zeros((1, 12))
    rec[0, :11] = [8, 8, 0.01, 0, 0.01, 0.9999, 1, 1, 1, 2.0, math.log(0.9999 / A_T)]
    rec[0, 11] = 1
    d_image = np.zeros((3, 16, 16))
    d_image[:, 8, 8] = 1.0
    d = oracle.render_bwd_brute(rec, cam, cfg, d_image)[0]
    assert d[5] == 0.0 and np.all(d[0:5] == 0.0)
    assert d[6] == pytest.approx(float(np.float32(0.99)))


def test_tiled_adjoint_equals_brute(oracle):
    cam = scenes.pinhole(64, 48, 64.0)
    cfg = scenes.RenderConfig(tile_w=8, tile_h=8, bg=(0.3, 0.3, 0.3))
    sc = scenes.uniform_scene(300, seed=7, xy_range=0.6)
    pr = oracle.project_scene(sc, cam, cfg)
    Wt, Ht = oracle.tiles_of(cam, cfg)
    _, keys, vals = oracle.bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False, key=pr["key"])
    _, vals, ranges = oracle.sort_pairs(keys, vals, Wt * Ht)
    w = np.random.default_rng(1).normal(size=(3, 48, 64))
    db = oracle.render_bwd_brute(pr["rec"], cam, cfg, w, key=pr["key"])
    dt = oracle.render_bwd_tiles(pr["rec"], vals, ranges, cam, cfg, w)
    np.testing.assert_allclose(dt, db, rtol=1e-10, atol=1e-12)
