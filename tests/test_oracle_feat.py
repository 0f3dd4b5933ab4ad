"""Pins of the oracle's rendered features (channels composited with the colour weights, depth as a
channel) and their adjoint: identities with the colour image, the telescoping sum, a closed-form
depth, and central differences."""
import math

import numpy as np
import pytest

from paper_2606_11529_gb300 import scenes


def _scene(seed=0, n=400, deg=0):
    sc = scenes.uniform_scene(n, seed=seed, sh_degree=deg)
    cam = scenes.pinhole(96, 80, 96.0)
    cfg = scenes.RenderConfig(sh_degree=deg, bg=(0.2, 0.4, 0.6), tile_w=16, tile_h=16)
    return sc, cam, cfg


def test_colours_as_features_reproduce_the_image(oracle):
    sc, cam, cfg = _scene()
    out = oracle.pipeline_tiled_feat(sc.arrays(), None, cam, cfg)
    rgb = out["proj"]["rec"][:, 6:9]
    f = oracle.render_tiles_feat(out["proj"]["rec"], rgb, out["vals"], out["ranges"], cam, cfg)
    bg = np.asarray(cfg.bg, np.float64)[:, None, None]
    np.testing.assert_allclose(f["features"], out["image"] - f["t_final"][None] * np.float32(bg), atol=1e-12)


def test_constant_feature_telescopes(oracle):
    sc, cam, cfg = _scene(1)
    ones = np.ones((sc.n, 2))
    ones[:, 1] = 3.0
    out = oracle.pipeline_tiled_feat(sc.arrays(), ones, cam, cfg)
    np.testing.assert_allclose(out["features"][0], 1.0 - out["t_final"], atol=1e-12)
    np.testing.assert_allclose(out["features"][1], 3.0 * (1.0 - out["t_final"]), atol=1e-12)
    assert (out["t_final"] < 0.9).mean() > 0.3


def test_single_gaussian_depth_closed_form(oracle):
    # isotropic Gaussian on the axis: the pixel at the principal point gets alpha = o G(0.5 px offset
    # from the raw-coordinate evaluation) and depth channel z alpha
    cam = scenes.pinhole(32, 32, 40.0)
    cfg = scenes.RenderConfig(tile_w=8, tile_h=8)
    z, s, o = 2.5, 0.1, 0.7
    P = [np.array([[0.0, 0.0, z]]), np.array([[s, s, s]]), np.array([[1.0, 0, 0, 0]]), np.array([o]),
         np.zeros((1, 1, 3))]
    out = oracle.pipeline_tiled_feat(P, None, cam, cfg, with_depth=True)
    k = (s * 40.0 / z) ** 2 + float(np.float32(0.3))
    for x, y in [(16, 16), (17, 15), (14, 18)]:
        dx, dy = x - 16.0, y - 16.0
        alpha = o * math.exp(-0.5 * (dx * dx + dy * dy) / k)
        assert out["features"][0, y, x] == pytest.approx(z * alpha, rel=1e-12)


@pytest.mark.parametrize("seed,deg,depth", [(0, 1, True), (1, 0, False), (2, 3, True)])
def test_feature_adjoint_matches_central_differences(oracle, seed, deg, depth):
    rng = np.random.default_rng(seed)
    cam = scenes.pinhole(32, 32, 32.0, scenes.yaw_view(5.0, t=(0.02, 0.0, 0.05)))
    cfg = scenes.RenderConfig(sh_degree=deg, bg=(0.1, 0.2, 0.3))
    n = 6
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2.5, 4.0, n)], 1)
    s = np.exp(rng.normal(-1.6, 0.3, (n, 3)))
    q = rng.normal(size=(n, 4))
    o = 1 / (1 + np.exp(-rng.normal(0.5, 0.8, n)))
    sh = rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3))
    sh[:, 0, :] = rng.uniform(0.5, 1.5, (n, 3))
    feat = rng.normal(size=(n, 3))
    P = [mu, s, q, o, sh, feat]
    nf = 3 + int(depth)
    wi = rng.normal(size=(3, 32, 32))
    wf = rng.normal(size=(nf, 32, 32))

    def loss(P):
        out = oracle.pipeline_tiled_feat(P[:5], P[5], cam, cfg, with_depth=depth)
        return float((wi * out["image"]).sum() + (wf * out["features"]).sum()), oracle.loss_brute(P[:5], cam, cfg, wi)[1]

    g = oracle.grads_tiled_feat(P[:5], P[5], cam, cfg, wi, wf, with_depth=depth)
    skipped = total = 0
    for a, name in enumerate(["mu", "scale", "quat", "opacity", "sh", "feat"]):
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
            lp, sp = loss(Pp)
            lm, sm = loss(Pm)
            total += 1
            if sp != sm:
                skipped += 1
                fd[idx] = g[name][idx]
                continue
            fd[idx] = (lp - lm) / (2 * h)
        err = np.linalg.norm(g[name] - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-5, (name, err)
    assert skipped <= 0.02 * total
