"""Pins of the oracle's LinPrim path (octahedron projection, slab-intersection evaluate, the per-tile
chord bound of the cull, and the adjoint) against closed forms, the exact ray-octahedron chord,
brute force and central differences."""
import math

import numpy as np
import pytest

from paper_2606_11529_gb300 import scenes

A_T = float(np.float32(1.0 / 255.0))


def _one(mu, s, q=(1.0, 0.0, 0.0, 0.0), o=0.8, deg=0, rgb=None):
    sh = np.zeros((1, (deg + 1) ** 2, 3))
    if rgb is not None:
        sh[0, 0] = (np.asarray(rgb) - 0.5) / 0.28209479177387814
    return (np.array([mu], np.float64), np.array([s], np.float64), np.array([q], np.float64), np.array([o]), sh)


def _cfg(**kw):
    base = dict(method=2)
    base.update(kw)
    return scenes.RenderConfig(**base)


def _exact_chord(mu, s, q, cam, X, Y):
    """Length of the chord of the ray through image point (X, Y) (pixel (x, y) has its centre at
    (x + 0.5, y + 0.5)) through the octahedron {||S^-1 R^T (x - mu)||_1 <= 1}, intersecting its
    eight face half-spaces exactly (world space, scipy rotation)."""
    from scipy.spatial.transform import Rotation
    V = np.asarray(cam.viewmat, np.float64)
    W, t = V[:, :3], V[:, 3]
    o = -W.T @ t
    dc = np.array([(X - cam.cx) / cam.fx, (Y - cam.cy) / cam.fy, 1.0])
    d = W.T @ (dc / np.linalg.norm(dc))
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    L = np.diag(1.0 / np.asarray(s)) @ R.T
    u0, ud = L @ (o - mu), L @ d
    lo, hi = -np.inf, np.inf
    for e1 in (-1, 1):
        for e2 in (-1, 1):
            for e3 in (-1, 1):
                e = np.array([e1, e2, e3], float)
                a, b = e @ ud, e @ u0
                if abs(a) < 1e-300:
                    if b > 1:
                        return 0.0
                    continue
                if a > 0:
                    hi = min(hi, (1 - b) / a)
                else:
                    lo = max(lo, (1 - b) / a)
    return max(0.0, hi - lo)


def test_axis_aligned_chord_closed_form(oracle):
    # identity view and rotation, centre on the axis: A = diag(f sx / z, f sy / z, sz), so the chord at
    # pixel offset (dX, dY) is 2 sz (1 - |dX| z / (f sx) - |dY| z / (f sy)) where positive
    f, z = 200.0, 4.0
    cam = scenes.pinhole(128, 128, f)
    s = (0.08, 0.05, 0.03)
    pr = oracle.project_lp(*_one([0.0, 0.0, z], s), cam, _cfg())
    sd = pr["sd"][0]
    np.testing.assert_allclose(pr["A"][0], np.diag([f * s[0] / z, f * s[1] / z, s[2]]), atol=1e-15)
    rng = np.random.default_rng(0)
    for dX, dY in rng.uniform(-5, 5, (200, 2)):
        want = max(0.0, 2 * s[2] * (1 - abs(dX) * z / (f * s[0]) - abs(dY) * z / (f * s[1])))
        assert oracle.lp_chord(sd, dX, dY) == pytest.approx(want, abs=1e-14)
    assert pr["ex"][0] == pytest.approx(f * s[0] / z) and pr["ey"][0] == pytest.approx(f * s[1] / z)
    assert pr["rec"][0, 9] == pytest.approx(z)  # Euclidean depth on the axis


@pytest.mark.parametrize("o", [0.3, 0.8, 0.9985])
def test_density_law_through_the_shortest_axis(oracle, o):
    # along the axis of the smallest half-extent the chord is 2 s_min, so alpha = 1 - exp(-sigma 2 s_min)
    # = 0.99 o (o clipped to 0.999)
    cam = scenes.pinhole(128, 128, 200.0)
    pr = oracle.project_lp(*_one([0.0, 0.0, 4.0], (0.07, 0.05, 0.02), o=o), cam, _cfg())
    sd = pr["sd"][0]
    alpha = 1 - math.exp(-sd[11] * oracle.lp_chord(sd, 0.0, 0.0))
    assert alpha == pytest.approx(0.99 * min(o, 0.999), rel=1e-12)


def test_linearised_chord_tends_to_the_exact_chord(oracle):
    # A linearises the projection at the centre; for octahedra small against their distance the chord
    # of the linearised slabs approaches the exact chord of the pixel ray (error falling with the size)
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(4)
    vm = scenes.yaw_view(18.0, t=(0.2, -0.1, 0.3))
    cam = scenes.pinhole(400, 300, 300.0, vm)
    V = np.asarray(vm, np.float64)
    for _ in range(6):
        q = rng.normal(size=4)
        pc = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(3.0, 5.0)])
        mu = V[:, :3].T @ (pc - V[:, 3])
        s0 = np.array([1.0, 0.6, 0.3]) * rng.uniform(0.7, 1.3, 3)
        errs = []
        for e in [0.04, 0.02, 0.01]:
            s = s0 * e
            pr = oracle.project_lp(*_one(mu, s, q), cam, _cfg())
            sd = pr["sd"][0]
            mx, my, ex, ey = sd[0], sd[1], pr["ex"][0], pr["ey"][0]
            worst = 0.0
            for a, b in [(0.0, 0.0), (0.2, -0.1), (-0.15, 0.25), (0.3, 0.3)]:
                exact = _exact_chord(mu, s, q, cam, mx + a * ex, my + b * ey)
                ln = oracle.lp_chord(sd, a * ex, b * ey)
                worst = max(worst, abs(ln - exact) / (2 * s.max()))
                if a == 0.0:
                    assert exact > 0
            errs.append(worst)
        assert errs[-1] < 0.02 and errs[0] > 1.5 * errs[-1], errs


def test_extents_bound_the_footprint(oracle):
    # ex, ey are the largest pixel offsets of the six vertices: the chord is zero beyond them and
    # positive close to them along the axis of the extreme vertex
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(2)
    cam = scenes.pinhole(400, 300, 300.0, scenes.yaw_view(-10.0, t=(0.1, 0.0, 0.0)))
    for _ in range(10):
        q = rng.normal(size=4)
        s = np.exp(rng.normal(-3, 0.4, 3))
        pr = oracle.project_lp(*_one([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 3.0], s, q), cam, _cfg())
        sd, A = pr["sd"][0], pr["A"][0]
        ex, ey = pr["ex"][0], pr["ey"][0]
        g = np.linspace(-1.2, 1.2, 121)
        inside = [(dx * ex, dy * ey) for dx in g for dy in g if oracle.lp_chord(sd, dx * ex, dy * ey) > 0]
        arr = np.array(inside)
        assert np.abs(arr[:, 0]).max() <= ex * (1 + 1e-12) and np.abs(arr[:, 1]).max() <= ey * (1 + 1e-12)
        k = int(np.argmax(np.abs(A[0])))
        assert oracle.lp_chord(sd, 0.98 * A[0, k], 0.98 * A[1, k]) > 0


def test_cull_is_conservative_and_bounded(oracle):
    cam = scenes.pinhole(96, 80, 96.0)
    cfg = _cfg()
    sc = scenes.uniform_scene(150, seed=6, xy_range=0.8)
    sc.scale *= 2.0
    pr = oracle.project_lp(*sc.arrays(), cam, cfg)
    _, keys, vals = oracle.bin_pairs_lp(pr["rec"], pr["sd"], pr["bbox"], cam, cfg, exact32=False)
    kept = set(zip((keys >> np.uint64(32)).astype(int).tolist(), vals.tolist()))
    req = -math.log1p(-A_T)
    Wt = 6
    checked = 0
    for i in range(sc.n):
        if pr["rec"][i, 11] == 0:
            continue
        sd = pr["sd"][i]
        for y in range(80):
            for x in range(96):
                dt = oracle.lp_chord(sd, x + 0.5 - sd[0], y + 0.5 - sd[1])
                if dt > 0 and sd[11] * dt >= req * (1 + 1e-9):
                    assert ((y // 16) * Wt + x // 16, i) in kept
                    checked += 1
        # the bound is at least every pixel's chord in a tile and at most the diagonal bound 2 min h
        n = [sd[2:5] + a * sd[5:8] + b * sd[8:11] for a, b in ((1, 1), (1, -1), (-1, 1), (-1, -1))]
        two_min_h = 2 * min(1 / abs(v[2]) for v in n)
        bx0, by0, bx1, by1 = pr["bbox"][i]
        for ty in range(by0, by1):
            for tx in range(bx0, bx1):
                b = oracle.lp_tile_bound(sd, tx, ty, cam, cfg)
                assert b <= two_min_h * (1 + 1e-12)
                best = max(oracle.lp_chord(sd, x + 0.5 - sd[0], y + 0.5 - sd[1])
                           for y in range(ty * 16, min(ty * 16 + 16, 80)) for x in range(tx * 16, min(tx * 16 + 16, 96)))
                assert best <= b * (1 + 1e-12) + 1e-15
    assert checked > 500


def _kernel_form(sd64, at):
    """The kernels' shader-data layout [n,20] from the oracle's (slab slopes p, q and half-widths h)."""
    n = sd64.shape[0]
    out = np.zeros((n, 20), np.float32)
    out[:, 0:2] = sd64[:, 0:2]
    out[:, 2] = sd64[:, 11]
    out[:, 3] = np.float32(-math.log1p(-at))
    for i, (a, b) in enumerate(((1, 1), (1, -1), (-1, 1), (-1, -1))):
        nv = sd64[:, 2:5] + a * sd64[:, 5:8] + b * sd64[:, 8:11]
        ok = np.abs(nv[:, 2]) >= 1e-10
        nz = np.where(ok, nv[:, 2], 1.0)
        out[:, 4 + 3 * i] = np.where(ok, nv[:, 0] / nz, 0.0)
        out[:, 5 + 3 * i] = np.where(ok, nv[:, 1] / nz, 0.0)
        out[:, 6 + 3 * i] = np.where(ok, 1.0 / np.abs(nz), np.inf)
    out[:, 16:19] = sd64[:, 12:15]
    return out


def test_fp32_cull_agrees_with_fp64_away_from_ties(oracle):
    rng = np.random.default_rng(9)
    flips = total = 0
    for tile in (8, 16):
        cam = scenes.pinhole(250, 170, 250.0, scenes.yaw_view(7.0))
        cfg = _cfg(tile_w=tile, tile_h=tile)
        sc = scenes.uniform_scene(2000, seed=int(rng.integers(1000)), xy_range=0.9)
        sc.scale *= np.exp(rng.normal(0.5, 0.5, (sc.n, 1)))
        pr = oracle.project_lp(*sc.arrays(), cam, cfg)
        c64, _, _ = oracle.bin_pairs_lp(pr["rec"], pr["sd"], pr["bbox"], cam, cfg, exact32=False)
        c32, _, _ = oracle.bin_pairs_lp(pr["rec"].astype(np.float32), _kernel_form(pr["sd"], A_T), pr["bbox"], cam, cfg,
                                        exact32=True)
        flips += np.abs(c64 - c32).sum()
        total += c64.sum()
    assert total > 15_000 and flips <= 1e-3 * total, (flips, total)


def _tiny_lp_scene(seed, n=6, deg=3):
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2.5, 4.0, n)], 1)
    s = np.exp(rng.normal(-1.5, 0.3, (n, 3)))
    q = rng.normal(size=(n, 4))
    o = 1 / (1 + np.exp(-rng.normal(0.0, 0.8, n)))
    K = (deg + 1) ** 2
    sh = rng.normal(0, 0.3, (n, K, 3))
    sh[:, 0, :] = rng.uniform(0.5, 1.5, (n, 3))
    return [mu, s, q, o, sh]


@pytest.mark.parametrize("seed,deg,yaw,tile", [(0, 3, 0.0, 16), (1, 1, 12.0, 8), (2, 0, -8.0, 16)])
def test_lp_adjoint_matches_central_differences(oracle, seed, deg, yaw, tile):
    cam = scenes.pinhole(32, 32, 32.0, scenes.yaw_view(yaw, t=(0.05, -0.03, 0.1)))
    cfg = _cfg(sh_degree=deg, bg=(0.1, 0.2, 0.3), tile_w=tile, tile_h=tile)
    P = _tiny_lp_scene(seed, deg=deg)
    w = np.random.default_rng(100 + seed).normal(size=(3, 32, 32))
    g = oracle.grads_tiled_lp(P, cam, cfg, w)
    skipped = total = 0
    for a, name in enumerate(["mu", "scale", "quat", "opacity", "sh"]):
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
            lp, sp = oracle.loss_tiled_lp(Pp, cam, cfg, w)
            lm, sm = oracle.loss_tiled_lp(Pm, cam, cfg, w)
            total += 1
            if sp != sm:
                skipped += 1
                fd[idx] = g[name][idx]
                continue
            fd[idx] = (lp - lm) / (2 * h)
        err = np.linalg.norm(g[name] - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-5, (name, err)
    assert skipped <= 0.03 * total
    assert np.abs(g["mu"]).max() > 0 and np.abs(g["quat"]).max() > 0 and np.abs(g["scale"]).max() > 0


def test_lp_single_primitive_opacity_derivative(oracle):
    # axis aligned, on the axis, the smallest half-extent along the view: at the centre pixel
    # C = c alpha with alpha = 0.99 o, so dC/do = 0.99 c
    cam = scenes.Camera(width=32, height=32, fx=40.0, fy=40.0, cx=16.5, cy=16.5,
                        viewmat=np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32), z_near=0.2)
    cfg = _cfg(tile_w=8, tile_h=8)
    P = list(_one([0.0, 0.0, 2.0], (0.12, 0.1, 0.05), o=0.6, rgb=(0.7, 0.2, 0.4)))
    w = np.zeros((3, 32, 32))
    w[0, 16, 16] = 1.0
    g = oracle.grads_tiled_lp(P, cam, cfg, w)
    assert g["opacity"][0] == pytest.approx(0.99 * 0.7, rel=1e-12)
    out = oracle.pipeline_tiled_lp(P, cam, cfg)
    assert out["image"][0, 16, 16] == pytest.approx(0.99 * 0.6 * 0.7, rel=1e-12)
