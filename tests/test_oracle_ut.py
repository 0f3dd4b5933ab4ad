"""Pins of the oracle's 3DGUT path (unscented-transform projection, ray evaluation, ray-offset
cull) against closed forms, brute force along the ray, and the EWA limit."""
import math

import numpy as np
import pytest

from paper_2606_11529_gb300 import scenes

A_T = float(np.float32(1.0 / 255.0))  # the configuration is held in float32 on both sides
DIL = float(np.float32(0.3))


def _one(mu, s, q=(1.0, 0.0, 0.0, 0.0), o=0.8, deg=0):
    return (np.array([mu], np.float64), np.array([s], np.float64), np.array([q], np.float64), np.array([o]),
            np.zeros((1, (deg + 1) ** 2, 3)))


def _cfg(**kw):
    base = dict(method=1, cov_dilation=0.3)
    base.update(kw)
    return scenes.RenderConfig(**base)


def test_on_axis_isotropic_covariance_is_exact(oracle):
    # on the optical axis the sigma points along x and y project symmetrically and the ones along z
    # project onto the centre: mean = principal point, Sigma_2D = (s f / z)^2 I exactly
    cam = scenes.pinhole(256, 256, 300.0)
    for s, z in [(0.05, 3.0), (0.2, 2.0), (0.01, 7.5)]:
        pr = oracle.project_ut(*_one([0.0, 0.0, z], [s, s, s]), cam, _cfg())
        np.testing.assert_allclose(pr["rec"][0, :2], [128.0, 128.0], atol=1e-9)
        c = (s * 300.0 / z) ** 2
        np.testing.assert_allclose(pr["cov0"][0], [c, 0.0, c], rtol=1e-12, atol=1e-12)


def test_mip_opacity_closed_form(oracle):
    cam = scenes.pinhole(256, 256, 300.0)
    s, z, o = 0.02, 4.0, 0.7
    pr = oracle.project_ut(*_one([0.0, 0.0, z], [s, s, s], o=o), cam, _cfg())
    c = (s * 300.0 / z) ** 2
    assert pr["rec"][0, 5] == pytest.approx(o * c / (c + DIL), rel=1e-12)
    assert pr["sd"][0, 12] == pytest.approx(o * c / (c + DIL), rel=1e-12)
    assert pr["rec"][0, 10] == pytest.approx(math.log(pr["rec"][0, 5] / A_T), rel=1e-12)


@pytest.mark.parametrize("xy", [(0.3, -0.2), (-0.5, 0.4)])
def test_unscented_covariance_tends_to_ewa(oracle, xy):
    # off axis the projection is non-linear; the UT covariance approaches the first-order (EWA,
    # unclamped, undilated) closed form s^2 (f/z)^2 [[1 + x^2/z^2, xy/z^2], [xy/z^2, 1 + y^2/z^2]]
    # with an error that falls like (s/z)^2
    f, z = 300.0, 4.0
    cam = scenes.pinhole(256, 256, f)
    x, y = xy
    errs = []
    for s in [0.04, 0.02, 0.01]:
        pr = oracle.project_ut(*_one([x, y, z], [s, s, s]), cam, _cfg())
        k = (s * f / z) ** 2
        ewa = np.array([k * (1 + x * x / z / z), k * x * y / z / z, k * (1 + y * y / z / z)])
        errs.append(np.abs(pr["cov0"][0] - ewa).max() / k)
    assert errs[-1] < 1e-4
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_ray_response_is_the_maximum_along_the_ray(oracle):
    from scipy.optimize import minimize_scalar
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    cam = scenes.pinhole(64, 64, 64.0)
    for _ in range(40):
        mu = rng.uniform([-0.5, -0.5, 2.0], [0.5, 0.5, 5.0])
        s = np.exp(rng.normal(-2.5, 0.5, 3))
        q = rng.normal(size=4)
        pr = oracle.project_ut(*_one(mu, s, q), cam, _cfg())
        sd = pr["sd"][0]
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is (x, y, z, w)
        Sinv = R @ np.diag(1.0 / s ** 2) @ R.T
        px, py = rng.integers(0, 64, 2)
        d = oracle.pixel_ray(px, py, cam)
        f = lambda t: 0.5 * (t * d - mu) @ Sinv @ (t * d - mu)
        best = minimize_scalar(f, bounds=(0.0, 50.0), method="bounded", options=dict(xatol=1e-12)).fun
        assert oracle.ut_response(sd, d) == pytest.approx(math.exp(-best), rel=1e-7, abs=1e-300)
    # a ray through the mean has response 1
    pr = oracle.project_ut(*_one([0.0, 0.0, 3.0], [0.1, 0.2, 0.05], (0.9, 0.1, -0.3, 0.2)), cam, _cfg())
    assert oracle.ut_response(pr["sd"][0], np.array([0.0, 0.0, 1.0])) == pytest.approx(1.0, abs=1e-15)


def test_pixel_ray_through_centre(oracle):
    cam = scenes.pinhole(64, 48, 50.0)
    d = oracle.pixel_ray(31, 23, cam)  # pixel centre (31.5, 23.5) is off the principal point by -0.5
    expect = np.array([-0.5 / 50.0, -0.5 / 50.0, 1.0])
    np.testing.assert_allclose(d, expect / np.linalg.norm(expect), rtol=1e-14)
    vm = scenes.yaw_view(20.0)
    camr = scenes.pinhole(64, 48, 50.0, vm)
    dr = oracle.pixel_ray(31, 23, camr)
    np.testing.assert_allclose(dr, np.asarray(vm, np.float64)[:, :3].T @ (expect / np.linalg.norm(expect)),
                               rtol=1e-6)


def test_single_gaussian_image_closed_form(oracle):
    # isotropic Gaussian: the response along a ray from the origin is exp(-|mu x d|^2 / (2 s^2))
    cam = scenes.pinhole(48, 40, 60.0)
    cfg = _cfg(tile_w=8, tile_h=8)
    mu, s, o = np.array([0.05, -0.03, 2.5]), 0.08, 0.9
    arrs = _one(mu, [s, s, s], o=o)
    arrs = arrs[:4] + (np.full((1, 1, 3), (0.7 - 0.5) / 0.28209479177387814),)
    out = oracle.pipeline_tiled_ut(arrs, cam, cfg)
    op = out["proj"]["rec"][0, 5]
    img = out["image"][0]
    checked = 0
    for py in range(40):
        for px in range(48):
            d = oracle.pixel_ray(px, py, cam)
            g = math.exp(-np.sum(np.cross(mu, d) ** 2) / (2 * s * s))
            a = min(0.99, op * g)
            ref = 0.7 * a if (g > 0.0113 and a >= A_T) else 0.0
            if abs(a - A_T) < 1e-9 or abs(g - 0.0113) < 1e-9:
                continue
            assert img[py, px] == pytest.approx(ref, abs=1e-12)
            checked += 1
    assert checked > 1800 and img.max() > 0.3


def test_offset_cull_is_conservative_for_the_footprint(oracle):
    # every pixel whose centre (x + 0.5, y + 0.5) reaches alpha_t under the UT 2D footprint lies in
    # a kept tile of its primitive
    cam = scenes.pinhole(96, 80, 96.0)
    cfg = _cfg()
    sc = scenes.uniform_scene(120, seed=5, xy_range=0.8)
    pr = oracle.project_ut(sc.mu, sc.scale, sc.quat, sc.opacity, sc.sh, cam, cfg)
    _, keys, vals = oracle.bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False)
    kept = set(zip((keys >> np.uint64(32)).astype(int).tolist(), vals.tolist()))
    ys, xs = np.mgrid[0:80, 0:96]
    Wt = 6
    for i in range(sc.n):
        R = pr["rec"][i]
        if R[11] == 0:
            continue
        dx, dy = xs + 0.5 - R[0], ys + 0.5 - R[1]
        q = R[2] * dx * dx + 2 * R[3] * dx * dy + R[4] * dy * dy
        hit = 0.5 * q < R[10] * (1 - 1e-9)
        for t in set(((ys[hit] // 16) * Wt + xs[hit] // 16).tolist()):
            assert (t, i) in kept


def test_row_form_with_ray_offset(oracle):
    rng = np.random.default_rng(12)
    cam = scenes.pinhole(250, 170, 250.0)
    flips = total = 0
    for tile in (8, 16):
        cfg = _cfg(tile_w=tile, tile_h=tile)
        Wt, Ht = (250 + tile - 1) // tile, (170 + tile - 1) // tile
        for _ in range(60):
            A = rng.normal(size=(2, 2))
            S = A @ A.T * rng.uniform(1, 40) + 0.3 * np.eye(2)
            C = np.linalg.inv(S)
            rec = np.zeros(12)
            rec[0], rec[1] = rng.uniform(-30, 280), rng.uniform(-30, 200)
            rec[2:5] = C[0, 0], C[0, 1], C[1, 1]
            rec[5] = rng.uniform(0.01, 1.0)
            rec[10] = math.log(rec[5] / A_T)
            rec[11] = 1.0
            for ty in range(Ht):
                for tx in range(Wt):
                    a = oracle.cull_one(rec, tx, ty, cam, cfg, form=0)
                    assert oracle.cull_one(rec, tx, ty, cam, cfg, form=1) == a
                    flips += oracle.cull_one(rec, tx, ty, cam, cfg, form=2) != a
                    total += 1
    assert total > 20_000 and flips <= total * 1e-4


def test_unscented_mean_is_exact_to_fourth_order_along_depth(oracle):
    # a Gaussian stretched only along the optical axis at lateral offset x0: u = f x0 / (z + t) + cx,
    # t ~ N(0, s^2).  Symmetric sigma points at +-sqrt(3) s match the moments of t up to the fifth, so
    # the UT mean differs from the true expectation (Gauss-Hermite quadrature) only at O(s^6)
    from numpy.polynomial.hermite_e import hermegauss
    f, z, x0 = 200.0, 4.0, 0.6
    cam = scenes.pinhole(256, 256, f)
    tq, wq = hermegauss(20)  # nodes within 8 sigma: the pole of 1/(z + t) stays outside
    wq = wq / wq.sum()
    errs = []
    for s in [0.4, 0.2, 0.1]:
        # no low-pass dilation: the Mip-Splatting factor would fade the degenerate footprint out
        pr = oracle.project_ut(*_one([x0, 0.0, z], [1e-9, 1e-9, s]), cam, _cfg(cov_dilation=0.0))
        true = np.sum(wq * (f * x0 / (z + s * tq))) + 128.0
        errs.append(abs(pr["rec"][0, 0] - true))
        assert abs(pr["rec"][0, 1] - 128.0) < 1e-9
    assert errs[0] / errs[1] > 40 and errs[1] / errs[2] > 40, errs


def test_unscented_covariance_depth_stretched_closed_form(oracle):
    # same configuration: the sigma points project to u0 = A / z (centre and the four lateral points)
    # and u_+- = A / (z +- h), h = sqrt(3) s, A = f x0.  With mean weights (0, 1/6 x 6) and covariance
    # weights (2, 1/6 x 6) the UT gives, with d = mean - u0 = A h^2 / (3 z (z^2 - h^2)):
    #   var = (2 + 4/6) d^2 + ((u_+ - u0 - d)^2 + (u_- - u0 - d)^2) / 6
    f, z, x0, s = 200.0, 4.0, 0.6, 0.3
    cam = scenes.pinhole(256, 256, f)
    pr = oracle.project_ut(*_one([x0, 0.0, z], [1e-9, 1e-9, s]), cam, _cfg(cov_dilation=0.0))
    A, h = f * x0, math.sqrt(3.0) * s
    d = A * h * h / (3 * z * (z * z - h * h))
    ep, em = -A * h / (z * (z + h)), A * h / (z * (z - h))
    var = (2 + 4 / 6) * d * d + ((ep - d) ** 2 + (em - d) ** 2) / 6
    assert pr["rec"][0, 0] == pytest.approx(128.0 + A / z + d, rel=1e-13)
    assert pr["cov0"][0, 0] == pytest.approx(var, rel=1e-9)
    assert abs(pr["cov0"][0, 1]) < 1e-12 and pr["cov0"][0, 2] == pytest.approx(2 * (f * 1e-9 / z) ** 2, rel=1e-3)


def test_unscented_covariance_rotated_anisotropic_tends_to_jacobian_form(oracle):
    # Sigma_2D -> J W R S^2 R^T W^T J^T (the first-order form) for small anisotropic, rotated Gaussians
    # seen through a rotated and translated camera; the rotation comes from scipy, not the oracle
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(8)
    f = 250.0
    vm = scenes.yaw_view(25.0, t=(0.3, -0.2, 0.5))
    cam = scenes.pinhole(256, 256, f, vm)
    V = np.asarray(vm, np.float64)
    for _ in range(6):
        q = rng.normal(size=4)
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        pc = np.array([rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(3.0, 5.0)])
        mu = V[:3, :3].T @ (pc - V[:3, 3])
        s0 = np.array([1.0, 0.4, 0.15]) * rng.uniform(0.5, 1.5, 3)
        errs = []
        for e in [0.02, 0.01, 0.005]:
            s = s0 * e
            pr = oracle.project_ut(*_one(mu, s, q), cam, _cfg())
            x, y, z = pc
            J = np.array([[f / z, 0, -f * x / z / z], [0, f / z, -f * y / z / z]])
            T = J @ V[:3, :3] @ Rm @ np.diag(s * s) @ Rm.T @ V[:3, :3].T @ J.T
            got = pr["cov0"][0]
            scale = np.abs(T).max()
            errs.append(max(abs(got[0] - T[0, 0]), abs(got[1] - T[0, 1]), abs(got[2] - T[1, 1])) / scale)
            np.testing.assert_allclose(pr["rec"][0, :2], [f * x / z + 128, f * y / z + 128], atol=scale ** 0.5 * e * 5)
        assert errs[-1] < 2e-4 and errs[0] / errs[1] > 3 and errs[1] / errs[2] > 3, errs


def test_ray_response_with_translated_camera(oracle):
    from scipy.optimize import minimize_scalar
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(4)
    vm = scenes.yaw_view(-30.0, t=(0.4, 0.1, -0.3))
    V = np.asarray(vm, np.float64)
    o = -V[:3, :3].T @ V[:3, 3]
    cam = scenes.pinhole(64, 64, 64.0, vm)
    for _ in range(20):
        pc = rng.uniform([-0.4, -0.4, 2.0], [0.4, 0.4, 4.0])
        mu = V[:3, :3].T @ (pc - V[:3, 3])
        s = np.exp(rng.normal(-2.0, 0.4, 3))
        q = rng.normal(size=4)
        pr = oracle.project_ut(*_one(mu, s, q), cam, _cfg())
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sinv = R @ np.diag(1.0 / s ** 2) @ R.T
        px, py = rng.integers(0, 64, 2)
        d = oracle.pixel_ray(px, py, cam)
        fn = lambda t: 0.5 * (o + t * d - mu) @ Sinv @ (o + t * d - mu)
        best = minimize_scalar(fn, bounds=(0.0, 50.0), method="bounded", options=dict(xatol=1e-12)).fun
        assert oracle.ut_response(pr["sd"][0], d) == pytest.approx(math.exp(-best), rel=1e-7, abs=1e-300)


def _tiny_ut_scene(seed, n=6, deg=3):
    rng = np.random.default_rng(seed)
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2.5, 4.0, n)], 1)
    s = np.exp(rng.normal(-1.6, 0.3, (n, 3)))
    q = rng.normal(size=(n, 4))
    o = 1 / (1 + np.exp(-rng.normal(0.5, 0.8, n)))
    K = (deg + 1) ** 2
    sh = rng.normal(0, 0.3, (n, K, 3))
    sh[:, 0, :] = rng.uniform(0.5, 1.5, (n, 3))  # colours stay away from the max(0, .) kink
    return [mu, s, q, o, sh]


@pytest.mark.parametrize("seed,deg,yaw,tile", [(0, 3, 0.0, 16), (1, 1, 12.0, 8), (2, 0, -8.0, 16)])
def test_ut_adjoint_matches_central_differences(oracle, seed, deg, yaw, tile):
    # FP64 central differences of the oracle's own tiled 3DGUT forward; a step that flips any
    # decision (a tile list, a gate) is left out and must stay rare
    cam = scenes.pinhole(32, 32, 32.0, scenes.yaw_view(yaw, t=(0.05, -0.03, 0.1)))
    cfg = _cfg(sh_degree=deg, bg=(0.1, 0.2, 0.3), tile_w=tile, tile_h=tile)
    P = _tiny_ut_scene(seed, deg=deg)
    w = np.random.default_rng(100 + seed).normal(size=(3, 32, 32))
    g = oracle.grads_tiled_ut(P, cam, cfg, w)
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
            lp, sp = oracle.loss_tiled_ut(Pp, cam, cfg, w)
            lm, sm = oracle.loss_tiled_ut(Pm, cam, cfg, w)
            total += 1
            if sp != sm:
                skipped += 1
                fd[idx] = g[name][idx]
                continue
            fd[idx] = (lp - lm) / (2 * h)
        err = np.linalg.norm(g[name] - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-5, (name, err)
    assert skipped <= 0.02 * total
    assert np.abs(g["mu"]).max() > 0 and np.abs(g["quat"]).max() > 0 and np.abs(g["scale"]).max() > 0


def test_ut_single_gaussian_opacity_derivative_closed_form(oracle):
    # one isotropic Gaussian on the axis, white-free colour c: C = c a, a = o m G, so
    # dC/do = c m G with m = k / (k + dil), k = (s f / z)^2, G = exp(-|mu x d|^2 / (2 s^2))
    cam = scenes.pinhole(32, 32, 40.0)
    cfg = _cfg(tile_w=8, tile_h=8)
    mu, s, o, c = np.array([0.0, 0.0, 2.0]), 0.1, 0.6, 0.7
    P = [np.array([mu]), np.array([[s, s, s]]), np.array([[1.0, 0, 0, 0]]), np.array([o]),
         np.full((1, 1, 3), (c - 0.5) / 0.28209479177387814)]
    w = np.zeros((3, 32, 32))
    w[0, 17, 18] = 1.0
    g = oracle.grads_tiled_ut(P, cam, cfg, w)
    k = (s * 40.0 / 2.0) ** 2
    d = oracle.pixel_ray(18, 17, cam)
    G = math.exp(-np.sum(np.cross(mu, d) ** 2) / (2 * s * s))
    assert g["opacity"][0] == pytest.approx(c * k / (k + DIL) * G, rel=1e-12)
    assert g["sh"][0, 0, 0] == pytest.approx(0.28209479177387814 * o * k / (k + DIL) * G, rel=1e-12)


def test_fisheye_equidistant_closed_form(oracle):
    # k = 0: a point at angle theta from the axis lands at radius f theta from the principal point
    cam = scenes.fisheye(400, 300, 150.0, dist=(0.0, 0.0, 0.0, 0.0))
    rng = np.random.default_rng(0)
    for _ in range(50):
        th, ph = rng.uniform(0, 1.2), rng.uniform(-math.pi, math.pi)
        d = rng.uniform(0.5, 5)
        pc = d * np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        uv = oracle.fisheye_project(pc, cam)[0]
        np.testing.assert_allclose(uv, [200 + 150 * th * math.cos(ph), 150 + 150 * th * math.sin(ph)], atol=1e-10)
    # the radial polynomial
    k = (0.05, -0.01, 0.001, 0.0002)
    cam = scenes.fisheye(400, 300, 150.0, dist=k)
    th = 0.9
    uv = oracle.fisheye_project(np.array([math.sin(th), 0.0, math.cos(th)]), cam)[0]
    kk = [float(np.float32(v)) for v in k]
    assert uv[0] - 200 == pytest.approx(150 * th * (1 + kk[0] * th ** 2 + kk[1] * th ** 4 + kk[2] * th ** 6 + kk[3] * th ** 8),
                                        rel=1e-12)


def test_fisheye_pixel_ray_projects_back_to_its_pixel(oracle):
    vm = scenes.yaw_view(12.0, t=(0.1, -0.2, 0.3))
    cam = scenes.fisheye(320, 240, 110.0, dist=(0.05, -0.01, 0.001, 0.0), viewmat=vm)
    V = np.asarray(cam.viewmat, np.float64)
    o = -V[:, :3].T @ V[:, 3]
    rng = np.random.default_rng(1)
    for _ in range(60):
        x, y = int(rng.integers(0, 320)), int(rng.integers(0, 240))
        d = oracle.pixel_ray(x, y, cam)
        # (the float32-rounded view rotation is orthonormal to ~1e-7)
        assert np.linalg.norm(d) == pytest.approx(1.0, abs=1e-6)
        p = o + rng.uniform(0.5, 8.0) * d
        pc = V[:, :3] @ p + V[:, 3]
        np.testing.assert_allclose(oracle.fisheye_project(pc, cam)[0], [x + 0.5, y + 0.5], atol=1e-4)
    # with the identity view (exact in float32) the round trip is exact to double rounding
    cam = scenes.fisheye(320, 240, 110.0, dist=(0.05, -0.01, 0.001, 0.0))
    for _ in range(60):
        x, y = int(rng.integers(0, 320)), int(rng.integers(0, 240))
        pc = rng.uniform(0.5, 8.0) * oracle.pixel_ray(x, y, cam)
        np.testing.assert_allclose(oracle.fisheye_project(pc, cam)[0], [x + 0.5, y + 0.5], atol=1e-9)


def test_single_gaussian_image_fisheye(oracle):
    cam = scenes.fisheye(48, 40, 40.0)
    cfg = _cfg(tile_w=8, tile_h=8)
    mu, s, o = np.array([0.35, -0.2, 2.0]), 0.08, 0.9
    arrs = _one(mu, [s, s, s], o=o)
    arrs = arrs[:4] + (np.full((1, 1, 3), (0.7 - 0.5) / 0.28209479177387814),)
    out = oracle.pipeline_tiled_ut(arrs, cam, cfg)
    op = out["proj"]["rec"][0, 5]
    img = out["image"][0]
    checked = 0
    for py in range(40):
        for px in range(48):
            d = oracle.pixel_ray(px, py, cam)
            g = math.exp(-np.sum(np.cross(mu, d) ** 2) / (2 * s * s))
            a = min(0.99, op * g)
            if abs(a - A_T) < 1e-9 or abs(g - 0.0113) < 1e-9:
                continue
            inside = out["ranges"][(py // 8) * 6 + px // 8]
            listed = 0 in out["vals"][inside[0]:inside[1]]
            ref = 0.7 * a if (listed and g > 0.0113 and a >= A_T) else 0.0
            assert img[py, px] == pytest.approx(ref, abs=1e-12)
            checked += 1
    assert checked > 1800 and img.max() > 0.3


def test_ut_adjoint_fisheye_central_differences(oracle):
    cam = scenes.fisheye(32, 32, 20.0, viewmat=scenes.yaw_view(9.0, t=(0.05, -0.03, 0.1)))
    cfg = _cfg(sh_degree=1, bg=(0.1, 0.2, 0.3), tile_w=8, tile_h=8)
    P = _tiny_ut_scene(7, deg=1)
    P[0][:, :2] *= 2.5  # off-axis, where the fisheye departs from the pinhole
    w = np.random.default_rng(17).normal(size=(3, 32, 32))
    g = oracle.grads_tiled_ut(P, cam, cfg, w)
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
            lp, sp = oracle.loss_tiled_ut(Pp, cam, cfg, w)
            lm, sm = oracle.loss_tiled_ut(Pm, cam, cfg, w)
            total += 1
            if sp != sm:
                skipped += 1
                fd[idx] = g[name][idx]
                continue
            fd[idx] = (lp - lm) / (2 * h)
        err = np.linalg.norm(g[name] - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err < 1e-5, (name, err)
    assert skipped <= 0.03 * total
    assert np.abs(g["mu"]).max() > 0
