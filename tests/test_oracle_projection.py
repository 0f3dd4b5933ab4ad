"""Pins of the oracle's projection and SH colour against closed forms,
invariants and library routines (no GPU)."""
import math

import numpy as np
import pytest
import scipy.special

from paper_2606_11529_gb300 import scenes


def _cfg(**kw):
    c = scenes.RenderConfig()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _one(oracle, mu, s, q, o=0.8, cam=None, cfg=None, sh=None):
    cam = cam or scenes.pinhole(256, 256, 256.0)
    cfg = cfg or _cfg(cov_dilation=0.0)
    K = (cfg.sh_degree + 1) ** 2
    sh = np.zeros((1, K, 3)) if sh is None else sh
    return oracle.project(np.array([mu], float), np.array([s], float), np.array([q], float), np.array([o]), sh,
                          cam, cfg)


def test_on_axis_isotropic_closed_form(oracle):
    # mu on the optical axis, isotropic sigma: Sigma_2D = (sigma f / z)^2 I, mu_2D = (cx, cy)
    for z, sig in [(2.0, 0.05), (5.0, 0.2), (11.0, 0.01)]:
        q = np.random.default_rng(1).normal(size=4)
        r = _one(oracle, [0.0, 0.0, z], [sig] * 3, q)
        cov = r["cov"][0]
        expect = (sig * 256.0 / z) ** 2
        assert abs(cov[0] - expect) <= 1e-12 * expect and abs(cov[2] - expect) <= 1e-12 * expect
        assert abs(cov[1]) <= 1e-12 * expect
        assert r["rec"][0, 0] == pytest.approx(128.0, abs=1e-12) and r["rec"][0, 1] == pytest.approx(128.0, abs=1e-12)
        assert r["rec"][0, 9] == pytest.approx(z)


def test_off_axis_isotropic_closed_form(oracle):
    # Sigma_2D = sigma^2 (f/z)^2 [[1 + x^2/z^2, xy/z^2], [xy/z^2, 1 + y^2/z^2]]
    x, y, z, sig, f = 0.3, -0.2, 3.0, 0.07, 256.0
    r = _one(oracle, [x, y, z], [sig] * 3, [1, 0, 0, 0])
    k = sig * sig * (f / z) ** 2
    exp = np.array([k * (1 + x * x / z ** 2), k * x * y / z ** 2, k * (1 + y * y / z ** 2)])
    np.testing.assert_allclose(r["cov"][0], exp, rtol=1e-12)
    np.testing.assert_allclose(r["rec"][0, :2], [f * x / z + 128, f * y / z + 128], rtol=1e-14)


def test_anisotropic_rotation_swaps_axes(oracle):
    sx, sy, z = 0.1, 0.03, 4.0
    f = 256.0
    r0 = _one(oracle, [0, 0, z], [sx, sy, 0.02], [1, 0, 0, 0])
    np.testing.assert_allclose(r0["cov"][0], [(sx * f / z) ** 2, 0, (sy * f / z) ** 2], atol=1e-12)
    # 90 degrees about the optical axis: q = (cos 45, 0, 0, sin 45); unnormalised input is normalised
    c = math.cos(math.pi / 4)
    r1 = _one(oracle, [0, 0, z], [sx, sy, 0.02], [3 * c, 0, 0, 3 * c])
    np.testing.assert_allclose(r1["cov"][0], [(sy * f / z) ** 2, 0, (sx * f / z) ** 2], atol=1e-12)
    # 90 degrees about the x axis swaps the y and z scales
    r2 = _one(oracle, [0, 0, z], [sx, sy, 0.02], [c, c, 0, 0])
    np.testing.assert_allclose(r2["cov"][0], [(sx * f / z) ** 2, 0, (0.02 * f / z) ** 2], atol=1e-12)


def test_isotropic_rotation_invariance_and_psd(oracle):
    rng = np.random.default_rng(3)
    base = _one(oracle, [0.2, 0.1, 3.0], [0.05] * 3, [1, 0, 0, 0])["cov"][0]
    for _ in range(5):
        r = _one(oracle, [0.2, 0.1, 3.0], [0.05] * 3, rng.normal(size=4))["cov"][0]
        np.testing.assert_allclose(r, base, rtol=1e-12)
    sc = scenes.uniform_scene(500, seed=4)
    pr = oracle.project_scene(sc, scenes.pinhole(256, 256, 256.0), _cfg())
    cov = pr["cov"][pr["rec"][:, 11] > 0]
    assert np.all(cov[:, 0] > 0) and np.all(cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2 > 0)


def test_conic_is_inverse_and_dilation(oracle):
    sc = scenes.uniform_scene(200, seed=5)
    cfg = _cfg(cov_dilation=0.3)
    pr = oracle.project_scene(sc, scenes.pinhole(256, 256, 256.0), cfg)
    pr0 = oracle.project_scene(sc, scenes.pinhole(256, 256, 256.0), _cfg(cov_dilation=0.0))
    vis = pr["rec"][:, 11] > 0
    for i in np.nonzero(vis)[0][:50]:
        a, b, c = pr["cov"][i]
        A = np.array([[a, b], [b, c]])
        cn = pr["rec"][i, 2:5]
        B = np.array([[cn[0], cn[1]], [cn[1], cn[2]]])
        np.testing.assert_allclose(A @ B, np.eye(2), atol=1e-9)
        # dilation adds float32(0.3) to the diagonal only
        np.testing.assert_allclose(pr["cov"][i] - pr0["cov"][i], [float(np.float32(0.3)), 0, float(np.float32(0.3))],
                                   atol=1e-9)


def test_view_transform_invariance(oracle):
    # moving the world rigidly and the camera with it leaves every footprint unchanged
    sc = scenes.uniform_scene(300, seed=6)
    cam0 = scenes.pinhole(256, 256, 256.0)
    cfg = _cfg()
    r0 = oracle.project_scene(sc, cam0, cfg)
    from scipy.spatial.transform import Rotation
    Rw = Rotation.from_euler("xyz", [0.3, -0.4, 0.2]).as_matrix()
    tw = np.array([0.5, -1.0, 2.0])
    # world' = Rw^T (world - tw): camera' viewmat = [Rw | tw] maps world' back to camera space
    mu2 = (sc.mu.astype(float) - tw) @ Rw
    qr = Rotation.from_matrix(Rw.T)
    qs = Rotation.from_quat(np.roll(sc.quat.astype(float), -1, axis=1))  # scipy is (x,y,z,w)
    q2 = np.roll((qr * qs).as_quat(), 1, axis=1)
    vm = np.hstack([Rw, tw[:, None]])
    cam1 = scenes.Camera(256, 256, 256.0, 256.0, 128.0, 128.0, vm.astype(np.float64), 0.2)

    class _Cam:  # keep float64 viewmat (no float32 rounding) for this exact check
        width, height, fx, fy, cx, cy, z_near = 256, 256, 256.0, 256.0, 128.0, 128.0, 0.2
        viewmat = vm
    ca = oracle.cam_array(_Cam)
    ca[6:18] = vm.reshape(12)
    import ctypes
    n = sc.n
    rec = np.zeros((n, 12))
    bb = np.zeros((n, 4), np.int32)
    tc = np.zeros(n, np.int32)
    f64 = lambda a: np.ascontiguousarray(a, np.float64)
    P = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int32)
    args = [f64(mu2), f64(sc.scale), f64(q2), f64(sc.opacity), f64(sc.sh)]
    fa = oracle.cfg_array(cfg)
    oracle.lib().oracle_project(n, *[a.ctypes.data_as(P) for a in args], ca.ctypes.data_as(P),
                                fa.ctypes.data_as(P), rec.ctypes.data_as(P), bb.ctypes.data_as(I),
                                tc.ctypes.data_as(I), None, None)
    vis = r0["rec"][:, 11] > 0
    np.testing.assert_allclose(rec[vis][:, :11], r0["rec"][vis][:, :11], rtol=1e-9, atol=1e-9)
    assert cam1.width == 256


def test_jacobian_clamp(oracle):
    # far off-axis: x/z beyond 1.3 * tan(half fov) is clamped inside the Jacobian only
    z, x, sig, f = 2.0, 2.0 * 1.3 * 0.5 * 1.5, 0.5, 256.0  # x/z = 0.975 > 1.3 * 0.5; wide enough to stay visible
    r = _one(oracle, [x, 0.0, z], [sig] * 3, [1, 0, 0, 0])
    lim = float(np.float32(1.3)) * 0.5
    J = np.array([[f / z, 0, -f * lim / z], [0, f / z, 0]])
    exp = sig * sig * J @ J.T
    np.testing.assert_allclose(r["cov"][0], [exp[0, 0], exp[0, 1], exp[1, 1]], rtol=1e-12)
    assert r["rec"][0, 0] == pytest.approx(f * x / z + 128.0)


def test_visibility_rules(oracle):
    r = _one(oracle, [0, 0, 0.1], [0.05] * 3, [1, 0, 0, 0])  # z < z_near
    assert r["tc"][0] == 0 and r["rec"][0, 11] == 0
    r = _one(oracle, [0, 0, 3.0], [0.05] * 3, [1, 0, 0, 0], o=0.5 / 255)  # o < alpha_t
    assert r["tc"][0] == 0
    r = _one(oracle, [50.0, 0, 3.0], [0.05] * 3, [1, 0, 0, 0])  # far outside the image
    assert r["tc"][0] == 0
    r = _one(oracle, [0, 0, 3.0], [0.05] * 3, [1, 0, 0, 0])
    assert r["tc"][0] > 0 and r["rec"][0, 11] == 1


def test_extent_is_exact_axis_extent_of_alpha_gate(oracle):
    # ex = max |dx| over the ellipse {o exp(-d^T conic d / 2) >= alpha_t}
    rng = np.random.default_rng(7)
    for _ in range(5):
        r = _one(oracle, [rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 3.0], np.exp(rng.normal(-3, 0.5, 3)),
                 rng.normal(size=4), o=0.7, cfg=_cfg())
        a, b, c = r["cov"][0]
        lt = r["rec"][0, 10]
        assert lt == pytest.approx(math.log(0.7 / float(np.float32(1 / 255))))
        # parametrise the boundary d = sqrt(2 lt) L u, Sigma = L L^T
        L = np.linalg.cholesky(np.array([[a, b], [b, c]]))
        th = np.linspace(0, 2 * np.pi, 200001)
        d = math.sqrt(2 * lt) * (L @ np.stack([np.cos(th), np.sin(th)]))
        ex = math.sqrt(2 * lt * a)
        ey = math.sqrt(2 * lt * c)
        assert np.abs(d[0]).max() == pytest.approx(ex, rel=1e-8)
        assert np.abs(d[1]).max() == pytest.approx(ey, rel=1e-8)
        w = 16
        assert r["pre"][0, 0] == pytest.approx((r["rec"][0, 0] - ex) / w)
        assert r["pre"][0, 3] == pytest.approx((r["rec"][0, 1] + ey) / w)


def test_bbox_contains_every_contributing_pixel(oracle):
    cam = scenes.pinhole(128, 96, 128.0)
    cfg = _cfg()
    sc = scenes.uniform_scene(60, seed=8, xy_range=0.6)
    pr = oracle.project_scene(sc, cam, cfg)
    ys, xs = np.mgrid[0:96, 0:128]
    for i in range(sc.n):
        R = pr["rec"][i]
        if R[11] == 0:
            continue
        dx, dy = xs - R[0], ys - R[1]
        power = -0.5 * (R[2] * dx * dx + 2 * R[3] * dx * dy + R[4] * dy * dy)
        alpha = np.minimum(float(np.float32(0.99)), R[5] * np.exp(power))
        hit = alpha >= float(np.float32(1 / 255))
        tx, ty = xs[hit] // 16, ys[hit] // 16
        bb = pr["bbox"][i]
        assert np.all((tx >= bb[0]) & (tx < bb[2]) & (ty >= bb[1]) & (ty < bb[3]))


def test_sh_orthonormal_by_quadrature(oracle):
    # int_{S^2} Y_i Y_j = delta_ij; Gauss-Legendre in z (exact to degree 39) x uniform phi
    zs, wz = np.polynomial.legendre.leggauss(20)
    nphi = 40
    M = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        s = math.sqrt(1 - z * z)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = oracle.sh_basis(3, np.array([s * math.cos(ph), s * math.sin(ph), z]))
            M += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(M, np.eye(16), atol=1e-12)


def test_sh_degree0_and_gradient(oracle):
    Y = oracle.sh_basis(0, np.array([0.3, -0.4, math.sqrt(1 - 0.25)]))
    assert Y[0] == pytest.approx(0.5 / math.sqrt(math.pi), rel=1e-15)
    rng = np.random.default_rng(9)
    for _ in range(5):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, G = oracle.sh_basis(3, d, with_grad=True)
        h = 1e-6
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            fd = (oracle.sh_basis(3, d + e) - oracle.sh_basis(3, d - e)) / (2 * h)
            np.testing.assert_allclose(G[:, j], fd, atol=1e-8)


def test_sh_degree1_is_linear_in_direction(oracle):
    # degree-1 real SH span {x, y, z}: each is a multiple of one coordinate, norm sqrt(3/(4 pi))
    rng = np.random.default_rng(10)
    d = rng.normal(size=(20, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Ys = np.array([oracle.sh_basis(1, x) for x in d])[:, 1:]
    coef, *_ = np.linalg.lstsq(d, Ys, rcond=None)
    np.testing.assert_allclose(d @ coef, Ys, atol=1e-13)
    np.testing.assert_allclose(np.sort(np.abs(coef).max(axis=0)), [math.sqrt(3 / (4 * math.pi))] * 3, rtol=1e-13)
    assert np.count_nonzero(np.abs(coef) > 1e-12) == 3


def test_sh_colour_degree0_recovers_rgb(oracle):
    sc = scenes.uniform_scene(50, seed=11)
    pr = oracle.project_scene(sc, scenes.pinhole(256, 256, 256.0), _cfg())
    rgb = sc.sh[:, 0, :] / math.sqrt(4 * math.pi) + 0.5
    vis = pr["rec"][:, 11] > 0
    np.testing.assert_allclose(pr["rec"][vis, 6:9], rgb[vis], atol=1e-6)


def _sh_closed_forms(x, y, z):
    """The 16 real spherical harmonics of degrees 0-3 written out as polynomials of the unit
    direction (x, y, z), index k = l^2 + l + m, from Y_l^m = sqrt(2) K_l^m P_l^|m|(z) cos(m phi)
    (m > 0), sin(|m| phi) (m < 0), K_l^m P_l^m(z) (m = 0), where P_l^m carries the Condon-Shortley
    phase (-1)^m: every odd |m| function changes sign relative to the phase-free table."""
    pi = math.pi
    return np.array([
        0.5 / math.sqrt(pi),
        -math.sqrt(3 / (4 * pi)) * y,
        math.sqrt(3 / (4 * pi)) * z,
        -math.sqrt(3 / (4 * pi)) * x,
        0.5 * math.sqrt(15 / pi) * x * y,
        -0.5 * math.sqrt(15 / pi) * y * z,
        0.25 * math.sqrt(5 / pi) * (3 * z * z - 1),
        -0.5 * math.sqrt(15 / pi) * x * z,
        0.25 * math.sqrt(15 / pi) * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
        0.5 * math.sqrt(105 / pi) * x * y * z,
        -0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
        0.25 * math.sqrt(7 / pi) * (5 * z ** 3 - 3 * z),
        -0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
        0.25 * math.sqrt(105 / pi) * z * (x * x - y * y),
        -0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y),
    ])


def test_sh_basis_closed_forms_every_function(oracle):
    # every one of the 16 functions, at axis directions and random ones: a swapped m <-> -m, a
    # flipped sign or an exchanged degree changes at least one value
    rng = np.random.default_rng(21)
    dirs = [np.eye(3)[i] for i in range(3)] + [-np.eye(3)[i] for i in range(3)]
    dirs += [v / np.linalg.norm(v) for v in rng.normal(size=(12, 3))]
    for d in dirs:
        np.testing.assert_allclose(oracle.sh_basis(3, d), _sh_closed_forms(*d), rtol=0, atol=1e-14)
    # hand values: Y_1^1 at +x is -sqrt(3/(4 pi)), Y_1^-1 at +y likewise, Y_2^0 at +z is sqrt(5/pi)/2
    assert oracle.sh_basis(1, np.array([1.0, 0, 0]))[3] == pytest.approx(-math.sqrt(3 / (4 * math.pi)), abs=1e-15)
    assert oracle.sh_basis(1, np.array([0, 1.0, 0]))[1] == pytest.approx(-math.sqrt(3 / (4 * math.pi)), abs=1e-15)
    assert oracle.sh_basis(2, np.array([0, 0, 1.0]))[6] == pytest.approx(0.5 * math.sqrt(5 / math.pi), abs=1e-15)


def test_sh_basis_equals_library_complex_harmonics(oracle):
    # scipy's complex Y_l^m carries the Condon-Shortley phase: the real functions are sqrt(2) Re Y_l^m
    # (index l^2 + l + m), sqrt(2) Im Y_l^m (index l^2 + l - m) and Y_l^0
    sph = getattr(scipy.special, "sph_harm_y", None)
    if sph is None:
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(22)
    for v in rng.normal(size=(25, 3)):
        d = v / np.linalg.norm(v)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = oracle.sh_basis(3, d)
        for l in range(4):
            for m in range(l + 1):
                c = complex(sph(l, m, theta, phi))
                if m == 0:
                    assert Y[l * l + l] == pytest.approx(c.real, abs=1e-13)
                else:
                    assert Y[l * l + l + m] == pytest.approx(math.sqrt(2) * c.real, abs=1e-13)
                    assert Y[l * l + l - m] == pytest.approx(math.sqrt(2) * c.imag, abs=1e-13)


def test_sh_basis_parity_gives_the_degree(oracle):
    # Y_k(-d) = (-1)^l Y_k(d) with l = floor(sqrt(k)): a function of the wrong degree fails
    rng = np.random.default_rng(23)
    for v in rng.normal(size=(10, 3)):
        d = v / np.linalg.norm(v)
        Yp, Yn = oracle.sh_basis(3, d), oracle.sh_basis(3, -d)
        for k in range(16):
            l = int(math.isqrt(k))
            assert Yn[k] == pytest.approx((-1) ** l * Yp[k], abs=1e-14), k
