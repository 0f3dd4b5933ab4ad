"""Seeded synthetic scenes and cameras for the 3DGS splatting path.

This module only draws random numbers and lays them out; it holds none of the
renderer's arithmetic.  Both the CUDA path and the CPU oracle read the same
float32 arrays produced here, so every parity check starts from identical
inputs.

Primitive parameters follow the 3DGS ``PrimitiveParams`` of the paper's
Appendix (3DGS implementation): mean ``mu`` (3), scales ``s`` (3), a rotation
quaternion ``q`` (4, w-first; it need not be unit, the renderer normalises it),
opacity ``o`` (1) and spherical-harmonic coefficients ``sh`` (K, 3) with
K = (degree + 1)^2.  Scales and opacity are passed already activated.

Cameras are pinhole with a world-to-camera matrix ``viewmat`` (3x4 row-major,
OpenCV axes: x right, y down, z forward), following the paper's camera /
view arguments of ``project`` (Sec. 3.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray = field(default_factory=lambda: np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32))
    z_near: float = 0.2
    model: int = 0             # 0 pinhole, 1 fisheye (equidistant with radial polynomial; 3DGUT only)
    dist: tuple = (0.0, 0.0, 0.0, 0.0)  # fisheye k1..k4: theta_d = theta (1 + k1 th^2 + k2 th^4 + k3 th^6 + k4 th^8)

    def as_tuple(self):
        return (self.width, self.height, self.fx, self.fy, self.cx, self.cy,
                np.asarray(self.viewmat, np.float32).reshape(12), self.z_near, self.model, tuple(self.dist))


@dataclass
class RenderConfig:
    """Renderer constants: tile size, alpha threshold 1/255, alpha clamp 0.99, transmittance stop
    1e-4, low-pass dilation 0.3, Jacobian clip 1.3 (3DGS), SH degree, background, batch depth and
    the method (0 3DGS, 1 3DGUT, 2 LinPrim)."""
    tile_w: int = 16
    tile_h: int = 16
    alpha_thresh: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_eps: float = 1e-4
    cov_dilation: float = 0.3
    clip_factor: float = 1.3
    sh_degree: int = 0
    bg: tuple = (0.0, 0.0, 0.0)
    batch_depth: int = 0  # 0 = kernel default
    method: int = 0       # 0 = 3DGS (EWA projection), 1 = 3DGUT (unscented transform + ray evaluation),
                          # 2 = LinPrim (octahedra, slab intersection)


@dataclass
class Scene:
    mu: np.ndarray      # [N,3] float32
    scale: np.ndarray   # [N,3] float32 (activated)
    quat: np.ndarray    # [N,4] float32 (w,x,y,z), not necessarily unit
    opacity: np.ndarray  # [N]  float32 (activated)
    sh: np.ndarray      # [N,K,3] float32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mu.shape[0])

    def arrays(self):
        return self.mu, self.scale, self.quat, self.opacity, self.sh

    def subset(self, idx) -> "Scene":
        return Scene(self.mu[idx], self.scale[idx], self.quat[idx], self.opacity[idx], self.sh[idx], self.sh_degree)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _finish(mu, log_s, q_raw, logit_o, sh, deg) -> Scene:
    return Scene(
        mu=np.ascontiguousarray(mu, np.float32),
        scale=np.ascontiguousarray(np.exp(log_s), np.float32),
        quat=np.ascontiguousarray(q_raw, np.float32),
        opacity=np.ascontiguousarray(_sigmoid(logit_o), np.float32),
        sh=np.ascontiguousarray(sh, np.float32),
        sh_degree=deg,
    )


def uniform_scene(n: int = 10_000, seed: int = 0, xy_range: float = 1.0, z_range=(2.0, 6.0),
                  log_scale_mean: float = -3.0, log_scale_std: float = 0.5, sh_degree: int = 0,
                  sh_std: float = 0.3) -> Scene:
    """Small-case workload: means uniform in [-1,1]^2 x [2,6] (camera space with an
    identity view), log-scales ~ N(-3, 0.5), random quaternions ~ N(0,1)^4,
    opacity = sigmoid(N(0,1)).  With ``sh_degree == 0`` the colour is drawn as
    RGB ~ U[0,1] and stored as the degree-0 coefficient whose rendered colour is
    that RGB (coefficient = (rgb - 0.5) * sqrt(4 pi)); otherwise every
    coefficient is drawn from N(0, sh_std^2).
    Draw order: mu_xy, mu_z, log_s, q, logit_o, colour."""
    rng = np.random.default_rng(seed)
    mu = np.empty((n, 3), np.float64)
    mu[:, :2] = rng.uniform(-xy_range, xy_range, size=(n, 2))
    mu[:, 2] = rng.uniform(z_range[0], z_range[1], size=n)
    log_s = rng.normal(log_scale_mean, log_scale_std, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    logit_o = rng.normal(0.0, 1.0, size=n)
    k = (sh_degree + 1) ** 2
    if sh_degree == 0:
        rgb = rng.uniform(0.0, 1.0, size=(n, 3))
        sh = ((rgb - 0.5) * math.sqrt(4.0 * math.pi)).reshape(n, 1, 3)
    else:
        sh = rng.normal(0.0, sh_std, size=(n, k, 3))
    return _finish(mu, log_s, q, logit_o, sh, sh_degree)


def clustered_scene(n: int = 1_000_000, seed: int = 0, n_centers: int = 200, spread: float = 0.5,
                    depth_range=(1.0, 20.0), width: int = 1920, height: int = 1080, focal: float = 1920.0,
                    sh_degree: int = 3, sh_std: float = 0.3) -> Scene:
    """Headline workload: ``n_centers`` cluster centres with depth ~ U[1,20] and
    x,y ~ U[-0.5,0.5] * depth * (W/fx, H/fy) (inside the view frustum of an
    identity camera); each primitive picks a centre uniformly and adds
    N(0, spread^2) per axis.  Scales, rotations and opacity as ``uniform_scene``;
    SH degree 3 coefficients (48 floats) ~ N(0, 0.3^2).
    Draw order: centre z, centre xy, centre choice, offsets, log_s, q, logit_o, sh."""
    rng = np.random.default_rng(seed)
    cz = rng.uniform(depth_range[0], depth_range[1], size=n_centers)
    cxy = rng.uniform(-0.5, 0.5, size=(n_centers, 2))
    cx = cxy[:, 0] * cz * (width / focal)
    cy = cxy[:, 1] * cz * (height / focal)
    centres = np.stack([cx, cy, cz], axis=1)
    pick = rng.integers(0, n_centers, size=n)
    mu = centres[pick] + rng.normal(0.0, spread, size=(n, 3))
    log_s = rng.normal(-3.0, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    logit_o = rng.normal(0.0, 1.0, size=n)
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, sh_std, size=(n, k, 3))
    return _finish(mu, log_s, q, logit_o, sh, sh_degree)


def pinhole(width: int, height: int, focal: float, viewmat=None, z_near: float = 0.2) -> Camera:
    """Pinhole camera with principal point at the image centre."""
    vm = np.hstack([np.eye(3), np.zeros((3, 1))]) if viewmat is None else np.asarray(viewmat, np.float64)
    return Camera(width, height, float(focal), float(focal), width / 2.0, height / 2.0,
                  np.ascontiguousarray(vm, np.float32).reshape(3, 4), z_near)


def fisheye(width: int, height: int, focal: float, dist=(0.05, -0.01, 0.001, 0.0), viewmat=None,
            z_near: float = 0.2) -> Camera:
    """Fisheye camera (equidistant projection with a 4-coefficient radial polynomial), principal point
    at the image centre: a camera-space point at angle theta from the axis lands at radius
    focal * theta (1 + k1 theta^2 + k2 theta^4 + k3 theta^6 + k4 theta^8) from the principal point."""
    cam = pinhole(width, height, focal, viewmat, z_near)
    cam.model = 1
    cam.dist = tuple(float(k) for k in dist)
    return cam


def yaw_view(yaw_deg: float, t=(0.0, 0.0, 0.0)) -> np.ndarray:
    """World-to-camera [R|t] for a camera yawed about the y axis by ``yaw_deg``."""
    a = math.radians(yaw_deg)
    r = np.array([[math.cos(a), 0.0, -math.sin(a)], [0.0, 1.0, 0.0], [math.sin(a), 0.0, math.cos(a)]])
    return np.hstack([r, np.asarray(t, np.float64).reshape(3, 1)]).astype(np.float32)


def small_case():
    """10,000 Gaussians, 256x256 pinhole, focal 256, 16x16 tiles, SH degree 0, seed 0."""
    return uniform_scene(10_000, seed=0), pinhole(256, 256, 256.0), RenderConfig(sh_degree=0)


def headline_case(n: int = 1_000_000, seed: int = 0):
    """1M SH-3 Gaussians in a clustered scene, 1920x1080 pinhole, focal 1920."""
    sc = clustered_scene(n, seed=seed)
    return sc, pinhole(1920, 1080, 1920.0), RenderConfig(sh_degree=3)


def linprim_case(n: int = 500_000, seed: int = 0):
    """LinPrim workload: 500k octahedra drawn as the headline scene (clustered means, half-extents
    e^N(-3, 0.5), rotations, opacity, SH degree 3) for a 1280x720 pinhole camera, focal 1280."""
    sc = clustered_scene(n, seed=seed, width=1280, height=720, focal=1280.0)
    return sc, pinhole(1280, 720, 1280.0), RenderConfig(sh_degree=3, method=2)


def multiview_cameras(n_views: int = 8, width: int = 1600, height: int = 1064, focal: float = 800.0,
                      seed: int = 0, fisheye_dist=None):
    """``n_views`` cameras yawed evenly over [-15, +15] degrees and translated by at most 0.1 along
    each axis: pinhole, or fisheye with radial coefficients ``fisheye_dist`` when given."""
    rng = np.random.default_rng(seed + 7)
    yaws = np.linspace(-15.0, 15.0, n_views) if n_views > 1 else np.zeros(1)
    cams = []
    for y in yaws:
        t = rng.uniform(-0.1, 0.1, size=3)
        vm = yaw_view(float(y), t)
        cams.append(pinhole(width, height, focal, vm) if fisheye_dist is None
                    else fisheye(width, height, focal, fisheye_dist, vm))
    return cams


# radial coefficients of the fisheye in the 3DGUT workload
FISHEYE_DIST = (0.05, -0.01, 0.001, 0.0)


def serving_scenes(n_scenes: int = 16, n_min: int = 100_000, n_max: int = 3_000_000, seed: int = 0,
                   scale_down: int = 1):
    """16 clustered SH-3 scenes with sizes log-uniform in [1e5, 3e6] (scene k uses seed k).
    ``scale_down`` divides every size (for quick runs)."""
    rng = np.random.default_rng(seed + 1000)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_scenes)).astype(np.int64) // scale_down
    return [clustered_scene(int(max(s, 1)), seed=k) for k, s in enumerate(sizes)]
