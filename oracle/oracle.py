"""ctypes binding of the FP64 CPU oracle (``xpr_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the package entry's
``smoke()`` check and by the benchmark's CPU-baseline leg.  The product path
never imports it.

Every function takes numpy arrays.  Camera and config constants are passed as
their float32 values widened to float64, so that thresholds (1/255, 0.99,
1e-4) are the same numbers on both sides; arithmetic is FP64 except the
exact-FP32 binning mode.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xpr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

_F64P = ctypes.POINTER(ctypes.c_double)
_F32P = ctypes.POINTER(ctypes.c_float)
_I32P = ctypes.POINTER(ctypes.c_int32)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_U64P = ctypes.POINTER(ctypes.c_uint64)
_I64P = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_project.argtypes = [ctypes.c_int64, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P,
                                     _I32P, _I32P, _F64P, _F64P]
        L.oracle_bin.argtypes = [ctypes.c_int64, _F64P, _F32P, _F32P, _I32P, _F64P, _F64P, ctypes.c_int, _I64P,
                                 _I32P, _U64P, _U32P]
        L.oracle_bin.restype = ctypes.c_int64
        L.oracle_sort.argtypes = [ctypes.c_int64, _U64P, _U32P, ctypes.c_int64, _I32P]
        L.oracle_depth_keys.argtypes = [ctypes.c_int64, _F64P, _F64P, ctypes.c_int, _F32P]
        L.oracle_project_unc.argtypes = [ctypes.c_int64, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_render_tiles.argtypes = [ctypes.c_int64, _F64P, _U32P, _I32P, _F64P, _F64P, _F64P, _F64P,
                                          _F64P, _F64P, _I32P, _I32P, _F64P]
        L.oracle_render_pixels.argtypes = [ctypes.c_int64, _F64P, _F32P, _I32P, ctypes.c_int64, _F64P, _F64P,
                                           _F64P, _F64P, _F64P, _I32P, _F64P, _U64P, _U64P]
        L.oracle_render_bwd_brute.argtypes = [ctypes.c_int64, _F64P, _F32P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_render_bwd_tiles.argtypes = [ctypes.c_int64, _F64P, _U32P, _I32P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_project_bwd.argtypes = [ctypes.c_int64, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P,
                                         _F64P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_sh_basis.argtypes = [ctypes.c_int, _F64P, _F64P, _F64P]
        L.oracle_cull_one.argtypes = [_F64P, ctypes.c_int, ctypes.c_int, _F64P, _F64P, ctypes.c_int]
        L.oracle_cull_one.restype = ctypes.c_int
        L.oracle_project_ut.argtypes = [ctypes.c_int64, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P,
                                        _F64P, _I32P, _I32P, _F64P, _F64P]
        L.oracle_render_tiles_ut.argtypes = [ctypes.c_int64, _F64P, _F64P, _U32P, _I32P, _F64P, _F64P,
                                             ctypes.c_double, _F64P, _F64P, _I32P, _I32P, _F64P, _U64P]
        L.oracle_render_bwd_tiles_ut.argtypes = [ctypes.c_int64, _F64P, _U32P, _I32P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_project_ut_bwd.argtypes = [ctypes.c_int64, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P,
                                            _F64P, _F64P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_render_pixels_ut.argtypes = [ctypes.c_int64, _F64P, _F64P, _F32P, _I32P, ctypes.c_int64, _F64P,
                                              _F64P, ctypes.c_double, _F64P, _F64P, _I32P, _F64P]
        L.oracle_ut_response.argtypes = [_F64P, _F64P]
        L.oracle_ut_response.restype = ctypes.c_double
        L.oracle_pixel_ray.argtypes = [ctypes.c_int, ctypes.c_int, _F64P, _F64P]
        L.oracle_project_lp.argtypes = [ctypes.c_int64, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P,
                                        _F64P, _I32P, _I32P, _F64P, _F64P]
        L.oracle_lp_chord.argtypes = [_F64P, ctypes.c_double, ctypes.c_double]
        L.oracle_lp_chord.restype = ctypes.c_double
        L.oracle_lp_keep.argtypes = [_F64P, ctypes.c_int, ctypes.c_int, _F64P, _F64P]
        L.oracle_lp_keep.restype = ctypes.c_int
        L.oracle_lp_tile_bound.argtypes = [_F64P, ctypes.c_int, ctypes.c_int, _F64P, _F64P]
        L.oracle_lp_tile_bound.restype = ctypes.c_double
        L.oracle_bin_lp.argtypes = [ctypes.c_int64, _F64P, _F64P, _F32P, _F32P, _F32P, _I32P, _F64P, _F64P,
                                    ctypes.c_int, _I64P, _I32P, _U64P, _U32P]
        L.oracle_bin_lp.restype = ctypes.c_int64
        L.oracle_render_tiles_lp.argtypes = [ctypes.c_int64, _F64P, _U32P, _I32P, _F64P, _F64P, ctypes.c_double,
                                             _F64P, _F64P, _I32P, _I32P, _F64P, _U64P]
        L.oracle_render_bwd_tiles_lp.argtypes = [ctypes.c_int64, _F64P, _U32P, _I32P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_project_lp_bwd.argtypes = [ctypes.c_int64, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P,
                                            _F64P, _F64P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_render_tiles_feat.argtypes = [ctypes.c_int64, _F64P, _F64P, ctypes.c_int, ctypes.c_int, _U32P,
                                               _I32P, _F64P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_render_bwd_tiles_feat.argtypes = [ctypes.c_int64, _F64P, _F64P, ctypes.c_int, ctypes.c_int, _U32P,
                                                   _I32P, _F64P, _F64P, _F64P, _F64P, _F64P, _F64P]
        L.oracle_fisheye_project.argtypes = [_F64P, _F64P, _F64P]
        L.oracle_abi_version.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32v(v) -> float:
    return float(np.float32(v))


def cam_array(cam) -> np.ndarray:
    """[W, H, fx, fy, cx, cy, V(12), z_near, model, k1..k4] with float32-rounded values."""
    vm = np.asarray(cam.viewmat, np.float32).reshape(12).astype(np.float64)
    dist = [_f32v(k) for k in getattr(cam, "dist", (0.0, 0.0, 0.0, 0.0))]
    return np.array([cam.width, cam.height, _f32v(cam.fx), _f32v(cam.fy), _f32v(cam.cx), _f32v(cam.cy), *vm,
                     _f32v(cam.z_near), int(getattr(cam, "model", 0)), *dist], np.float64)


def cfg_array(cfg) -> np.ndarray:
    """[tile_w, tile_h, alpha_t, alpha_max, t_eps, dilation, clip, sh_degree, bg(3), method]."""
    return np.array([cfg.tile_w, cfg.tile_h, _f32v(cfg.alpha_thresh), _f32v(cfg.alpha_max), _f32v(cfg.t_eps),
                     _f32v(cfg.cov_dilation), _f32v(cfg.clip_factor), cfg.sh_degree,
                     *[_f32v(b) for b in cfg.bg], getattr(cfg, "method", 0)], np.float64)


class Band(NamedTuple):
    """Uncertainty model of the 3DGS ambiguity band (the compositing walk of xpr_oracle.c).

    eps: relative precision of a float32 evaluation of the exponent and the exponential.
    mu_abs, conic_rel: multipliers of the per-primitive uncertainty scales of a float32 projection
    (``fp32_uncertainty``: the centre's rounding in pixels and the conic's cancellation factor);
    both are zero when the float32 side reads the same float32 records as the oracle (stage-wise
    parity), and bound the float32 projection's rounding when it computed its own records
    (end-to-end parity).  Without per-primitive scales mu_abs is in pixels."""
    eps: float = 1e-6
    mu_abs: float = 0.0
    conic_rel: float = 0.0


#: stage-wise parity: both sides composite the same float32 records
BAND_STAGE = Band(1e-6, 0.0, 0.0)
#: end-to-end parity: the float32 projection's own records (twice the rounding-error model of the
#: centres; the Sigma_2D entries uncertain to 2e-6 of their absolute-value sums, about 32 units of
#: float32 roundoff, against at most 14 measured on a float32 restatement of the projection)
BAND_E2E = Band(1e-6, 2.0, 2e-6)


def _cmax(rec, cfg) -> float:
    """Largest colour or background magnitude (the scale of the jump bound)."""
    r = np.asarray(rec, np.float64)
    c = float(np.abs(r[:, 6:9]).max()) if r.size else 0.0
    return max(c, max(abs(float(b)) for b in cfg.bg), 1e-30)


def _bandp(band, rec, cfg):
    if band is None or (not isinstance(band, Band) and float(band) == 0.0):
        return None
    if not isinstance(band, Band):
        band = Band(eps=float(band))
    return np.array([band.eps, band.mu_abs, band.conic_rel, _cmax(rec, cfg)], np.float64)


def tiles_of(cam, cfg):
    return (cam.width + cfg.tile_w - 1) // cfg.tile_w, (cam.height + cfg.tile_h - 1) // cfg.tile_h


# --------------------------------------------------------------------------- projection

def project(mu, scale, quat, opac, sh, cam, cfg):
    """Projection (Listing 1 project).  Returns dict with rec[n,12] (f64),
    bbox[n,4], tc[n], pre[n,4] (values before floor, tile units), cov[n,3] and
    key[n] (float32 depth sort keys, depth_keys)."""
    mu, scale, quat, opac, sh = map(_f64, (mu, scale, quat, opac, sh))
    n = mu.shape[0]
    rec = np.zeros((n, 12), np.float64)
    bbox = np.zeros((n, 4), np.int32)
    tc = np.zeros(n, np.int32)
    pre = np.zeros((n, 4), np.float64)
    cov = np.zeros((n, 3), np.float64)
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_project(n, _p(mu, _F64P), _p(scale, _F64P), _p(quat, _F64P), _p(opac, _F64P), _p(sh, _F64P),
                         _p(ca, _F64P), _p(fa, _F64P), _p(rec, _F64P), _p(bbox, _I32P), _p(tc, _I32P),
                         _p(pre, _F64P), _p(cov, _F64P))
    return dict(rec=rec, bbox=bbox, tc=tc, pre=pre, cov=cov, key=depth_keys(mu, cam),
                unc=fp32_uncertainty(mu, scale, quat, opac, sh, cam, cfg))


def depth_keys(mu, cam, euclid: bool = False):
    """Depth sort keys (float32): camera z (or, euclid, the Euclidean distance to the camera) of
    the float32 means, every operation rounded to float32 in a fixed order without FMA; the tile
    lists are ordered by (tile, key bits, index)."""
    mu = _f64(np.asarray(mu, np.float32))
    key = np.zeros(mu.shape[0], np.float32)
    ca = cam_array(cam)
    lib().oracle_depth_keys(mu.shape[0], _p(mu, _F64P), _p(ca, _F64P), int(bool(euclid)), _p(key, _F32P))
    return key


def fp32_uncertainty(mu, scale, quat, opac, sh, cam, cfg):
    """Per-primitive scales of a float32 projection's rounding, unc[n,5] (oracle_project_unc):
    the centre's rounding model in pixels, the 2x2 inverse's cancellation factor, and the
    absolute-value sums of the Sigma_2D entries.  Test infrastructure for the ambiguity band."""
    mu, scale, quat, opac, sh = map(_f64, (mu, scale, quat, opac, sh))
    n = mu.shape[0]
    unc = np.zeros((n, 5))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_project_unc(n, _p(mu, _F64P), _p(scale, _F64P), _p(quat, _F64P), _p(opac, _F64P), _p(sh, _F64P),
                             _p(ca, _F64P), _p(fa, _F64P), _p(unc, _F64P))
    return unc


def project_scene(scene, cam, cfg):
    return project(scene.mu, scene.scale, scene.quat, scene.opacity, scene.sh, cam, cfg)


def project_bwd(mu, scale, quat, opac, sh, cam, cfg, d_rec):
    mu, scale, quat, opac, sh, d_rec = map(_f64, (mu, scale, quat, opac, sh, d_rec))
    n = mu.shape[0]
    dmu = np.zeros((n, 3))
    ds = np.zeros((n, 3))
    dq = np.zeros((n, 4))
    do = np.zeros(n)
    dsh = np.zeros_like(sh)
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_project_bwd(n, _p(mu, _F64P), _p(scale, _F64P), _p(quat, _F64P), _p(opac, _F64P),
                             _p(sh, _F64P), _p(ca, _F64P), _p(fa, _F64P), _p(d_rec, _F64P), _p(dmu, _F64P),
                             _p(ds, _F64P), _p(dq, _F64P), _p(do, _F64P), _p(dsh, _F64P))
    return dict(mu=dmu, scale=ds, quat=dq, opacity=do, sh=dsh)


# --------------------------------------------------------------------------- binning / sort

def bin_pairs(rec, bbox, cam, cfg, exact32: bool, order=None, key=None):
    """Replicate + tile ID + cull, visiting primitives in ``order`` (index order when None);
    counts are per visited position.  With exact32, ``rec`` must be float32 records (the decision
    is taken in FP32, the depths are the records' own); else the keys carry ``key`` (depth_keys;
    None = the FP64 depth rounded to float32)."""
    bbox = np.ascontiguousarray(bbox, np.int32)
    n = bbox.shape[0]
    od = None if order is None else np.ascontiguousarray(order, np.int64)
    ca, fa = cam_array(cam), cfg_array(cfg)
    r64 = None if exact32 else _f64(rec)
    r32 = np.ascontiguousarray(rec, np.float32) if exact32 else None
    kk = None if (exact32 or key is None) else np.ascontiguousarray(key, np.float32)
    counts = np.zeros(n, np.int32)
    total = lib().oracle_bin(n, _p(r64, _F64P), _p(r32, _F32P), _p(kk, _F32P), _p(bbox, _I32P), _p(ca, _F64P),
                             _p(fa, _F64P), int(exact32), _p(od, _I64P), _p(counts, _I32P), None, None)
    keys = np.zeros(max(total, 1), np.uint64)
    vals = np.zeros(max(total, 1), np.uint32)
    lib().oracle_bin(n, _p(r64, _F64P), _p(r32, _F32P), _p(kk, _F32P), _p(bbox, _I32P), _p(ca, _F64P),
                     _p(fa, _F64P), int(exact32), _p(od, _I64P), _p(counts, _I32P), _p(keys, _U64P), _p(vals, _U32P))
    return counts, keys[:total].copy(), vals[:total].copy()


def depth_order(rec, tc, key=None):
    """Primitives with tiles by (float32 depth key, index), then the rest in index order (key None:
    the records' depths rounded to float32)."""
    d32 = np.asarray(rec, np.float64)[:, 9].astype(np.float32) if key is None else np.asarray(key, np.float32)
    has = np.asarray(tc) > 0
    idx = np.arange(len(has))
    vis = idx[has][np.lexsort((idx[has], d32[has]))]
    return np.concatenate([vis, idx[~has]]).astype(np.int64)


def sort_pairs(keys, vals, n_tiles):
    keys = np.array(keys, np.uint64, copy=True)
    vals = np.array(vals, np.uint32, copy=True)
    ranges = np.zeros((n_tiles, 2), np.int32)
    kk = keys if keys.size else np.zeros(1, np.uint64)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    lib().oracle_sort(keys.size, _p(kk, _U64P), _p(vv, _U32P), n_tiles, _p(ranges, _I32P))
    return kk[:keys.size], vv[:vals.size], ranges


def cull_one(rec_row, tx, ty, cam, cfg, form: int = 0) -> bool:
    """Tile cull decision for one record and tile.  form 0: per-tile minimum (FP64); 1: row form
    (FP64); 2: row form in FP32 on the float-rounded record (the kernels' decision)."""
    r = _f64(rec_row)
    ca, fa = cam_array(cam), cfg_array(cfg)
    return bool(lib().oracle_cull_one(_p(r, _F64P), tx, ty, _p(ca, _F64P), _p(fa, _F64P), form))


# --------------------------------------------------------------------------- compositing

def _band_out(bd, jump):
    """band: pixels whose value may differ (bit 1); gband: pixels whose gradient may differ as well
    (any flag); jump: bound of the colour change through the flagged decisions."""
    return dict(band=(bd & 1).astype(bool), gband=bd != 0, jump=jump)


def render_tiles(rec, vals, ranges, cam, cfg, band=None, unc=None):
    """Per-tile walk over given lists.  ``band``: a Band (or a float eps) turns on the ambiguity
    band of the walk; ``unc``: the per-primitive scales of fp32_uncertainty."""
    rec = _f64(rec)
    un = None if unc is None else _f64(unc)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    H, W = cam.height, cam.width
    image = np.zeros((3, H, W))
    tfin = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    bd = np.zeros((H, W), np.int32)
    jump = np.zeros((H, W))
    ca, fa = cam_array(cam), cfg_array(cfg)
    bp = _bandp(band, rec, cfg)
    lib().oracle_render_tiles(rec.shape[0], _p(rec, _F64P), _p(vv, _U32P), _p(ranges, _I32P), _p(ca, _F64P),
                              _p(fa, _F64P), _p(bp, _F64P), _p(un, _F64P), _p(image, _F64P), _p(tfin, _F64P),
                              _p(nc, _I32P), _p(bd, _I32P), _p(jump, _F64P))
    return dict(image=image, t_final=tfin, n_contrib=nc, **_band_out(bd, jump))


def render_pixels(rec, pix, cfg, band=None, key=None, unc=None):
    """Brute-force walk over every visible primitive at the listed pixels, in the order of the
    depth keys ``key`` (depth_keys; None = the records' depths rounded to float32)."""
    rec = _f64(rec)
    un = None if unc is None else _f64(unc)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    m = pix.shape[0]
    color = np.zeros((m, 3))
    tfin = np.zeros(m)
    bd = np.zeros(m, np.int32)
    jump = np.zeros(m)
    sig = np.zeros(1, np.uint64)
    psig = np.zeros(m, np.uint64)
    fa = cfg_array(cfg)
    kk = None if key is None else np.ascontiguousarray(key, np.float32)
    bp = _bandp(band, rec, cfg)
    lib().oracle_render_pixels(rec.shape[0], _p(rec, _F64P), _p(kk, _F32P), _p(pix, _I32P), m, _p(fa, _F64P),
                               _p(bp, _F64P), _p(un, _F64P), _p(color, _F64P), _p(tfin, _F64P), _p(bd, _I32P),
                               _p(jump, _F64P), _p(psig, _U64P), _p(sig, _U64P))
    return dict(color=color, t_final=tfin, sig=int(sig[0]), pixel_sig=psig, **_band_out(bd, jump))


def render_brute(rec, cam, cfg, band=None, key=None, unc=None):
    """Brute-force image (every pixel, every visible primitive; Sec. 3.1)."""
    H, W = cam.height, cam.width
    ys, xs = np.mgrid[0:H, 0:W]
    pix = np.stack([xs.ravel(), ys.ravel()], 1)
    r = render_pixels(rec, pix, cfg, band, key, unc)
    return dict(image=r["color"].T.reshape(3, H, W), t_final=r["t_final"].reshape(H, W),
                band=r["band"].reshape(H, W), gband=r["gband"].reshape(H, W), jump=r["jump"].reshape(H, W),
                sig=r["sig"])


def render_bwd_brute(rec, cam, cfg, d_image, key=None):
    rec = _f64(rec)
    d_image = _f64(d_image)
    d_rec = np.zeros((rec.shape[0], 12))
    ca, fa = cam_array(cam), cfg_array(cfg)
    kk = None if key is None else np.ascontiguousarray(key, np.float32)
    lib().oracle_render_bwd_brute(rec.shape[0], _p(rec, _F64P), _p(kk, _F32P), _p(ca, _F64P), _p(fa, _F64P),
                                  _p(d_image, _F64P), _p(d_rec, _F64P))
    return d_rec


def render_bwd_tiles(rec, vals, ranges, cam, cfg, d_image):
    rec = _f64(rec)
    d_image = _f64(d_image)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    d_rec = np.zeros((rec.shape[0], 12))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_render_bwd_tiles(rec.shape[0], _p(rec, _F64P), _p(vv, _U32P), _p(ranges, _I32P),
                                  _p(ca, _F64P), _p(fa, _F64P), _p(d_image, _F64P), _p(d_rec, _F64P))
    return d_rec


def sh_basis(deg, d, with_grad=False):
    d = _f64(d)
    K = (deg + 1) ** 2
    Y = np.zeros(16)
    G = np.zeros(48) if with_grad else None
    lib().oracle_sh_basis(deg, _p(d, _F64P), _p(Y, _F64P), _p(G, _F64P))
    return (Y[:K], G[:3 * K].reshape(K, 3)) if with_grad else Y[:K]


# --------------------------------------------------------------------------- whole pipelines

def pipeline_tiled(scene, cam, cfg, band=None):
    """FP64 tiled pipeline: project -> bin (FP64 cull, float32 depth keys) -> sort -> per-tile walk."""
    pr = project_scene(scene, cam, cfg)
    Wt, Ht = tiles_of(cam, cfg)
    _, keys, vals = bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False, key=pr["key"])
    keys, vals, ranges = sort_pairs(keys, vals, Wt * Ht)
    out = render_tiles(pr["rec"], vals, ranges, cam, cfg, band, pr["unc"])
    out.update(proj=pr, keys=keys, vals=vals, ranges=ranges)
    return out


# --------------------------------------------------------------------------- 3DGUT

def project_ut(mu, scale, quat, opac, sh, cam, cfg):
    """3DGUT projection (unscented transform).  Returns rec[n,12] (3DGS layout with the UT mean and
    conic, Mip-Splatting opacity), sd[n,16] (ro_c, M row-major, o', rgb), bbox, tc, pre, cov0."""
    mu, scale, quat, opac, sh = map(_f64, (mu, scale, quat, opac, sh))
    n = mu.shape[0]
    rec = np.zeros((n, 12))
    sd = np.zeros((n, 16))
    bbox = np.zeros((n, 4), np.int32)
    tc = np.zeros(n, np.int32)
    pre = np.zeros((n, 4))
    cov0 = np.zeros((n, 3))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_project_ut(n, _p(mu, _F64P), _p(scale, _F64P), _p(quat, _F64P), _p(opac, _F64P),
                            _p(sh, _F64P), _p(ca, _F64P), _p(fa, _F64P), _p(rec, _F64P), _p(sd, _F64P),
                            _p(bbox, _I32P), _p(tc, _I32P), _p(pre, _F64P), _p(cov0, _F64P))
    return dict(rec=rec, sd=sd, bbox=bbox, tc=tc, pre=pre, cov0=cov0, key=depth_keys(mu, cam))


def project_ut_scene(scene, cam, cfg):
    return project_ut(scene.mu, scene.scale, scene.quat, scene.opacity, scene.sh, cam, cfg)


def render_tiles_ut(rec, sd, vals, ranges, cam, cfg, delta: float = 0.0):
    rec, sd = _f64(rec), _f64(sd)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    H, W = cam.height, cam.width
    image = np.zeros((3, H, W))
    tfin = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    bd = np.zeros((H, W), np.int32)
    jump = np.zeros((H, W))
    psig = np.zeros((H, W), np.uint64)
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_render_tiles_ut(rec.shape[0], _p(rec, _F64P), _p(sd, _F64P), _p(vv, _U32P), _p(ranges, _I32P),
                                 _p(ca, _F64P), _p(fa, _F64P), delta, _p(image, _F64P), _p(tfin, _F64P),
                                 _p(nc, _I32P), _p(bd, _I32P), _p(jump, _F64P), _p(psig, _U64P))
    return dict(image=image, t_final=tfin, n_contrib=nc, pixel_sig=psig,
                **_band_out(bd, jump * _cmax(sd[:, 7:], cfg)))


def render_bwd_tiles_ut(sd, vals, ranges, cam, cfg, d_image):
    """Adjoint of the per-tile 3DGUT walk: d_sd[n,16] = (dro_c, dM, do', drgb)."""
    sd, d_image = _f64(sd), _f64(d_image)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    d_sd = np.zeros((sd.shape[0], 16))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_render_bwd_tiles_ut(sd.shape[0], _p(sd, _F64P), _p(vv, _U32P), _p(ranges, _I32P), _p(ca, _F64P),
                                     _p(fa, _F64P), _p(d_image, _F64P), _p(d_sd, _F64P))
    return d_sd


def project_ut_bwd(mu, scale, quat, opac, sh, cam, cfg, d_sd):
    """Adjoint of the 3DGUT projection from d_sd[n,16] to the primitive parameters."""
    mu, scale, quat, opac, sh, d_sd = map(_f64, (mu, scale, quat, opac, sh, d_sd))
    n = mu.shape[0]
    dmu, ds, dq, do, dsh = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros(n), np.zeros_like(sh)
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_project_ut_bwd(n, _p(mu, _F64P), _p(scale, _F64P), _p(quat, _F64P), _p(opac, _F64P),
                                _p(sh, _F64P), _p(ca, _F64P), _p(fa, _F64P), _p(d_sd, _F64P), _p(dmu, _F64P),
                                _p(ds, _F64P), _p(dq, _F64P), _p(do, _F64P), _p(dsh, _F64P))
    return dict(mu=dmu, scale=ds, quat=dq, opacity=do, sh=dsh)


def render_pixels_ut(rec, sd, pix, cam, cfg, delta: float = 0.0, key=None):
    """Every visible primitive (depth-key order) at the listed pixels, no tiles."""
    rec, sd = _f64(rec), _f64(sd)
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 2)
    m = pix.shape[0]
    color = np.zeros((m, 3))
    tfin = np.zeros(m)
    bd = np.zeros(m, np.int32)
    jump = np.zeros(m)
    ca, fa = cam_array(cam), cfg_array(cfg)
    kk = None if key is None else np.ascontiguousarray(key, np.float32)
    lib().oracle_render_pixels_ut(rec.shape[0], _p(rec, _F64P), _p(sd, _F64P), _p(kk, _F32P), _p(pix, _I32P), m,
                                  _p(ca, _F64P), _p(fa, _F64P), delta, _p(color, _F64P), _p(tfin, _F64P),
                                  _p(bd, _I32P), _p(jump, _F64P))
    return dict(color=color, t_final=tfin, **_band_out(bd, jump * _cmax(sd[:, 7:], cfg)))


def ut_response(sd_row, rd) -> float:
    s, r = _f64(sd_row), _f64(rd)
    return float(lib().oracle_ut_response(_p(s, _F64P), _p(r, _F64P)))


def fisheye_project(pc, cam):
    """Pixel coordinates of camera-space points pc[m,3] under the camera's fisheye model."""
    pc = _f64(np.atleast_2d(pc))
    out = np.zeros((pc.shape[0], 2))
    ca = cam_array(cam)
    for i in range(pc.shape[0]):
        lib().oracle_fisheye_project(_p(np.ascontiguousarray(pc[i]), _F64P), _p(ca, _F64P),
                                     _p(out[i:i + 1].reshape(2), _F64P))
    return out


def pixel_ray(x, y, cam):
    rd = np.zeros(3)
    ca = cam_array(cam)
    lib().oracle_pixel_ray(int(x), int(y), _p(ca, _F64P), _p(rd, _F64P))
    return rd


def pipeline_tiled_ut(scene_arrays, cam, cfg, delta: float = 0.0):
    """FP64 3DGUT pipeline: UT projection -> bin (FP64 cull, ray-offset tile bounds) -> sort ->
    per-tile ray walk.  scene_arrays = (mu, scale, quat, opacity, sh)."""
    pr = project_ut(*scene_arrays, cam, cfg)
    Wt, Ht = tiles_of(cam, cfg)
    _, keys, vals = bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False, key=pr["key"])
    keys, vals, ranges = sort_pairs(keys, vals, Wt * Ht)
    out = render_tiles_ut(pr["rec"], pr["sd"], vals, ranges, cam, cfg, delta)
    out.update(proj=pr, keys=keys, vals=vals, ranges=ranges)
    return out


def loss_tiled_ut(scene_arrays, cam, cfg, w):
    """sum(w * image) of the FP64 3DGUT pipeline and a hash of every decision it took (the tile
    lists and each pixel's gates), to tell a smooth change from a flipped decision."""
    import hashlib
    out = pipeline_tiled_ut(scene_arrays, cam, cfg)
    h = hashlib.sha1()
    for a in (out["vals"], out["ranges"], out["pixel_sig"]):
        h.update(np.ascontiguousarray(a).tobytes())
    return float((w * out["image"]).sum()), h.hexdigest()


def grads_tiled_ut(scene_arrays, cam, cfg, d_image):
    """Analytic FP64 gradients of sum(d_image * image) of the 3DGUT pipeline."""
    mu, s, q, o, sh = scene_arrays
    out = pipeline_tiled_ut(scene_arrays, cam, cfg)
    d_sd = render_bwd_tiles_ut(out["proj"]["sd"], out["vals"], out["ranges"], cam, cfg, d_image)
    g = project_ut_bwd(mu, s, q, o, sh, cam, cfg, d_sd)
    g["d_sd"] = d_sd
    return g


def loss_brute(scene_arrays, cam, cfg, w):
    """sum(w * image) of the brute-force FP64 render; also the decision hash."""
    mu, s, q, o, sh = scene_arrays
    pr = project(mu, s, q, o, sh, cam, cfg)
    r = render_brute(pr["rec"], cam, cfg, key=pr["key"])
    return float((w * r["image"]).sum()), r["sig"]


def grads_brute(scene_arrays, cam, cfg, d_image):
    """Analytic FP64 gradients of sum(d_image * image) w.r.t. all parameters."""
    mu, s, q, o, sh = scene_arrays
    pr = project(mu, s, q, o, sh, cam, cfg)
    d_rec = render_bwd_brute(pr["rec"], cam, cfg, d_image, key=pr["key"])
    g = project_bwd(mu, s, q, o, sh, cam, cfg, d_rec)
    g["d_rec"] = d_rec
    return g


# --------------------------------------------------------------------------- LinPrim

def project_lp(mu, scale, quat, opac, sh, cam, cfg):
    """LinPrim projection.  rec[n,12] (mu_2D, rgb, Euclidean depth, visible), sd[n,16] = (mu_2D,
    c0, c1, c2 (rows of A^-1), sigma, rgb), bbox, tc, pre, aux[n,12] = (A row-major, ex, ey, camera z)."""
    mu, scale, quat, opac, sh = map(_f64, (mu, scale, quat, opac, sh))
    n = mu.shape[0]
    rec, sd, aux = np.zeros((n, 12)), np.zeros((n, 16)), np.zeros((n, 12))
    bbox, tc, pre = np.zeros((n, 4), np.int32), np.zeros(n, np.int32), np.zeros((n, 4))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_project_lp(n, _p(mu, _F64P), _p(scale, _F64P), _p(quat, _F64P), _p(opac, _F64P), _p(sh, _F64P),
                            _p(ca, _F64P), _p(fa, _F64P), _p(rec, _F64P), _p(sd, _F64P), _p(bbox, _I32P),
                            _p(tc, _I32P), _p(pre, _F64P), _p(aux, _F64P))
    return dict(rec=rec, sd=sd, bbox=bbox, tc=tc, pre=pre, A=aux[:, :9].reshape(-1, 3, 3), ex=aux[:, 9],
                ey=aux[:, 10], z=aux[:, 11], key=depth_keys(mu, cam, euclid=True))


def lp_chord(sd_row, dX, dY) -> float:
    return float(lib().oracle_lp_chord(_p(_f64(sd_row), _F64P), float(dX), float(dY)))


def lp_keep(sd_row, tx, ty, cam, cfg) -> bool:
    ca, fa = cam_array(cam), cfg_array(cfg)
    return bool(lib().oracle_lp_keep(_p(_f64(sd_row), _F64P), tx, ty, _p(ca, _F64P), _p(fa, _F64P)))


def lp_tile_bound(sd_row, tx, ty, cam, cfg) -> float:
    ca, fa = cam_array(cam), cfg_array(cfg)
    return float(lib().oracle_lp_tile_bound(_p(_f64(sd_row), _F64P), tx, ty, _p(ca, _F64P), _p(fa, _F64P)))


def bin_pairs_lp(rec, sd, bbox, cam, cfg, exact32: bool, order=None, key=None):
    """LinPrim replicate + tile ID + cull.  exact32: rec float32 records and sd the kernels'
    float32 shader data [n,20] (their FP32 decision); else rec/sd the oracle's FP64 ones and the
    depth keys ``key`` (depth_keys with euclid; None = rec's depth rounded to float32)."""
    bbox = np.ascontiguousarray(bbox, np.int32)
    n = bbox.shape[0]
    od = None if order is None else np.ascontiguousarray(order, np.int64)
    ca, fa = cam_array(cam), cfg_array(cfg)
    r64 = None if exact32 else _f64(rec)
    s64 = None if exact32 else _f64(sd)
    r32 = np.ascontiguousarray(rec, np.float32) if exact32 else None
    s32 = np.ascontiguousarray(sd, np.float32) if exact32 else None
    counts = np.zeros(n, np.int32)
    kk = None if (exact32 or key is None) else np.ascontiguousarray(key, np.float32)
    args = (n, _p(r64, _F64P), _p(s64, _F64P), _p(r32, _F32P), _p(s32, _F32P), _p(kk, _F32P), _p(bbox, _I32P),
            _p(ca, _F64P), _p(fa, _F64P), int(exact32), _p(od, _I64P), _p(counts, _I32P))
    total = lib().oracle_bin_lp(*args, None, None)
    keys = np.zeros(max(total, 1), np.uint64)
    vals = np.zeros(max(total, 1), np.uint32)
    lib().oracle_bin_lp(*args, _p(keys, _U64P), _p(vals, _U32P))
    return counts, keys[:total].copy(), vals[:total].copy()


def render_tiles_lp(sd, vals, ranges, cam, cfg, delta: float = 0.0):
    sd = _f64(sd)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    H, W = cam.height, cam.width
    image, tfin = np.zeros((3, H, W)), np.zeros((H, W))
    nc, bd, psig = np.zeros((H, W), np.int32), np.zeros((H, W), np.int32), np.zeros((H, W), np.uint64)
    jump = np.zeros((H, W))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_render_tiles_lp(sd.shape[0], _p(sd, _F64P), _p(vv, _U32P), _p(ranges, _I32P), _p(ca, _F64P),
                                 _p(fa, _F64P), delta, _p(image, _F64P), _p(tfin, _F64P), _p(nc, _I32P),
                                 _p(bd, _I32P), _p(jump, _F64P), _p(psig, _U64P))
    return dict(image=image, t_final=tfin, n_contrib=nc, pixel_sig=psig,
                **_band_out(bd, jump * _cmax(sd[:, 6:], cfg)))


def condition_band_lp(sd, vals, ranges, cam, cfg, eta_px=1e-4, rel=2e-6, tol=5e-5, trials=4, seed=0):
    """Pixels whose LinPrim image is ill-conditioned at float32 scale: the FP64 image moves by more
    than ``tol`` when the projected centres are shifted by N(0, eta_px^2) pixels and the slab rows
    and densities scaled by 1 + N(0, rel^2) (independently per primitive, ``trials`` draws).  Near
    the silhouette of a face seen almost edge-on the chord is a steep function of the pixel
    position, so there the rounding of any float32 evaluation decides the value at the 1e-4 level."""
    sd = _f64(sd)
    base = render_tiles_lp(sd, vals, ranges, cam, cfg)["image"]
    rng = np.random.default_rng(seed)
    worst = np.zeros(base.shape[1:])
    for _ in range(trials):
        p = sd.copy()
        p[:, 0:2] += eta_px * rng.normal(size=(p.shape[0], 2))
        p[:, 2:12] *= 1 + rel * rng.normal(size=(p.shape[0], 10))
        img = render_tiles_lp(p, vals, ranges, cam, cfg)["image"]
        worst = np.maximum(worst, np.abs(img - base).max(0))
    return worst > tol


def render_bwd_tiles_lp(sd, vals, ranges, cam, cfg, d_image):
    sd, d_image = _f64(sd), _f64(d_image)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    d_sd = np.zeros((sd.shape[0], 16))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_render_bwd_tiles_lp(sd.shape[0], _p(sd, _F64P), _p(vv, _U32P), _p(ranges, _I32P), _p(ca, _F64P),
                                     _p(fa, _F64P), _p(d_image, _F64P), _p(d_sd, _F64P))
    return d_sd


def project_lp_bwd(mu, scale, quat, opac, sh, cam, cfg, d_sd):
    mu, scale, quat, opac, sh, d_sd = map(_f64, (mu, scale, quat, opac, sh, d_sd))
    n = mu.shape[0]
    dmu, ds, dq, do, dsh = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros(n), np.zeros_like(sh)
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_project_lp_bwd(n, _p(mu, _F64P), _p(scale, _F64P), _p(quat, _F64P), _p(opac, _F64P),
                                _p(sh, _F64P), _p(ca, _F64P), _p(fa, _F64P), _p(d_sd, _F64P), _p(dmu, _F64P),
                                _p(ds, _F64P), _p(dq, _F64P), _p(do, _F64P), _p(dsh, _F64P))
    return dict(mu=dmu, scale=ds, quat=dq, opacity=do, sh=dsh)


def pipeline_tiled_lp(scene_arrays, cam, cfg, delta: float = 0.0):
    """FP64 LinPrim pipeline: projection -> bin (FP64 per-tile bound) -> sort -> per-tile walk."""
    pr = project_lp(*scene_arrays, cam, cfg)
    Wt, Ht = tiles_of(cam, cfg)
    _, keys, vals = bin_pairs_lp(pr["rec"], pr["sd"], pr["bbox"], cam, cfg, exact32=False, key=pr["key"])
    keys, vals, ranges = sort_pairs(keys, vals, Wt * Ht)
    out = render_tiles_lp(pr["sd"], vals, ranges, cam, cfg, delta)
    out.update(proj=pr, keys=keys, vals=vals, ranges=ranges)
    return out


def loss_tiled_lp(scene_arrays, cam, cfg, w):
    import hashlib
    out = pipeline_tiled_lp(scene_arrays, cam, cfg)
    h = hashlib.sha1()
    for a in (out["vals"], out["ranges"], out["pixel_sig"]):
        h.update(np.ascontiguousarray(a).tobytes())
    return float((w * out["image"]).sum()), h.hexdigest()


def grads_tiled_lp(scene_arrays, cam, cfg, d_image):
    mu, s, q, o, sh = scene_arrays
    out = pipeline_tiled_lp(scene_arrays, cam, cfg)
    d_sd = render_bwd_tiles_lp(out["proj"]["sd"], out["vals"], out["ranges"], cam, cfg, d_image)
    g = project_lp_bwd(mu, s, q, o, sh, cam, cfg, d_sd)
    g["d_sd"] = d_sd
    return g


# --------------------------------------------------------------------------- rendered features

def _feat_args(rec, feat):
    rec = _f64(rec)
    nfeat = 0 if feat is None else int(np.asarray(feat).reshape(rec.shape[0], -1).shape[1])
    f = np.zeros(1) if nfeat == 0 else _f64(np.asarray(feat).reshape(rec.shape[0], nfeat))
    return rec, f, nfeat


def render_tiles_feat(rec, feat, vals, ranges, cam, cfg, with_depth=False):
    """3DGS image plus rendered features [nfeat + with_depth, H, W] over given lists: each channel is
    sum_i f_ic alpha_i T_i (the depth channel's values are the records' depths)."""
    rec, f, nfeat = _feat_args(rec, feat)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    H, W = cam.height, cam.width
    nf = nfeat + int(bool(with_depth))
    image, feats, tfin = np.zeros((3, H, W)), np.zeros((max(nf, 1), H, W)), np.zeros((H, W))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_render_tiles_feat(rec.shape[0], _p(rec, _F64P), _p(f, _F64P), nfeat, int(bool(with_depth)),
                                   _p(vv, _U32P), _p(ranges, _I32P), _p(ca, _F64P), _p(fa, _F64P), _p(image, _F64P),
                                   _p(feats, _F64P), _p(tfin, _F64P))
    return dict(image=image, features=feats[:nf], t_final=tfin)


def render_bwd_tiles_feat(rec, feat, vals, ranges, cam, cfg, d_image, d_features, with_depth=False):
    """Adjoint of render_tiles_feat: (d_rec[n,12] with the depth gradient in entry 9, d_feat[n,nfeat])."""
    rec, f, nfeat = _feat_args(rec, feat)
    vals = np.ascontiguousarray(vals, np.uint32)
    vv = vals if vals.size else np.zeros(1, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.int32)
    d_image, d_features = _f64(d_image), _f64(d_features)
    d_rec, d_feat = np.zeros((rec.shape[0], 12)), np.zeros((rec.shape[0], max(nfeat, 1)))
    ca, fa = cam_array(cam), cfg_array(cfg)
    lib().oracle_render_bwd_tiles_feat(rec.shape[0], _p(rec, _F64P), _p(f, _F64P), nfeat, int(bool(with_depth)),
                                       _p(vv, _U32P), _p(ranges, _I32P), _p(ca, _F64P), _p(fa, _F64P),
                                       _p(d_image, _F64P), _p(d_features, _F64P), _p(d_rec, _F64P),
                                       _p(d_feat, _F64P))
    return d_rec, d_feat[:, :nfeat]


def pipeline_tiled_feat(scene_arrays, feat, cam, cfg, with_depth=False):
    pr = project(*scene_arrays, cam, cfg)
    Wt, Ht = tiles_of(cam, cfg)
    _, keys, vals = bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False, key=pr["key"])
    keys, vals, ranges = sort_pairs(keys, vals, Wt * Ht)
    out = render_tiles_feat(pr["rec"], feat, vals, ranges, cam, cfg, with_depth)
    out.update(proj=pr, vals=vals, ranges=ranges)
    return out


def grads_tiled_feat(scene_arrays, feat, cam, cfg, d_image, d_features, with_depth=False):
    out = pipeline_tiled_feat(scene_arrays, feat, cam, cfg, with_depth)
    d_rec, d_feat = render_bwd_tiles_feat(out["proj"]["rec"], feat, out["vals"], out["ranges"], cam, cfg, d_image,
                                          d_features, with_depth)
    g = project_bwd(*scene_arrays, cam, cfg, d_rec)
    g["feat"] = d_feat
    return g


def threads_used() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB, lib().oracle_abi_version())
