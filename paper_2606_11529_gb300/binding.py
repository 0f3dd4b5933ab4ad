"""ctypes binding of libxpr.so (C ABI in include/xpr.h).

Argument marshalling only: every function here passes device pointers of
torch tensors to the entry point of the same name and raises ``XprError`` on a
non-zero status.  Output tensors are allocated with ``torch.empty`` when the
caller does not pass them (PyTorch is the allocator; the library never
allocates).  There is no CPU fallback: if the library cannot be loaded the
first call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

c_i32, c_i64, c_f32, c_vp, c_sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_size_t


class XprCamera(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("fx", c_f32), ("fy", c_f32), ("cx", c_f32), ("cy", c_f32),
                ("viewmat", c_f32 * 12), ("z_near", c_f32), ("model", c_i32), ("dist", c_f32 * 4)]


class XprConfig(ctypes.Structure):
    _fields_ = [("tile_w", c_i32), ("tile_h", c_i32), ("alpha_thresh", c_f32), ("alpha_max", c_f32),
                ("t_eps", c_f32), ("cov_dilation", c_f32), ("clip_factor", c_f32), ("sh_degree", c_i32),
                ("bg", c_f32 * 3), ("batch_depth", c_i32), ("method", c_i32)]


class XprPrims(ctypes.Structure):
    _fields_ = [("mu", c_vp), ("scale", c_vp), ("quat", c_vp), ("opacity", c_vp), ("sh", c_vp)]


class XprPrimsGrad(ctypes.Structure):
    _fields_ = [("mu", c_vp), ("scale", c_vp), ("quat", c_vp), ("opacity", c_vp), ("sh", c_vp)]


class XprItem(ctypes.Structure):
    _fields_ = [("prim_offset", c_i64), ("n", c_i64), ("rec_offset", c_i64), ("tile_offset", c_i64),
                ("pix_offset", c_i64)]


XPR_OK, XPR_ERR_INVALID, XPR_ERR_CAPACITY, XPR_ERR_CUDA, XPR_ERR_TIMEOUT, XPR_ERR_INTERNAL = range(6)
XPR_METHOD_3DGS, XPR_METHOD_3DGUT, XPR_METHOD_LINPRIM = 0, 1, 2
REC = 12
SD = 16     # 3DGUT shader data per record
LP_SD = 20  # LinPrim shader data per record

# (name, restype, argtypes) of every exported entry point
SIGNATURES = {
    "xpr_project": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                            c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_tile_bin_workspace": (c_sz, [c_i64]),
    "xpr_depth_order_workspace": (c_sz, [c_i64]),
    "xpr_depth_order": (c_i32, [c_vp, c_vp, c_i64, c_vp, c_vp, c_sz, c_vp]),
    "xpr_tile_bin": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(XprCamera),
                             ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64), c_vp,
                             c_sz, c_vp]),
    "xpr_tile_bin_noalloc": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(XprCamera),
                                     ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64),
                                     c_vp]),
    "xpr_sort_workspace": (c_sz, [c_i64, c_i32]),
    "xpr_sort": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "xpr_sort_tiles_workspace": (c_sz, [c_i64, c_i32]),
    "xpr_sort_tiles": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp]),
    "xpr_render_fwd": (c_i32, [c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig), c_vp,
                               c_vp, c_vp, c_vp]),
    "xpr_render_bwd": (c_i32, [c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig), c_vp,
                               c_vp, c_vp, c_vp, ctypes.POINTER(XprPrims), ctypes.POINTER(XprPrimsGrad), c_vp]),
    "xpr_project_bwd": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera),
                                ctypes.POINTER(XprConfig), c_vp, ctypes.POINTER(XprPrimsGrad), c_vp]),
    "xpr_project_views": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera), c_i32,
                                  ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_depth_order_views": (c_i32, [c_vp, c_vp, c_i64, c_i32, c_vp, c_vp, c_sz, c_vp]),
    "xpr_tile_bin_views": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, ctypes.POINTER(XprCamera),
                                   ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64), c_vp,
                                   c_sz, c_vp]),
    "xpr_tile_worklist_workspace": (c_sz, [c_i32]),
    "xpr_tile_worklist": (c_i32, [c_vp, c_i32, c_vp, c_vp, c_sz, c_vp]),
    "xpr_render_fwd_views": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_vp, ctypes.POINTER(XprCamera),
                                     ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_bwd_views": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_vp, ctypes.POINTER(XprCamera),
                                     ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_project_bwd_views": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera), c_i32,
                                      ctypes.POINTER(XprConfig), c_vp, ctypes.POINTER(XprPrimsGrad), c_vp]),
    "xpr_project_color": (c_i32, [c_vp, c_vp, c_i64, ctypes.POINTER(XprCamera), c_i32, ctypes.POINTER(XprConfig),
                                  c_vp, c_vp]),
    "xpr_bin_sorted_workspace": (c_sz, [c_i64, c_i32, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig)]),
    "xpr_bin_rows_workspace": (c_sz, [c_i64, c_i64, c_i64, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig)]),
    "xpr_bin_rows": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                             c_vp, c_vp, c_i64, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), c_vp, c_sz, c_vp]),
    "xpr_bin_rows_views_workspace": (c_sz, [c_i64, c_i32, c_i64, c_i64, ctypes.POINTER(XprCamera),
                                            ctypes.POINTER(XprConfig)]),
    "xpr_bin_rows_views": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, ctypes.POINTER(XprCamera),
                                   ctypes.POINTER(XprConfig), c_vp, c_vp, c_i64, ctypes.POINTER(c_i64),
                                   ctypes.POINTER(c_i64), c_vp, c_sz, c_vp]),
    "xpr_bin_rows_items_workspace": (c_sz, [ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem), c_i32,
                                            ctypes.POINTER(XprConfig), c_i64, c_i64]),
    "xpr_bin_rows_items": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem),
                                   c_i32, ctypes.POINTER(XprConfig), c_vp, c_vp, c_i64, ctypes.POINTER(c_i64),
                                   ctypes.POINTER(c_i64), c_vp, c_sz, c_vp]),
    "xpr_bin_sorted": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, ctypes.POINTER(XprCamera),
                               ctypes.POINTER(XprConfig), c_vp, c_vp, c_i64, ctypes.POINTER(c_i64), c_vp, c_sz,
                               c_vp]),
    "xpr_project_ut": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                               c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_ut_fwd": (c_i32, [c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                                  c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_ut_bwd": (c_i32, [c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                                  c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_project_ut_bwd": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera),
                                   ctypes.POINTER(XprConfig), c_vp, ctypes.POINTER(XprPrimsGrad), c_vp]),
    "xpr_project_ut_views": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera), c_i32,
                                     ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_ut_fwd_views": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_vp, ctypes.POINTER(XprCamera),
                                        ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_ut_bwd_views": (c_i32, [c_vp, c_i64, c_i32, c_vp, c_vp, ctypes.POINTER(XprCamera),
                                        ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_project_ut_bwd_views": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera), c_i32,
                                         ctypes.POINTER(XprConfig), c_vp, ctypes.POINTER(XprPrimsGrad), c_vp]),
    "xpr_project_lp": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                               c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_tile_bin_lp": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(XprCamera),
                                ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64),
                                c_vp, c_sz, c_vp]),
    "xpr_render_lp_fwd": (c_i32, [c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                                  c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_lp_bwd": (c_i32, [c_vp, c_i64, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprConfig),
                                  c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_project_lp_bwd": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera),
                                   ctypes.POINTER(XprConfig), c_vp, ctypes.POINTER(XprPrimsGrad), c_vp]),
    "xpr_render_fwd_feat": (c_i32, [c_vp, c_i64, c_vp, c_i32, c_i32, c_vp, c_vp, ctypes.POINTER(XprCamera),
                                    ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_bwd_feat": (c_i32, [c_vp, c_i64, c_vp, c_i32, c_i32, c_vp, c_vp, ctypes.POINTER(XprCamera),
                                    ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_project_items": (c_i32, [ctypes.POINTER(XprPrims), ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem), c_i32,
                                  ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp]),
    "xpr_depth_order_items": (c_i32, [c_vp, c_vp, ctypes.POINTER(XprItem), c_i32, c_vp, c_vp, c_sz, c_vp]),
    "xpr_bin_sorted_items_workspace": (c_sz, [ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem), c_i32,
                                              ctypes.POINTER(XprConfig)]),
    "xpr_bin_sorted_items": (c_i32, [c_vp, c_vp, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem),
                                     c_i32, ctypes.POINTER(XprConfig), c_vp, c_vp, c_i64, ctypes.POINTER(c_i64), c_vp,
                                     c_sz, c_vp]),
    "xpr_render_fwd_items": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem), c_i32,
                                     ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_render_bwd_items": (c_i32, [c_vp, c_vp, c_vp, ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem), c_i32,
                                     ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "xpr_project_bwd_items": (c_i32, [ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera),
                                      ctypes.POINTER(XprItem), c_i32, ctypes.POINTER(XprConfig), c_vp,
                                      ctypes.POINTER(XprPrimsGrad), c_vp]),
    "xpr_forward_items_workspace": (c_sz, [ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem), c_i32,
                                           ctypes.POINTER(XprConfig), c_i64]),
    "xpr_forward_items": (c_i32, [ctypes.POINTER(XprPrims), ctypes.POINTER(XprCamera), ctypes.POINTER(XprItem), c_i32,
                                  ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_i64, ctypes.POINTER(c_i64), c_vp, c_sz,
                                  c_vp]),
    "xpr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "xpr_last_error": (ctypes.c_char_p, []),
    "xpr_version": (ctypes.c_int, []),
    "xpr_launch_count": (ctypes.c_ulonglong, []),
    "xpr_device_check": (c_i32, []),
    "xpr_selftest_wait": (c_i32, [c_vp, c_i32, c_vp]),
    "xpr_project_host": (c_i32, [ctypes.POINTER(XprPrims), ctypes.POINTER(XprPrims), c_i64, ctypes.POINTER(XprCamera),
                                 ctypes.POINTER(XprConfig), c_vp, c_vp, c_vp, c_vp, c_vp]),
}

_lib = None


class XprError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn} failed with status {status}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libxpr.so (building it first if needed and allowed)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libxpr.so not found at {path}; run paper_2606_11529_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, fn: str):
    if status != XPR_OK:
        msg = load().xpr_last_error().decode(errors="replace")
        raise XprError(status, fn, msg)


def xpr_device_check():
    """Synchronises the device and raises XprError if a kernel recorded a timed-out wait or an
    inconsistent intermediate since the last check (the flags are cleared)."""
    _check(load().xpr_device_check(), "xpr_device_check")


def xpr_selftest_wait(polls=1000, stream=None):
    """Runs the sort's bounded look-back wait against words nothing publishes (see xpr.h); returns
    the 256 counts it ended with.  The timeout is then reported by xpr_device_check."""
    z = torch.zeros(512, dtype=torch.int32, device="cuda")
    _check(load().xpr_selftest_wait(_ptr(z), int(polls), _stream(stream)), "xpr_selftest_wait")
    return z[256:]


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_camera(cam) -> XprCamera:
    """From a ``scenes.Camera``-like object."""
    c = XprCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    vm = [float(v) for v in __import__("numpy").asarray(cam.viewmat, dtype="float32").reshape(12)]
    c.viewmat[:] = vm
    c.z_near = float(cam.z_near)
    c.model = int(getattr(cam, "model", 0))
    c.dist[:] = [float(k) for k in getattr(cam, "dist", (0.0, 0.0, 0.0, 0.0))]
    return c


def make_config(cfg) -> XprConfig:
    g = XprConfig()
    g.tile_w, g.tile_h = int(cfg.tile_w), int(cfg.tile_h)
    g.alpha_thresh, g.alpha_max, g.t_eps = float(cfg.alpha_thresh), float(cfg.alpha_max), float(cfg.t_eps)
    g.cov_dilation, g.clip_factor = float(cfg.cov_dilation), float(cfg.clip_factor)
    g.sh_degree = int(cfg.sh_degree)
    g.bg[:] = [float(b) for b in cfg.bg]
    g.batch_depth = int(getattr(cfg, "batch_depth", 0))
    g.method = int(getattr(cfg, "method", XPR_METHOD_3DGS))
    return g


def _as_c(x, C):
    return x if isinstance(x, C) else (make_camera(x) if C is XprCamera else make_config(x))


def _dev(t):
    return t.device


def _prims(mu, scale, quat, opacity, sh) -> XprPrims:
    """sh may be None (geometry-only projection)."""
    for name, t in (("mu", mu), ("scale", scale), ("quat", quat), ("opacity", opacity), ("sh", sh)):
        if t is None and name == "sh":
            continue
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return XprPrims(mu.data_ptr(), scale.data_ptr(), quat.data_ptr(), opacity.data_ptr(),
                    None if sh is None else sh.data_ptr())


def tiles_of(cam, cfg):
    return (int(cam.width) + int(cfg.tile_w) - 1) // int(cfg.tile_w), \
           (int(cam.height) + int(cfg.tile_h) - 1) // int(cfg.tile_h)


# ---------------------------------------------------------------------------------------- entry points

def xpr_project(mu, scale, quat, opacity, sh, cam, cfg, rec=None, bbox=None, tile_count=None, stream=None,
                isect_count=None, with_isect_count=False):
    """Returns (rec, bbox, tile_count), plus isect_count when ``with_isect_count`` (or a buffer) is given."""
    L = load()
    n = mu.shape[0]
    dev = _dev(mu)
    rec = torch.empty((n, REC), dtype=torch.float32, device=dev) if rec is None else rec
    bbox = torch.empty((n, 4), dtype=torch.int32, device=dev) if bbox is None else bbox
    tile_count = torch.empty(n, dtype=torch.int32, device=dev) if tile_count is None else tile_count
    if isect_count is None and with_isect_count:
        isect_count = torch.empty(n, dtype=torch.int32, device=dev)
    p = _prims(mu, scale, quat, opacity, sh)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_project(ctypes.byref(p), n, ctypes.byref(c), ctypes.byref(g), _ptr(rec), _ptr(bbox),
                         _ptr(tile_count), _ptr(isect_count), _stream(stream)), "xpr_project")
    return (rec, bbox, tile_count) if isect_count is None else (rec, bbox, tile_count, isect_count)


def xpr_project_host(host, dst, cam, cfg, stream=None, with_isect_count=False):
    """xpr_project reading the geometry from pinned host tensors host = (mu, scale, quat, opacity)
    and writing its copy into the device tensors dst = (mu, scale, quat, opacity, sh or None) in the
    same pass.  Returns (rec, bbox, tile_count[, isect_count])."""
    L = load()
    n = dst[0].shape[0]
    for t, d in zip(host, dst[:4]):
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.shape != d.shape:
            raise ValueError("host geometry must be contiguous float32 host tensors shaped like the device ones")
    dev = dst[0].device
    rec = torch.empty((n, REC), dtype=torch.float32, device=dev)
    bbox = torch.empty((n, 4), dtype=torch.int32, device=dev)
    tile_count = torch.empty(n, dtype=torch.int32, device=dev)
    isect_count = torch.empty(n, dtype=torch.int32, device=dev) if with_isect_count else None
    hp = XprPrims(*[t.data_ptr() for t in host], None)
    dp = _prims(*dst)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_project_host(ctypes.byref(hp), ctypes.byref(dp), n, ctypes.byref(c), ctypes.byref(g), _ptr(rec),
                              _ptr(bbox), _ptr(tile_count), _ptr(isect_count), _stream(stream)), "xpr_project_host")
    return (rec, bbox, tile_count) if isect_count is None else (rec, bbox, tile_count, isect_count)


def xpr_depth_order(rec, tile_count, order=None, workspace=None, stream=None):
    L = load()
    n = rec.shape[0]
    order = torch.empty(n, dtype=torch.int32, device=rec.device) if order is None else order
    need = int(L.xpr_depth_order_workspace(n))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=rec.device)
    _check(L.xpr_depth_order(_ptr(rec), _ptr(tile_count), n, _ptr(order), _ptr(workspace), workspace.numel(),
                             _stream(stream)), "xpr_depth_order")
    return order


def xpr_tile_bin(rec, bbox, tile_count, cam, cfg, capacity=None, offsets=None, keys=None, vals=None,
                 workspace=None, stream=None, order=None, isect_count=None, tile_ids=False):
    """Returns (offsets[n+1], pairs[I], vals[I], I) where pairs are u64 keys (int64 storage) or, with
    ``tile_ids``, u32 tile ids (int32 storage).  ``order``: optional emission order (int32
    permutation); ``isect_count``: per-primitive kept-tile counts from xpr_project.  ``capacity``:
    initial guess for the pair buffers; on XPR_ERR_CAPACITY they are re-allocated to the reported
    size and the call is repeated."""
    L = load()
    n = rec.shape[0]
    dev = rec.device
    kdt = torch.int32 if tile_ids else torch.int64
    offsets = torch.empty(n + 1, dtype=torch.int32, device=dev) if offsets is None else offsets
    ws_need = int(L.xpr_tile_bin_workspace(n))
    if workspace is None or workspace.numel() < ws_need:
        workspace = torch.empty(max(ws_need, 256), dtype=torch.uint8, device=dev)
    if keys is None or capacity is None:
        cap = int(capacity) if capacity is not None else max(4 * n, 1024)
        keys = torch.empty(cap, dtype=kdt, device=dev)
        vals = torch.empty(cap, dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    for _ in range(2):
        n_isect = c_i64(0)
        s = L.xpr_tile_bin(_ptr(rec), _ptr(bbox), _ptr(tile_count), _ptr(isect_count), _ptr(order), n,
                           ctypes.byref(c), ctypes.byref(g), _ptr(offsets), None if tile_ids else _ptr(keys),
                           _ptr(keys) if tile_ids else None, _ptr(vals), keys.numel(), ctypes.byref(n_isect),
                           _ptr(workspace), workspace.numel(), _stream(stream))
        if s == XPR_ERR_CAPACITY and n_isect.value <= 0x7FFFFFFF:
            keys = torch.empty(n_isect.value, dtype=kdt, device=dev)
            vals = torch.empty(n_isect.value, dtype=torch.int32, device=dev)
            continue
        _check(s, "xpr_tile_bin")
        I = int(n_isect.value)
        return offsets, keys[:I], vals[:I], I
    raise XprError(XPR_ERR_CAPACITY, "xpr_tile_bin", "capacity retry failed")


def xpr_sort_tiles(tiles, vals, n_tiles, tiles_out=None, vals_out=None, ranges=None, workspace=None, stream=None,
                   want_tiles=True):
    """Returns (tiles_sorted or None, vals_sorted, ranges).  want_tiles=False skips writing the
    sorted tile ids (and lets the sort use `tiles` as scratch when it needs more than 2 passes)."""
    L = load()
    n = tiles.numel()
    dev = tiles.device
    if want_tiles:
        tiles_out = torch.empty_like(tiles) if tiles_out is None else tiles_out
    else:
        tiles_out = None
    vals_out = torch.empty_like(vals) if vals_out is None else vals_out
    ranges = torch.empty((n_tiles, 2), dtype=torch.int32, device=dev) if ranges is None else ranges
    need = int(L.xpr_sort_tiles_workspace(n, n_tiles))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    _check(L.xpr_sort_tiles(_ptr(tiles), _ptr(vals), n, n_tiles, _ptr(tiles_out), _ptr(vals_out), _ptr(ranges),
                            _ptr(workspace), workspace.numel(), _stream(stream)), "xpr_sort_tiles")
    return tiles_out, vals_out, ranges


def xpr_sort(keys, vals, n_tiles, keys_out=None, vals_out=None, ranges=None, workspace=None, stream=None,
             begin_bit=0):
    L = load()
    n = keys.numel()
    dev = keys.device
    keys_out = torch.empty_like(keys) if keys_out is None else keys_out
    vals_out = torch.empty_like(vals) if vals_out is None else vals_out
    ranges = torch.empty((n_tiles, 2), dtype=torch.int32, device=dev) if ranges is None else ranges
    need = int(L.xpr_sort_workspace(n, n_tiles))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    _check(L.xpr_sort(_ptr(keys), _ptr(vals), n, n_tiles, begin_bit, _ptr(keys_out), _ptr(vals_out), _ptr(ranges),
                      _ptr(workspace), workspace.numel(), _stream(stream)), "xpr_sort")
    return keys_out, vals_out, ranges


def xpr_render_fwd(rec, vals, ranges, cam, cfg, image=None, t_final=None, n_contrib=None, stream=None):
    L = load()
    dev = rec.device
    H, W = int(cam.height), int(cam.width)
    image = torch.empty((3, H, W), dtype=torch.float32, device=dev) if image is None else image
    t_final = torch.empty((H, W), dtype=torch.float32, device=dev) if t_final is None else t_final
    n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev) if n_contrib is None else n_contrib
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_fwd(_ptr(rec), rec.shape[0], _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                            _ptr(image), _ptr(t_final), _ptr(n_contrib), _stream(stream)), "xpr_render_fwd")
    return image, t_final, n_contrib


def xpr_render_bwd(rec, vals, ranges, cam, cfg, t_final, n_contrib, d_image, prims=None, d_rec=None,
                   d_prims=None, stream=None):
    """prims: optional (mu, scale, quat, opacity, sh) to also run the projection adjoint.
    Returns d_rec[n,12] and, if prims is given, (dmu, dscale, dquat, dopacity, dsh)."""
    L = load()
    n = rec.shape[0]
    dev = rec.device
    d_rec = torch.empty((n, REC), dtype=torch.float32, device=dev) if d_rec is None else d_rec
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    pp = gp = None
    grads = None
    if prims is not None:
        pp = _prims(*prims)
        grads = d_prims if d_prims is not None else tuple(torch.empty_like(t) for t in prims)
        gp = XprPrimsGrad(*[t.data_ptr() for t in grads])
    _check(L.xpr_render_bwd(_ptr(rec), n, _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                            _ptr(t_final), _ptr(n_contrib), _ptr(d_image.contiguous()), _ptr(d_rec),
                            ctypes.byref(pp) if pp is not None else None,
                            ctypes.byref(gp) if gp is not None else None, _stream(stream)), "xpr_render_bwd")
    return (d_rec, grads) if prims is not None else d_rec


def xpr_project_bwd(mu, scale, quat, opacity, sh, cam, cfg, d_rec, d_prims=None, stream=None):
    L = load()
    grads = d_prims if d_prims is not None else tuple(torch.empty_like(t) for t in (mu, scale, quat, opacity, sh))
    p = _prims(mu, scale, quat, opacity, sh)
    gp = XprPrimsGrad(*[t.data_ptr() for t in grads])
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_project_bwd(ctypes.byref(p), mu.shape[0], ctypes.byref(c), ctypes.byref(g), _ptr(d_rec),
                             ctypes.byref(gp), _stream(stream)), "xpr_project_bwd")
    return grads


# ---------------------------------------------------------------------------------------- multi-view form

def camera_array(cams):
    arr = (XprCamera * len(cams))()
    for v, c in enumerate(cams):
        arr[v] = c if isinstance(c, XprCamera) else make_camera(c)
    return arr


def xpr_project_views(mu, scale, quat, opacity, sh, cams, cfg, stream=None, with_isect_count=True):
    """Returns rec[V*n,12], bbox[V*n,4], tile_count[V*n], isect_count[V*n] (view-major; None when
    not asked for)."""
    L = load()
    n, V = mu.shape[0], len(cams)
    dev = mu.device
    rec = torch.empty((V * n, REC), dtype=torch.float32, device=dev)
    bbox = torch.empty((V * n, 4), dtype=torch.int32, device=dev)
    tc = torch.empty(V * n, dtype=torch.int32, device=dev)
    cnt = torch.empty(V * n, dtype=torch.int32, device=dev) if with_isect_count else None
    p = _prims(mu, scale, quat, opacity, sh)
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_project_views(ctypes.byref(p), n, camera_array(cams), V, ctypes.byref(g), _ptr(rec), _ptr(bbox),
                               _ptr(tc), _ptr(cnt), _stream(stream)), "xpr_project_views")
    return rec, bbox, tc, cnt


def xpr_depth_order_views(rec, tile_count, n, n_views, workspace=None, stream=None):
    L = load()
    order = torch.empty(n * n_views, dtype=torch.int32, device=rec.device)
    need = int(L.xpr_depth_order_workspace(n * n_views))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=rec.device)
    _check(L.xpr_depth_order_views(_ptr(rec), _ptr(tile_count), n, n_views, _ptr(order), _ptr(workspace),
                                   workspace.numel(), _stream(stream)), "xpr_depth_order_views")
    return order


def xpr_tile_bin_views(rec, bbox, tile_count, isect_count, order, n, n_views, cam, cfg, capacity=None,
                       workspace=None, stream=None):
    """Returns (offsets[V*n+1], tiles[I] (global u32 ids, int32 storage), vals[I], I)."""
    L = load()
    dev = rec.device
    N = n * n_views
    offsets = torch.empty(N + 1, dtype=torch.int32, device=dev)
    need = int(L.xpr_tile_bin_workspace(N))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    cap = int(capacity) if capacity is not None else max(4 * N, 1024)
    tiles = torch.empty(cap, dtype=torch.int32, device=dev)
    vals = torch.empty(cap, dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    for _ in range(2):
        got = c_i64(0)
        s = L.xpr_tile_bin_views(_ptr(rec), _ptr(bbox), _ptr(tile_count), _ptr(isect_count), _ptr(order), n,
                                 n_views, ctypes.byref(c), ctypes.byref(g), _ptr(offsets), _ptr(tiles), _ptr(vals),
                                 tiles.numel(), ctypes.byref(got), _ptr(workspace), workspace.numel(),
                                 _stream(stream))
        if s == XPR_ERR_CAPACITY and got.value <= 0x7FFFFFFF:
            tiles = torch.empty(got.value, dtype=torch.int32, device=dev)
            vals = torch.empty(got.value, dtype=torch.int32, device=dev)
            continue
        _check(s, "xpr_tile_bin_views")
        I = int(got.value)
        return offsets, tiles[:I], vals[:I], I
    raise XprError(XPR_ERR_CAPACITY, "xpr_tile_bin_views", "capacity retry failed")


def xpr_project_color(mu, sh, rec, cams, cfg, stream=None):
    """Fills rec[V*n, 6:9] (colours of visible records) from the SH coefficients; cams: a camera or a list."""
    L = load()
    cams = list(cams) if isinstance(cams, (list, tuple)) else [cams]
    for name, t in (("mu", mu), ("sh", sh), ("rec", rec)):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_project_color(_ptr(mu), _ptr(sh), mu.shape[0], camera_array(cams), len(cams), ctypes.byref(g),
                               _ptr(rec), _stream(stream)), "xpr_project_color")


def binsort_ok(cam, cfg, n_views=1):
    """Whether xpr_bin_sorted takes this grid: at most 4096 tile columns (its per-row cursors in
    shared memory) and 1..16 views."""
    Wt, Ht = tiles_of(cam, cfg)
    return Wt <= 4096 and 1 <= n_views <= 16


def bin_sorted_workspace_bytes(n, n_views, cam, cfg):
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    return int(load().xpr_bin_sorted_workspace(n, n_views, ctypes.byref(c), ctypes.byref(g)))


def xpr_bin_sorted(rec, bbox, tile_count, order, n, cam, cfg, n_views=1, capacity=None, workspace=None,
                   stream=None):
    """Fused bin + sort: returns (ranges[V*T,2], vals[I] (record indices, int32 storage), I).
    ``capacity``: initial size of vals; on XPR_ERR_CAPACITY it is re-allocated to I and the call
    repeated."""
    L = load()
    dev = rec.device
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    Wt, Ht = tiles_of(cam, cfg)
    ranges = torch.empty((n_views * Wt * Ht, 2), dtype=torch.int32, device=dev)
    need = int(L.xpr_bin_sorted_workspace(n, n_views, ctypes.byref(c), ctypes.byref(g)))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    cap = int(capacity) if capacity is not None else max(4 * n * n_views, 1024)
    vals = torch.empty(cap, dtype=torch.int32, device=dev)
    for _ in range(2):
        got = c_i64(0)
        s = L.xpr_bin_sorted(_ptr(rec), _ptr(bbox), _ptr(tile_count), _ptr(order), n, n_views, ctypes.byref(c),
                             ctypes.byref(g), _ptr(ranges), _ptr(vals), vals.numel(), ctypes.byref(got),
                             _ptr(workspace), workspace.numel(), _stream(stream))
        if s == XPR_ERR_CAPACITY and got.value <= 0x7FFFFFFF:
            vals = torch.empty(max(got.value, 1), dtype=torch.int32, device=dev)
            continue
        _check(s, "xpr_bin_sorted")
        I = int(got.value)
        return ranges, vals[:I], I
    raise XprError(XPR_ERR_CAPACITY, "xpr_bin_sorted", "capacity retry failed")


def bin_rows_ok(cam, cfg) -> bool:
    """The rows binning takes grids of at most 128 x 128 tiles (3DGS and 3DGUT; one view, the views
    of one camera, or items whose every camera fits)."""
    Wt, Ht = tiles_of(cam, cfg)
    return Wt <= 128 and Ht <= 128 and int(getattr(cfg, "method", XPR_METHOD_3DGS)) != XPR_METHOD_LINPRIM


def bin_rows_items_ok(layout, cfg) -> bool:
    return all(bin_rows_ok(c, cfg) for c in layout.cams)


def bin_rows_workspace_bytes(n, n_spans, n_isect, cam, cfg):
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    return int(load().xpr_bin_rows_workspace(int(n), int(n_spans), int(n_isect), ctypes.byref(c), ctypes.byref(g)))


def bin_rows_views_workspace_bytes(n, n_views, n_spans, n_isect, cam, cfg):
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    return int(load().xpr_bin_rows_views_workspace(int(n), int(n_views), int(n_spans), int(n_isect), ctypes.byref(c),
                                                   ctypes.byref(g)))


def bin_rows_items_workspace_bytes(layout, n_spans, n_isect, cfg):
    g = _as_c(cfg, XprConfig)
    return int(load().xpr_bin_rows_items_workspace(layout.carr, layout.arr, layout.K, ctypes.byref(g), int(n_spans),
                                                   int(n_isect)))


def _bin_rows_retry(name, call, need, n_tiles, dev, cap, workspace):
    """The capacity protocol of the rows binning calls: call(ranges, vals, workspace, got_i, got_s) runs
    the C entry, need(S, I) gives the workspace it wants.  On XPR_ERR_CAPACITY vals and the workspace
    are re-allocated to the reported counts and the call repeated; returns (ranges, vals[:I], I, S,
    workspace)."""
    ranges = torch.empty((max(n_tiles, 1), 2), dtype=torch.int32, device=dev)[:n_tiles]
    vals = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    n0 = need(0, 0)
    if workspace is None or workspace.numel() < n0:
        workspace = torch.empty(max(n0, 256), dtype=torch.uint8, device=dev)
    for _ in range(3):
        got_i, got_s = c_i64(0), c_i64(0)
        s = call(ranges, vals, workspace, got_i, got_s)
        if s == XPR_ERR_CAPACITY and got_i.value <= 0x7FFFFFFF and got_s.value <= 0x7FFFFFFF:
            if got_i.value > vals.numel():
                vals = torch.empty(got_i.value, dtype=torch.int32, device=dev)
            # room for a quarter more span slots beside the pairs: the calls that follow (the next
            # frame) then find it and queue their work ahead of the counts they read back
            n1 = need(int(got_s.value * 1.25) + 1024, max(got_i.value, vals.numel()))
            if workspace.numel() < n1:
                workspace = torch.empty(n1, dtype=torch.uint8, device=dev)
            continue
        _check(s, name)
        I = int(got_i.value)
        return ranges, vals[:I], I, int(got_s.value), workspace
    raise XprError(XPR_ERR_CAPACITY, name, "capacity retry failed")


def xpr_bin_rows(rec, bbox, tile_count, order, n, cam, cfg, isect_count=None, capacity=None, workspace=None,
                 stream=None):
    """Bin + sort by tile rows: returns (ranges[T,2], vals[I] (record indices, int32 storage), I, S,
    workspace), S the span slots.  ``capacity``: initial size of vals; ``workspace``: initial
    scratch.  On XPR_ERR_CAPACITY either is re-allocated to the reported counts and the call repeated;
    the workspace returned is the one used (keep it for the next call)."""
    L = load()
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    Wt, Ht = tiles_of(cam, cfg)
    cap = int(capacity) if capacity is not None else max(4 * n, 1024)

    def call(ranges, vals, ws, gi, gs):
        return L.xpr_bin_rows(_ptr(rec), _ptr(bbox), _ptr(tile_count), _ptr(isect_count), _ptr(order), n,
                              ctypes.byref(c), ctypes.byref(g), _ptr(ranges), _ptr(vals), vals.numel(),
                              ctypes.byref(gi), ctypes.byref(gs), _ptr(ws), ws.numel(), _stream(stream))

    return _bin_rows_retry("xpr_bin_rows", call, lambda S, I: bin_rows_workspace_bytes(n, S, I, cam, cfg), Wt * Ht,
                           rec.device, cap, workspace)


def xpr_bin_rows_views(rec, bbox, tile_count, order, n, n_views, cam, cfg, isect_count=None, capacity=None,
                       workspace=None, stream=None):
    """xpr_bin_rows over V views of one camera (records view-major): ranges[V*T,2], the rest as
    xpr_bin_rows."""
    L = load()
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    Wt, Ht = tiles_of(cam, cfg)
    cap = int(capacity) if capacity is not None else max(4 * n * n_views, 1024)

    def call(ranges, vals, ws, gi, gs):
        return L.xpr_bin_rows_views(_ptr(rec), _ptr(bbox), _ptr(tile_count), _ptr(isect_count), _ptr(order), n,
                                    n_views, ctypes.byref(c), ctypes.byref(g), _ptr(ranges), _ptr(vals), vals.numel(),
                                    ctypes.byref(gi), ctypes.byref(gs), _ptr(ws), ws.numel(), _stream(stream))

    return _bin_rows_retry("xpr_bin_rows_views", call,
                           lambda S, I: bin_rows_views_workspace_bytes(n, n_views, S, I, cam, cfg),
                           n_views * Wt * Ht, rec.device, cap, workspace)


def xpr_bin_rows_items(rec, bbox, tile_count, order, layout, cfg, isect_count=None, capacity=None, workspace=None,
                       stream=None):
    """xpr_bin_rows over the items of a multi-scene batch: ranges[S,2] over all items' tiles, the rest
    as xpr_bin_rows."""
    L = load()
    g = _as_c(cfg, XprConfig)
    cap = int(capacity) if capacity is not None else max(4 * layout.R, 1024)

    def call(ranges, vals, ws, gi, gs):
        return L.xpr_bin_rows_items(_ptr(rec), _ptr(bbox), _ptr(tile_count), _ptr(isect_count), _ptr(order),
                                    layout.carr, layout.arr, layout.K, ctypes.byref(g), _ptr(ranges), _ptr(vals),
                                    vals.numel(), ctypes.byref(gi), ctypes.byref(gs), _ptr(ws), ws.numel(),
                                    _stream(stream))

    return _bin_rows_retry("xpr_bin_rows_items", call, lambda S, I: bin_rows_items_workspace_bytes(layout, S, I, g),
                           layout.S, rec.device, cap, workspace)


def xpr_tile_worklist(ranges, workspace=None, stream=None):
    L = load()
    nt = ranges.shape[0]
    wl = torch.empty(nt, dtype=torch.int32, device=ranges.device)
    need = int(L.xpr_tile_worklist_workspace(nt))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=ranges.device)
    _check(L.xpr_tile_worklist(_ptr(ranges), nt, _ptr(wl), _ptr(workspace), workspace.numel(), _stream(stream)),
           "xpr_tile_worklist")
    return wl


def xpr_render_fwd_views(rec, n, n_views, vals, ranges, cam, cfg, worklist=None, counter=None, stream=None):
    L = load()
    dev = rec.device
    H, W = int(cam.height), int(cam.width)
    image = torch.empty((n_views, 3, H, W), dtype=torch.float32, device=dev)
    tfin = torch.empty((n_views, H, W), dtype=torch.float32, device=dev)
    ncon = torch.empty((n_views, H, W), dtype=torch.int32, device=dev)
    if worklist is not None and counter is None:
        counter = torch.empty(1, dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_fwd_views(_ptr(rec), n, n_views, _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                                  _ptr(image), _ptr(tfin), _ptr(ncon), _ptr(worklist), _ptr(counter),
                                  _stream(stream)), "xpr_render_fwd_views")
    return image, tfin, ncon


def xpr_render_bwd_views(rec, n, n_views, vals, ranges, cam, cfg, t_final, n_contrib, d_image, worklist=None,
                         counter=None, stream=None):
    L = load()
    dev = rec.device
    d_rec = torch.empty((n * n_views, REC), dtype=torch.float32, device=dev)
    if worklist is not None and counter is None:
        counter = torch.empty(1, dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_bwd_views(_ptr(rec), n, n_views, _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                                  _ptr(t_final), _ptr(n_contrib), _ptr(d_image.contiguous()), _ptr(d_rec),
                                  _ptr(worklist), _ptr(counter), _stream(stream)), "xpr_render_bwd_views")
    return d_rec


def xpr_project_bwd_views(mu, scale, quat, opacity, sh, cams, cfg, d_rec, stream=None):
    L = load()
    grads = tuple(torch.empty_like(t) for t in (mu, scale, quat, opacity, sh))
    p = _prims(mu, scale, quat, opacity, sh)
    gp = XprPrimsGrad(*[t.data_ptr() for t in grads])
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_project_bwd_views(ctypes.byref(p), mu.shape[0], camera_array(cams), len(cams), ctypes.byref(g),
                                   _ptr(d_rec), ctypes.byref(gp), _stream(stream)), "xpr_project_bwd_views")
    return grads


# ---------------------------------------------------------------------------------------- multi-scene items

class ItemLayout:
    """Offsets of a multi-scene batch (XprItem): item k = (scene of primitives [prim_offset,
    prim_offset + n), camera k).  Records are item-major in blocks padded to 32, tiles and pixels
    follow item order."""

    def __init__(self, prim_offsets, counts, cams, cfg):
        self.cams = list(cams)
        K = len(self.cams)
        if not 1 <= K <= 16:
            raise ValueError(f"{K} items: a batch holds 1..16")
        self.arr = (XprItem * K)()
        rec = tile = pix = 0
        self.rec_offsets, self.tile_offsets, self.pix_offsets, self.shapes = [], [], [], []
        for k, (p0, n, cam) in enumerate(zip(prim_offsets, counts, self.cams)):
            Wt, Ht = tiles_of(cam, cfg)
            self.arr[k] = XprItem(int(p0), int(n), rec, tile, pix)
            self.rec_offsets.append(rec)
            self.tile_offsets.append(tile)
            self.pix_offsets.append(pix)
            self.shapes.append((int(cam.height), int(cam.width)))
            rec += (int(n) + 31) // 32 * 32
            tile += Wt * Ht
            pix += int(cam.width) * int(cam.height)
        self.K, self.R, self.S, self.pixels = K, rec, tile, pix
        self.carr = camera_array(self.cams)

    def images(self, flat):
        """Per-item [3, H, W] views of a flat image buffer."""
        return [flat[3 * p0:3 * p0 + 3 * h * w].view(3, h, w) for p0, (h, w) in zip(self.pix_offsets, self.shapes)]

    def planes(self, flat):
        """Per-item [H, W] views of a flat per-pixel buffer."""
        return [flat[p0:p0 + h * w].view(h, w) for p0, (h, w) in zip(self.pix_offsets, self.shapes)]


def xpr_project_items(mu, scale, quat, opacity, sh, layout, cfg, stream=None):
    L = load()
    dev = mu.device
    rec = torch.empty((layout.R, REC), dtype=torch.float32, device=dev)
    bbox = torch.empty((layout.R, 4), dtype=torch.int32, device=dev)
    tc = torch.empty(layout.R, dtype=torch.int32, device=dev)
    p = _prims(mu, scale, quat, opacity, sh)
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_project_items(ctypes.byref(p), layout.carr, layout.arr, layout.K, ctypes.byref(g), _ptr(rec),
                               _ptr(bbox), _ptr(tc), _stream(stream)), "xpr_project_items")
    return rec, bbox, tc


def xpr_depth_order_items(rec, tile_count, layout, workspace=None, stream=None):
    L = load()
    order = torch.empty(layout.R, dtype=torch.int32, device=rec.device)
    need = int(L.xpr_depth_order_workspace(layout.R))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=rec.device)
    _check(L.xpr_depth_order_items(_ptr(rec), _ptr(tile_count), layout.arr, layout.K, _ptr(order), _ptr(workspace),
                                   workspace.numel(), _stream(stream)), "xpr_depth_order_items")
    return order


def bin_sorted_items_workspace_bytes(layout, cfg):
    g = _as_c(cfg, XprConfig)
    return int(load().xpr_bin_sorted_items_workspace(layout.carr, layout.arr, layout.K, ctypes.byref(g)))


def xpr_bin_sorted_items(rec, bbox, tile_count, order, layout, cfg, capacity=None, workspace=None, stream=None):
    """Fused bin + sort over all items: (ranges[S,2], vals[I] (int32 storage), I)."""
    L = load()
    dev = rec.device
    g = _as_c(cfg, XprConfig)
    ranges = torch.empty((max(layout.S, 1), 2), dtype=torch.int32, device=dev)[:layout.S]
    need = bin_sorted_items_workspace_bytes(layout, g)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    cap = int(capacity) if capacity is not None else max(4 * layout.R, 1024)
    vals = torch.empty(cap, dtype=torch.int32, device=dev)
    for _ in range(2):
        got = c_i64(0)
        s = L.xpr_bin_sorted_items(_ptr(rec), _ptr(bbox), _ptr(tile_count), _ptr(order), layout.carr, layout.arr,
                                   layout.K, ctypes.byref(g), _ptr(ranges), _ptr(vals), vals.numel(),
                                   ctypes.byref(got), _ptr(workspace), workspace.numel(), _stream(stream))
        if s == XPR_ERR_CAPACITY and got.value <= 0x7FFFFFFF:
            vals = torch.empty(max(got.value, 1), dtype=torch.int32, device=dev)
            continue
        _check(s, "xpr_bin_sorted_items")
        I = int(got.value)
        return ranges, vals[:I], I
    raise XprError(XPR_ERR_CAPACITY, "xpr_bin_sorted_items", "capacity retry failed")


def xpr_render_fwd_items(rec, vals, ranges, layout, cfg, worklist=None, counter=None, stream=None):
    """Flat outputs: image[3 * pixels] (item k's planes at 3 pix_offset), t_final[pixels], n_contrib[pixels]."""
    L = load()
    dev = rec.device
    image = torch.empty(3 * layout.pixels, dtype=torch.float32, device=dev)
    tfin = torch.empty(layout.pixels, dtype=torch.float32, device=dev)
    ncon = torch.empty(layout.pixels, dtype=torch.int32, device=dev)
    if worklist is not None and counter is None:
        counter = torch.empty(1, dtype=torch.int32, device=dev)
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_render_fwd_items(_ptr(rec), _ptr(vals), _ptr(ranges), layout.carr, layout.arr, layout.K,
                                  ctypes.byref(g), _ptr(image), _ptr(tfin), _ptr(ncon), _ptr(worklist), _ptr(counter),
                                  _stream(stream)), "xpr_render_fwd_items")
    return image, tfin, ncon


def xpr_render_bwd_items(rec, vals, ranges, layout, cfg, t_final, n_contrib, d_image, worklist=None, counter=None,
                         stream=None):
    L = load()
    dev = rec.device
    d_rec = torch.empty((layout.R, REC), dtype=torch.float32, device=dev)
    if worklist is not None and counter is None:
        counter = torch.empty(1, dtype=torch.int32, device=dev)
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_render_bwd_items(_ptr(rec), _ptr(vals), _ptr(ranges), layout.carr, layout.arr, layout.K,
                                  ctypes.byref(g), _ptr(t_final), _ptr(n_contrib), _ptr(d_image.contiguous()),
                                  _ptr(d_rec), _ptr(worklist), _ptr(counter), _stream(stream)), "xpr_render_bwd_items")
    return d_rec


def xpr_project_bwd_items(mu, scale, quat, opacity, sh, layout, cfg, d_rec, stream=None):
    L = load()
    grads = tuple(torch.empty_like(t) for t in (mu, scale, quat, opacity, sh))
    p = _prims(mu, scale, quat, opacity, sh)
    gp = XprPrimsGrad(*[t.data_ptr() for t in grads])
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_project_bwd_items(ctypes.byref(p), mu.shape[0], layout.carr, layout.arr, layout.K, ctypes.byref(g),
                                   _ptr(d_rec), ctypes.byref(gp), _stream(stream)), "xpr_project_bwd_items")
    return grads


def xpr_forward_items(mu, scale, quat, opacity, sh, layout, cfg, capacity, workspace=None, out=None, stream=None):
    """The whole forward of a multi-scene batch in one C call.  Returns (image, t_final, n_contrib,
    n_isect, workspace) with flat per-pixel outputs (``layout.images``); ``workspace`` (uint8,
    grown here when too small, to be passed again) holds every intermediate.  On a capacity
    shortfall the call is repeated once with room for the reported pair count."""
    L = load()
    dev = mu.device
    g = _as_c(cfg, XprConfig)
    p = _prims(mu, scale, quat, opacity, sh)
    if out is None:
        out = (torch.empty(3 * layout.pixels, dtype=torch.float32, device=dev),
               torch.empty(layout.pixels, dtype=torch.float32, device=dev),
               torch.empty(layout.pixels, dtype=torch.int32, device=dev))
    image, tfin, ncon = out
    cap = int(capacity)
    for _ in range(2):
        need = int(L.xpr_forward_items_workspace(layout.carr, layout.arr, layout.K, ctypes.byref(g), cap))
        if workspace is None or workspace.numel() < need:
            workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
        got = c_i64(0)
        s = L.xpr_forward_items(ctypes.byref(p), layout.carr, layout.arr, layout.K, ctypes.byref(g), _ptr(image),
                                _ptr(tfin), _ptr(ncon), cap, ctypes.byref(got), _ptr(workspace), workspace.numel(),
                                _stream(stream))
        if s == XPR_ERR_CAPACITY and got.value <= 0x7FFFFFFF:
            cap = int(got.value * 1.25) + 1024
            continue
        _check(s, "xpr_forward_items")
        return image, tfin, ncon, int(got.value), workspace
    raise XprError(XPR_ERR_CAPACITY, "xpr_forward_items", "capacity retry failed")


# ---------------------------------------------------------------------------------------- 3DGUT

def xpr_project_ut(mu, scale, quat, opacity, sh, cam, cfg, stream=None, with_isect_count=True):
    """Unscented projection: returns rec[n,12], sd[n,16], bbox[n,4], tile_count[n], isect_count[n] (or None)."""
    L = load()
    n = mu.shape[0]
    dev = mu.device
    rec = torch.empty((n, REC), dtype=torch.float32, device=dev)
    sd = torch.empty((n, SD), dtype=torch.float32, device=dev)
    bbox = torch.empty((n, 4), dtype=torch.int32, device=dev)
    tc = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev) if with_isect_count else None
    p = _prims(mu, scale, quat, opacity, sh)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_project_ut(ctypes.byref(p), n, ctypes.byref(c), ctypes.byref(g), _ptr(rec), _ptr(sd), _ptr(bbox),
                            _ptr(tc), _ptr(cnt), _stream(stream)), "xpr_project_ut")
    return rec, sd, bbox, tc, cnt


def xpr_render_ut_fwd(sd, vals, ranges, cam, cfg, stream=None):
    L = load()
    dev = sd.device
    H, W = int(cam.height), int(cam.width)
    image = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    t_final = torch.empty((H, W), dtype=torch.float32, device=dev)
    n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_ut_fwd(_ptr(sd), sd.shape[0], _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                               _ptr(image), _ptr(t_final), _ptr(n_contrib), _stream(stream)), "xpr_render_ut_fwd")
    return image, t_final, n_contrib


def xpr_render_ut_bwd(sd, vals, ranges, cam, cfg, t_final, n_contrib, d_image, stream=None):
    L = load()
    d_sd = torch.empty((sd.shape[0], SD), dtype=torch.float32, device=sd.device)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_ut_bwd(_ptr(sd), sd.shape[0], _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                               _ptr(t_final), _ptr(n_contrib), _ptr(d_image.contiguous()), _ptr(d_sd),
                               _stream(stream)), "xpr_render_ut_bwd")
    return d_sd


def xpr_project_ut_bwd(mu, scale, quat, opacity, sh, cam, cfg, d_sd, stream=None):
    L = load()
    grads = tuple(torch.empty_like(t) for t in (mu, scale, quat, opacity, sh))
    p = _prims(mu, scale, quat, opacity, sh)
    gp = XprPrimsGrad(*[t.data_ptr() for t in grads])
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_project_ut_bwd(ctypes.byref(p), mu.shape[0], ctypes.byref(c), ctypes.byref(g), _ptr(d_sd),
                                ctypes.byref(gp), _stream(stream)), "xpr_project_ut_bwd")
    return grads


def xpr_project_ut_views(mu, scale, quat, opacity, sh, cams, cfg, stream=None, with_isect_count=True):
    """Returns rec[V*n,12], sd[V*n,16], bbox[V*n,4], tile_count[V*n], isect_count[V*n] (or None)."""
    L = load()
    n, V = mu.shape[0], len(cams)
    dev = mu.device
    rec = torch.empty((V * n, REC), dtype=torch.float32, device=dev)
    sd = torch.empty((V * n, SD), dtype=torch.float32, device=dev)
    bbox = torch.empty((V * n, 4), dtype=torch.int32, device=dev)
    tc = torch.empty(V * n, dtype=torch.int32, device=dev)
    cnt = torch.empty(V * n, dtype=torch.int32, device=dev) if with_isect_count else None
    p = _prims(mu, scale, quat, opacity, sh)
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_project_ut_views(ctypes.byref(p), n, camera_array(cams), V, ctypes.byref(g), _ptr(rec), _ptr(sd),
                                  _ptr(bbox), _ptr(tc), _ptr(cnt), _stream(stream)), "xpr_project_ut_views")
    return rec, sd, bbox, tc, cnt


def xpr_render_ut_fwd_views(sd, n, n_views, vals, ranges, cam, cfg, worklist=None, counter=None, stream=None):
    L = load()
    dev = sd.device
    H, W = int(cam.height), int(cam.width)
    image = torch.empty((n_views, 3, H, W), dtype=torch.float32, device=dev)
    tfin = torch.empty((n_views, H, W), dtype=torch.float32, device=dev)
    ncon = torch.empty((n_views, H, W), dtype=torch.int32, device=dev)
    if worklist is not None and counter is None:
        counter = torch.empty(1, dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_ut_fwd_views(_ptr(sd), n, n_views, _ptr(vals), _ptr(ranges), ctypes.byref(c),
                                     ctypes.byref(g), _ptr(image), _ptr(tfin), _ptr(ncon), _ptr(worklist),
                                     _ptr(counter), _stream(stream)), "xpr_render_ut_fwd_views")
    return image, tfin, ncon


def xpr_render_ut_bwd_views(sd, n, n_views, vals, ranges, cam, cfg, t_final, n_contrib, d_image, worklist=None,
                            counter=None, stream=None):
    L = load()
    dev = sd.device
    d_sd = torch.empty((n * n_views, SD), dtype=torch.float32, device=dev)
    if worklist is not None and counter is None:
        counter = torch.empty(1, dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_ut_bwd_views(_ptr(sd), n, n_views, _ptr(vals), _ptr(ranges), ctypes.byref(c),
                                     ctypes.byref(g), _ptr(t_final), _ptr(n_contrib), _ptr(d_image.contiguous()),
                                     _ptr(d_sd), _ptr(worklist), _ptr(counter), _stream(stream)),
           "xpr_render_ut_bwd_views")
    return d_sd


def xpr_project_ut_bwd_views(mu, scale, quat, opacity, sh, cams, cfg, d_sd, stream=None):
    L = load()
    grads = tuple(torch.empty_like(t) for t in (mu, scale, quat, opacity, sh))
    p = _prims(mu, scale, quat, opacity, sh)
    gp = XprPrimsGrad(*[t.data_ptr() for t in grads])
    g = _as_c(cfg, XprConfig)
    _check(L.xpr_project_ut_bwd_views(ctypes.byref(p), mu.shape[0], camera_array(cams), len(cams), ctypes.byref(g),
                                      _ptr(d_sd), ctypes.byref(gp), _stream(stream)), "xpr_project_ut_bwd_views")
    return grads


# ---------------------------------------------------------------------------------------- LinPrim

def xpr_project_lp(mu, scale, quat, opacity, sh, cam, cfg, stream=None, with_isect_count=True):
    """Returns rec[n,12], sd[n,20], bbox[n,4], tile_count[n], isect_count[n] (or None)."""
    L = load()
    n = mu.shape[0]
    dev = mu.device
    rec = torch.empty((n, REC), dtype=torch.float32, device=dev)
    sd = torch.empty((n, LP_SD), dtype=torch.float32, device=dev)
    bbox = torch.empty((n, 4), dtype=torch.int32, device=dev)
    tc = torch.empty(n, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev) if with_isect_count else None
    p = _prims(mu, scale, quat, opacity, sh)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_project_lp(ctypes.byref(p), n, ctypes.byref(c), ctypes.byref(g), _ptr(rec), _ptr(sd), _ptr(bbox),
                            _ptr(tc), _ptr(cnt), _stream(stream)), "xpr_project_lp")
    return rec, sd, bbox, tc, cnt


def xpr_tile_bin_lp(rec, sd, bbox, tile_count, cam, cfg, capacity=None, workspace=None, stream=None, order=None,
                    isect_count=None):
    """LinPrim binning (tile ids): returns (offsets[n+1], tiles[I] (int32 storage), vals[I], I)."""
    L = load()
    n = rec.shape[0]
    dev = rec.device
    offsets = torch.empty(n + 1, dtype=torch.int32, device=dev)
    need = int(L.xpr_tile_bin_workspace(n))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    cap = int(capacity) if capacity is not None else max(4 * n, 1024)
    tiles = torch.empty(cap, dtype=torch.int32, device=dev)
    vals = torch.empty(cap, dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    for _ in range(2):
        got = c_i64(0)
        s = L.xpr_tile_bin_lp(_ptr(rec), _ptr(sd), _ptr(bbox), _ptr(tile_count), _ptr(isect_count), _ptr(order), n,
                              ctypes.byref(c), ctypes.byref(g), _ptr(offsets), None, _ptr(tiles), _ptr(vals),
                              tiles.numel(), ctypes.byref(got), _ptr(workspace), workspace.numel(), _stream(stream))
        if s == XPR_ERR_CAPACITY and got.value <= 0x7FFFFFFF:
            tiles = torch.empty(got.value, dtype=torch.int32, device=dev)
            vals = torch.empty(got.value, dtype=torch.int32, device=dev)
            continue
        _check(s, "xpr_tile_bin_lp")
        I = int(got.value)
        return offsets, tiles[:I], vals[:I], I
    raise XprError(XPR_ERR_CAPACITY, "xpr_tile_bin_lp", "capacity retry failed")


def xpr_render_lp_fwd(sd, vals, ranges, cam, cfg, stream=None):
    L = load()
    dev = sd.device
    H, W = int(cam.height), int(cam.width)
    image = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    t_final = torch.empty((H, W), dtype=torch.float32, device=dev)
    n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_lp_fwd(_ptr(sd), sd.shape[0], _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                               _ptr(image), _ptr(t_final), _ptr(n_contrib), _stream(stream)), "xpr_render_lp_fwd")
    return image, t_final, n_contrib


def xpr_render_lp_bwd(sd, vals, ranges, cam, cfg, t_final, n_contrib, d_image, stream=None):
    L = load()
    d_sd = torch.empty((sd.shape[0], LP_SD), dtype=torch.float32, device=sd.device)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_lp_bwd(_ptr(sd), sd.shape[0], _ptr(vals), _ptr(ranges), ctypes.byref(c), ctypes.byref(g),
                               _ptr(t_final), _ptr(n_contrib), _ptr(d_image.contiguous()), _ptr(d_sd),
                               _stream(stream)), "xpr_render_lp_bwd")
    return d_sd


def xpr_project_lp_bwd(mu, scale, quat, opacity, sh, cam, cfg, d_sd, stream=None):
    L = load()
    grads = tuple(torch.empty_like(t) for t in (mu, scale, quat, opacity, sh))
    p = _prims(mu, scale, quat, opacity, sh)
    gp = XprPrimsGrad(*[t.data_ptr() for t in grads])
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_project_lp_bwd(ctypes.byref(p), mu.shape[0], ctypes.byref(c), ctypes.byref(g), _ptr(d_sd),
                                ctypes.byref(gp), _stream(stream)), "xpr_project_lp_bwd")
    return grads


# ---------------------------------------------------------------------------------------- rendered features

def _feat_dims(feat, with_depth):
    nfeat = 0 if feat is None else int(feat.shape[1])
    if feat is not None and not (feat.is_cuda and feat.dtype == torch.float32 and feat.is_contiguous()):
        raise ValueError("feat must be a contiguous float32 CUDA tensor [n, n_feat]")
    return nfeat, nfeat + (1 if with_depth else 0)


def xpr_render_fwd_feat(rec, feat, vals, ranges, cam, cfg, with_depth=False, stream=None):
    """Returns (image[3,H,W], features[n_feat + with_depth, H, W], t_final, n_contrib)."""
    L = load()
    dev = rec.device
    nfeat, nf = _feat_dims(feat, with_depth)
    H, W = int(cam.height), int(cam.width)
    image = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    features = torch.empty((nf, H, W), dtype=torch.float32, device=dev)
    t_final = torch.empty((H, W), dtype=torch.float32, device=dev)
    n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_fwd_feat(_ptr(rec), rec.shape[0], _ptr(feat), nfeat, int(bool(with_depth)), _ptr(vals),
                                 _ptr(ranges), ctypes.byref(c), ctypes.byref(g), _ptr(image), _ptr(features),
                                 _ptr(t_final), _ptr(n_contrib), _stream(stream)), "xpr_render_fwd_feat")
    return image, features, t_final, n_contrib


def xpr_render_bwd_feat(rec, feat, vals, ranges, cam, cfg, t_final, n_contrib, d_image, d_features, with_depth=False,
                        stream=None):
    """Returns (d_rec[n,12] with the depth gradient in entry 9, d_feat[n, n_feat] or None)."""
    L = load()
    n = rec.shape[0]
    dev = rec.device
    nfeat, _ = _feat_dims(feat, with_depth)
    d_rec = torch.empty((n, REC), dtype=torch.float32, device=dev)
    d_feat = torch.empty((n, nfeat), dtype=torch.float32, device=dev) if nfeat > 0 else None
    c, g = _as_c(cam, XprCamera), _as_c(cfg, XprConfig)
    _check(L.xpr_render_bwd_feat(_ptr(rec), n, _ptr(feat), nfeat, int(bool(with_depth)), _ptr(vals), _ptr(ranges),
                                 ctypes.byref(c), ctypes.byref(g), _ptr(t_final), _ptr(n_contrib),
                                 _ptr(d_image.contiguous()), _ptr(d_features.contiguous()), _ptr(d_rec), _ptr(d_feat),
                                 _stream(stream)), "xpr_render_bwd_feat")
    return d_rec, d_feat
