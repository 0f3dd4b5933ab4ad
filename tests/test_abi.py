"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
entry point declared in include/xpr.h, and rejects invalid arguments on the
host before any device work (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _device_visible() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


# The host-validation checks below pass placeholder addresses (16, 256, ...) that validation rejects
# before any launch.  They run only where no CUDA device is visible, so that a check reordered by a
# later change can never send a placeholder address to a GPU.
host_only = pytest.mark.skipif(_device_visible(), reason="placeholder addresses: run only without a CUDA device")


def _declared():
    txt = open(os.path.join(ROOT, "include", "xpr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(xpr_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_11529_gb300 import binding, build
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2606_11529_gb300 import binding, build
    names = _declared()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(xpr_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the binding knows the signature of each of them
    assert set(names) <= set(binding.SIGNATURES)


def test_library_is_sm103a(lib):
    from paper_2606_11529_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert lib.xpr_version() == 1


def test_status_strings(lib):
    assert lib.xpr_status_string(0) == b"ok"
    assert b"capacity" in lib.xpr_status_string(2)
    assert lib.xpr_status_string(99) == b"unknown status"


def _cam_cfg(**over):
    from paper_2606_11529_gb300 import binding, scenes
    cam = binding.make_camera(scenes.pinhole(64, 48, 64.0))
    cfg = binding.make_config(scenes.RenderConfig())
    for k, v in over.items():
        if hasattr(cam, k):
            setattr(cam, k, v)
        else:
            setattr(cfg, k, v)
    return cam, cfg


@host_only
@pytest.mark.parametrize("over,frag", [
    (dict(tile_w=7), b"tile size"),
    (dict(tile_h=32), b"tile size"),
    (dict(width=0), b"image size"),
    (dict(sh_degree=4), b"sh_degree"),
    (dict(alpha_max=1.0), b"alpha_max"),
    (dict(model=2), b"camera model"),
    (dict(model=1), b"fisheye camera needs the 3DGUT"),
])
def test_invalid_arguments_rejected_on_host(lib, over, frag):
    from paper_2606_11529_gb300 import binding
    cam, cfg = _cam_cfg(**over)
    # NULL device pointers: the camera / config check fails first, and a check reordered after the
    # NULL-pointer check would still stop on the host
    p = binding.XprPrims(None, None, None, None, None)
    s = lib.xpr_project(ctypes.byref(p), 1, ctypes.byref(cam), ctypes.byref(cfg), None, None, None, None, None)
    assert s == binding.XPR_ERR_INVALID
    assert frag in lib.xpr_last_error()


@host_only
def test_null_and_alias_rejected(lib):
    from paper_2606_11529_gb300 import binding
    cam, cfg = _cam_cfg()
    s = lib.xpr_project(None, 5, ctypes.byref(cam), ctypes.byref(cfg), None, None, None, None, None)
    assert s == binding.XPR_ERR_INVALID
    s = lib.xpr_sort(256, 256, 10, 4, 0, 256, 512, 1024, 4096, 1 << 20, None)
    assert s == binding.XPR_ERR_INVALID and b"alias" in lib.xpr_last_error()
    s = lib.xpr_sort(256, 256, 10, 4, 33, 512, 768, 1024, 4096, 1 << 20, None)
    assert s == binding.XPR_ERR_INVALID and b"begin_bit" in lib.xpr_last_error()
    n = ctypes.c_int64(0)
    s = lib.xpr_tile_bin(256, 256, 256, None, None, 10, ctypes.byref(cam), ctypes.byref(cfg), 256, 256, None, 256,
                         -1, ctypes.byref(n), 256, 1 << 20, None)
    assert s == binding.XPR_ERR_INVALID and b"capacity" in lib.xpr_last_error()
    s = lib.xpr_project(None, -1, ctypes.byref(cam), ctypes.byref(cfg), None, None, None, None, None)
    assert s == binding.XPR_ERR_INVALID


def test_workspace_sizes_monotone(lib):
    a = lib.xpr_sort_workspace(1000, 256)
    b = lib.xpr_sort_workspace(100000, 256)
    assert 0 < a < b
    assert lib.xpr_tile_bin_workspace(10) >= 16
    assert lib.xpr_tile_bin_workspace(10_000_000) > lib.xpr_tile_bin_workspace(10)


@host_only
def test_bin_sorted_host_checks(lib):
    from paper_2606_11529_gb300 import binding
    cam, cfg = _cam_cfg()
    ws = lib.xpr_bin_sorted_workspace(100_000, 1, ctypes.byref(cam), ctypes.byref(cfg))
    assert ws > 0
    assert lib.xpr_bin_sorted_workspace(100_000, 3, ctypes.byref(cam), ctypes.byref(cfg)) > ws
    assert lib.xpr_bin_sorted_workspace(1000, 17, ctypes.byref(cam), ctypes.byref(cfg)) == 0
    n = ctypes.c_int64(0)
    s = lib.xpr_bin_sorted(256, 256, 256, 256, 10, 1, ctypes.byref(cam), ctypes.byref(cfg), None, 256, 100,
                           ctypes.byref(n), 256, 1 << 20, None)
    assert s == binding.XPR_ERR_INVALID and b"NULL" in lib.xpr_last_error()
    s = lib.xpr_bin_sorted(256, 256, 256, 256, 10, 1, ctypes.byref(cam), ctypes.byref(cfg), 256, 256, -1,
                           ctypes.byref(n), 256, 1 << 20, None)
    assert s == binding.XPR_ERR_INVALID and b"capacity" in lib.xpr_last_error()
    # every valid camera (width <= 32768, 8x8 tiles: 4096 columns) fits the per-band counters
    widest, cfg8 = _cam_cfg(width=32768, tile_w=8, tile_h=8)
    assert binding.binsort_ok(widest, cfg8) and binding.binsort_ok(cam, cfg)


@host_only
def test_project_color_host_checks(lib):
    from paper_2606_11529_gb300 import binding
    cam, cfg = _cam_cfg()
    cams = (binding.XprCamera * 1)(cam)
    s = lib.xpr_project_color(None, 256, 10, cams, 1, ctypes.byref(cfg), 256, None)
    assert s == binding.XPR_ERR_INVALID and b"NULL" in lib.xpr_last_error()
    s = lib.xpr_project_color(256, 256, 10, cams, 0, ctypes.byref(cfg), 256, None)
    assert s == binding.XPR_ERR_INVALID


@host_only
def test_project_host_checks(lib):
    from paper_2606_11529_gb300 import binding
    cam, cfg = _cam_cfg()
    p = binding.XprPrims(16, 16, 16, 16, None)
    s = lib.xpr_project_host(None, ctypes.byref(p), 10, ctypes.byref(cam), ctypes.byref(cfg), 16, 16, 16, None, None)
    assert s == binding.XPR_ERR_INVALID and b"NULL" in lib.xpr_last_error()
    q = binding.XprPrims(16, 16, 20, 16, None)  # quat not 16-byte aligned
    s = lib.xpr_project_host(ctypes.byref(q), ctypes.byref(p), 10, ctypes.byref(cam), ctypes.byref(cfg), 16, 16, 16,
                             None, None)
    assert s == binding.XPR_ERR_INVALID and b"aligned" in lib.xpr_last_error()
    ut = binding.XprConfig.from_buffer_copy(cfg)
    ut.method = binding.XPR_METHOD_3DGUT
    s = lib.xpr_project_host(ctypes.byref(p), ctypes.byref(p), 10, ctypes.byref(cam), ctypes.byref(ut), 16, 16, 16,
                             None, None)
    assert s == binding.XPR_ERR_INVALID


@host_only
def test_selftest_wait_host_checks(lib):
    from paper_2606_11529_gb300 import binding
    assert lib.xpr_selftest_wait(None, 10, None) == binding.XPR_ERR_INVALID
    for polls in (0, (1 << 20) + 1):
        assert lib.xpr_selftest_wait(16, polls, None) == binding.XPR_ERR_INVALID


@host_only
def test_items_host_checks(lib):
    # offsets that are not the running sums, or too many items, are refused before any device work
    from paper_2606_11529_gb300 import binding, scenes
    cfg = binding.make_config(scenes.RenderConfig())
    cams = [scenes.pinhole(64, 48, 64.0), scenes.pinhole(32, 32, 32.0)]
    lay = binding.ItemLayout([0, 100], [100, 50], cams, cfg)
    assert lay.R == 128 + 64 and lay.S == 4 * 3 + 2 * 2 and lay.pixels == 64 * 48 + 32 * 32
    assert lib.xpr_bin_sorted_items_workspace(lay.carr, lay.arr, 2, ctypes.byref(cfg)) > 0
    lay.arr[1].rec_offset = 100  # not padded to a multiple of 32
    assert lib.xpr_bin_sorted_items_workspace(lay.carr, lay.arr, 2, ctypes.byref(cfg)) == 0
    p = binding.XprPrims(None, None, None, None, None)
    s = lib.xpr_project_items(ctypes.byref(p), lay.carr, lay.arr, 2, ctypes.byref(cfg), None, None, None, None)
    assert s == binding.XPR_ERR_INVALID and b"running sums" in lib.xpr_last_error()
    s = lib.xpr_project_items(ctypes.byref(p), lay.carr, lay.arr, 17, ctypes.byref(cfg), None, None, None, None)
    assert s == binding.XPR_ERR_INVALID
