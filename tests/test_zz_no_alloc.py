"""xpr_tile_bin_noalloc, the binning entry point for callers that cannot
allocate device memory (its prefix-sum scratch is a static array inside the
library), must give exactly what xpr_tile_bin gives with a caller-provided
workspace, on consecutive calls that reuse the shared static scratch.

This file is collected last on purpose: a failure here leaves every other test
already run."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

pytestmark = pytest.mark.gpu


def _noalloc(rec, bbox, tc, cam, cfg, capacity, order=None):
    L = B.load()
    n = rec.shape[0]
    off = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    keys = torch.full((max(capacity, 1),), -1, dtype=torch.int64, device="cuda")
    vals = torch.full((max(capacity, 1),), -1, dtype=torch.int32, device="cuda")
    got = ctypes.c_int64(0)
    c, g = B.make_camera(cam), B.make_config(cfg)
    s = L.xpr_tile_bin_noalloc(rec.data_ptr(), bbox.data_ptr(), tc.data_ptr(), None,
                               None if order is None else order.data_ptr(), n, ctypes.byref(c), ctypes.byref(g),
                               off.data_ptr(), keys.data_ptr(), None, vals.data_ptr(), capacity, ctypes.byref(got),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return s, off, keys[:got.value], vals[:got.value], got.value


def test_noalloc_matches_tile_bin_on_consecutive_calls():
    cases = [(scenes.uniform_scene(12_345, seed=3), scenes.pinhole(250, 170, 250.0), scenes.RenderConfig()),
             (scenes.uniform_scene(40_000, seed=4, sh_degree=1), scenes.pinhole(320, 240, 320.0),
              scenes.RenderConfig(tile_w=8, tile_h=8, sh_degree=1))]
    for sc, cam, cfg in cases:  # two calls in a row share (and overwrite) the static scratch
        rec, bbox, tc = B.xpr_project(*R.scene_to_device(sc), cam, cfg)
        order = B.xpr_depth_order(rec, tc)
        off_ref, k_ref, v_ref, I = B.xpr_tile_bin(rec, bbox, tc, cam, cfg, order=order)
        s, off, k, v, got = _noalloc(rec, bbox, tc, cam, cfg, I + 100, order)
        assert s == B.XPR_OK, B.load().xpr_last_error()
        assert got == I > 1000
        assert torch.equal(off, off_ref)
        assert torch.equal(k, k_ref)
        assert torch.equal(v, v_ref)


def test_noalloc_capacity_and_size_limit():
    sc, cam, cfg = scenes.small_case()
    rec, bbox, tc = B.xpr_project(*R.scene_to_device(sc), cam, cfg)
    _, _, _, I = B.xpr_tile_bin(rec, bbox, tc, cam, cfg)
    s, _, _, _, got = _noalloc(rec, bbox, tc, cam, cfg, 16)
    assert s == B.XPR_ERR_CAPACITY and got == I
    L = B.load()
    c, g = B.make_camera(cam), B.make_config(cfg)
    n_out = ctypes.c_int64(0)
    # every device pointer is NULL: the size limit is checked first, and if it ever were not, the
    # call would stop at the NULL-pointer check instead of reaching the GPU
    s = L.xpr_tile_bin_noalloc(None, None, None, None, None, (1 << 26) + 1, ctypes.byref(c), ctypes.byref(g), None,
                               None, None, None, 0, ctypes.byref(n_out), None)
    assert s == B.XPR_ERR_INVALID and b"limit" in L.xpr_last_error()
