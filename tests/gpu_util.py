"""Helpers shared by the GPU tests (not collected by pytest)."""
import numpy as np
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from oracle.oracle import BAND_E2E, BAND_STAGE  # noqa: F401  (3DGS ambiguity-band models)

IMG_TOL = 1e-4    # max abs image error outside the ambiguity band
GRAD_TOL = 1e-3   # per-tensor relative L2 error of gradients
BAND = 1e-5       # 3DGUT / LinPrim: relative margin of a gate decision that counts as ambiguous


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def dev_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).to("cuda")


def dev_i64(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to("cuda")


def host_u64(t):
    return t.cpu().numpy().view(np.uint64)


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def rel_err(g, ref):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(g - ref) / (den if den > 0 else 1.0)


def oracle_lists(oracle, rec32, bbox, cam, cfg):
    """Oracle bin (exact FP32 decisions) + sort of float32 records."""
    Wt, Ht = oracle.tiles_of(cam, cfg)
    counts, keys, vals = oracle.bin_pairs(rec32, bbox, cam, cfg, exact32=True)
    sk, sv, ranges = oracle.sort_pairs(keys, vals, Wt * Ht)
    return counts, keys, vals, sk, sv, ranges


def near_integer_bbox(pre, tol=1e-4):
    return np.any(np.abs(pre - np.round(pre)) < tol, axis=1)


def check_band(got, ref, mask=None, max_frac=1e-4, tol=IMG_TOL, what=""):
    """Image parity against an oracle result with an ambiguity band.

    got, ref["image"] (or ref["color"]): [3, ...] / [..., 3] arrays of the same pixels; ref["band"]
    marks pixels where a gate decision lies within its float32 uncertainty, ref["jump"] bounds how
    far those decisions can move the colour.  Asserts: the band covers at most ``max_frac`` of the
    (masked) pixels; outside it every channel is within ``tol``; inside it within jump + tol.
    Returns the boolean mask of unambiguous pixels."""
    img = ref["image"] if "image" in ref else ref["color"].T
    got = np.asarray(got, np.float64)
    if got.shape != img.shape:
        got = got.T
    band = ref["band"]
    m = np.ones(band.shape, bool) if mask is None else mask
    frac = float(band[m].mean()) if m.any() else 0.0
    print(f"{what} ambiguity band: {int(band[m].sum())} of {int(m.sum())} pixels ({frac:.2e})")
    assert frac <= max_frac, f"{what}: band fraction {frac:.2e} > {max_frac:.1e}"
    err = np.abs(got - img).max(0)
    ok = m & ~band
    if ok.any():
        assert err[ok].max() <= tol, f"{what}: max error {err[ok].max():.3e} outside the band"
    bad = m & band
    if bad.any():
        excess = err[bad] - (ref["jump"][bad] + tol)
        assert excess.max() <= 0, f"{what}: band pixel beyond its jump bound by {excess.max():.3e}"
    return ok


def tile_lists_row_major(vals, ranges):
    """The sorted record indices re-gathered tile by tile in row-major tile order, and the list
    lengths (layout-independent: the ranges locate each tile's segment)."""
    import torch
    v = torch.as_tensor(vals).cuda().to(torch.int64)
    r = torch.as_tensor(ranges).cuda().to(torch.int64)
    lens = r[:, 1] - r[:, 0]
    total = int(lens.sum().item())
    starts_out = torch.cumsum(lens, 0) - lens
    idx = torch.repeat_interleave(r[:, 0] - starts_out, lens) + torch.arange(total, device="cuda")
    return v[idx], lens


def assert_same_tile_lists(v_a, r_a, v_b, r_b):
    """Every tile's list (record indices in order) is the same in both (vals, ranges) pairs."""
    import torch
    a, la = tile_lists_row_major(v_a, r_a)
    b, lb = tile_lists_row_major(v_b, r_b)
    assert torch.equal(la, lb), "tile list lengths differ"
    assert torch.equal(a, b), "tile lists differ"
