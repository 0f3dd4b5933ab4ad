"""Helpers shared by the GPU tests (not collected by pytest)."""
import numpy as np
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

IMG_TOL = 1e-4    # max abs image error outside the ambiguity band
GRAD_TOL = 1e-3   # per-tensor relative L2 error of gradients
BAND = 1e-5       # relative margin of a gate decision that counts as ambiguous


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
