"""Time the FP64 oracle, as it stands, on a bounded sample of a workload.

TEST INFRASTRUCTURE ONLY (used by the benchmark's CPU-baseline leg and its
reference arm).  One forward+backward of the tiled oracle pipeline is
estimated from:
  - projection of a fraction ``prim_frac`` of the primitives (scaled up linearly),
  - binning (FP64 cull) and sorting of those primitives' pairs (scaled up linearly),
  - per-tile compositing and its adjoint on ``n_tiles`` tiles chosen at random
    from the full-scene tile lists (scaled by total tiles / sampled tiles),
  - the projection adjoint on the sampled primitives (scaled up linearly).
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import oracle as O


# The full scene's per-tile lists, built once per (scene, camera, config) and reused by every
# estimate on them: only the compositing of the sampled tiles is timed, the lists are set-up.
_lists: dict = {}


def _full_lists(scene, cam, cfg, T: int):
    if not (_lists.get("scene") is scene and _lists.get("cam") is cam and _lists.get("cfg") is cfg):
        _lists.clear()
        full = O.project_scene(scene, cam, cfg)
        _, k2, v2 = O.bin_pairs(full["rec"], full["bbox"], cam, cfg, exact32=False)
        _, v2, r2 = O.sort_pairs(k2, v2, T)
        _lists.update(scene=scene, cam=cam, cfg=cfg, rec=full["rec"], vals=v2, ranges=r2)
    return _lists["rec"], _lists["vals"], _lists["ranges"]


def release_lists() -> None:
    """Drops the cached full-scene lists (several hundred MB of host memory on a 1M scene)."""
    _lists.clear()


def estimate_fwd_bwd_seconds(scene, cam, cfg, prim_frac: float = 0.1, n_tiles: int = 48, seed: int = 0):
    rng = np.random.default_rng(seed)
    n = scene.n
    m = max(1, int(round(n * prim_frac)))
    sub = np.sort(rng.choice(n, size=m, replace=False))
    ss = scene.subset(sub)
    Wt, Ht = O.tiles_of(cam, cfg)
    T = Wt * Ht

    t0 = time.perf_counter()
    pr = O.project_scene(ss, cam, cfg)
    t_proj = time.perf_counter() - t0

    t0 = time.perf_counter()
    _, keys, vals = O.bin_pairs(pr["rec"], pr["bbox"], cam, cfg, exact32=False)
    keys, vals, ranges = O.sort_pairs(keys, vals, T)
    t_bin = time.perf_counter() - t0

    # compositing on sampled tiles of the FULL scene: the sampled primitives' lists hold a fraction
    # prim_frac of each tile's entries, so the walk is shorter than the real one; to stay honest the
    # per-tile work is measured on the full-length lists of the sampled tiles.
    tiles = rng.choice(T, size=min(n_tiles, T), replace=False)
    rec_c, v2, r_all = _full_lists(scene, cam, cfg, T)
    r2 = np.zeros_like(r_all)
    r2[tiles] = r_all[tiles]
    t0 = time.perf_counter()
    fw = O.render_tiles(rec_c, v2, r2, cam, cfg)
    w = np.ones((3, cam.height, cam.width))
    d_rec = O.render_bwd_tiles(rec_c, v2, r2, cam, cfg, w)
    t_render = time.perf_counter() - t0
    del fw

    t0 = time.perf_counter()
    d_sub = np.zeros((m, 12))
    d_sub[:, :9] = 1e-3
    O.project_bwd(*ss.arrays(), cam, cfg, d_sub)
    t_pbwd = time.perf_counter() - t0

    est = (t_proj + t_bin + t_pbwd) * (n / m) + t_render * (T / len(tiles))
    measured = t_proj + t_bin + t_render + t_pbwd
    desc = (f"oracle (FP64, C) on a bounded sample: project+bin+sort+project-adjoint of {m} of {n} primitives "
            f"(x{n / m:.1f}), per-tile compositing fwd+adjoint on {len(tiles)} of {T} tiles (x{T / len(tiles):.1f}); "
            f"{measured:.1f} s measured, "
            f"{'the whole workload' if m == n and len(tiles) == T else 'extrapolated to one full fwd+bwd'}; "
            f"projection and forward compositing "
            f"use OpenMP, binning/sort/adjoint compositing are serial")
    return est, measured, desc


def threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)
