"""Batched (multi-view) form of the splatting path and its autotuner.

V views of one scene (V <= 16, one image size) run through one launch per
stage: the projection reads each primitive once for all views, binning and
the tile sort see the V x T tiles as one grid, and the render forward and
adjoint run as persistent grids whose blocks take tiles from a list sorted by
descending segment length (the paper's trip-count binning, Sec. 4.3, made
dynamic) through an atomic counter.  Per view the result is exactly the
single-view computation.

The autotuner follows the paper's hyperparameter selection (Sec. 5,
"Hyperparameters"): it renders the target views with each candidate tile size
(8x8, 16x16, the paper's GPU search space) and shared-memory batch depth
(entries staged per batch, the analogue of the paper's batch divisor), takes
the median of repeated timed runs and caches the best setting per (device,
scene, resolution).
"""
from __future__ import annotations

import dataclasses
import math
import statistics

import torch

from . import binding as B

TILE_CANDIDATES = ((8, 8), (16, 16))
BATCH_CANDIDATES = (16, 32, 64, 128, 256)


@dataclasses.dataclass
class ViewsFrame:
    rec: torch.Tensor
    tile_count: torch.Tensor
    n_isect: int
    vals_sorted: torch.Tensor
    ranges: torch.Tensor
    worklist: torch.Tensor | None
    image: torch.Tensor
    t_final: torch.Tensor
    n_contrib: torch.Tensor
    sd: torch.Tensor | None = None  # 3DGUT shader data [V*n, 16]


def _is_ut(cfg) -> bool:
    return int(getattr(cfg, "method", B.XPR_METHOD_3DGS)) == B.XPR_METHOD_3DGUT


class ViewsWorkspace:
    def __init__(self):
        self.last_isect = 0
        self.last_spans = 0
        self.bufs = {}
        # consecutive view chunks a batch of these views is split into (grown when one batch would
        # hold more than 2^31 - 1 pairs, the limit of the 32-bit pair index)
        self.chunks = 1

    def scratch(self, name, nbytes, device):
        t = self.bufs.get(name)
        if t is None or t.numel() < nbytes or t.device != device:
            t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
            self.bufs[name] = t
        return t


def forward_views(mu, scale, quat, opacity, sh, cams, cfg, ws: ViewsWorkspace | None = None, persistent=True,
                  stream=None, fused=False, rows=True) -> ViewsFrame:
    """Projection, depth order, binning and tile sort, work list and render of V views.  The binning
    and tile sort is the rows form (`xpr_bin_rows_views`) where every view's grid has at most 128 x
    128 tiles (``rows``), else the fused counting sort (``fused``) or the key path (tile ids, then
    the tile sort); every form gives the same lists."""
    L = B.load()
    ws = ws or ViewsWorkspace()
    n, V = mu.shape[0], len(cams)
    dev = mu.device
    cam0 = cams[0]
    for c in cams:
        if (c.width, c.height) != (cam0.width, cam0.height):
            raise ValueError("all views of one batch must share the image size")
    ccfg = B.make_config(cfg)
    rows = rows and B.bin_rows_ok(cam0, cfg)
    fused = fused and not rows and B.binsort_ok(cam0, cfg, V)
    ut = _is_ut(cfg)
    sd = None
    # the key path needs the kept-tile counts; the rows binning finds the pair total in its span scan
    want_cnt = not fused and not rows
    if ut:
        rec, sd, bbox, tc, cnt = B.xpr_project_ut_views(mu, scale, quat, opacity, sh, cams, ccfg, stream=stream,
                                                        with_isect_count=want_cnt)
    else:
        rec, bbox, tc, cnt = B.xpr_project_views(mu, scale, quat, opacity, sh, cams, ccfg, stream=stream,
                                                 with_isect_count=want_cnt)
    order = B.xpr_depth_order_views(rec, tc, n, V, workspace=ws.scratch("depth", L.xpr_depth_order_workspace(n * V),
                                                                         dev), stream=stream)
    cap = max(int(ws.last_isect * 1.25) + 1024, 1024)
    Wt, Ht = B.tiles_of(cam0, cfg)
    nt = V * Wt * Ht
    if rows:
        # room for the pairs asked for and a quarter more span slots than last time, so that the
        # binning queues its work ahead of the counts it reads back
        need = B.bin_rows_views_workspace_bytes(n, V, int(ws.last_spans * 1.25) + 1024, cap, cam0, ccfg)
        ranges, vs, I, S, ws.bufs["rows"] = B.xpr_bin_rows_views(rec, bbox, tc, order, n, V, cam0, ccfg,
                                                                 isect_count=cnt, capacity=cap,
                                                                 workspace=ws.scratch("rows", need, dev),
                                                                 stream=stream)
        ws.last_spans = S
    elif fused:
        ranges, vs, I = B.xpr_bin_sorted(rec, bbox, tc, order, n, cam0, ccfg, n_views=V, capacity=cap,
                                         workspace=ws.scratch("binsort", B.bin_sorted_workspace_bytes(
                                             n, V, cam0, ccfg), dev), stream=stream)
    else:
        _, tiles, vals, I = B.xpr_tile_bin_views(rec, bbox, tc, cnt, order, n, V, cam0, ccfg, capacity=cap,
                                                 workspace=ws.scratch("bin", L.xpr_tile_bin_workspace(n * V), dev),
                                                 stream=stream)
        _, vs, ranges = B.xpr_sort_tiles(tiles, vals, nt, workspace=ws.scratch(
            "sort", L.xpr_sort_tiles_workspace(I, nt), dev), stream=stream, want_tiles=False)
    ws.last_isect = I
    wl = B.xpr_tile_worklist(ranges, workspace=ws.scratch("wl", L.xpr_tile_worklist_workspace(nt), dev),
                             stream=stream) if persistent else None
    if ut:
        image, tfin, ncon = B.xpr_render_ut_fwd_views(sd, n, V, vs, ranges, cam0, ccfg, worklist=wl, stream=stream)
    else:
        image, tfin, ncon = B.xpr_render_fwd_views(rec, n, V, vs, ranges, cam0, ccfg, worklist=wl, stream=stream)
    return ViewsFrame(rec, tc, I, vs, ranges, wl, image, tfin, ncon, sd)


class MultiViewSplat(torch.autograd.Function):
    """images[V,3,H,W] = splat of one scene from V cameras; backward sums over views."""

    @staticmethod
    def forward(ctx, mu, scale, quat, opacity, sh, cams, cfg, ws, persistent):
        fr = forward_views(mu, scale, quat, opacity, sh, cams, cfg, ws, persistent)
        shade = fr.sd if fr.sd is not None else fr.rec  # 3DGUT renders from the shader data
        ctx.save_for_backward(mu, scale, quat, opacity, sh, shade, fr.vals_sorted, fr.ranges, fr.t_final,
                              fr.n_contrib, *(() if fr.worklist is None else (fr.worklist,)))
        ctx.cams, ctx.cfg = cams, cfg
        return fr.image

    @staticmethod
    def backward(ctx, d_image):
        saved = ctx.saved_tensors
        mu, scale, quat, opacity, sh, shade, vals, ranges, tfin, ncon = saved[:10]
        wl = saved[10] if len(saved) > 10 else None
        cams, ccfg = ctx.cams, B.make_config(ctx.cfg)
        n, V = mu.shape[0], len(cams)
        if _is_ut(ctx.cfg):
            d_sd = B.xpr_render_ut_bwd_views(shade, n, V, vals, ranges, cams[0], ccfg, tfin, ncon,
                                             d_image.contiguous(), worklist=wl)
            grads = B.xpr_project_ut_bwd_views(mu, scale, quat, opacity, sh, cams, ccfg, d_sd)
        else:
            d_rec = B.xpr_render_bwd_views(shade, n, V, vals, ranges, cams[0], ccfg, tfin, ncon,
                                           d_image.contiguous(), worklist=wl)
            grads = B.xpr_project_bwd_views(mu, scale, quat, opacity, sh, cams, ccfg, d_rec)
        return (*grads, None, None, None, None)


def view_chunks(cams, k):
    """``cams`` split into ``k`` consecutive chunks of near-equal size (none empty)."""
    cams = list(cams)
    k = max(1, min(int(k), len(cams)))
    q, m = divmod(len(cams), k)
    out, o = [], 0
    for i in range(k):
        c = q + (1 if i < m else 0)
        out.append(cams[o:o + c])
        o += c
    return out


def render_views(mu, scale, quat, opacity, sh, cams, cfg, ws: ViewsWorkspace | None = None, persistent=True):
    """Differentiable render of V views in one launch per stage: returns images [V, 3, H, W].

    When one batch of the V views would hold more than 2^31 - 1 (tile, primitive) pairs (the pair
    index is 32-bit), the views run as consecutive chunks, each one batch (the chunk count is
    doubled until every chunk fits and kept in ``ws`` for the next call); a single view above the
    limit raises."""
    ws = ws or ViewsWorkspace()
    cams = list(cams)
    while True:
        parts = view_chunks(cams, ws.chunks)
        try:
            imgs = [MultiViewSplat.apply(mu, scale, quat, opacity, sh, part, cfg, ws, persistent) for part in parts]
        except B.XprError as e:
            if e.status != B.XPR_ERR_CAPACITY or len(parts) >= len(cams):
                raise
            ws.chunks = min(2 * len(parts), len(cams))
            ws.last_isect = 0
            continue
        return imgs[0] if len(imgs) == 1 else torch.cat(imgs)


# ------------------------------------------------------------------------------------------- autotuner

_CACHE: dict = {}


def _time_ms(fn, reps):
    times = []
    for _ in range(reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
    return statistics.median(times)


def autotune(params, cams, cfg, scene_id="scene", backward=True, reps=5, tiles=TILE_CANDIDATES,
             batches=BATCH_CANDIDATES, chunks=None):
    """Returns (best_cfg, table) where table maps (tile_w, tile_h, batch) -> median ms of one batched
    forward (+ backward) over all `cams` (a candidate whose batch exceeds 2^31 - 1 pairs runs the
    views in chunks, as `render_views` does; inf only where a single view exceeds it).  ``chunks``
    (a dict, optional) receives the chunk count each candidate ran with.  Results are cached per
    (device, scene_id, resolution)."""
    key = (torch.cuda.get_device_name(), scene_id, cams[0].width, cams[0].height, len(cams), backward,
           int(getattr(cfg, "method", 0)))
    if key in _CACHE:
        if chunks is not None:
            chunks.update(_CACHE[key][2])
        return _CACHE[key][:2]
    table, nchunks = {}, {}
    d_img = None
    for tw, th in tiles:
        for bd in batches:
            c = dataclasses.replace(cfg, tile_w=tw, tile_h=th, batch_depth=bd)
            ws = ViewsWorkspace()
            P = [p.detach().requires_grad_(backward) for p in params]

            def run():
                img = render_views(*P, cams, c, ws)
                if backward:
                    img.backward(d_img if d_img is not None else torch.ones_like(img))

            try:
                run()  # warm-up (and capacity sizing)
            except B.XprError as e:
                if e.status != B.XPR_ERR_CAPACITY:
                    raise
                table[(tw, th, bd)] = math.inf  # a single view above 2^31 - 1 pairs: this tile size does not fit
                continue
            table[(tw, th, bd)] = _time_ms(run, reps)
            nchunks[(tw, th, bd)] = ws.chunks
    best = min(table, key=table.get)
    out = (dataclasses.replace(cfg, tile_w=best[0], tile_h=best[1], batch_depth=best[2]), table, nchunks)
    _CACHE[key] = out
    if chunks is not None:
        chunks.update(nchunks)
    return out[:2]


# ------------------------------------------------------------------------------------------- scenes

@dataclasses.dataclass
class ItemsFrame:
    layout: "B.ItemLayout"
    rec: torch.Tensor
    tile_count: torch.Tensor
    n_isect: int
    vals_sorted: torch.Tensor
    ranges: torch.Tensor
    worklist: torch.Tensor | None
    image: torch.Tensor      # flat: item k's planes [3, H, W] at 3 pix_offset[k]
    t_final: torch.Tensor    # flat: item k's [H, W] at pix_offset[k]
    n_contrib: torch.Tensor

    def images(self):
        return self.layout.images(self.image)


class SceneSet:
    """Scenes of any size held as one set of concatenated parameter arrays (the batch's primitive
    space): scene s owns primitives [offsets[s], offsets[s] + counts[s])."""

    def __init__(self, scenes):
        scenes = [tuple(t.contiguous() for t in s) for s in scenes]
        self.counts = [int(s[0].shape[0]) for s in scenes]
        self.offsets = [0]
        for c in self.counts[:-1]:
            self.offsets.append(self.offsets[-1] + c)
        self.params = [torch.cat([s[j] for s in scenes]) for j in range(5)]

    def views(self):
        """Per-scene (mu, scale, quat, opacity, sh) tensors: contiguous slices of the set."""
        return [tuple(t[o:o + n] for t in self.params) for o, n in zip(self.offsets, self.counts)]

    def layout(self, scene_of_item, cams, cfg) -> "B.ItemLayout":
        return B.ItemLayout([self.offsets[s] for s in scene_of_item], [self.counts[s] for s in scene_of_item], cams, cfg)


def forward_items(mu, scale, quat, opacity, sh, layout, cfg, ws: ViewsWorkspace | None = None, persistent=True,
                  stream=None, rows=True) -> ItemsFrame:
    """K (scene, camera) items of uneven scene and image sizes through one launch per stage (3DGS):
    projection, depth order, binning and tile sort (by rows where every item's grid has at most 128
    x 128 tiles and ``rows``, else the fused counting sort: the same lists), work list over every
    item's tiles, render."""
    L = B.load()
    ws = ws or ViewsWorkspace()
    dev = mu.device
    ccfg = B.make_config(cfg)
    rec, bbox, tc = B.xpr_project_items(mu, scale, quat, opacity, sh, layout, ccfg, stream=stream)
    order = B.xpr_depth_order_items(rec, tc, layout, workspace=ws.scratch("depth", L.xpr_depth_order_workspace(
        layout.R), dev), stream=stream)
    cap = max(int(ws.last_isect * 1.25) + 1024, 1024)
    if rows and B.bin_rows_items_ok(layout, cfg):
        need = B.bin_rows_items_workspace_bytes(layout, int(ws.last_spans * 1.25) + 1024, cap, ccfg)
        ranges, vs, I, S, ws.bufs["rows"] = B.xpr_bin_rows_items(rec, bbox, tc, order, layout, ccfg, capacity=cap,
                                                                 workspace=ws.scratch("rows", need, dev),
                                                                 stream=stream)
        ws.last_spans = S
    else:
        ranges, vs, I = B.xpr_bin_sorted_items(rec, bbox, tc, order, layout, ccfg, capacity=cap,
                                               workspace=ws.scratch("binsort", B.bin_sorted_items_workspace_bytes(
                                                   layout, ccfg), dev), stream=stream)
    ws.last_isect = I
    wl = B.xpr_tile_worklist(ranges, workspace=ws.scratch("wl", L.xpr_tile_worklist_workspace(layout.S), dev),
                             stream=stream) if persistent else None
    image, tfin, ncon = B.xpr_render_fwd_items(rec, vs, ranges, layout, ccfg, worklist=wl, stream=stream)
    return ItemsFrame(layout, rec, tc, I, vs, ranges, wl, image, tfin, ncon)


class MultiSceneSplat(torch.autograd.Function):
    """Flat images of K (scene, camera) items; backward sums each scene primitive's gradient over
    the items that see it."""

    @staticmethod
    def forward(ctx, mu, scale, quat, opacity, sh, layout, cfg, ws, persistent):
        fr = forward_items(mu, scale, quat, opacity, sh, layout, cfg, ws, persistent)
        ctx.save_for_backward(mu, scale, quat, opacity, sh, fr.rec, fr.vals_sorted, fr.ranges, fr.t_final,
                              fr.n_contrib, *(() if fr.worklist is None else (fr.worklist,)))
        ctx.layout, ctx.cfg = layout, cfg
        return fr.image

    @staticmethod
    def backward(ctx, d_image):
        saved = ctx.saved_tensors
        mu, scale, quat, opacity, sh, rec, vals, ranges, tfin, ncon = saved[:10]
        wl = saved[10] if len(saved) > 10 else None
        ccfg = B.make_config(ctx.cfg)
        d_rec = B.xpr_render_bwd_items(rec, vals, ranges, ctx.layout, ccfg, tfin, ncon, d_image.contiguous(),
                                       worklist=wl)
        grads = B.xpr_project_bwd_items(mu, scale, quat, opacity, sh, ctx.layout, ccfg, d_rec)
        return (*grads, None, None, None, None)


def render_items(mu, scale, quat, opacity, sh, layout, cfg, ws: ViewsWorkspace | None = None, persistent=True):
    """Differentiable render of a multi-scene batch: returns the per-item images [3, H_k, W_k]
    (views of one flat output)."""
    flat = MultiSceneSplat.apply(mu, scale, quat, opacity, sh, layout, cfg, ws or ViewsWorkspace(), persistent)
    return layout.images(flat)
