"""Tile-splatting path on the GPU (3DGS, and 3DGUT when ``cfg.method == 1``): the plain
per-stage calls and the ``torch.autograd.Function`` that chains them.

Forward  = xpr_project -> xpr_depth_order -> xpr_bin_sorted -> xpr_render_fwd
           (or xpr_tile_bin -> xpr_sort_tiles in place of xpr_bin_sorted)
Backward = xpr_render_bwd (compositing adjoint, then projection adjoint)
3DGUT    = xpr_project_ut / xpr_render_ut_fwd / xpr_render_ut_bwd + xpr_project_ut_bwd around the
           same depth order, binning (ray-offset cull) and sort
LinPrim  = xpr_project_lp / xpr_tile_bin_lp (chord-bound cull) / xpr_render_lp_fwd / xpr_render_lp_bwd
           + xpr_project_lp_bwd around the same depth order and sort (``cfg.method == 2``)

The Function takes activated parameters (mu, scale, quat, opacity, sh), as in
the paper's PrimitiveParams, and returns the image [3, H, W].  Gradients are
produced for all five parameter tensors.  Buffers are allocated by PyTorch's
caching allocator; the intersection buffers start at the size seen on the
previous call with the same ``Workspace`` so the capacity retry of
xpr_tile_bin is rare.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B


class Workspace:
    """Per-stream state of the forward: the last intersection count (initial capacity guess for
    xpr_tile_bin) and the transient scratch of xpr_tile_bin / xpr_sort.  Per-frame outputs are
    fresh tensors from PyTorch's caching allocator, so a Frame stays valid after later calls."""

    def __init__(self, fused: bool = False, rows: bool = True, rows_counts: bool = False):
        self.last_isect = 0
        self.last_spans = 0
        self.bufs = {}
        self.fused = fused  # xpr_bin_sorted (True) or xpr_tile_bin + xpr_sort_tiles (False)
        # with fused False: xpr_bin_rows where the grid allows it (True), else the key path
        self.rows = rows
        # binning by rows: the projection also counts each primitive's kept tiles (True: the pair
        # total is read back with the span total), or the pair total comes from the span scan (False,
        # the default: the count costs the projection 35 us on the 1M / 1080p headline, the second
        # read-back the binning 7 us)
        self.rows_counts = rows_counts
        self.sh_events = None  # set by a caller whose SH copy is still in flight (consumed by one forward)
        # set by a caller whose inputs are still in pinned host memory: (host (mu, scale, quat,
        # opacity, sh), copy stream); the forward brings them over itself (consumed by one forward)
        self.host_inputs = None

    def take_sh_events(self):
        ev, self.sh_events = self.sh_events, None
        return ev

    def take_host_inputs(self):
        h, self.host_inputs = self.host_inputs, None
        return h

    def scratch(self, name, nbytes, device):
        t = self.bufs.get(name)
        if t is None or t.numel() < nbytes or t.device != device:
            t = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
            self.bufs[name] = t
        return t


class StageTimers:
    """Optional CUDA-event brackets around each C-ABI call (recorded on the launching stream)."""

    def __init__(self):
        self.events = {}

    def start(self, name, stream=None):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        self.events.setdefault(name, []).append((e0, e1))

    def stop(self, name, stream=None):
        self.events[name][-1][1].record(stream)

    def mean_ms(self):
        torch.cuda.synchronize()
        return {k: sum(a.elapsed_time(b) for a, b in v) / len(v) for k, v in self.events.items()}

    def reset(self):
        self.events = {}


class _NoTimers:
    def start(self, name, stream=None):
        pass

    def stop(self, name, stream=None):
        pass


_NO_TIMERS = _NoTimers()


@dataclass
class Frame:
    """Everything the forward produces (kept for the backward and for tests).  On the key path the
    pairs are emitted in depth order, so `tiles` (u32 tile ids, int32 storage) sorted stably by
    tile give the (tile, depth) order of Sec. 4.2; the fused path and the binning by rows produce
    `vals_sorted` and `ranges` directly and leave offsets, tiles, vals and tiles_sorted as None (and
    isect_count, unless the workspace asks the rows path for the kept counts)."""
    rec: torch.Tensor
    bbox: torch.Tensor
    tile_count: torch.Tensor
    isect_count: torch.Tensor
    order: torch.Tensor
    offsets: torch.Tensor
    tiles: torch.Tensor
    vals: torch.Tensor
    n_isect: int
    tiles_sorted: torch.Tensor
    vals_sorted: torch.Tensor
    ranges: torch.Tensor
    image: torch.Tensor
    t_final: torch.Tensor
    n_contrib: torch.Tensor
    sd: torch.Tensor | None = None  # 3DGUT shader data [n, 16]


def method_of(cfg) -> int:
    return int(getattr(cfg, "method", B.XPR_METHOD_3DGS))


def is_ut(cfg) -> bool:
    return method_of(cfg) == B.XPR_METHOD_3DGUT


def is_lp(cfg) -> bool:
    return method_of(cfg) == B.XPR_METHOD_LINPRIM


def forward_frame(mu, scale, quat, opacity, sh, cam, cfg, ws: Workspace | None = None, stream=None,
                  timers=None, fused: bool = False, keep_sorted_tiles: bool = False, sh_events=None,
                  render: bool = True, host_inputs=None) -> Frame:
    """The forward stages, each one C-ABI call: project, depth order, then the binning and tile sort:
    by tile rows (xpr_bin_rows, the default where the grid has at most 128 x 128 tiles), the key
    path (xpr_tile_bin emitting u32 tile ids in depth order + xpr_sort_tiles: larger grids, LinPrim,
    or keep_sorted_tiles) or the fused bin + sort (xpr_bin_sorted); then render.  All give the same
    sorted lists bit for bit.
    sh_events: events of an SH copy still in flight; then the projection runs without colours,
    and the stream waits for the events just before xpr_project_color fills them in.
    host_inputs: (pinned host (mu, scale, quat, opacity, sh), copy stream): the parameters are brought
    into the given device tensors here.  3DGS: the projection reads the geometry over the host link
    and writes its device copy in the same pass (xpr_project_host); then the SH coefficients are
    copied on the copy stream under the depth order, binning and sort, and the colours are filled
    in after the sort (as with sh_events).  3DGUT / LinPrim: everything is copied first."""
    L = B.load()
    tm = timers or _NO_TIMERS
    ccam, ccfg = B.make_camera(cam), B.make_config(cfg)
    fused = fused and B.binsort_ok(cam, cfg)
    n = mu.shape[0]
    dev = mu.device
    ws = ws or Workspace()
    ut, lp = is_ut(cfg), is_lp(cfg)
    fused = fused and not lp  # LinPrim is binned by xpr_tile_bin_lp
    rows = not fused and not keep_sorted_tiles and getattr(ws, "rows", True) and B.bin_rows_ok(cam, cfg)
    want_cnt = not fused and (not rows or getattr(ws, "rows_counts", True))
    sd = None
    deferred = sh_events is not None and not (ut or lp)
    from_host = host_inputs is not None and not (ut or lp)
    if host_inputs is not None and not from_host:  # these projections need every input first
        _wait_events(stream, _copy_on(host_inputs[1], (mu, scale, quat, opacity, sh), host_inputs[0], stream))
    if from_host:
        deferred = True
    if sh_events is not None and (ut or lp):  # these projections take the colours in the same pass
        _wait_events(stream, sh_events)
    tm.start("project", stream)
    if ut:
        rec, sd, bbox, tc, cnt = B.xpr_project_ut(mu, scale, quat, opacity, sh, ccam, ccfg, stream=stream,
                                                  with_isect_count=want_cnt)
    elif lp:
        rec, sd, bbox, tc, cnt = B.xpr_project_lp(mu, scale, quat, opacity, sh, ccam, ccfg, stream=stream)
    elif from_host:
        hs, cs = host_inputs
        out = B.xpr_project_host(hs[:4], (mu, scale, quat, opacity, None), ccam, ccfg, stream=stream,
                                 with_isect_count=want_cnt)
        rec, bbox, tc = out[:3]
        cnt = out[3] if len(out) > 3 else None
        sh_events = _copy_on(cs, (sh,), hs[4:], stream)  # after the projection: the host link is free
    else:
        out = B.xpr_project(mu, scale, quat, opacity, None if deferred else sh, ccam, ccfg, stream=stream,
                            with_isect_count=want_cnt)
        rec, bbox, tc = out[:3]
        cnt = out[3] if len(out) > 3 else None
    tm.stop("project", stream)
    # emit intersections in (depth, index) order so that only tile ids remain to be ordered
    tm.start("depth_order", stream)
    order = B.xpr_depth_order(rec, tc, workspace=ws.scratch("depth", L.xpr_depth_order_workspace(n), dev),
                              stream=stream)
    tm.stop("depth_order", stream)
    cap = max(int(ws.last_isect * 1.25) + 1024, 1024)
    Wt, Ht = B.tiles_of(cam, cfg)
    nt = Wt * Ht
    if fused:
        bs_ws = ws.scratch("binsort", B.bin_sorted_workspace_bytes(n, 1, ccam, ccfg), dev)
        tm.start("bin_sort", stream)
        ranges, vs, I = B.xpr_bin_sorted(rec, bbox, tc, order, n, ccam, ccfg, capacity=cap, workspace=bs_ws,
                                         stream=stream)
        tm.stop("bin_sort", stream)
        offsets = tiles = vals = ks = None
    elif rows:
        need = B.bin_rows_workspace_bytes(n, int(ws.last_spans * 1.25) + 1024, cap, ccam, ccfg)
        rows_ws = ws.scratch("rows", need, dev)
        tm.start("bin_sort", stream)
        ranges, vs, I, S, used = B.xpr_bin_rows(rec, bbox, tc, order, n, ccam, ccfg, isect_count=cnt, capacity=cap,
                                                workspace=rows_ws, stream=stream)
        tm.stop("bin_sort", stream)
        ws.bufs["rows"] = used
        ws.last_spans = S
        offsets = tiles = vals = ks = None
    else:
        bin_ws = ws.scratch("bin", L.xpr_tile_bin_workspace(n), dev)
        tm.start("tile_bin", stream)
        if lp:
            offsets, tiles, vals, I = B.xpr_tile_bin_lp(rec, sd, bbox, tc, ccam, ccfg, capacity=cap, workspace=bin_ws,
                                                        stream=stream, order=order, isect_count=cnt)
        else:
            offsets, tiles, vals, I = B.xpr_tile_bin(rec, bbox, tc, ccam, ccfg, capacity=cap, workspace=bin_ws,
                                                     stream=stream, order=order, isect_count=cnt, tile_ids=True)
        tm.stop("tile_bin", stream)
        sort_ws = ws.scratch("sort", L.xpr_sort_tiles_workspace(I, nt), dev)
        tm.start("sort", stream)
        ks, vs, ranges = B.xpr_sort_tiles(tiles, vals, nt, workspace=sort_ws, stream=stream,
                                          want_tiles=keep_sorted_tiles)
        tm.stop("sort", stream)
    ws.last_isect = I
    if deferred:
        _wait_events(stream, sh_events)
        tm.start("color", stream)
        B.xpr_project_color(mu, sh, rec, ccam, ccfg, stream=stream)
        tm.stop("color", stream)
    if not render:  # the caller composites the lists itself (rendered features)
        return Frame(rec, bbox, tc, cnt, order, offsets, tiles, vals, I, ks, vs, ranges, None, None, None, sd)
    tm.start("render_fwd", stream)
    if ut:
        image, t_final, n_contrib = B.xpr_render_ut_fwd(sd, vs, ranges, ccam, ccfg, stream=stream)
    elif lp:
        image, t_final, n_contrib = B.xpr_render_lp_fwd(sd, vs, ranges, ccam, ccfg, stream=stream)
    else:
        image, t_final, n_contrib = B.xpr_render_fwd(rec, vs, ranges, ccam, ccfg, stream=stream)
    tm.stop("render_fwd", stream)
    return Frame(rec, bbox, tc, cnt, order, offsets, tiles, vals, I, ks, vs, ranges, image, t_final, n_contrib, sd)


def _copy_on(copy_stream, dst, src, stream):
    """Copies src (host) into dst (device) on copy_stream after the work enqueued on `stream` (None:
    the current stream) so far; returns the event of the copies."""
    cur = stream if stream is not None else torch.cuda.current_stream()
    copy_stream.wait_stream(cur)
    with torch.cuda.stream(copy_stream), torch.no_grad():
        for d, h in zip(dst, src):
            d.copy_(h, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(copy_stream)
    return ev


def _wait_events(stream, events):
    cur = stream if stream is not None else torch.cuda.current_stream()
    for e in (events if isinstance(events, (list, tuple)) else [events]):
        cur.wait_event(e)


class SplatFunction(torch.autograd.Function):
    """image = splat(mu, scale, quat, opacity, sh); backward gives all five gradients."""

    @staticmethod
    def forward(ctx, mu, scale, quat, opacity, sh, cam, cfg, ws, timers):
        fr = forward_frame(mu, scale, quat, opacity, sh, cam, cfg, ws, timers=timers, fused=ws.fused,
                           sh_events=ws.take_sh_events(), host_inputs=ws.take_host_inputs())
        # 3DGUT and LinPrim render from the shader data, 3DGS from the records
        shade = fr.sd if fr.sd is not None else fr.rec
        ctx.save_for_backward(mu, scale, quat, opacity, sh, shade, fr.vals_sorted, fr.ranges, fr.t_final,
                              fr.n_contrib)
        ctx.cam, ctx.cfg, ctx.timers = cam, cfg, timers
        return fr.image

    @staticmethod
    def backward(ctx, d_image):
        mu, scale, quat, opacity, sh, shade, vals, ranges, t_final, n_contrib = ctx.saved_tensors
        tm = ctx.timers or _NO_TIMERS
        ccam, ccfg = B.make_camera(ctx.cam), B.make_config(ctx.cfg)
        ut, lp = is_ut(ctx.cfg), is_lp(ctx.cfg)
        tm.start("render_bwd")
        if ut:
            d_shade = B.xpr_render_ut_bwd(shade, vals, ranges, ccam, ccfg, t_final, n_contrib, d_image.contiguous())
        elif lp:
            d_shade = B.xpr_render_lp_bwd(shade, vals, ranges, ccam, ccfg, t_final, n_contrib, d_image.contiguous())
        else:
            d_shade = B.xpr_render_bwd(shade, vals, ranges, ccam, ccfg, t_final, n_contrib, d_image.contiguous())
        tm.stop("render_bwd")
        tm.start("project_bwd")
        if ut:
            grads = B.xpr_project_ut_bwd(mu, scale, quat, opacity, sh, ccam, ccfg, d_shade)
        elif lp:
            grads = B.xpr_project_lp_bwd(mu, scale, quat, opacity, sh, ccam, ccfg, d_shade)
        else:
            grads = B.xpr_project_bwd(mu, scale, quat, opacity, sh, ccam, ccfg, d_shade)
        tm.stop("project_bwd")
        return (*grads, None, None, None, None)


class FeatSplatFunction(torch.autograd.Function):
    """(image, features) = splat with rendered feature channels (3DGS): feat[n, F] per-primitive rows
    (or None) and, with with_depth, the expected-depth channel; backward gives the five parameter
    gradients and d feat."""

    @staticmethod
    def forward(ctx, mu, scale, quat, opacity, sh, feat, cam, cfg, with_depth, ws):
        fr = forward_frame(mu, scale, quat, opacity, sh, cam, cfg, ws, render=False)
        image, features, t_final, n_contrib = B.xpr_render_fwd_feat(fr.rec, feat, fr.vals_sorted, fr.ranges,
                                                                    B.make_camera(cam), B.make_config(cfg),
                                                                    with_depth=with_depth)
        ctx.has_feat = feat is not None
        ctx.save_for_backward(mu, scale, quat, opacity, sh, *( (feat,) if feat is not None else ()), fr.rec,
                              fr.vals_sorted, fr.ranges, t_final, n_contrib)
        ctx.cam, ctx.cfg, ctx.with_depth = cam, cfg, with_depth
        return image, features

    @staticmethod
    def backward(ctx, d_image, d_features):
        saved = list(ctx.saved_tensors)
        mu, scale, quat, opacity, sh = saved[:5]
        feat = saved[5] if ctx.has_feat else None
        rec, vals, ranges, t_final, n_contrib = saved[-5:]
        ccam, ccfg = B.make_camera(ctx.cam), B.make_config(ctx.cfg)
        if d_image is None:
            d_image = torch.zeros((3, ctx.cam.height, ctx.cam.width), dtype=torch.float32, device=mu.device)
        nf = (0 if feat is None else feat.shape[1]) + int(bool(ctx.with_depth))
        if d_features is None:
            d_features = torch.zeros((nf, ctx.cam.height, ctx.cam.width), dtype=torch.float32, device=mu.device)
        d_rec, d_feat = B.xpr_render_bwd_feat(rec, feat, vals, ranges, ccam, ccfg, t_final, n_contrib,
                                              d_image.contiguous(), d_features.contiguous(),
                                              with_depth=ctx.with_depth)
        grads = B.xpr_project_bwd(mu, scale, quat, opacity, sh, ccam, ccfg, d_rec)
        return (*grads, d_feat, None, None, None, None)


def render_features(mu, scale, quat, opacity, sh, feat, cam, cfg, with_depth: bool = False,
                    ws: Workspace | None = None):
    """Differentiable 3DGS render with rendered features: returns (image [3,H,W], features
    [F + with_depth, H, W]); feat is [n, F] (or None for depth alone)."""
    return FeatSplatFunction.apply(mu, scale, quat, opacity, sh, feat, cam, cfg, with_depth, ws or Workspace())


def render(mu, scale, quat, opacity, sh, cam, cfg, ws: Workspace | None = None, timers: StageTimers | None = None):
    """Differentiable render of one view: returns image [3, H, W]."""
    return SplatFunction.apply(mu, scale, quat, opacity, sh, cam, cfg, ws or Workspace(), timers)


class Uploader:
    """Host -> device copies of pinned parameter tensors on a copy stream, off the compute stream.

    `start(dst, src, after=None)` enqueues the copies (after the compute stream's earlier work, and
    after the events in `after`) and returns an event that fires when they are done; `upload`
    does the same and makes the current stream wait.  The splatting forward only needs the SH
    coefficients for the colours, after binning and sorting: giving it the SH copy's event
    (``Workspace.sh_events``) lets those stages run while the coefficients are still in flight."""

    def __init__(self):
        self.stream = torch.cuda.Stream()

    def start(self, dst, src, after=()):
        cur = torch.cuda.current_stream()
        self.stream.wait_stream(cur)  # earlier compute is done with the destination buffers
        for e in after:
            self.stream.wait_event(e)
        with torch.cuda.stream(self.stream):
            for d, h in zip(dst, src):
                d.copy_(h, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        return ev

    def upload(self, dst, src):
        ev = self.start(dst, src)
        torch.cuda.current_stream().wait_event(ev)


def scene_to_device(scene, device="cuda"):
    """Float32 contiguous device tensors (mu, scale, quat, opacity, sh) of a scenes.Scene."""
    return tuple(torch.from_numpy(a).to(device).contiguous() for a in scene.arrays())
