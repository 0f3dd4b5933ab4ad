"""Serving form of the splatting path: scenes resident in HBM, a stream of
render requests, admission by HBM footprint and continuous batching.

The paper describes no serving system (it times single renders, Sec. 5); this
module is the request loop around the same forward stages:

* every scene's parameters stay on the device for the server's lifetime;
* a request (scene id, camera, image size) is admitted when the working memory
  its forward needs (projected records, intersection and sort buffers, image)
  fits in the pool that the in-flight requests have not reserved; admission is
  FIFO, so a large request is not starved by smaller ones behind it, and a
  request larger than the whole pool is rejected;
* one host thread runs the loop: it takes arrivals as they come, and whenever
  one of ``slots`` CUDA streams is free and requests are admitted, it takes the
  oldest admitted request and the admitted requests after it, whatever their
  scene and image size (up to 16, while the batch's summed footprint stays
  within ``batch_cost_cap`` times the oldest one's, so that a small request is
  not held back by a large one), and launches them as one multi-scene batch (one launch per stage for all of them,
  the tiles of every request in one persistent work list), then copies the
  images to pinned host memory and records an event; so several batches are in
  flight at once, on different streams, and a request arriving while the GPU is
  busy joins the next batch instead of queueing behind single renders;
* the loop polls the batches' events; a request is ready when its image has
  reached pinned host memory; its reservation is then freed and what now fits
  is admitted.  One thread with no hand-off between threads keeps the dispatch
  latency of an isolated request at the plain path's.

The plain baseline renders the same trace one request at a time, in arrival
order, through the per-stage single-view path.

The scheduling state (``Scheduler``, ``HBMBudget``) is plain host code with no
device dependence, so its behaviour is testable without a GPU.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import math
import time

import numpy as np

RESOLUTIONS = ((512, 512), (1280, 720), (1920, 1080))
MAX_VIEWS = 16


@dataclasses.dataclass
class Request:
    rid: int
    scene: int
    width: int
    height: int
    yaw_deg: float
    trans: tuple
    arrival: float  # seconds after the start of the trace
    nbytes: int = 0  # reserved working memory
    status: str = "new"  # new -> pending -> admitted -> running -> done | rejected
    admitted: float = math.nan
    start: float = math.nan
    ready: float = math.nan
    batch_views: int = 0
    n_isect: int = 0
    image: object = None  # the delivered image (None once a client that keeps no images has it)
    delivered: bool = False

    @property
    def key(self):
        return (self.scene, self.width, self.height)

    @property
    def latency(self):
        return self.ready - self.arrival


def make_trace(n_requests: int, n_scenes: int = 16, rate_hz: float = 200.0, seed: int = 0,
               resolutions=RESOLUTIONS, max_yaw_deg: float = 5.0, max_trans: float = 0.05) -> list[Request]:
    """Open-loop Poisson arrivals: inter-arrival times ~ Exp(mean 1/rate_hz); each request picks a
    scene and a resolution uniformly and a pose with yaw ~ U[-max_yaw, max_yaw] degrees and a
    translation ~ U[-max_trans, max_trans] per axis.
    Draw order: inter-arrival times, scenes, resolutions, yaws, translations."""
    rng = np.random.default_rng(seed + 2000)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    scene = rng.integers(0, n_scenes, size=n_requests)
    res = rng.integers(0, len(resolutions), size=n_requests)
    yaw = rng.uniform(-max_yaw_deg, max_yaw_deg, size=n_requests)
    tr = rng.uniform(-max_trans, max_trans, size=(n_requests, 3))
    out = []
    for i in range(n_requests):
        w, h = resolutions[int(res[i])]
        out.append(Request(i, int(scene[i]), int(w), int(h), float(yaw[i]), tuple(float(x) for x in tr[i]),
                           float(arrivals[i])))
    return out


def camera_of(req: Request):
    """Pinhole camera of a request: focal length = image width (the same field of view at every
    size), principal point at the image centre, the request's yaw and translation."""
    from . import scenes
    return scenes.pinhole(req.width, req.height, float(req.width), scenes.yaw_view(req.yaw_deg, req.trans))


class HBMBudget:
    """Byte accounting of the working-memory pool shared by the in-flight requests."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.used = 0
        self.peak = 0

    def fits(self, nbytes: int) -> bool:
        return self.used + nbytes <= self.capacity

    def reserve(self, nbytes: int) -> bool:
        if not self.fits(nbytes):
            return False
        self.used += int(nbytes)
        self.peak = max(self.peak, self.used)
        return True

    def release(self, nbytes: int):
        self.used -= int(nbytes)
        assert self.used >= 0, "released more than reserved"


class Scheduler:
    """FIFO admission by footprint and batch formation.  Not thread-safe by itself: the server
    calls it under one lock."""

    def __init__(self, budget: HBMBudget, max_views: int = MAX_VIEWS, batch_cost_cap: float | None = None):
        self.budget = budget
        self.max_views = max_views
        # None: a batch takes the oldest admitted requests up to max_views; a number c: requests
        # join the oldest one only while the batch's summed footprint (the cost proxy) stays within
        # c times the oldest request's, so that small requests are not held back by large ones
        self.batch_cost_cap = batch_cost_cap
        self.pending = collections.deque()  # arrived, not yet admitted (FIFO)
        self.admitted = collections.deque()  # admitted, not yet taken by a worker (FIFO)
        self.in_flight = 0
        self.rejected = 0

    def arrive(self, req: Request, now: float):
        if req.nbytes > self.budget.capacity:
            req.status = "rejected"
            self.rejected += 1
            return
        req.status = "pending"
        self.pending.append(req)
        self.admit(now)

    def admit(self, now: float):
        while self.pending and self.budget.reserve(self.pending[0].nbytes):
            r = self.pending.popleft()
            r.status, r.admitted = "admitted", now
            self.admitted.append(r)

    def take_batch(self, now: float) -> list[Request]:
        """The oldest admitted requests, any scene and size, up to max_views of them."""
        if not self.admitted:
            return []
        batch = [self.admitted.popleft()]
        cap = None if self.batch_cost_cap is None else self.batch_cost_cap * max(batch[0].nbytes, 1)
        cost = batch[0].nbytes
        while self.admitted and len(batch) < self.max_views:
            if cap is not None and cost + self.admitted[0].nbytes > cap:
                break
            cost += self.admitted[0].nbytes
            batch.append(self.admitted.popleft())
        for r in batch:
            r.status, r.start, r.batch_views = "running", now, len(batch)
        self.in_flight += 1
        return batch

    def complete(self, batch: list[Request], now: float):
        for r in batch:
            r.status, r.ready = "done", now
            self.budget.release(r.nbytes)
        self.in_flight -= 1
        self.admit(now)

    def idle(self) -> bool:
        return not self.pending and not self.admitted and self.in_flight == 0


def latency_stats(reqs: list[Request], warmup: int = 0) -> dict:
    """p50 / p99 arrival-to-ready latency (ms) and views/s over the requests after ``warmup``."""
    done = [r for r in reqs[warmup:] if r.status == "done"]
    if not done:
        return {"p50_ms": None, "p99_ms": None, "views_per_s": 0.0, "completed": 0,
                "rejected": sum(r.status == "rejected" for r in reqs[warmup:])}
    lat = np.array([r.latency for r in done]) * 1e3
    span = max(r.ready for r in done) - min(r.arrival for r in done)
    return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "mean_ms": round(float(lat.mean()), 3), "views_per_s": round(len(done) / span, 2) if span > 0 else None,
            "completed": len(done), "rejected": sum(r.status == "rejected" for r in reqs[warmup:]),
            "mean_batch_views": round(float(np.mean([r.batch_views for r in done])), 3)}


# ------------------------------------------------------------------------------------------ device side

def footprint_bytes_items(n_prims: int, width: int, height: int, n_isect: int, cfg) -> int:
    """Device working memory of one request rendered as an item of a multi-scene batch: the
    workspace `xpr_forward_items` asks for one item of this size at a capacity of ``n_isect`` pairs
    (records, boxes, counts, depth order and its scratch, the binning's scratch, the sorted pairs,
    the tile ranges and work list), plus the image planes, t_final and n_contrib."""
    from . import binding as B
    from . import scenes as S
    L = B.load()
    layout = B.ItemLayout([0], [int(n_prims)], [S.pinhole(int(width), int(height), float(width))], cfg)
    g = B.make_config(cfg)
    ws = int(L.xpr_forward_items_workspace(layout.carr, layout.arr, 1, ctypes.byref(g), int(n_isect)))
    return ws + int(width) * int(height) * (3 * 4 + 4 + 4)


def footprint_bytes(n_prims: int, width: int, height: int, n_isect: int, cfg, n_views: int = 1) -> int:
    """Device working memory of one forward of ``n_views`` views (every buffer the stages
    allocate: records, bounding boxes, counts, depth order, offsets, the pair buffers at the
    capacity the forward asks for, the sorted pairs, the scratch of each C-ABI call, the tile
    ranges and work list, and the image planes)."""
    from . import binding as B
    L = B.load()
    nv = n_prims * n_views
    tw, th = int(cfg.tile_w), int(cfg.tile_h)
    nt = n_views * ((width + tw - 1) // tw) * ((height + th - 1) // th)
    cap = int(n_isect * 1.25) + 1024
    per_prim = nv * (12 * 4 + 16 + 4 + 4 + 4 + 4) + 4
    pairs = 2 * cap * 4 + 2 * n_isect * 4
    scratch = (int(L.xpr_depth_order_workspace(nv)) + int(L.xpr_tile_bin_workspace(nv)) +
               int(L.xpr_sort_tiles_workspace(n_isect, nt)) + int(L.xpr_tile_worklist_workspace(nt)))
    image = n_views * width * height * (3 * 4 + 4 + 4)
    return int(per_prim + pairs + scratch + nt * 12 + image)


def _wait_until(t_abs: float):
    while True:
        d = t_abs - time.perf_counter()
        if d <= 0:
            return
        time.sleep(min(d, 2e-4))


class Server:
    """Continuous-batching renderer over resident scenes (see the module docstring).

    ``scenes``: a ``batched.SceneSet`` (the resident scenes as one concatenated parameter set; its
    ``views()`` are the per-scene tensors), or a list of per-scene (mu, scale, quat, opacity, sh)
    tuples, concatenated here.  ``pool_bytes``: working-memory pool for the in-flight requests
    (the resident scenes are outside it).  ``slots``: batches in flight, one CUDA stream each."""

    def __init__(self, scenes, cfg, pool_bytes: int, slots: int = 2, capacity_factor: float = 1.3,
                 max_views: int = MAX_VIEWS, deliver_host: bool = True, keep_images: bool = True,
                 batch_cost_cap: float | None = 2.0):
        if scenes is not None and not hasattr(scenes, "views") and len(scenes) and scenes[0] is not None:
            from . import batched as BT
            scenes = BT.SceneSet(scenes)
        self.scene_set = scenes if hasattr(scenes, "views") else None
        self.scenes = self.scene_set.views() if self.scene_set is not None else scenes
        self.cfg = cfg
        self.slots = slots
        self.capacity_factor = capacity_factor
        self.deliver_host = deliver_host
        # keep_images False: a request drops its image once delivered (a client that consumes
        # results), so the pinned host buffers are recycled instead of pinning new memory per request
        self.keep_images = keep_images
        self.budget = HBMBudget(pool_bytes)
        self.sched = Scheduler(self.budget, max_views, batch_cost_cap)
        self.calib = {}
        self.errors = []
        self._ws = {}
        self._pinned = {}
        self._ccfg = None
        if cfg is not None:
            from . import binding as B
            self._ccfg = B.make_config(cfg)

    # intersections at the canonical pose of each (scene, size): the admission estimate
    def calibrate(self, resolutions=RESOLUTIONS):
        import torch
        from . import binding as B
        from . import scenes as S
        for k, P in enumerate(self.scenes):
            for (w, h) in resolutions:
                cam = S.pinhole(w, h, float(w))
                _, _, _, cnt = B.xpr_project(*P, B.make_camera(cam), B.make_config(self.cfg), with_isect_count=True)
                self.calib[(k, w, h)] = int(cnt.sum(dtype=torch.int64).item())

    def n_isect_estimate(self, req: Request) -> int:
        return int(math.ceil(self.calib[req.key] * self.capacity_factor)) + 1024

    def estimate(self, req: Request) -> int:
        n = int(self.scenes[req.scene][0].shape[0])
        return footprint_bytes_items(n, req.width, req.height, self.n_isect_estimate(req), self.cfg)

    def new_stream(self):
        import torch
        return torch.cuda.Stream()

    def _pinned_buffer(self, stream, nfloats):
        import torch
        key = id(stream)
        buf = self._pinned.get(key)
        if buf is None or buf.numel() < nfloats:
            buf = torch.empty(int(nfloats), dtype=torch.float32).pin_memory()
            self._pinned[key] = buf
        return buf[:nfloats]

    def launch(self, batch: list[Request], stream):
        """Enqueues one multi-scene batch on ``stream`` through one native call (projection, depth
        order, fused bin + sort, persistent render over every request's tiles), then the copy of
        the images to pinned host memory, and returns the pending handle.  The native call reads
        the pair count back, so it returns once the binning is done; the render and the copy run
        on."""
        import torch
        from . import binding as B
        ss = self.scene_set
        cams = [camera_of(r) for r in batch]
        layout = ss.layout([r.scene for r in batch], cams, self._ccfg)
        key = id(stream)
        cap = sum(self.n_isect_estimate(r) for r in batch)
        with torch.cuda.stream(stream):
            image, _, _, n_isect, ws = B.xpr_forward_items(*ss.params, layout, self._ccfg, cap,
                                                           workspace=self._ws.get(key), stream=stream)
            self._ws[key] = ws
            if self.deliver_host:
                out = self._pinned_buffer(stream, image.numel()) if not self.keep_images else \
                    torch.empty(image.numel(), dtype=torch.float32, pin_memory=True)
                out.copy_(image, non_blocking=True)
            else:
                out = image
            ev = torch.cuda.Event()
            ev.record(stream)
        return ev, out, layout, n_isect

    def is_done(self, handle) -> bool:
        return handle[0].query()

    def finish(self, batch: list[Request], handle):
        _, out, layout, n_isect = handle
        imgs = layout.images(out)
        for r, im in zip(batch, imgs):
            r.image = im if self.keep_images else None
            r.n_isect = n_isect
            r.delivered = True

    def run(self, trace: list[Request]) -> list[Request]:
        """Replays ``trace`` open-loop against the wall clock; returns it with times filled in."""
        if not self.calib:
            self.calibrate(sorted({(r.width, r.height) for r in trace}))
        for r in trace:
            r.nbytes = self.estimate(r)
        streams = [self.new_stream() for _ in range(self.slots)]
        free = list(range(self.slots))
        inflight = []  # (batch, handle, stream index)
        t0 = time.perf_counter()
        nxt = 0
        while True:
            now = time.perf_counter() - t0
            # completions (in launch order per stream; any order across streams)
            still = []
            for batch, handle, si in inflight:
                if self.is_done(handle):
                    try:
                        self.finish(batch, handle)
                    except Exception as e:  # recorded and re-raised below
                        self.errors.append(e)
                    now = time.perf_counter() - t0
                    self.sched.complete(batch, now)
                    for r in batch:
                        if not r.delivered:
                            r.status = "error"
                    free.append(si)
                else:
                    still.append((batch, handle, si))
            inflight = still
            # arrivals
            while nxt < len(trace) and trace[nxt].arrival <= now:
                self.sched.arrive(trace[nxt], now)
                nxt += 1
            # dispatch: every free stream takes the oldest admitted requests
            while free and self.sched.admitted and not self.errors:
                batch = self.sched.take_batch(time.perf_counter() - t0)
                si = free.pop(0)
                try:
                    inflight.append((batch, self.launch(batch, streams[si]), si))
                except Exception as e:
                    self.errors.append(e)
                    self.sched.complete(batch, time.perf_counter() - t0)
                    for r in batch:
                        r.status = "error"
                    free.append(si)
            if self.errors and not inflight:
                break
            if nxt >= len(trace) and self.sched.idle():
                break
            if not inflight and not self.sched.admitted and nxt < len(trace):
                # idle until the next arrival (sleep, then spin the last 0.3 ms)
                wake = t0 + trace[nxt].arrival
                d = wake - time.perf_counter()
                if d > 3e-4:
                    time.sleep(d - 3e-4)
        if self.errors:
            raise self.errors[0]
        return trace


def run_plain(scenes, cfg, trace: list[Request], server: Server | None = None, deliver_host: bool = True,
              keep_images: bool = True):
    """The plain per-request queue: one request at a time, in arrival order, through the
    single-view per-stage path on the current stream (keep_images as for Server)."""
    import torch
    from . import binding as B
    from . import render as R
    t0 = time.perf_counter()
    for r in trace:
        _wait_until(t0 + r.arrival)
        r.start = time.perf_counter() - t0
        ws = R.Workspace()
        if server is not None:
            ws.last_isect = int(server.n_isect_estimate(r) / 1.25)
        fr = R.forward_frame(*scenes[r.scene], camera_of(r), cfg, ws)
        if deliver_host:
            out = torch.empty(tuple(fr.image.shape), dtype=fr.image.dtype, pin_memory=True)
            out.copy_(fr.image, non_blocking=True)
        else:
            out = fr.image
        torch.cuda.current_stream().synchronize()
        r.ready = time.perf_counter() - t0
        r.status, r.batch_views, r.n_isect, r.delivered = "done", 1, fr.n_isect, True
        r.image = out if keep_images else None
    return trace
