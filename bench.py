"""Benchmark of the 3DGS tile-splatting path on GB300.

Workload: forward + backward through the torch.autograd.Function at 1M SH-3
Gaussians in a clustered synthetic scene, 1920x1080 pinhole (focal 1920),
16x16 tiles, gradients w.r.t. all primitive parameters.  One step = one view:
project -> tile bin -> sort -> render forward -> render adjoint -> projection
adjoint.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle as it stands on the host cores on a
bounded sample of the same workload (there is no installable reference
implementation: the paper's system is described only in its text).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/iter @1M Gaussians 1080p vs plain path; serve p50/p99 ms, views/s"
UNIT = "ms/iter"
WORKLOAD = "3DGS fwd+bwd, 1M SH-3 Gaussians clustered (200 centres, spread 0.5, depth 1-20), 1920x1080 pinhole f=1920, 16x16 tiles, seed 0"

# Per-unit algorithmic work of each stage: bytes a stage must move, or FP32-pipe operations per
# (pixel, entry) pair counted from the kernels' arithmetic.
SH_FLOATS = 48
PARAM_BYTES = 4 * (3 + 3 + 4 + 1 + SH_FLOATS)  # 236 B per primitive
REC_BYTES = 48
# FP32-pipe operations per (pixel, entry) pair of the method's compositing arithmetic written per
# pair (power from the pixel offset, alpha, gates, blend; the adjoint counted on a contributing
# unclamped pair with the colour behind a pixel as one scalar): the algorithmic work of the render
# stages.
FWD_OPS_PER_PAIR = 16
BWD_OPS_PER_PAIR = 39
# What the kernels execute per pair after factoring the power by pixel column (A dx^2 and B dx once
# per entry and column) and, in the adjoint, applying the mean partials' conic factors once per
# (tile, entry): forward 12 + 4 per column of 4 pixels, adjoint 28 + 4 per column of 8 pixels.
FWD_EXEC_OPS_PER_PAIR = 13.0
BWD_EXEC_OPS_PER_PAIR = 28.5
# stages that are one kernel launch (the render adjoint's bracket also holds the zero-fill of d_rec)
SINGLE_KERNEL = {"project": "project_fwd_kernel<3>", "render_fwd": "render_fwd_kernel<16,16>",
                 "render_bwd": "render_bwd_kernel<16,16>", "project_bwd": "project_bwd_kernel<3>"}
# DRAM bytes (read + write) per launch of a kernel from one ncu capture, the profile summary that
# holds it, and the sha256 (first 16 hex digits) of the kernel's source file when it was captured:
# the figure is reported only while that source is unchanged (null once the kernel has changed).
TRAFFIC = {
    "render_bwd_kernel<16,16>": (45_117_952, "profiles/render_bwd_headline.md",
                                 "paper_2606_11529_gb300/csrc/render.cu", "f7da4ab3040d0655"),
}
FP32_LANES = 128  # FP32 lanes per SM (4 partitions x 32)
DEFAULT_SM_MHZ = 2070.0  # maximum SM clock, used when no clock sample exists
# 3DGUT ray evaluation: FP32-pipe operations per (pixel, entry) pair
UT_FWD_OPS_PER_PAIR = 31
UT_BWD_OPS_PER_PAIR = 66
# LinPrim slab intersection: FP32-pipe operations per (pixel, entry) pair
LP_FWD_OPS_PER_PAIR = 39
LP_BWD_OPS_PER_PAIR = 97


# SM count read from the device and the SM clock the ALU peak is taken at (the median sampled
# under load in the timed region once known)
_ALU = {"sms": None, "mhz": DEFAULT_SM_MHZ, "mhz_source": "maximum SM clock (no sample yet)"}


def set_alu_peak(dev, sm_mhz=None, source=None):
    import torch
    _ALU["sms"] = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    if sm_mhz:
        _ALU["mhz"], _ALU["mhz_source"] = float(sm_mhz), source or "median sampled SM clock in the timed region"


def peaks():
    p = {"hbm_gbs": 6800.0, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        p = {"hbm_gbs": float(j["hbm_gbs"]), "source": "measured"}
    except Exception:
        pass
    sms = _ALU["sms"] or 152
    # FP32 lane-ops/s (an FMA counted as one operation): SMs x 128 lanes x SM clock
    p["alu_ops"] = sms * FP32_LANES * _ALU["mhz"] * 1e6
    p["alu_desc"] = (f"{sms} SMs (device properties) x {FP32_LANES} FP32 lanes x {_ALU['mhz']:.0f} MHz "
                     f"({_ALU['mhz_source']}), FP32 lane-ops/s, derived")
    return p


def traffic_of(kernel):
    """ncu DRAM bytes per launch of ``kernel`` if its source is unchanged since the capture."""
    import hashlib
    t = TRAFFIC.get(kernel)
    if t is None:
        return None, None
    nbytes, profile, src, sha = t
    try:
        with open(os.path.join(ROOT, src), "rb") as f:
            cur = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        return None, None
    return (nbytes, profile) if cur == sha else (None, None)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 50 ms, timestamped) taken from before the warm-up to after the
    timed region; the report uses the samples inside the timed window when there are any, else
    all samples of the run (and says so)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None
        self.window = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, t0, t1):
        self.window = (t0, t1)

    @staticmethod
    def _epoch(ts):
        import datetime
        try:
            dt = datetime.datetime.strptime(ts.strip(), "%Y/%m/%d %H:%M:%S.%f")
            return time.mktime(dt.timetuple()) + dt.microsecond * 1e-6
        except ValueError:
            return None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [[x.strip() for x in r.split(",")] for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        samples = []
        for r in rows:
            if len(r) < 10:
                continue
            try:
                samples.append((self._epoch(r[0]), float(r[2]), float(r[3]), r[6:10]))
            except ValueError:
                continue
        scope = "timed region"
        sel = samples
        if self.window:
            inside = [s for s in samples if s[0] is not None and self.window[0] - 0.05 <= s[0] <= self.window[1] + 0.05]
            if inside:
                sel = inside
            else:
                scope = "whole run (timed region shorter than the sampling interval)"
        reasons = set()
        for s in sel:
            for nm, v in zip(names, s[3]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm = [s[1] for s in sel]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(s[2] for s in sel) if sel else None, "reasons": sorted(reasons),
                "samples": len(sel), "scope": scope}


def workload_config(sc, cam, cfg):
    """The workload's description, the same dict on both arms."""
    return {"workload": WORKLOAD, "primitives": sc.n, "sh_degree": cfg.sh_degree,
            "resolution": [cam.width, cam.height], "tile": [cfg.tile_w, cfg.tile_h]}


# --------------------------------------------------------------------------- reference arm (oracle on CPU)
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import baseline
    from paper_2606_11529_gb300 import scenes
    sc, cam, cfg = scenes.headline_case()
    # every step is one whole forward + backward of the workload (all primitives, all tiles), timed
    # on the host cores as the oracle stands: nothing is sampled or extrapolated
    for _ in range(args.warmup):
        baseline.estimate_fwd_bwd_seconds(sc, cam, cfg, prim_frac=1.0, n_tiles=1 << 30, seed=0)
    ests = []
    desc = ""
    for k in range(args.steps):
        est, m, desc = baseline.estimate_fwd_bwd_seconds(sc, cam, cfg, prim_frac=1.0, n_tiles=1 << 30, seed=k)
        ests.append(est)
    baseline.release_lists()
    ms = 1000.0 * statistics.mean(ests)
    cores = baseline.threads()
    out = {"impl": "reference", "metric": METRIC, "value": ms, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(sc, cam, cfg),
           "cpu_baseline": {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
           "e2e": {"value": ms, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


# --------------------------------------------------------------------------- GPU arm
def cpu_baseline_leg():
    from oracle import baseline
    from paper_2606_11529_gb300 import scenes
    sc, cam, cfg = scenes.headline_case()
    est, meas, desc = baseline.estimate_fwd_bwd_seconds(sc, cam, cfg, prim_frac=1.0, n_tiles=1 << 30, seed=0)
    baseline.release_lists()
    return {"value": 1000.0 * est, "unit": UNIT, "cores": baseline.threads(), "kind": "oracle", "sample": desc}


def _median_ms(fn, reps, flush=None):
    import torch
    times = []
    for k in range(reps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        times.append(s.elapsed_time(e))
    return statistics.median(times)


def batched_leg(dev, reps, flush, method=0):
    """Batched form: 3M uniform Gaussians seen by 8 pinhole cameras (1600x1064, focal 800, yaw
    -15..+15 degrees), forward + backward of all 8 views; one batched pass (autotuned tile size and
    batch depth, persistent render grids) against 8 plain single-view passes.  method 1: 3DGUT."""
    import numpy as np
    import torch
    from paper_2606_11529_gb300 import batched as BT
    from paper_2606_11529_gb300 import render as R
    from paper_2606_11529_gb300 import scenes
    sc = scenes.uniform_scene(3_000_000, seed=0)
    # 3DGUT sees the views through the fisheye of its configuration (it needs no linearisation)
    cams = scenes.multiview_cameras(8, 1600, 1064, 800.0, seed=0,
                                    fisheye_dist=scenes.FISHEYE_DIST if method == 1 else None)
    base = scenes.RenderConfig(sh_degree=0, method=method)
    P = [t.to(dev) for t in R.scene_to_device(sc)]
    w = torch.from_numpy(np.random.default_rng(2).normal(size=(8, 3, 1064, 1600)).astype(np.float32)).to(dev)
    chunks = {}
    best, table = BT.autotune(P, cams, base, scene_id=f"uniform-3M-m{method}", reps=5, chunks=chunks)
    Pg = [p.detach().requires_grad_(True) for p in P]
    ws = BT.ViewsWorkspace()

    def batched():
        for p in Pg:
            p.grad = None
        (BT.render_views(*Pg, cams, best, ws) * w).sum().backward()

    wss = [R.Workspace() for _ in cams]

    def plain():
        for p in Pg:
            p.grad = None
        for v, cam in enumerate(cams):
            (R.render(*Pg, cam, base, wss[v]) * w[v]).sum().backward()

    for _ in range(3):
        batched()
        plain()
    torch.cuda.synchronize()
    tb = _median_ms(batched, reps, flush)
    tp = _median_ms(plain, reps, flush)
    # pairs of the chosen setting, summed over the view chunks it runs in
    n_isect = sum(BT.forward_views(*P, part, best, BT.ViewsWorkspace()).n_isect
                  for part in BT.view_chunks(cams, ws.chunks))
    what = "3DGUT (unscented projection, ray evaluation)" if method == 1 else "3DGS"
    lens = ("fisheye (k = 0.05, -0.01, 0.001, 0)" if method == 1 else "pinhole")
    return {"workload": f"{what}: 3M uniform SH-0 Gaussians (xy U[-1,1], z U[2,6]), 8 {lens} views 1600x1064 "
                        "f=800, yaw -15..+15 deg, fwd+bwd of all 8 views, seed 0",
            "ms_batched": round(tb, 3), "ms_plain_8x": round(tp, 3), "speedup": round(tp / tb, 3),
            "intersections": n_isect, "tile": [best.tile_w, best.tile_h], "batch_depth": best.batch_depth,
            "view_chunks": ws.chunks,
            "autotune_ms": {f"{k[0]}x{k[1]}/b{k[2]}": (round(v, 3) if v != float("inf") else None)
                            for k, v in table.items()},
            "autotune_view_chunks": {f"{k[0]}x{k[1]}/b{k[2]}": c for k, c in chunks.items()},
            "timing": f"median of {reps} (L2 flushed before each)"}


def scenes_leg(dev, reps, flush):
    """Multi-scene batched form: 4 clustered SH-3 scenes of uneven size (drawn as the serving
    workload's) seen by 2 cameras each at different resolutions (8 items), forward + backward of all
    8 in one launch per stage, against 8 plain single-view passes."""
    import numpy as np
    import torch
    from paper_2606_11529_gb300 import batched as BT
    from paper_2606_11529_gb300 import render as R
    from paper_2606_11529_gb300 import scenes
    from paper_2606_11529_gb300 import serve as SV
    scs = scenes.serving_scenes(16, seed=0)[:4]
    cfg = scenes.RenderConfig(sh_degree=3)
    sset = BT.SceneSet([tuple(t.to(dev) for t in R.scene_to_device(s)) for s in scs])
    res = [(1920, 1080), (512, 512), (1280, 720), (1920, 1080), (512, 512), (1280, 720), (1280, 720), (512, 512)]
    soi = [0, 0, 1, 1, 2, 2, 3, 3]
    cams = [scenes.pinhole(w, h, float(w), scenes.yaw_view(3.0 * (k - 4), (0.01 * k, 0.0, 0.0)))
            for k, (w, h) in enumerate(res)]
    layout = sset.layout(soi, cams, cfg)
    rng = np.random.default_rng(4)
    wts = [torch.from_numpy(rng.normal(size=(3, h, w)).astype(np.float32)).to(dev) for (w, h) in res]
    P = [p.detach().requires_grad_(True) for p in sset.params]
    views = [tuple(t[o:o + n] for t in P) for o, n in zip(sset.offsets, sset.counts)]
    ws = BT.ViewsWorkspace()

    def batched():
        for p in P:
            p.grad = None
        imgs = BT.render_items(*P, layout, cfg, ws)
        sum((im * w).sum() for im, w in zip(imgs, wts)).backward()

    wss = [R.Workspace() for _ in cams]

    def plain():
        for p in P:
            p.grad = None
        for k, (s_, cam) in enumerate(zip(soi, cams)):
            (R.render(*views[s_], cam, cfg, wss[k]) * wts[k]).sum().backward()

    for _ in range(3):
        batched()
        plain()
    torch.cuda.synchronize()
    tb = _median_ms(batched, reps, flush)
    tp = _median_ms(plain, reps, flush)
    fr = BT.forward_items(*sset.params, layout, cfg, BT.ViewsWorkspace())
    return {"workload": f"4 clustered SH-3 scenes of uneven size ({', '.join(str(c) for c in sset.counts)} Gaussians), "
                        "2 cameras each at 1920x1080 / 512x512 / 1280x720 (f = width): 8 (scene, camera) items, "
                        "fwd+bwd of all 8, seed 0",
            "ms_batched": round(tb, 3), "ms_plain_8x": round(tp, 3), "speedup": round(tp / tb, 3),
            "intersections": fr.n_isect, "timing": f"median of {reps} (L2 flushed before each)"}


def ut_leg(dev, n, reps, flush, fisheye=False):
    """3DGUT form: the headline scene (1M clustered SH-3 Gaussians, 1920x1080 pinhole, or the fisheye
    of the 3DGUT configuration with the same focal length) with the unscented projection, ray-offset
    binning and ray-evaluated compositing, forward + backward through the autograd Function."""
    import dataclasses
    import numpy as np
    import torch
    from paper_2606_11529_gb300 import render as R
    from paper_2606_11529_gb300 import scenes
    sc, cam, cfg = scenes.headline_case(n)
    cfg = dataclasses.replace(cfg, method=1)
    if fisheye:
        cam = scenes.fisheye(cam.width, cam.height, cam.fx, scenes.FISHEYE_DIST)
    P = [t.to(dev).requires_grad_(True) for t in R.scene_to_device(sc)]
    w = torch.from_numpy(np.random.default_rng(1).normal(size=(3, cam.height, cam.width)).astype(np.float32)).to(dev)
    ws = R.Workspace()

    def step(timers=None):
        for p in P:
            p.grad = None
        (R.render(*P, cam, cfg, ws, timers) * w).sum().backward()

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ms = _median_ms(step, reps, flush)
    timers = R.StageTimers()
    for k in range(reps):
        flush.fill_(k & 0xFF)
        step(timers)
    st = timers.mean_ms()
    fr = R.forward_frame(*[p.detach() for p in P], cam, cfg, ws)
    pairs = int(fr.n_contrib.to(torch.int64).sum().item())
    alu = peaks()["alu_ops"]
    roof = {}
    for name, ops in (("render_fwd", UT_FWD_OPS_PER_PAIR), ("render_bwd", UT_BWD_OPS_PER_PAIR)):
        ach = pairs * ops / (st[name] * 1e-3)
        roof[name] = {"kernel": f"ut_{name}_kernel<16,16>", "bound": "alu", "achieved_tops": round(ach / 1e12, 3),
                      "frac": round(ach / alu, 4)}
    lens = "fisheye f=1920 (k = 0.05, -0.01, 0.001, 0)" if fisheye else "pinhole f=1920"
    return {"workload": f"3DGUT fwd+bwd, the headline scene (1M SH-3 Gaussians clustered, 1920x1080 {lens}, "
                        "16x16 tiles, seed 0), unscented projection with 7 sigma points",
            "ms_per_iter": round(ms, 4), "stages_ms": {k: round(v, 4) for k, v in st.items()},
            "intersections": fr.n_isect, "pairs_blended": pairs, "render_roofline": roof,
            "timing": f"median of {reps} (L2 flushed before each)"}


def lp_leg(dev, reps, flush):
    """LinPrim form: 500k octahedra drawn as the headline scene (clustered means, half-extents
    e^N(-3, 0.5), SH degree 3), 1280x720 pinhole f=1280, 16x16 tiles, forward + backward through the
    autograd Function."""
    import numpy as np
    import torch
    from paper_2606_11529_gb300 import render as R
    from paper_2606_11529_gb300 import scenes
    sc, cam, cfg = scenes.linprim_case()
    P = [t.to(dev).requires_grad_(True) for t in R.scene_to_device(sc)]
    w = torch.from_numpy(np.random.default_rng(1).normal(size=(3, cam.height, cam.width)).astype(np.float32)).to(dev)
    ws = R.Workspace()

    def step(timers=None):
        for p in P:
            p.grad = None
        (R.render(*P, cam, cfg, ws, timers) * w).sum().backward()

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    ms = _median_ms(step, reps, flush)
    timers = R.StageTimers()
    for k in range(reps):
        flush.fill_(k & 0xFF)
        step(timers)
    st = timers.mean_ms()
    fr = R.forward_frame(*[p.detach() for p in P], cam, cfg, ws)
    pairs = int(fr.n_contrib.to(torch.int64).sum().item())
    alu = peaks()["alu_ops"]
    roof = {}
    for name, ops in (("render_fwd", LP_FWD_OPS_PER_PAIR), ("render_bwd", LP_BWD_OPS_PER_PAIR)):
        ach = pairs * ops / (st[name] * 1e-3)
        roof[name] = {"kernel": f"lp_{name}_kernel<16,16>", "bound": "alu", "achieved_tops": round(ach / 1e12, 3),
                      "frac": round(ach / alu, 4)}
    return {"workload": "LinPrim fwd+bwd: 500k octahedra (clustered means, half-extents e^N(-3,0.5), SH-3), "
                        "1280x720 pinhole f=1280, 16x16 tiles, seed 0",
            "ms_per_iter": round(ms, 4), "stages_ms": {k: round(v, 4) for k, v in st.items()},
            "intersections": fr.n_isect, "pairs_blended": pairs, "render_roofline": roof,
            "timing": f"median of {reps} (L2 flushed before each)"}


def feat_leg(dev, n, reps, flush):
    """Rendered features: the headline scene (1M SH-3 Gaussians, 1920x1080) with 8 per-primitive
    semantic channels and the expected-depth channel composited in the colour's blend loop,
    forward + backward through render_features, against the plain colour-only step."""
    import numpy as np
    import torch
    from paper_2606_11529_gb300 import render as R
    from paper_2606_11529_gb300 import scenes
    sc, cam, cfg = scenes.headline_case(n)
    P = [t.to(dev).requires_grad_(True) for t in R.scene_to_device(sc)]
    feat = torch.from_numpy(np.random.default_rng(5).normal(size=(sc.n, 8)).astype(np.float32)).to(dev)
    feat.requires_grad_(True)
    rng = np.random.default_rng(6)
    wi = torch.from_numpy(rng.normal(size=(3, cam.height, cam.width)).astype(np.float32)).to(dev)
    wf = torch.from_numpy(rng.normal(size=(9, cam.height, cam.width)).astype(np.float32)).to(dev)
    ws = R.Workspace()

    def step():
        for p in P + [feat]:
            p.grad = None
        img, feats = R.render_features(*P, feat, cam, cfg, with_depth=True, ws=ws)
        ((img * wi).sum() + (feats * wf).sum()).backward()

    def plain():
        for p in P:
            p.grad = None
        (R.render(*P, cam, cfg, ws) * wi).sum().backward()

    for _ in range(3):
        step()
        plain()
    torch.cuda.synchronize()
    ms = _median_ms(step, reps, flush)
    ms_plain = _median_ms(plain, reps, flush)
    return {"workload": "rendered features: the headline scene (1M SH-3 Gaussians, 1920x1080, 16x16 tiles) with 8 "
                        "semantic channels + expected depth, fwd+bwd of image and features",
            "ms_per_iter": round(ms, 4), "ms_colour_only": round(ms_plain, 4),
            "timing": f"median of {reps} (L2 flushed before each)"}


def serve_leg(dev, n_requests, warmup, cap_gb, scale_down):
    """Serving form: 16 resident clustered SH-3 scenes (sizes log-uniform in [1e5, 3e6]), Poisson
    arrivals at 200 requests/s, sizes 512x512 / 1280x720 / 1920x1080; the continuous-batching server
    against the plain one-at-a-time queue on the same trace, then the server under a small pool."""
    import torch
    from paper_2606_11529_gb300 import batched as BT
    from paper_2606_11529_gb300 import render as R
    from paper_2606_11529_gb300 import scenes
    from paper_2606_11529_gb300 import serve as SV
    t0 = time.perf_counter()
    # the resident scenes as one concatenated parameter set; both paths read its per-scene views
    sset = BT.SceneSet([tuple(t.to(dev) for t in R.scene_to_device(s))
                        for s in scenes.serving_scenes(16, seed=0, scale_down=scale_down)])
    resident = sset.views()
    gen_s = time.perf_counter() - t0
    cfg = scenes.RenderConfig(sh_degree=3)
    free, _ = torch.cuda.mem_get_info(dev)
    pool = int(max(free - (16 << 30), 8 << 30))
    # the client consumes each image once delivered (pinned output buffers are recycled)
    srv = SV.Server(sset, cfg, pool_bytes=pool, slots=2, keep_images=False)
    srv.calibrate()
    # warm every (scene, size) once so lazy module loading and allocator growth stay outside
    SV.run_plain(resident, cfg, SV.make_trace(48, rate_hz=1e6, seed=99), srv, keep_images=False)
    # and a burst through the server, so that each stream's allocator pool has grown too
    srv.run(SV.make_trace(192, rate_hz=1e6, seed=98))
    srv.run(SV.make_trace(192, rate_hz=2000.0, seed=97))
    trace = SV.make_trace(n_requests + warmup, rate_hz=200.0, seed=0)
    srv.run(trace)
    ours = SV.latency_stats(trace, warmup)
    ours["pool_peak_gb"] = round(srv.budget.peak / 2 ** 30, 3)
    ptrace = SV.make_trace(n_requests + warmup, rate_hz=200.0, seed=0)
    SV.run_plain(resident, cfg, ptrace, srv, keep_images=False)
    plain = SV.latency_stats(ptrace, warmup)
    # the same comparison at twice the rate, where the queue of the plain path builds up
    n_hi = max(n_requests // 2, 100)
    htrace = SV.make_trace(n_hi + warmup // 2, rate_hz=400.0, seed=2)
    srv.run(htrace)
    hi = {"rate_hz": 400.0, "requests": n_hi, "server": SV.latency_stats(htrace, warmup // 2)}
    hptrace = SV.make_trace(n_hi + warmup // 2, rate_hz=400.0, seed=2)
    SV.run_plain(resident, cfg, hptrace, srv, keep_images=False)
    hi["plain_queue"] = SV.latency_stats(hptrace, warmup // 2)
    n_cap = max(n_requests // 4, 100)
    capped = SV.Server(sset, cfg, pool_bytes=int(cap_gb * 2 ** 30), slots=2, keep_images=False)
    capped.calib = srv.calib
    ctrace = SV.make_trace(n_cap + warmup // 4, rate_hz=200.0, seed=1)
    capped.run(ctrace)
    cst = SV.latency_stats(ctrace, warmup // 4)
    cst["pool_gb"], cst["pool_peak_gb"] = cap_gb, round(capped.budget.peak / 2 ** 30, 3)
    scene_prims = [int(s[0].shape[0]) for s in resident]
    return {"workload": f"16 resident clustered SH-3 scenes ({sum(scene_prims)} Gaussians, "
                        f"{min(scene_prims)}-{max(scene_prims)} per scene), Poisson 200 req/s, "
                        "512x512 / 1280x720 / 1920x1080 (f = width), forward only, image delivered to pinned host",
            "requests": n_requests, "warmup_requests": warmup, "slots": 2, "batch_cost_cap": 2.0,
            "p50_ms": ours["p50_ms"], "p99_ms": ours["p99_ms"], "views_per_s": ours["views_per_s"],
            "server": ours, "plain_queue": plain, "capped_pool": cst, "rate_400": hi,
            "resident_gb": round(sum(sum(t.numel() * 4 for t in s) for s in resident) / 2 ** 30, 3),
            "scene_gen_s": round(gen_s, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=1_000_000, help="primitive count (default: the headline 1M)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 8-view batched leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-ut", action="store_true", help="skip the 3DGUT leg")
    ap.add_argument("--ut-only", action="store_true",
                    help="run only the 3DGUT leg and print it as its own JSON line (for profiling captures)")
    ap.add_argument("--no-lp", action="store_true", help="skip the LinPrim leg")
    ap.add_argument("--no-feat", action="store_true", help="skip the rendered-features leg")
    ap.add_argument("--feat-only", action="store_true",
                    help="run only the rendered-features leg and print it as its own JSON line (for profiling)")
    ap.add_argument("--ut-fisheye", action="store_true", help="with --ut-only: render through the fisheye camera")
    ap.add_argument("--lp-only", action="store_true",
                    help="run only the LinPrim leg and print it as its own JSON line (for profiling captures)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving leg and print it as its own JSON line")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-warmup", type=int, default=200)
    ap.add_argument("--serve-cap-gb", type=float, default=4.0)
    ap.add_argument("--serve-scale-down", type=int, default=1)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2606_11529_gb300 import binding as B
    from paper_2606_11529_gb300 import render as R
    from paper_2606_11529_gb300 import scenes

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = B.load()
    set_alu_peak(dev)

    if args.serve_only:
        out = {"leg": "serve", "serve": serve_leg(dev, args.serve_requests, args.serve_warmup, args.serve_cap_gb,
                                                  args.serve_scale_down)}
        if rank == 0:
            print(json.dumps(out))
        return 0

    if args.ut_only or args.lp_only or args.feat_only:
        flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
        if args.ut_only:
            out = {"leg": "3dgut", "ut": ut_leg(dev, args.n, max(args.steps, 1), flush, fisheye=args.ut_fisheye)}
        elif args.lp_only:
            out = {"leg": "linprim", "linprim": lp_leg(dev, max(args.steps, 1), flush)}
        else:
            out = {"leg": "features", "features": feat_leg(dev, args.n, max(args.steps, 1), flush)}
        if rank == 0:
            print(json.dumps(out))
        return 0

    sc, cam, cfg = scenes.headline_case(args.n)
    if world > 1:
        # view-parallel training step: rank r renders view r of the step (the headline camera turned
        # by r degrees), then one packed NCCL all-reduce sums the primitive gradients over the ranks
        cam = scenes.pinhole(cam.width, cam.height, cam.fx, scenes.yaw_view(float(rank)))
    from paper_2606_11529_gb300 import parallel as PL
    host = [torch.from_numpy(a).pin_memory() for a in sc.arrays()]
    P = [h.to(dev).requires_grad_(True) for h in host]
    w = torch.from_numpy(np.random.default_rng(1).normal(size=(3, cam.height, cam.width)).astype(np.float32)).to(dev)
    ws = R.Workspace()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(timers=None):
        for p in P:
            p.grad = None
        img = R.render(*P, cam, cfg, ws, timers)
        loss = (img * w).sum()
        loss.backward()
        if world > 1:
            PL.allreduce_sum([p.grad for p in P])
        return loss

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    timers = R.StageTimers()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = L.xpr_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    t_epoch0 = time.time()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict L2 between steps (outside the timed events)
        starts[k].record()
        step()
        ends[k].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clocks.mark(t_epoch0, time.time())
    launches = int(L.xpr_launch_count() - launches0)
    # the stage times come from a second pass of the same steps with CUDA events around each C-ABI
    # call (the events' recording would otherwise be part of the timed steps)
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        step(timers)
    clk = clocks.stop()
    if clk.get("sm_mhz"):
        set_alu_peak(dev, clk["sm_mhz"])
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        if world > 1:
            dist.barrier()
    stage_ms = timers.mean_ms()

    # algorithmic work of the last step (from its own outputs, outside the timed region)
    fr = R.forward_frame(*[p.detach() for p in P], cam, cfg, ws)
    pairs = int(fr.n_contrib.to(torch.int64).sum().item())
    I = fr.n_isect
    n = sc.n
    T = int(fr.ranges.shape[0])
    passes = math.ceil(max(1, (T - 1).bit_length()) / 8)  # tile bits only (depth-ordered input)
    pk = peaks()
    # Algorithmic bytes per stage (what the method must move, the per-unit figures of the design
    # notes); "impl" is what the implementation moves when it differs.
    work = {
        "project": ("hbm", n * (PARAM_BYTES + REC_BYTES + 16 + 4), None),
        # one radix pass over (key, index) pairs: read the depth and tile count, read + write 8 B
        # pairs, write the order
        "depth_order": ("hbm", n * (8 + 16 + 4), None),
        # bin: read each primitive's record, box and count, write 12 B per kept pair (u64 key + u32
        # value) and the offsets
        "tile_bin": ("hbm", n * (REC_BYTES + 16 + 4 + 4) + I * 12, None),
        # sort: one read and one write of 12 B per kept pair (the lower bound of one pass)
        "sort": ("hbm", 24 * I, {"passes": passes, "bytes": passes * 16 * I + passes * 4 * I}),
        # fused bin + sort: the bin's reads plus one write of the sorted lists (4 B per kept pair) and
        # the tile ranges
        "bin_sort": ("hbm", n * (REC_BYTES + 16 + 4 + 4) + I * 4 + T * 8, None),
        "render_fwd": ("alu", pairs * FWD_OPS_PER_PAIR, {"ops_per_pair": FWD_EXEC_OPS_PER_PAIR}),
        "render_bwd": ("alu", pairs * BWD_OPS_PER_PAIR, {"ops_per_pair": BWD_EXEC_OPS_PER_PAIR}),
        "project_bwd": ("hbm", n * (2 * PARAM_BYTES + REC_BYTES), None),
    }
    stages = {}
    for name, (bound, amount, impl) in work.items():
        t = stage_ms.get(name)
        if not t:
            continue
        if bound == "hbm":
            ach = amount / (t * 1e-3) / 1e9
            stages[name] = {"ms": round(t, 4), "bound": "hbm", "achieved_gbs": round(ach, 1),
                            "frac": round(ach / pk["hbm_gbs"], 4)}
            if impl:
                ib = impl["bytes"] / (t * 1e-3) / 1e9
                stages[name]["impl"] = {"passes": impl["passes"], "bytes": impl["bytes"], "gbs": round(ib, 1),
                                        "frac": round(ib / pk["hbm_gbs"], 4)}
        else:
            ach = amount / (t * 1e-3)
            stages[name] = {"ms": round(t, 4), "bound": "alu", "achieved_tops": round(ach / 1e12, 3),
                            "frac": round(ach / pk["alu_ops"], 4)}
            if impl:
                ex = pairs * impl["ops_per_pair"] / (t * 1e-3)
                stages[name]["executed"] = {"ops_per_pair": impl["ops_per_pair"], "tops": round(ex / 1e12, 3),
                                            "frac": round(ex / pk["alu_ops"], 4)}
    # roofline of the dominant kernel: the largest stage that is a single kernel launch
    single = {k: v for k, v in stages.items() if k in SINGLE_KERNEL}
    dom = max(single, key=lambda k: single[k]["ms"])
    d = stages[dom]
    kname = SINGLE_KERNEL[dom]
    traffic, traffic_src = traffic_of(kname)
    if d["bound"] == "hbm":
        roof = {"kernel": kname, "bound": "hbm", "achieved": d["achieved_gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": d["frac"], "traffic": traffic,
                "peak_source": pk["source"] + " (MEASURED_PEAKS.json hbm_gbs)"}
    else:
        roof = {"kernel": kname, "bound": "alu", "achieved": d["achieved_tops"],
                "peak": round(pk["alu_ops"] / 1e12, 2), "unit": "TOP/s", "frac": d["frac"], "traffic": traffic,
                "peak_source": pk["alu_desc"], "sms": _ALU["sms"], "peak_sm_mhz": _ALU["mhz"]}
        if "executed" in d:
            roof["executed"] = d["executed"]
    roof["timing"] = ("CUDA events around the C-ABI call on the launching stream, mean over a second pass of the "
                      "timed steps (the headline steps run without these events)")
    roof["traffic_source"] = traffic_src or "null: no ncu capture of the kernel's current source"

    # end to end through the public API: pinned H2D of the step's inputs, fwd+bwd, D2H of the loss
    e2e_s = torch.cuda.Event(enable_timing=True)
    e2e_e = torch.cuda.Event(enable_timing=True)
    h2d = sum(h.numel() * h.element_size() for h in host)
    up = R.Uploader()

    def upload_inputs():
        # the forward brings the inputs over itself: the projection reads the geometry from pinned
        # host memory and writes its device copy in the same pass, then the SH coefficients are
        # copied under the depth order, binning and sort (the colours are needed only after them)
        ws.host_inputs = (host, up.stream)

    upload_inputs()
    step()
    torch.cuda.synchronize()
    e2e_s.record()
    for k in range(args.steps):
        upload_inputs()
        loss = step()
        _ = loss.item()
    e2e_e.record()
    torch.cuda.synchronize()
    e2e_ms = e2e_s.elapsed_time(e2e_e) / args.steps

    # the same, also bringing every output back: the image and all five parameter gradients copied
    # into pinned host buffers inside each step (for a caller whose optimiser runs on the host)
    img_host = torch.empty((3, cam.height, cam.width), dtype=torch.float32).pin_memory()
    grad_host = [torch.empty_like(h).pin_memory() for h in host]
    d2h_full = img_host.numel() * 4 + sum(g.numel() * 4 for g in grad_host)

    def step_out():
        for p in P:
            p.grad = None
        img = R.render(*P, cam, cfg, ws)
        loss = (img * w).sum()
        loss.backward()
        if world > 1:
            PL.allreduce_sum([p.grad for p in P])
        img_host.copy_(img.detach(), non_blocking=True)
        for g, p in zip(grad_host, P):
            g.copy_(p.grad, non_blocking=True)
        return loss

    upload_inputs()
    step_out()
    torch.cuda.synchronize()
    e2e_s.record()
    for k in range(args.steps):
        upload_inputs()
        loss = step_out()
        _ = loss.item()
    e2e_e.record()
    torch.cuda.synchronize()
    e2e_full_ms = e2e_s.elapsed_time(e2e_e) / args.steps
    if world > 1:
        t = torch.tensor([e2e_ms, e2e_full_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms, e2e_full_ms = float(t[0].item()), float(t[1].item())

    del fr
    # the same step with the other binning paths in place of xpr_bin_rows: the fused bin + sort
    # (xpr_bin_sorted) and the key path (xpr_tile_bin + xpr_sort_tiles, with its stage times)
    ws_fused, ws_key = R.Workspace(fused=True), R.Workspace(rows=False)

    def alt_step(wsx, t=None):
        for p in P:
            p.grad = None
        (R.render(*P, cam, cfg, wsx, t) * w).sum().backward()

    for _ in range(3):
        alt_step(ws_fused)
        alt_step(ws_key)
    fused_ms = _median_ms(lambda: alt_step(ws_fused), args.steps, flush)
    key_ms = _median_ms(lambda: alt_step(ws_key), args.steps, flush)
    key_timers = R.StageTimers()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        alt_step(ws_key, key_timers)
    key_stages = {k: round(v, 4) for k, v in key_timers.mean_ms().items()}
    ut = None if args.no_ut else ut_leg(dev, args.n, max(args.steps, 5), flush)
    lp = None if args.no_lp else lp_leg(dev, max(args.steps, 5), flush)
    feat = None if args.no_feat else feat_leg(dev, args.n, max(args.steps, 5), flush)
    batched = None if args.no_batched else batched_leg(dev, max(args.steps // 2, 5), flush)
    batched_ut = None if (args.no_batched or args.no_ut) else batched_leg(dev, max(args.steps // 2, 5), flush, 1)
    batched_scenes = None if args.no_batched else scenes_leg(dev, max(args.steps // 2, 5), flush)
    serve = None
    if not args.no_serve:
        torch.cuda.empty_cache()
        serve = serve_leg(dev, args.serve_requests, args.serve_warmup, args.serve_cap_gb, args.serve_scale_down)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg()

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(ms, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(sc, cam, cfg),
            "workload_stats": {"intersections": I, "pairs_blended": pairs,
                               "views_per_s_total": round(world * 1000.0 / ms, 2),
                               "fused_bin_sort_path_ms": round(fused_ms, 4), "key_path_ms": round(key_ms, 4),
                               "key_path_stages_ms": key_stages},
            "l2": "flushed between steps (256 MB write outside the timed events)",
            "parallelism": (f"view-parallel x{world}: one view per rank, one packed NCCL all-reduce of the "
                            f"{sum(p.numel() for p in P) * 4 // 2 ** 20} MB of gradients per step") if world > 1
            else "single GPU",
            "roofline": roof,
            "stages": stages,
            "batched": batched,
            "batched_3dgut": batched_ut,
            "batched_scenes": batched_scenes,
            "serve": serve,
            "ut": ut,
            "linprim": lp,
            "features": feat,
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_ms, 4), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4,
                    "note": "the gradients stay on the device (for an on-device optimiser); only the loss is read back",
                    "with_outputs_d2h": {"value": round(e2e_full_ms, 4), "unit": UNIT, "h2d_bytes_per_step": h2d,
                                         "d2h_bytes_per_step": d2h_full + 4,
                                         "note": "image and all five parameter gradients copied to pinned host "
                                                 "memory inside each step"}},
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s": round(wall, 3),
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
