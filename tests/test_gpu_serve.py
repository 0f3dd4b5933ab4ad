"""Serving form on the GPU: every served image is bit-identical to the same
request rendered alone through the plain single-view path, with and without
batching, under a pool that gates admission, and with several streams busy."""
import dataclasses

import pytest
import torch

from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes
from paper_2606_11529_gb300 import serve as SV

pytestmark = pytest.mark.gpu

RES = ((128, 128), (160, 96), (96, 64))


@pytest.fixture(scope="module")
def resident():
    scs = [scenes.clustered_scene(n, seed=k, n_centers=20, width=160, height=96, focal=160.0, sh_degree=deg)
           for k, (n, deg) in enumerate([(3000, 3), (12000, 3), (800, 3), (20000, 3)])]
    return [R.scene_to_device(s) for s in scs]


def _alone(resident, cfg, r):
    return R.forward_frame(*resident[r.scene], SV.camera_of(r), cfg).image.cpu()


def _check_identical(resident, cfg, trace):
    for r in trace:
        assert r.status == "done", (r.rid, r.status)
        ref = _alone(resident, cfg, r)
        assert torch.equal(r.image.cpu(), ref), f"request {r.rid} (batch of {r.batch_views}) differs"


def test_served_equals_alone(resident):
    cfg = scenes.RenderConfig(sh_degree=3)
    trace = SV.make_trace(80, n_scenes=len(resident), rate_hz=3000.0, seed=5, resolutions=RES)
    srv = SV.Server(resident, cfg, pool_bytes=8 << 30, slots=3)
    srv.run(trace)
    _check_identical(resident, cfg, trace)
    st = SV.latency_stats(trace)
    assert st["completed"] == 80 and st["p99_ms"] > 0


def test_batched_requests_equal_alone(resident):
    cfg = scenes.RenderConfig(sh_degree=3)
    # a burst of requests for two (scene, size) classes: they are batched several views at a time
    base = SV.make_trace(24, n_scenes=1, rate_hz=1e6, seed=6, resolutions=((128, 128),))
    trace = [dataclasses.replace(r, scene=1 + (i % 2), arrival=0.0) for i, r in enumerate(base)]
    srv = SV.Server(resident, cfg, pool_bytes=8 << 30, slots=2)
    srv.run(trace)
    assert max(r.batch_views for r in trace) > 1
    _check_identical(resident, cfg, trace)


def test_pool_gates_and_rejects(resident):
    cfg = scenes.RenderConfig(sh_degree=3)
    trace = SV.make_trace(30, n_scenes=len(resident), rate_hz=5000.0, seed=7, resolutions=RES)
    srv = SV.Server(resident, cfg, pool_bytes=1, slots=2)
    srv.calibrate(RES)
    sizes = sorted(srv.estimate(r) for r in trace)
    srv.budget.capacity = sizes[-3]  # the largest requests do not fit at all; at most one large in flight
    srv.run(trace)
    rejected = [r for r in trace if r.status == "rejected"]
    assert rejected and all(r.nbytes > srv.budget.capacity for r in rejected)
    served = [r for r in trace if r.status != "rejected"]
    assert srv.budget.peak <= srv.budget.capacity and srv.budget.used == 0
    _check_identical(resident, cfg, served)


def test_plain_queue_matches(resident):
    cfg = scenes.RenderConfig(sh_degree=3)
    trace = SV.make_trace(20, n_scenes=len(resident), rate_hz=3000.0, seed=8, resolutions=RES)
    SV.run_plain(resident, cfg, trace)
    _check_identical(resident, cfg, trace)


def test_served_equals_alone_at_the_serving_workload_size():
    # the serving workload's sizes: its smallest and largest scenes (clustered SH-3, about 1.9e5 and
    # 2.8e6 Gaussians) at 512x512, 1280x720 and 1920x1080, three worker streams, requests arriving
    # together: every image equals the same request rendered alone, bit for bit
    import math
    import numpy as np
    rng = np.random.default_rng(1000)
    sizes = np.exp(rng.uniform(math.log(100_000), math.log(3_000_000), size=16)).astype(np.int64)
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    resident = [R.scene_to_device(scenes.clustered_scene(int(sizes[k]), seed=k)) for k in pick]
    cfg = scenes.RenderConfig(sh_degree=3)
    trace = SV.make_trace(18, n_scenes=2, rate_hz=1e5, seed=6)
    srv = SV.Server(resident, cfg, pool_bytes=24 << 30, slots=3)
    srv.run(trace)
    _check_identical(resident, cfg, trace)
    assert {(r.width, r.height) for r in trace} == set(SV.RESOLUTIONS)
