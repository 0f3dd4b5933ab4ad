"""Host logic of the serving form, without a GPU: the Poisson trace, footprint
accounting, FIFO admission, batch formation, and the single-thread dispatch loop
driven by a fake executor (a deadline standing in for the render)."""
import time

import numpy as np
import pytest

from paper_2606_11529_gb300 import serve as SV


def _req(rid, scene=0, w=512, h=512, nbytes=10, arrival=0.0):
    r = SV.Request(rid, scene, w, h, 0.0, (0.0, 0.0, 0.0), arrival)
    r.nbytes = nbytes
    return r


def test_trace_is_poisson_and_seeded():
    t = SV.make_trace(20000, n_scenes=16, rate_hz=200.0, seed=3)
    arr = np.array([r.arrival for r in t])
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 200.0) < 0.03 / 200.0  # 20k exponential draws: ~0.7% s.e.
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05  # exponential: CV = 1
    assert set(r.scene for r in t) == set(range(16))
    assert set((r.width, r.height) for r in t) == set(SV.RESOLUTIONS)
    assert all(abs(r.yaw_deg) <= 5.0 and max(map(abs, r.trans)) <= 0.05 for r in t)
    t2 = SV.make_trace(20000, n_scenes=16, rate_hz=200.0, seed=3)
    assert [(r.scene, r.width, r.arrival) for r in t] == [(r.scene, r.width, r.arrival) for r in t2]


def test_budget_accounting():
    b = SV.HBMBudget(100)
    assert b.reserve(60) and not b.reserve(41) and b.reserve(40)
    assert b.used == 100 and b.peak == 100
    b.release(60)
    assert b.used == 40 and b.peak == 100
    with pytest.raises(AssertionError):
        b.release(41)


def test_fifo_admission_blocks_behind_a_large_head():
    s = SV.Scheduler(SV.HBMBudget(100))
    s.arrive(_req(0, nbytes=70), 0.0)
    s.arrive(_req(1, nbytes=50), 0.0)  # does not fit beside request 0
    s.arrive(_req(2, nbytes=10), 0.0)  # would fit, but must wait behind request 1
    assert [r.rid for r in s.admitted] == [0] and [r.rid for r in s.pending] == [1, 2]
    b = s.take_batch(0.0)
    s.complete(b, 1.0)
    assert [r.rid for r in s.admitted] == [1, 2] and s.budget.used == 60


def test_too_large_is_rejected():
    s = SV.Scheduler(SV.HBMBudget(100))
    r = _req(0, nbytes=101)
    s.arrive(r, 0.0)
    assert r.status == "rejected" and s.rejected == 1 and s.idle()


def test_batches_take_the_oldest_admitted_of_any_scene_and_size():
    s = SV.Scheduler(SV.HBMBudget(10 ** 9), max_views=3)
    keys = [(0, 512), (1, 512), (0, 512), (0, 1280), (0, 512), (0, 512), (1, 512)]
    for i, (sc, w) in enumerate(keys):
        s.arrive(_req(i, scene=sc, w=w, h=w), 0.0)
    b1 = s.take_batch(0.0)
    assert [r.rid for r in b1] == [0, 1, 2]  # capped at max_views, oldest first, scenes and sizes mixed
    assert all(r.batch_views == 3 and r.status == "running" for r in b1)
    assert [r.rid for r in s.admitted] == [3, 4, 5, 6]
    b2 = s.take_batch(0.0)
    assert [r.rid for r in b2] == [3, 4, 5]
    assert s.in_flight == 2


class FakeServer(SV.Server):
    """Server whose batch "runs" for a time proportional to its pixel count (no device)."""

    def __init__(self, pool, slots, service_s=0.002, **kw):
        super().__init__(scenes=[None] * 4, cfg=None, pool_bytes=pool, slots=slots, **kw)
        self.service_s = service_s
        self.calib = {"fake": 1}
        self.running = 0
        self.max_running = 0
        self.batches = []

    def estimate(self, req):
        return req.width * req.height  # bytes ~ pixels

    def new_stream(self):
        return None

    def launch(self, batch, stream):
        assert self.budget.used <= self.budget.capacity
        self.running += 1
        self.max_running = max(self.max_running, self.running)
        self.batches.append(len(batch))
        pixels = sum(r.width * r.height for r in batch)
        return time.perf_counter() + self.service_s * pixels / 512 ** 2

    def is_done(self, handle):
        done = time.perf_counter() >= handle
        if done:
            self.running -= 1
        return done

    def finish(self, batch, handle):
        for r in batch:
            r.image = r.rid
            r.delivered = True


@pytest.mark.parametrize("slots", [1, 3])
def test_dispatch_loop_completes_everything(slots):
    trace = SV.make_trace(300, n_scenes=4, rate_hz=2000.0, seed=1)
    srv = FakeServer(pool=2 * 1920 * 1080, slots=slots)
    srv.run(trace)
    assert all(r.status == "done" and r.image == r.rid for r in trace)
    assert srv.budget.used == 0 and srv.budget.peak <= srv.budget.capacity
    assert srv.max_running <= slots
    for r in trace:
        assert r.arrival <= r.admitted <= r.start <= r.ready
    st = SV.latency_stats(trace, warmup=20)
    assert st["completed"] == 280 and st["p50_ms"] <= st["p99_ms"]
    assert max(srv.batches) > 1  # requests that arrive while the streams are busy are batched


def test_pool_gates_concurrency():
    # a pool that holds one 1080p request: 1080p requests never overlap one another
    trace = [_req(i, w=1920, h=1080, arrival=0.0) for i in range(6)]
    srv = FakeServer(pool=1920 * 1080 + 512 * 512, slots=4, service_s=0.001)
    srv.run(trace)
    spans = sorted((r.start, r.ready) for r in trace)
    assert all(b[0] >= a[1] for a, b in zip(spans, spans[1:]))
    assert srv.budget.peak <= srv.budget.capacity


def test_latency_stats_on_known_values():
    reqs = []
    for i in range(100):
        r = _req(i, arrival=float(i))
        r.status, r.ready = "done", float(i) + (i + 1) * 1e-3  # latencies 1..100 ms
        reqs.append(r)
    st = SV.latency_stats(reqs)
    assert st["p50_ms"] == pytest.approx(50.5) and st["p99_ms"] == pytest.approx(99.01)
    assert st["views_per_s"] == pytest.approx(100 / 99.1, abs=0.006)  # rounded to 0.01


def test_undelivered_request_is_an_error():
    # a batch that completes without delivering its images is marked failed
    class Undelivering(FakeServer):
        def finish(self, batch, handle):
            pass

    trace = SV.make_trace(20, n_scenes=2, rate_hz=5000.0, seed=3)
    srv = Undelivering(pool=2 * 1920 * 1080, slots=2)
    srv.run(trace)
    assert all(r.status == "error" for r in trace)


def test_cost_capped_batches_keep_small_requests_apart_from_large():
    s = SV.Scheduler(SV.HBMBudget(10 ** 9), max_views=8, batch_cost_cap=2.0)
    for i, nb in enumerate([10, 5, 5, 100, 4, 4]):
        s.arrive(_req(i, nbytes=nb), 0.0)
    assert [r.rid for r in s.take_batch(0.0)] == [0, 1, 2]     # 10 + 5 + 5 <= 2 x 10
    assert [r.rid for r in s.take_batch(0.0)] == [3, 4, 5]     # a large head takes the small ones along
    s = SV.Scheduler(SV.HBMBudget(10 ** 9), max_views=8, batch_cost_cap=1.0)
    for i, nb in enumerate([10, 5, 5]):
        s.arrive(_req(i, nbytes=nb), 0.0)
    assert [r.rid for r in s.take_batch(0.0)] == [0]           # cap 1: one request per batch
