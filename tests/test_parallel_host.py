"""View-parallel training step (several ranks) on CPU with the gloo backend: the partition of views
over ranks, the packed all-reduce, and the step's gradients equal the single-process sum over all
views.  The per-view gradients come from the FP64 oracle (no GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_11529_gb300 import parallel as PL
from paper_2606_11529_gb300 import scenes


def test_partition_is_balanced_and_complete():
    for n in range(0, 20):
        for world in range(1, 6):
            parts = [PL.partition_views(n, world, r) for r in range(world)]
            assert sum(parts, []) == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        PL.partition_views(4, 2, 2)


def test_pack_roundtrip():
    ts = [torch.randn(5, 3), torch.randn(7), torch.randn(2, 4, 3)]
    flat = PL.pack(ts)
    assert flat.numel() == 15 + 7 + 24
    out = [torch.empty_like(t) for t in ts]
    PL.unpack_into(flat, out)
    assert all(torch.equal(a, b) for a, b in zip(ts, out))
    with pytest.raises(ValueError):
        PL.unpack_into(torch.zeros(3), [torch.zeros(2)])


def _setup():
    sc = scenes.uniform_scene(60, seed=5, xy_range=0.6, sh_degree=1)
    cams = scenes.multiview_cameras(5, 40, 32, 40.0, seed=2)
    cfg = scenes.RenderConfig(sh_degree=1, bg=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(9)
    targets = [rng.uniform(0, 1, size=(3, 32, 40)) for _ in cams]
    return sc, cams, cfg, targets


def _oracle_grad_fn(oracle, sc, cams, cfg, targets):
    def fn(view_ids):
        loss, acc = 0.0, None
        for v in view_ids:
            img = oracle.pipeline_tiled(sc, cams[v], cfg)["image"]
            ls, (d_img,) = PL.l2_loss_grad([torch.from_numpy(img)], [torch.from_numpy(targets[v])])
            loss += float(ls)
            g = oracle.grads_brute(sc.arrays(), cams[v], cfg, d_img.numpy())
            gs = [torch.from_numpy(np.ascontiguousarray(g[k])) for k in ("mu", "scale", "quat", "opacity", "sh")]
            acc = gs if acc is None else [a + b for a, b in zip(acc, gs)]
        if acc is None:
            acc = [torch.zeros(sc.arrays()[j].shape, dtype=torch.float64) for j in range(5)]
        return loss, acc
    return fn


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        sc, cams, cfg, targets = _setup()
        step = PL.ViewParallelStep(_oracle_grad_fn(O, sc, cams, cfg, targets), world=world, rank=rank)
        loss, grads = step.step(len(cams))
        q.put((rank, loss, [g.numpy() for g in grads]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_view_parallel_step_equals_single_process_sum(oracle, world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc, cams, cfg, targets = _setup()
    loss_all, ref = _oracle_grad_fn(oracle, sc, cams, cfg, targets)(list(range(len(cams))))
    assert abs(sum(o[1] for o in out) - loss_all) <= 1e-12 * max(1.0, abs(loss_all))
    for rank, _, grads in out:  # every rank holds the whole step's gradient
        for g, r in zip(grads, ref):
            np.testing.assert_allclose(g, r.numpy(), rtol=1e-12, atol=1e-15)
