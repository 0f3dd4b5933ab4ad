"""View-parallel training step across ranks (one process per GPU).

The paper's stages parallelise per view: every view of a training step is an independent render
of the same primitives, and the primitives' gradient is the sum of the views' gradients.  So the
step is split by view: rank r renders its share of the step's views (one launch per stage for all
of them, the batched form) and back-propagates their loss, then ONE sum all-reduce of the
primitive gradients over all ranks (all five parameter tensors packed into one flat buffer: N x
(11 + 3K) floats, 236 MB at 1M SH-3 primitives) leaves every rank with the gradient of the whole
step.  No other data crosses ranks: the primitives are replicated and every rank applies the same
optimiser step to its copy.

The partition and the packing are host logic, tested with the gloo backend on CPU ranks; on GPUs
the collective is NCCL's all-reduce over the packed device buffer.
"""
from __future__ import annotations

import torch


def partition_views(n_views: int, world: int, rank: int) -> list[int]:
    """Contiguous, balanced blocks of view indices: rank r gets views [r q + min(r, m), ...) with
    q, m = divmod(n_views, world); ranks beyond the view count get none."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    q, m = divmod(n_views, world)
    start = rank * q + min(rank, m)
    return list(range(start, start + q + (1 if rank < m else 0)))


def pack(tensors) -> torch.Tensor:
    """One flat buffer holding every tensor (in order), for a single collective."""
    return torch.cat([t.reshape(-1) for t in tensors])


def unpack_into(flat: torch.Tensor, tensors) -> None:
    """Copies consecutive slices of ``flat`` back into ``tensors`` (shapes as given)."""
    o = 0
    for t in tensors:
        n = t.numel()
        t.copy_(flat[o:o + n].view_as(t))
        o += n
    if o != flat.numel():
        raise ValueError(f"packed {flat.numel()} values, unpacked {o}")


def allreduce_sum(grads, group=None) -> None:
    """In place: every tensor of ``grads`` becomes its sum over the ranks of ``group`` (one packed
    all-reduce; a no-op when torch.distributed is not initialised or has one rank)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return
    flat = pack(grads)
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    unpack_into(flat, grads)


def l2_loss_grad(images, targets):
    """Loss sum_v mean((image_v - target_v)^2) and its gradient w.r.t. each image."""
    loss, grads = 0.0, []
    for im, tg in zip(images, targets):
        d = im - tg
        loss = loss + (d * d).mean()
        grads.append(2.0 * d / d.numel())
    return loss, grads


class ViewParallelStep:
    """One training step of a view-parallel job.

    ``grad_fn(view_ids) -> (loss, [grad tensors])`` renders the given views of the step and
    returns their loss and the primitive gradients (summed over those views); the default is the
    GPU path (batched render + autograd).  ``step(views)`` runs this rank's share of ``views`` and
    the all-reduce, and returns (the summed loss of this rank's views, the step's gradients)."""

    def __init__(self, grad_fn, world: int = 1, rank: int = 0, group=None):
        self.grad_fn = grad_fn
        self.world, self.rank, self.group = world, rank, group

    def step(self, n_views: int):
        mine = partition_views(n_views, self.world, self.rank)
        loss, grads = self.grad_fn(mine)
        allreduce_sum(grads, self.group)
        return loss, grads


def gpu_grad_fn(params, cams, cfg, targets, ws=None):
    """The GPU path of ViewParallelStep: the selected views of ``cams`` through the batched form
    (one launch per stage), L2 loss against ``targets`` (one image per view), autograd backward."""
    from . import batched as BT

    def fn(view_ids):
        P = [p.detach().requires_grad_(True) for p in params]
        if not view_ids:
            return 0.0, [torch.zeros_like(p) for p in P]
        imgs = BT.render_views(*P, [cams[v] for v in view_ids], cfg, ws)
        loss, _ = l2_loss_grad(list(imgs), [targets[v] for v in view_ids])
        loss.backward()
        return float(loss.item()), [p.grad for p in P]

    return fn
