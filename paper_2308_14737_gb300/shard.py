"""Data-parallel sharding of a render batch over ranks (one process per GPU).

Views are independent in the forward pass, so a batch is split by views: each
rank renders and differentiates its own views with the library's batched calls,
and the backward needs one exchange -- the sum over ranks of the per-Gaussian
gradients (and of the pose gradients, since a flow target may be another rank's
view).  ``shard_views`` balances the ranks by cost (pixels x Gaussians, largest
first onto the least-loaded rank); ``allreduce_gradients`` is that exchange, one
``torch.distributed.all_reduce`` (NCCL on GPUs, gloo on the host) per gradient
tensor.  A rank whose shard is empty still joins the all-reduce with zeros.
"""

from __future__ import annotations

import numpy as np


def view_cost(scene, v) -> int:
    """Ray-Gaussian pairs of a view (its rays x its object's Gaussians)."""
    n = len(v["rays"]) if v.get("rays") is not None else int(v["W"]) * int(v["H"])
    return n * scene.K(v["object"])


def shard_views(scene, world_size: int) -> list[list[int]]:
    """Indices of the views of each rank: longest-processing-time greedy on the
    view costs (deterministic: ties go to the lower rank, views in index order)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    costs = [view_cost(scene, v) for v in scene.views]
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world_size
    shards: list[list[int]] = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in shards]


def sub_scene(scene, view_idx):
    """The scene restricted to the given views (same objects and poses; the views'
    planes repacked contiguously)."""
    from . import synth

    objs = [(scene.means[scene.object_slice(o)], scene.chol[scene.object_slice(o)],
             scene.weights[scene.object_slice(o)]) for o in range(scene.n_objects)]
    views = [{k: val for k, val in scene.views[i].items() if k != "pix_offset"} for i in view_idx]
    return synth.make_scene(objs, views, scene.poses, name=scene.name + f"_shard{len(view_idx)}")


def allreduce_gradients(grads: dict, group=None) -> dict:
    """Sums every gradient tensor of ``grads`` (None entries skipped) over the
    ranks of ``group`` in place and returns the dict."""
    import torch.distributed as dist

    for k in sorted(grads):
        if grads[k] is not None:
            dist.all_reduce(grads[k], op=dist.ReduceOp.SUM, group=group)
    return grads


def shard_loads(scene, shards) -> np.ndarray:
    """Pairs per rank of a sharding (for reporting balance)."""
    return np.array([sum(view_cost(scene, scene.views[i]) for i in s) for s in shards], dtype=np.int64)
