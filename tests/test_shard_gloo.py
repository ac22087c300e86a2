"""Data-parallel sharding on the host (two gloo ranks on CPU): views split by cost,
each rank differentiates its shard with the FP64 oracle, and the one exchange step
(an all-reduce of the gradients) reproduces the whole batch's gradients.  The GPU
path runs the same exchange with NCCL; this box has one GPU, so it is exercised
here with gloo."""

import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2308_14737_gb300 import shard, synth


def _scene():
    """Five orbit views whose flow targets (the next view) cross the shards."""
    return synth.object_orbit(K=7, n_views=5, W=9, H=7)


def _view_upstream(scene, vi, v):
    P = synth.view_entries(v)
    gd, ga, gn, gf = synth.upstream_grads(np.random.default_rng(100 + vi), P, 1)
    return gd, ga, gn.reshape(-1), gf.reshape(-1)


def _grads(scene, view_idx):
    import oracle

    sub = shard.sub_scene(scene, view_idx)
    if not view_idx:
        return dict(means=np.zeros(scene.means.shape), chol=np.zeros(scene.chol.shape),
                    weights=np.zeros(scene.weights.shape), poses=np.zeros(scene.poses.shape))
    parts = [_view_upstream(scene, i, scene.views[i]) for i in view_idx]
    gd, ga, gn, gf = (np.concatenate([p[j] for p in parts]) for j in range(4))
    return oracle.backward_scene(sub, gd, ga, gn, gf, n_flow=1)


def _worker(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        scene = _scene()
        shards = shard.shard_views(scene, world)
        g = {k: torch.as_tensor(v) for k, v in _grads(scene, shards[rank]).items()}
        shard.allreduce_gradients(g)
        if rank == 0:
            out_q.put({k: v.numpy() for k, v in g.items()})
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_views_balances_and_covers():
    s = synth.ragged_batch(n_objects=6, views_per_object=2, sides=(16, 24, 32))
    for world in (1, 2, 3, 5):
        sh = shard.shard_views(s, world)
        assert sorted(i for x in sh for i in x) == list(range(len(s.views)))
        loads = shard.shard_loads(s, sh)
        biggest = max(shard.view_cost(s, v) for v in s.views)
        assert loads.max() - loads.min() <= biggest  # greedy LPT bound


def test_two_rank_allreduce_reproduces_full_batch():
    """world_size 2 over gloo: the sum of the ranks' shard gradients equals the
    gradient of the whole batch (poses included: a view's flow target may be
    rendered on the other rank)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = q.get(timeout=180)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    scene = _scene()
    full = _grads(scene, list(range(len(scene.views))))
    for k in full:
        np.testing.assert_allclose(got[k], full[k], rtol=1e-12, atol=1e-12 * max(1.0, np.abs(full[k]).max()))
