"""Tile autotuner: times forward + backward of a batch layout for each candidate
(rays per forward thread, backward threads, backward ray tile, launch mode) and
keeps the fastest, cached in a JSON file keyed by the layout's shape class
(Gaussian counts, pixel count, flow slots, normals, pose gradients)."""

from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import fmb

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "fmb_gb300", "autotune.json")

# Grid launches only: the persistent mode (use_persistent = 1) measured slower than
# the grid launch on every configuration and tile on the GB300 (orbit 3-19 %, large
# K 0.05-0.4 %, ragged batch see the design notes): it cannot use the backward's
# 2-CTA clusters, and each work item costs two CTA barriers and a global atomic
# round trip, where the hardware starts the next CTA of a grid in a freed slot
# directly and already takes the cost-ordered items most expensive first.
CANDIDATES = [dict(fwd_rays_per_thread=r, bwd_threads=t, bwd_ray_tile=t * m, use_persistent=0)
              for r in (2, 4) for t in (128, 160) for m in (2, 3)]

# Extra candidates for small batches (fewer 256-ray tiles than two waves of the
# GPU's SMs): short ray tiles and narrow CTAs spread a few thousand rays over more
# SMs, at the price of more per-tile overhead; the forward's Gaussian split
# (fwd_ksplit, two rays per thread), which shortens each thread's serial walk over
# the Gaussians at the price of the merge launch; and more Gaussian blocks per ray
# tile in the backward (bwd_gblocks), which does the same for the adjoint at the
# price of one set of per-ray records per block (50 000-ray minibatch at K = 256:
# backward 0.0606 -> 0.0571 ms with 4 blocks at 256-ray tiles; one 64x64 view at
# K = 40: 0.0167 -> 0.0146 ms with 2).
SMALL_BWD_TILES = ((64, 64), (64, 128), (128, 128))
SMALL_CANDIDATES = [dict(fwd_rays_per_thread=r, bwd_threads=t, bwd_ray_tile=m, use_persistent=0)
                    for r in (1, 2) for t, m in SMALL_BWD_TILES] + \
                   [dict(fwd_rays_per_thread=2, fwd_ksplit=s, bwd_threads=t, bwd_ray_tile=m, use_persistent=0)
                    for s in (2, 4) for t, m in SMALL_BWD_TILES] + \
                   [dict(fwd_rays_per_thread=r, bwd_threads=128, bwd_ray_tile=m, bwd_gblocks=g, use_persistent=0)
                    for r in (1, 2) for m in (128, 256) for g in (2, 4)]


def candidates_for(views, n_sms: int) -> list:
    """Candidate tiles of a batch: ``CANDIDATES``, plus ``SMALL_CANDIDATES`` when
    the batch has fewer rays than two waves of 256-ray tiles on ``n_sms`` SMs."""
    P = sum(fmb.view_entries(v) for v in views)
    return list(CANDIDATES) + (list(SMALL_CANDIDATES) if P < 2 * n_sms * 256 else [])


# The alpha-compositing variant has fixed 32-ray tiles: only the launch mode is tuned.
CANDIDATES_AC = [dict(use_persistent=p) for p in (0, 1)]

TUNED_FIELDS = ("fwd_rays_per_thread", "bwd_threads", "bwd_ray_tile", "use_persistent", "fwd_ksplit", "bwd_gblocks")


def layout_key(obj_offsets, views, params: fmb.FmbParams, want_pose: bool) -> str:
    """Shape class of a batch: log2 buckets of the per-view pair counts and of the
    total pixel count, plus the render options."""
    offs = np.asarray(obj_offsets, dtype=np.int64)
    Ks = sorted({int(offs[v["object"] + 1] - offs[v["object"]]) for v in views})
    kb = sorted({int(np.log2(max(k, 1))) for k in Ks})
    P = int(sum(fmb.view_entries(v) for v in views))
    return json.dumps(dict(k=kb, p=int(np.log2(max(P, 1))), v=len(views), f=int(params.n_flow),
                           n=int(params.want_normals), pose=bool(want_pose), variant=int(params.variant)),
                      sort_keys=True)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(params: fmb.FmbParams, choice: dict) -> fmb.FmbParams:
    p = fmb.FmbParams()
    ctypes_copy = {name: getattr(params, name) for name, _ in fmb.FmbParams._fields_}
    for k, v in ctypes_copy.items():
        setattr(p, k, v)
    for k in TUNED_FIELDS:
        if k in choice:
            setattr(p, k, int(choice[k]))
    return p


def tune(obj_offsets, views, n_poses, params: fmb.FmbParams, means, chol, weights, poses, upstream: dict,
         want_pose=True, candidates=None, reps=3, cache_path=None, force=False, device="cuda"):
    """Returns (params with the fastest tile choice, timings).  ``upstream`` holds
    device tensors g_depth, g_alpha, g_normal, g_flow for the backward."""
    path = cache_path or os.environ.get("FMB_AUTOTUNE_CACHE", DEFAULT_CACHE)
    key = layout_key(obj_offsets, views, params, want_pose)
    cache = _load(path)
    if key in cache and not force:
        return apply(params, cache[key]["best"]), cache[key]["timings"]
    if candidates is None:
        n_sms = torch.cuda.get_device_properties(torch.device(device)).multi_processor_count
        candidates = CANDIDATES_AC if int(params.variant) == 1 else candidates_for(views, n_sms)
    cands = candidates
    G = int(np.asarray(obj_offsets)[-1])
    out = dict(means=torch.empty(G, 3, device=device), chol=torch.empty(G, 6, device=device),
               weights=torch.empty(G, device=device),
               poses=torch.empty(int(n_poses), 12, device=device) if want_pose else None)
    timings = []
    for c in cands:
        p = apply(params, c)
        try:
            r = fmb.Renderer(obj_offsets, views, n_poses, p, device=device)
        except fmb.FmbError:
            continue
        eager = lambda: (r.forward(means, chol, weights, poses),
                         r.backward(means, chol, weights, poses, upstream["g_depth"], upstream["g_alpha"],
                                    upstream["g_normal"], upstream["g_flow"], want_pose=want_pose, out=out))
        # Each candidate is timed as the batched path runs it: forward + backward
        # captured in one CUDA graph and replayed, so that the host's per-call cost
        # (which decides eager timings of small batches) does not choose the tiles.
        side = torch.cuda.Stream(device)
        side.wait_stream(torch.cuda.current_stream(device))
        with torch.cuda.stream(side):
            eager()  # lazy set-up happens outside the capture
        torch.cuda.current_stream(device).wait_stream(side)
        torch.cuda.synchronize(device)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            eager()
        step = graph.replay
        step()
        torch.cuda.synchronize(device)
        # short steps (a few hundred microseconds or less) are timed over more
        # repetitions, so that each timed block lasts about 2 ms and the choice does
        # not follow the timing noise of a handful of tiny launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize(device)
        n_rep = max(reps, min(64, int(2.0 / max(e0.elapsed_time(e1), 1e-3))))
        best_ms = None
        for _ in range(3):  # best of three timed runs: robust to the GPU's other work
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(n_rep):
                step()
            e1.record()
            torch.cuda.synchronize(device)
            ms = e0.elapsed_time(e1) / n_rep
            best_ms = ms if best_ms is None else min(best_ms, ms)
        timings.append(dict(choice=c, ms=best_ms))
        del graph, r
    if not timings:
        raise RuntimeError("no autotune candidate could be run")
    best = min(timings, key=lambda x: x["ms"])
    cache[key] = dict(best=best["choice"], timings=timings)
    _store(path, cache)
    return apply(params, best["choice"]), timings
