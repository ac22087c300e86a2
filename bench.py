"""Benchmark of the Fuzzy Metaballs render path: ray-Gaussian pairs/s for one
forward + backward pass over a batch of views, batched versus plain per-view
launches.

Headline workload (one step): the large-K stress configuration -- 8 sphere views
at 1024x768 (f = 1024), K = 4096 diagonal-precision Gaussians, depth + alpha +
normal planes, flow to the next view, and the full backward (means, Cholesky
factors, weights, poses) from random upstream gradients: 2.58e10 pairs per step.
Inputs are seeded synthetic data; L2 is flushed (256 MiB write) between timed
steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload largek|orbit|single|ragged|recon|minibatch]
                    [--configs all|none]

At N = 1 the same JSON line carries, under "configs", one record for each of the
other configurations, measured the same way in the same run: a single 64x64 view
with K = 40 (depth + alpha, Gaussian gradients); the 16-view 320x240 orbit with
K = 100 (all planes, flow, pose gradients); the ragged batch of 64 objects (K from
20 to 400, square images of side 64..512, 4 views each); and the reconstruction
workload (100 views at 640x480, K = 256, two flow slots) with the full
reconstruction step (forward, loss, backward and Adam replayed from one CUDA
graph) and the stored-intermediate adjoint beside the recomputing one.  Each
record has its batched and plain rates, the roofline fractions, the oracle timed
on a bounded sample and the parity of the GPU result on that sample.
``--workload`` makes another configuration the headline; ``--configs none``
leaves the records out.

The batched arm's tiles come from the autotuner, run before the timed region; set
FMB_AUTOTUNE_CACHE to a file to reuse a previous run's choice (e.g. when
profiling, so the profiled run launches no tuning candidates).

Prints one JSON line.  Under torchrun (N > 1) every rank renders its own replica
of the headline batch (weak scaling) and rank 0 prints the aggregate.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ray-Gaussian pairs/s fwd+bwd, batched vs plain, at <=1e-4 rel err vs FP64"
DEFAULT_WORKLOAD = "largek"
SUB_CONFIGS = ("single", "orbit", "ragged", "recon")
# Timed steps of each configuration's record (at least --steps): about a second of
# GPU work each, enough for stable CUDA-event means.
SUB_STEPS = {"single": 400, "orbit": 400, "ragged": 40, "recon": 30, "largek": 20, "minibatch": 400}

# Algorithmic per-pair work of the implemented formulation: FP32 add/mul/fma lane
# operations (an FMA counts once; negations, comparisons, loads and control
# excluded) and MUFU operations (ex2, rcp, rsqrt), counted operation by operation
# in docs/opcount.md from the formulas, with and without the normal plane.
OPS = {  # normals -> (fwd FP32, fwd MUFU, bwd FP32, bwd MUFU), with pose gradients
    True: (56, 4, 110, 4),
    False: (35, 3, 63, 3),  # without normals the second projection of u is skipped (7 operations)
}
# The algorithmic minimum of the whitened formulation (docs/opcount.md): the
# executed counts above less the operations of the compensated geometry (16 with
# normals, 9 without) and the rsqrt guard of the normal.
ALGO_OPS = {True: (39, 93), False: (26, 54)}  # normals -> (fwd FP32, bwd FP32), with pose gradients
# Without pose gradients the two-parameter adjoint needs only the lower triangle of
# sum v abar^T (6 of its 9 accumulations per pair).
NO_POSE_SAVING = 3
# Alpha-compositing variant (Sec. 3.3): per pair, the same geometry plus the
# transmittance and weight arithmetic (prefix sums, T = e^-S, 1 - e^-delta by its
# series), and in the backward a re-render, the per-pair weight adjoint and the
# packed pair loop; the per-ray 64-bit sort network (integer compares and
# shuffles) is extra and not counted.  The backward count has one re-render: the
# keep_order adjoint evaluates each pair twice in its per-ray phase (about 60 FP32
# operations more), so its fraction against this count is a lower bound.
OPS_AC = {True: (82, 4, 206, 7), False: (67, 3, 146, 5)}
MUFU_MIX = {True: {"ex2": 2, "rcp": 1, "rsqrt": 1}, False: {"ex2": 2, "rcp": 1}}  # per pair, each pass
N_SM = 152
LANES_PER_SM = 128
# MUFU results per SM and clock, measured by the ALU probe on the GB300 at 2070 MHz
# (profiles/alu_probe_rates.md): ex2 31.8, rcp and rsqrt 16.0.
MUFU_RATE = {"ex2": 31.8, "rcp": 16.0, "rsqrt": 16.0}


# The paper's runtime-per-ray table (its Table 2): one whole iteration (forward,
# backward and memory transfers) per ray with 40 Gaussians, JAX on an i5-7267U CPU and
# a GTX 1080 GPU.  Context only: other hardware, unstated precision.
PAPER_RUNTIME_PER_RAY = {"weighted blending": {"cpu_us": 4.94, "gpu_ns": 226.6},
                         "alpha compositing": {"cpu_us": 12.7, "gpu_ns": 377.6}}
PAPER_RUNTIME_GAUSSIANS = 40


def paper_context(variant: str) -> dict:
    name = "alpha compositing" if variant == "ac" else "weighted blending"
    ns = PAPER_RUNTIME_PER_RAY[name]["gpu_ns"]
    return {"what": "Table 2: whole iteration (forward, backward, memory transfers) per ray, 40 Gaussians, JAX; "
                    "other hardware, context only",
            "gtx1080_ns_per_ray": ns, "gtx1080_pairs_per_s": PAPER_RUNTIME_GAUSSIANS / (ns * 1e-9), "variant": name}


def peak_fp32_gops(clock_mhz: float) -> float:
    """FP32-pipe peak in G lane-operations per second (152 SMs x 128 lanes x clock)."""
    return N_SM * LANES_PER_SM * clock_mhz * 1e6 / 1e9


def mufu_busy_frac(pairs_per_s: float, clock_mhz: float, normals: bool = True) -> float:
    """Fraction of the MUFU pipe's time the per-pair ex2/rcp/rsqrt need at this rate."""
    sm_clocks_per_pair = sum(n / MUFU_RATE[k] for k, n in MUFU_MIX[bool(normals)].items())
    return pairs_per_s * sm_clocks_per_pair / (N_SM * clock_mhz * 1e6)


# Committed ncu summaries of the backward kernel, per workload.  Each records the
# DRAM bytes of one captured launch and the factor that scales them to one launch
# of the workload (the large-K capture is a 3-view case of the same kernel, within
# the size rule for full ncu captures; its plane traffic grows with the pixels).
PROFILES = {"orbit": os.path.join(ROOT, "profiles", "backward_kernel_orbit16x320x240_K100.md"),
            "largek": os.path.join(ROOT, "profiles", "backward_kernel_largek8x1024x768_K4096.md")}


def csrc_sha256() -> str:
    """Hash of the sources that define the backward kernel, and of its compile flags."""
    import hashlib

    from paper_2308_14737_gb300 import build

    d = os.path.join(ROOT, "paper_2308_14737_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("fmb_backward.cu", "fmb_internal.cuh", "fmb_f32x2.cuh"):
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(build.EXTRA_FLAGS.get("fmb_backward.cu", [])).encode())
    return h.hexdigest()


def profiled_traffic(tiles=None, workload="orbit"):
    """DRAM bytes (read + write) per launch of the backward kernel on a workload,
    from the committed ncu summary (scaled to a full launch by the summary's
    scale_to_full factor), or None if there is no summary for the workload or the
    kernel sources or the launch tiles changed since the capture."""
    try:
        txt = open(PROFILES[workload]).read()
    except (OSError, KeyError):
        return None
    vals = dict(line.split(":", 1) for line in txt.splitlines()
                if line.startswith(("dram_bytes_per_launch", "source_sha256", "tiles", "scale_to_full")))
    sha = next((v for k, v in vals.items() if k.startswith("source_sha256")), "").strip()
    if not sha or sha.split()[-1] != csrc_sha256():
        return None
    if tiles is not None:  # the backward kernel's tiles (the forward's do not change its traffic)
        want = " ".join(f"{k}={int(v)}" for k, v in sorted(tiles.items())
                        if k in ("bwd_ray_tile", "bwd_threads", "use_persistent"))
        if vals.get("tiles", "").strip() != want:
            return None
    try:
        frac = vals.get("scale_to_full", "1").split("(")[0].strip()  # e.g. "8/3 (pixels)"
        num, _, den = frac.partition("/")
        scale = float(num) / (float(den) if den else 1.0)
        return int(round(int(vals["dram_bytes_per_launch"]) * scale))
    except (KeyError, ValueError, SyntaxError, TypeError, ZeroDivisionError):
        return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


WORKLOADS = {
    "orbit": dict(scene="object_orbit", n_flow=1, normals=1, want_pose=True,
                  desc="object orbit: 16 views 320x240 (f=320) on a radius-4 ring, K=100 Gaussians, "
                       "depth+alpha+normal planes, flow to the next view, backward w.r.t. means, Cholesky "
                       "factors, weights and poses"),
    "single": dict(scene="single_view", n_flow=0, normals=0, want_pose=False,
                   desc="single view 64x64 (f=64), camera at distance 4, K=40 Gaussians, depth+alpha planes, "
                        "backward w.r.t. means, Cholesky factors and weights"),
    "ragged": dict(scene="ragged_batch", n_flow=0, normals=1, want_pose=True,
                   desc="ragged batch: 64 objects, K ~ U{20..400}, square images of side in {64,128,256,512} "
                        "(f = side), 4 sphere views each (256 views), depth+alpha+normal planes, backward "
                        "w.r.t. all Gaussian parameters and poses"),
    "recon": dict(scene="reconstruction", n_flow=2, normals=0, want_pose=False,
                  desc="reconstruction workload: 100 sphere views 640x480 (f=640), K=256 Gaussians, "
                       "depth+alpha planes, flow to the next and the previous view, backward w.r.t. means, "
                       "Cholesky factors and weights"),
    "minibatch": dict(scene="reconstruction", n_flow=2, normals=0, want_pose=False, rays=50000,
                      desc="ray minibatch: 50 000 rays drawn uniformly across the 100 sphere views 640x480 (f=640) "
                           "of the reconstruction workload, K=256, depth+alpha planes, flow to the next and the "
                           "previous view, backward w.r.t. means, Cholesky factors and weights"),
    "largek": dict(scene="large_k", n_flow=1, normals=1, want_pose=True,
                   desc="large-K stress: 8 sphere views 1024x768 (f=1024), K=4096 diagonal-precision Gaussians, "
                        "all four planes, backward w.r.t. Gaussians and poses"),
}


def scene_and_inputs(seed=0, workload="orbit", views=None):
    """The workload's seeded scene and upstream gradients; ``views``: keep only the
    first that many views (a smaller case of the same kernels, for profiling)."""
    from paper_2308_14737_gb300 import synth

    wl = WORKLOADS[workload]
    s = synth.SCENES[wl["scene"]](seed=seed)
    if views:
        objs = [(s.means[s.object_slice(o)], s.chol[s.object_slice(o)], s.weights[s.object_slice(o)])
                for o in range(s.n_objects)]
        s = synth.make_scene(objs, [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views[:views]],
                             s.poses, name=s.name + f"_first{views}")
    if wl.get("rays"):
        s = synth.ray_batch(s, wl["rays"], seed=seed)
    rng = np.random.default_rng(seed + 1)
    nf = max(wl["n_flow"], 1)
    gd, ga, gn, gf = synth.upstream_grads(rng, s.n_pixels, nf)
    ups = dict(g_depth=gd, g_alpha=ga, g_normal=gn.reshape(-1) if wl["normals"] else None,
               g_flow=gf.reshape(-1) if wl["n_flow"] else None)
    return s, ups


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, val in zip(names, p[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(s, wl, variant="two-param"):
    """The `config` object of a workload: what it renders and its shape (the same
    object in both arms of the benchmark)."""
    if wl.get("rays"):
        c = {"workload": wl["desc"], "views": len(s.views), "rays": s.n_pixels, "width": s.views[0]["W"],
             "height": s.views[0]["H"], "K": s.K(0)}
    else:
        sizes = sorted({(v["W"], v["H"]) for v in s.views})
        Ks = sorted({s.K(v["object"]) for v in s.views})
        c = {"workload": wl["desc"], "views": len(s.views)}
        if len(sizes) == 1:
            c.update(width=sizes[0][0], height=sizes[0][1])
        else:
            c.update(sizes=f"{len(sizes)} sizes from {sizes[0][0]}x{sizes[0][1]} to {sizes[-1][0]}x{sizes[-1][1]}")
        c["K"] = Ks[0] if len(Ks) == 1 else f"{len(Ks)} values from {Ks[0]} to {Ks[-1]}"
    c["variant"] = "alpha compositing (Eq. 9-10)" if variant == "ac" else "two-parameter model (Eq. 7)"
    c["pairs_per_step"] = s.n_pairs
    c["l2"] = "flushed between timed steps (256 MiB write, outside the timed events)"
    return c


def measure_workload(args, name, steps, warmup, dev, ws=1, extras=True, cpu=True):
    """Measures one configuration: the batched arm (one call per pass for all
    views, autotuned tiles, the step's two calls replayed from one CUDA graph; each
    call also from a graph of its own for the forward / backward split) timed per
    step with CUDA events, the plain arm (one forward and one backward call per view),
    the host-fed end-to-end rate, the roofline fractions and, with ``cpu``, the
    oracle on a bounded sample with the parity of the GPU result there.  Returns a
    dict (rates are this rank's; the caller aggregates over ranks)."""
    import torch

    from paper_2308_14737_gb300 import autotune, fmb, synth

    wl = WORKLOADS[name]
    nf, want_pose = wl["n_flow"], wl["want_pose"]
    s, ups = scene_and_inputs(workload=name, views=getattr(args, "views", None) if name == args.workload else None)
    pairs = s.n_pairs
    T = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    means, chol, weights, poses = T(s.means), T(s.chol), T(s.weights), T(s.poses)
    gd, ga, gn, gf = (T(ups[k]) for k in ("g_depth", "g_alpha", "g_normal", "g_flow"))
    ac = args.variant == "ac"
    # alpha compositing: the forward keeps each ray's depth order for the backward (both arms)
    params = fmb.default_params(n_flow=nf, want_normals=wl["normals"], variant=1 if ac else 0,
                                keep_order=1 if ac else 0)
    batched = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params, device=dev)
    G = means.shape[0]
    grads = dict(means=torch.empty(G, 3, device=dev), chol=torch.empty(G, 6, device=dev),
                 weights=torch.empty(G, device=dev),
                 poses=torch.empty(len(s.poses), 12, device=dev) if want_pose else None)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    # Like the paper's losses (Sec. 4), weight the depth, normal and flow upstream
    # gradients by the object mask: here the rendered alpha >= 1e-2.
    # The normal gradient is also weighted by |N| >= 0.05 (normal quality): the
    # renormalised blended normal is ill-conditioned where per-Gaussian normals
    # cancel.
    batched.forward(means, chol, weights, poses)
    m = (batched.alpha >= 1e-2).float()
    gd.mul_(m)
    for v in s.views:
        o, P = v["pix_offset"], synth.view_entries(v)
        if gn is not None:
            mn = m[o:o + P] * (batched.saved[3 * o + 2 * P:3 * o + 3 * P] >= 0.05).float()
            gn[3 * o:3 * (o + P)].view(3, P).mul_(mn)
        if gf is not None:
            gf[2 * nf * o:2 * nf * (o + P)].view(2 * nf, P).mul_(m[o:o + P])
    for k, t in (("g_depth", gd), ("g_normal", gn), ("g_flow", gf)):
        ups[k] = None if t is None else t.cpu().numpy()

    # Batched arm: tiles chosen by the autotuner (before the timed region), forward and
    # backward each replayed from a CUDA graph.
    tuned_params, _ = autotune.tune(
        s.obj_offsets, s.views, len(s.poses), params, means, chol, weights, poses,
        dict(g_depth=gd, g_alpha=ga, g_normal=gn, g_flow=gf), want_pose=want_pose,
        candidates=autotune.CANDIDATES_AC if ac else None,
        cache_path=os.environ.get("FMB_AUTOTUNE_CACHE") or
        os.path.join(tempfile.gettempdir(), f"fmb_autotune_{os.getpid()}.json"))
    batched = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), tuned_params, device=dev)
    ksplit = fmb.fmb_forward_ksplit(tuned_params, s.obj_offsets, batched.c_views)
    launches = (fmb.fmb_launch_count(tuned_params, s.obj_offsets, batched.c_views, backward=False) +
                fmb.fmb_launch_count(tuned_params, s.obj_offsets, batched.c_views, backward=True,
                                     want_pose=want_pose))
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(2):
            batched.forward(means, chol, weights, poses)
            batched.backward(means, chol, weights, poses, gd, ga, gn, gf, want_pose=want_pose, out=grads)
    torch.cuda.current_stream(dev).wait_stream(side)
    # the step (forward and backward) as one graph, as a training loop replays it; each
    # call in a graph of its own for the forward / backward split
    graph_s, graph_f, graph_b = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_s):
        batched.forward(means, chol, weights, poses)
        batched.backward(means, chol, weights, poses, gd, ga, gn, gf, want_pose=want_pose, out=grads)
    with torch.cuda.graph(graph_f):
        batched.forward(means, chol, weights, poses)
    with torch.cuda.graph(graph_b):
        batched.backward(means, chol, weights, poses, gd, ga, gn, gf, want_pose=want_pose, out=grads)

    # plain arm: one forward and one backward call per view (default tiles, no graph)
    plain = []
    for v in s.views:
        vv = dict(v, pix_offset=0)  # each single-view renderer owns its own planes
        plain.append((fmb.Renderer(s.obj_offsets, [vv], len(s.poses), params, device=dev), v["pix_offset"],
                      synth.view_entries(v)))

    # per-view gradient buffers, summed over the views after the calls (as a caller of
    # per-view launches has to)
    pgrads = [{k: None if v is None else torch.empty_like(v) for k, v in grads.items()} for _ in plain]
    psum = {k: torch.empty_like(v) for k, v in grads.items() if v is not None}
    sl = lambda t, c, o, P: None if t is None else t[c * o:c * (o + P)]

    def plain_step():
        for (r, o, P), g in zip(plain, pgrads):
            r.forward(means, chol, weights, poses)
            r.backward(means, chol, weights, poses, gd[o:o + P], ga[o:o + P], sl(gn, 3, o, P),
                       sl(gf, 2 * nf, o, P), want_pose=want_pose, out=g)
        for k in psum:
            torch.sum(torch.stack([g[k] for g in pgrads]), dim=0, out=psum[k])

    def timed(fn, n_steps, n_warm, split=False):
        for _ in range(n_warm):
            if split:
                graph_f.replay()
                graph_b.replay()
            else:
                fn()
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(n_steps):
            flush.zero_()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            if split:
                graph_f.replay()
                e1.record(stream)
                graph_b.replay()
            else:
                fn()
                e1.record(stream)
            e2.record(stream)
            evs.append((e0, e1, e2))
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        tot = sum(a.elapsed_time(c) for a, b, c in evs)
        fwd = sum(a.elapsed_time(b) for a, b, c in evs)
        bwd = sum(b.elapsed_time(c) for a, b, c in evs)
        return tot, fwd, bwd

    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        t_b, _, _ = timed(graph_s.replay, steps, warmup)
        _, t_f, t_bw = timed(None, steps, warmup, split=True)
    clocks = clk.summary()
    plain_steps = max(steps // 4, 3)
    t_p, _, _ = timed(plain_step, plain_steps, max(warmup, 3))
    assert fmb.fmb_read_device_status(batched.ws) == 0

    ms_step = t_b / steps
    ms_plain = t_p / plain_steps
    if ws > 1:
        import torch.distributed as dist

        x = torch.tensor([ms_step, ms_plain], device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)  # the slowest rank sets the whole job's time
        ms_step, ms_plain = float(x[0]), float(x[1])
    fwd_ms, bwd_ms = t_f / steps, t_bw / steps
    value = ws * pairs / (ms_step * 1e-3)

    # e2e: through the public API with host buffers (pinned), copies inside the timed region;
    # every rank runs it (replicas), the slowest rank's step time sets the whole-job rate
    if ws > 1:
        torch.distributed.barrier()
    e2e = e2e_measure(args, name, s, ups, tuned_params, dev)
    if ws > 1:
        x = torch.tensor([e2e["ms_per_step"]], device=dev)
        torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
        e2e["ms_per_step"] = float(x[0])
        e2e["value"] = ws * pairs / (e2e["ms_per_step"] * 1e-3)
        e2e["h2d_bytes_per_step"] *= ws
        e2e["d2h_bytes_per_step"] *= ws

    clock_for_peak = 2070.0
    peak = peak_fp32_gops(clock_for_peak)
    f32f, mf, f32b, mb = (OPS_AC if ac else OPS)[bool(wl["normals"])]
    if not ac and not want_pose:
        f32b -= NO_POSE_SAVING
    roofline = {
        "bound": "alu",
        "kernel": ("backward_ac_kernel" if ac else "backward_kernel") + " (fmb_render_backward call)",
        "achieved": pairs * f32b / (bwd_ms * 1e-3) / 1e9,
        "peak": peak,
        "unit": "G FP32 lane-ops/s",
        "frac": None,
        "traffic": None,
        "per_pair_ops": {"fwd_fp32": f32f, "fwd_mufu": mf, "bwd_fp32": f32b, "bwd_mufu": mb},
        "peak_basis": "152 SMs x 128 FP32 lanes x 2070 MHz max SM clock (an FMA counts as one operation; "
                      "the nominal issue bound, above the probe's measured FFMA2 rate); the MUFU pipe is the "
                      "lesser bound (mufu_busy_frac, from the probe's measured MUFU rates)",
        "mufu_busy_frac": mufu_busy_frac(pairs / (bwd_ms * 1e-3), clock_for_peak, wl["normals"]),
        "forward": {"achieved": pairs * f32f / (fwd_ms * 1e-3) / 1e9,
                    "frac": pairs * f32f / (fwd_ms * 1e-3) / 1e9 / peak},
        "step_frac": pairs * (f32f + f32b) / (ms_step * 1e-3) / 1e9 / peak,
    }
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    if not ac:
        # the same times against the method's own operations only (the compensated
        # geometry's extra operations left out of the count)
        cf, cb = ALGO_OPS[bool(wl["normals"])]
        if not want_pose:
            cb -= NO_POSE_SAVING
        roofline["method_ops_only"] = {
            "bwd_fp32": cb, "fwd_fp32": cf,
            "frac": pairs * cb / (bwd_ms * 1e-3) / 1e9 / peak,
            "forward_frac": pairs * cf / (fwd_ms * 1e-3) / 1e9 / peak,
            "step_frac": pairs * (cf + cb) / (ms_step * 1e-3) / 1e9 / peak}
    # the committed ncu summaries cover the two-parameter backward on the orbit and large-K workloads
    roofline["traffic"] = (profiled_traffic({k: int(getattr(tuned_params, k)) for k in autotune.TUNED_FIELDS},
                                            workload=name)
                           if not ac and not getattr(args, "views", None) else None)
    rec = {
        "workload": name,
        "config": workload_config(s, wl, args.variant),
        "value": value,
        "unit": "pairs/s",
        "ms_per_step": ms_step,
        "steps": steps,
        "warmup": warmup,
        "fwd_ms": fwd_ms,
        "bwd_ms": bwd_ms,
        "plain": {"value": ws * pairs / (ms_plain * 1e-3), "ms_per_step": ms_plain, "steps": plain_steps,
                  "launch": "one forward and one backward call per view, default tiles, no graph"},
        "batched_over_plain": ms_plain / ms_step,
        "frames_per_s": ws * len(s.views) / (ms_step * 1e-3),
        "launch": {"batched": "one forward and one backward call for all views, autotuned tiles, the step "
                              "replayed from one CUDA graph (fwd_ms / bwd_ms: each call from a graph of its own)",
                   "tiles": {k: int(getattr(tuned_params, k)) for k in autotune.TUNED_FIELDS},
                   "fwd_ksplit": ksplit, "kernel_launches_per_step": launches},
        "roofline": roofline,
        "clocks": clocks,
        "e2e": e2e,
    }
    if extras and args.points:
        rec["points_export"] = timed_call(lambda: batched.points(means, chol, weights, poses), steps, dev, pairs,
                                          "points, normals at the rendered depth, Eq. 16 screen normals and the "
                                          "max-weight quality of every pixel (fmb_render_points)")
    if extras and args.attribution:
        ray_loss = gd.abs()  # the per-ray loss: the magnitude of the synthetic upstream depth gradient
        att = torch.empty(G, dtype=torch.float32, device=dev)
        rec["loss_attribution"] = timed_call(
            lambda: batched.attribution(means, chol, weights, poses, ray_loss, out=att), steps, dev, pairs,
            "per-Gaussian sum of ray loss x normalised weight over every ray of the batch "
            "(fmb_loss_attribution, Sec. 8 splitting criterion)")
    if extras and (name == "recon" or args.stored):
        rec["stored_vs_recompute"] = stored_adjoint_measure(args, name, s, (gd, ga, gn, gf), tuned_params, dev)
    if extras and name == "recon":
        rec["recon_step"] = recon_step_measure(args, name, s, dev)
    if cpu:
        rec["plain_vs_batched_grad_max_rel"] = {
            k: float((psum[k] - grads[k]).abs().max() / grads[k].abs().max()) for k in psum}
        rec["cpu_baseline"] = cpu_baseline(name, s, batched, (means, chol, weights, poses), want_pose, args)
    del plain, pgrads, graph_s, graph_f, graph_b, batched, flush
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    return rec


def timed_call(fn, steps, dev, pairs, what):
    """A call timed alone after three warm-up calls: mean of max(steps / 4, 3)."""
    import torch

    for _ in range(3):
        fn()
    torch.cuda.synchronize(dev)
    n = max(steps // 4, 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        fn()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / n
    return {"ms": ms, "value": pairs / (ms * 1e-3), "unit": "pairs/s", "steps": n, "what": what}


def run_gpu(args):
    import torch

    from paper_2308_14737_gb300 import fmb

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    fmb.load_library()

    head = measure_workload(args, args.workload, args.steps, args.warmup, dev, ws=ws,
                            cpu=(ws == 1 and not args.no_cpu_baseline))
    subs = {}
    if ws == 1 and args.configs == "all" and args.variant == "two-param":
        for name in SUB_CONFIGS:
            if name == args.workload:
                continue
            subs[name] = measure_workload(args, name, max(args.steps, SUB_STEPS[name]), args.warmup, dev,
                                          cpu=not args.no_cpu_baseline)
    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": "pairs/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded; stands in for the paper's CO3D sequences)",
        "config": dict(head["config"], parallelism="replicas" if ws > 1 else "single GPU"),
        "launch": head["launch"],
        "plain": head["plain"],
        "batched_over_plain": head["batched_over_plain"],
        "fwd_ms": head["fwd_ms"],
        "bwd_ms": head["bwd_ms"],
        "frames_per_s": head["frames_per_s"],
        "paper_context": paper_context(args.variant),
        "roofline": head["roofline"],
        "clocks": head["clocks"],
        # the library's own count of its launches per forward + backward call, times the timed steps
        "gpu_launches": head["launch"]["kernel_launches_per_step"] * args.steps,
        "e2e": head["e2e"],
    }
    for k in ("points_export", "loss_attribution", "stored_vs_recompute", "recon_step",
              "plain_vs_batched_grad_max_rel", "cpu_baseline"):
        if k in head:
            line[k] = head[k]
    if subs:
        line["configs"] = subs
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def stored_adjoint_measure(args, name, s, ups_dev, tuned_params, dev):
    """Recompute-adjoint versus stored-intermediate adjoint on the same batch and
    tiles: the stored variant's forward also writes 12 bytes per pair (t, log2
    weight, density) into its workspace and its backward reads them.  Both arms are
    timed the same way (plain calls, CUDA events, L2 flushed between steps)."""
    import torch

    from paper_2308_14737_gb300 import autotune, fmb

    wl = WORKLOADS[name]
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    m, c, w, po = T(s.means), T(s.chol), T(s.weights), T(s.poses)
    gd, ga, gn, gf = ups_dev
    G = m.shape[0]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    n = max(args.steps // 4, 3)
    res, grads = {}, {}
    for arm, store in (("recompute", 0), ("stored", 1)):
        p = autotune.apply(tuned_params, {})
        p.store_pairs = store
        p.fwd_rays_per_thread = 2
        r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), p, device=dev)
        out = dict(means=torch.empty(G, 3, device=dev), chol=torch.empty(G, 6, device=dev),
                   weights=torch.empty(G, device=dev),
                   poses=torch.empty(len(s.poses), 12, device=dev) if wl["want_pose"] else None)
        for _ in range(3):
            r.forward(m, c, w, po)
            r.backward(m, c, w, po, gd, ga, gn, gf, want_pose=wl["want_pose"], out=out)
        torch.cuda.synchronize(dev)
        tf = tb = 0.0
        for _ in range(n):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record()
            r.forward(m, c, w, po)
            e[1].record()
            r.backward(m, c, w, po, gd, ga, gn, gf, want_pose=wl["want_pose"], out=out)
            e[2].record()
            torch.cuda.synchronize(dev)
            tf += e[0].elapsed_time(e[1])
            tb += e[1].elapsed_time(e[2])
        tf, tb = tf / n, tb / n
        res[arm] = {"fwd_ms": tf, "bwd_ms": tb, "value": s.n_pairs / ((tf + tb) * 1e-3), "unit": "pairs/s",
                    "workspace_bytes": int(r.ws.numel() * r.ws.element_size())}
        grads[arm] = out
        del r
        torch.cuda.empty_cache()
    res["stored"]["per_pair_bytes"] = 12
    res["recompute"]["saved_bytes_per_pixel"] = 12
    res["grad_max_rel_diff"] = {k: float((grads["stored"][k] - grads["recompute"][k]).abs().max() /
                                         grads["recompute"][k].abs().max())
                                for k in grads["stored"] if grads["stored"][k] is not None}
    res["steps"] = n
    res["timing"] = "plain calls (no graph) with the autotuned tiles, CUDA events, L2 flushed between steps"
    return res


def recon_step_measure(args, name, s, dev):
    """The full reconstruction step (render, loss, adjoint, fused Adam, replayed
    from one CUDA graph) on the reconstruction workload.  The target planes are
    rendered by the same GPU renderer from a second seed's Gaussians seen by the
    same cameras."""
    import torch

    from paper_2308_14737_gb300 import fmb, synth
    from paper_2308_14737_gb300.step import ReconstructionStep

    nf = WORKLOADS[name]["n_flow"]
    params = fmb.default_params(n_flow=nf, want_normals=0)
    tgt_obj = synth.random_gaussians(np.random.default_rng(1), s.K(0), "cholesky")
    ts = synth.make_scene([tgt_obj], [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views],
                          s.poses)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    r = fmb.Renderer(ts.obj_offsets, ts.views, len(ts.poses), params, device=dev)
    out = r.forward(T(ts.means), T(ts.chol), T(ts.weights), T(ts.poses))
    targets = {k: out[k].cpu().numpy() for k in ("depth", "alpha", "flow")}
    del r, out
    st = ReconstructionStep(s, targets, params=params, lr=1e-2, device=dev)
    st.capture(warmup=2)
    for _ in range(3):
        st.replay()
    torch.cuda.synchronize(dev)
    loss0 = float(st.loss)
    n = max(args.steps // 20, 5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        st.replay()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / n
    return {"ms_per_step": ms, "value": s.n_pairs / (ms * 1e-3), "unit": "pairs/s", "steps": n,
            "loss_first": loss0, "loss_last": float(st.loss),
            "what": "forward, L1 depth + BCE alpha + L2 flow loss, backward, Adam (lr 1e-2), one CUDA graph; "
                    "targets rendered by the GPU renderer from a second seed"}


def e2e_measure(args, name, s, ups, params, dev):
    """Same metric through the public host-fed API (``pipeline.HostPipeline``) with
    pinned host buffers: every step copies its inputs (scene, poses, upstream
    gradient planes) host -> device and its results (depth, alpha, normal, flow
    planes and all gradients) device -> host inside the timed region, overlapped with
    the neighbouring steps' kernels.  Two modes of the API: ``submit`` (any host
    tensors each step; a launch per copy) and the fixed-buffer graphs
    (``capture_fixed`` / ``submit_fixed``: each buffer set's copies in and out
    replayed as graphs, around the render's graph, on the same three streams).  ``value`` is the fixed-buffer mode's; both
    modes' last steps are checked against a plain device call."""
    import torch

    from paper_2308_14737_gb300 import fmb, pipeline

    want_pose = WORKLOADS[name]["want_pose"]
    pin = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).pin_memory()
    h_in = dict(means=pin(s.means), chol=pin(s.chol), weights=pin(s.weights), poses=pin(s.poses),
                g_depth=pin(ups["g_depth"]), g_alpha=pin(ups["g_alpha"]), g_normal=pin(ups["g_normal"]),
                g_flow=pin(ups["g_flow"]))
    pipe = pipeline.HostPipeline(s.obj_offsets, s.views, len(s.poses), params, h_in, want_pose=want_pose, device=dev)
    h_outs = [pipe.host_outputs(), pipe.host_outputs()]
    h2d = sum(h.numel() * 4 for h in h_in.values() if h is not None)
    d2h = sum(o.numel() * 4 for o in h_outs[0].values())
    # at least 20 steps: the pipeline's fill (the first step's inputs in) and drain
    # (the last step's results out) are paid once per timed run, as in a training loop
    n = max(args.steps, 20)
    cur = torch.cuda.current_stream(dev)

    def timed(step, streams):
        for _ in range(4):
            step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        for st in streams:
            st.wait_stream(cur)
        for _ in range(n):
            step()
        for st in streams:
            cur.wait_stream(st)
        e1.record(cur)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    k_call = [0]

    def call_step():
        pipe.submit(h_in, h_outs[k_call[0] % 2])
        k_call[0] += 1

    ms_call = timed(call_step, pipe.streams())
    got_call = {k: v.clone() for k, v in h_outs[(k_call[0] - 1) % 2].items()}
    h_fixed = [pipe.host_outputs(), pipe.host_outputs()]
    pipe.capture_fixed(h_in, h_fixed)
    ms_fixed = timed(pipe.submit_fixed, pipe.streams())
    got_fixed = h_fixed[(pipe.i_fixed - 1) % 2]

    # the last step's host results against a plain device-resident call on the same
    # inputs: planes bitwise, gradients up to the order of fp32 atomic additions
    d = {k: None if v is None else v.to(dev) for k, v in h_in.items()}
    r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params, device=dev)
    out = r.forward(d["means"], d["chol"], d["weights"], d["poses"])
    g = r.backward(d["means"], d["chol"], d["weights"], d["poses"], d["g_depth"], d["g_alpha"], d["g_normal"],
                   d["g_flow"], want_pose=want_pose)
    want = dict(depth=out["depth"], alpha=out["alpha"], normal=out["normal"], flow=out["flow"],
                grad_means=g["means"], grad_chol=g["chol"], grad_weights=g["weights"], grad_poses=g["poses"])
    for mode, got in (("submit", got_call), ("fixed-buffer", got_fixed)):
        for k, v in want.items():
            if v is None:
                continue
            a, b = got[k].reshape(-1), v.reshape(-1).cpu()
            ok = torch.equal(a, b) if not k.startswith("grad") else \
                bool((a - b).abs().max() <= 1e-5 * float(b.abs().max()) + 1e-30)
            if not ok:
                raise RuntimeError(f"host-fed pipeline ({mode}) result {k} differs from the plain call's")
    return {"value": s.n_pairs / (ms_fixed * 1e-3), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms_fixed, "steps": n,
            "per_call_submit": {"value": s.n_pairs / (ms_call * 1e-3), "ms_per_step": ms_call, "steps": n},
            "parity": "both modes' last step's host results vs a plain device call: planes bitwise, gradients "
                      "within 1e-5 of the largest entry",
            "api": "pipeline.HostPipeline, two device buffer sets, three streams (copies in, forward + backward, "
                   "copies out) overlapped across steps; with fixed pinned host buffers (capture_fixed / "
                   "submit_fixed) each set's copies in and copies out are CUDA graphs too (three graph launches "
                   "per step); per_call_submit: submit() with a launch per copy"}


def cpu_model() -> str:
    """The host CPU's model name as /proc/cpuinfo gives it (x86: "model name";
    Arm: implementer and part numbers), or the platform string."""
    import platform

    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.processor() or platform.machine()
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    fields = {}
    for line in info:
        if ":" in line:
            k, v = (x.strip() for x in line.split(":", 1))
            fields.setdefault(k, v)
    if "CPU part" in fields:
        # Arm's published part numbers for the server cores this may run on
        known = {"0xd4f": "Neoverse-V2", "0xd40": "Neoverse-V1", "0xd0c": "Neoverse-N1", "0xd49": "Neoverse-N2",
                 "0xd8e": "Neoverse-N3", "0xd84": "Neoverse-V3"}
        part = fields["CPU part"].lower()
        name = known.get(part, f"part {part}") if fields.get("CPU implementer", "").lower() == "0x41" else part
        return f"{platform.machine()} {name} (implementer {fields.get('CPU implementer', '?')}, part {part})"
    return platform.machine()


def oracle_single_thread(name, s, args):
    """The oracle on one thread over a small sample (the central 64x48 crop of the
    first view), forward + backward, in pairs/s."""
    import oracle

    from paper_2308_14737_gb300 import synth

    wl = WORKLOADS[name]
    nf = wl["n_flow"]
    v0 = {k: v for k, v in s.views[0].items() if k != "pix_offset"}
    first = synth.make_scene([(s.means[s.object_slice(v0["object"])], s.chol[s.object_slice(v0["object"])],
                               s.weights[s.object_slice(v0["object"])])], [dict(v0, object=0)], s.poses)
    sub = synth.crop_views(first, 64, 48) if v0.get("rays") is None else first
    gd, ga, gn, gf = synth.upstream_grads(np.random.default_rng(7), sub.n_pixels, max(nf, 1))
    var = 1 if args.variant == "ac" else 0
    t0 = time.perf_counter()
    oracle.render_scene(sub, n_flow=nf, variant=var, n_threads=1)
    oracle.backward_scene(sub, gd, ga, gn.reshape(-1) if wl["normals"] else None, gf.reshape(-1) if nf else None,
                          n_flow=nf, variant=var, n_threads=1)
    dt = time.perf_counter() - t0
    return {"value": sub.n_pairs / dt, "unit": "pairs/s", "threads": 1,
            "sample": f"{sub.n_pixels} rays of the first view x K={sub.means.shape[0]}, forward + backward"}


def oracle_sample(workload, s):
    """Bounded sample of a workload for the oracle: two of the orbit's views, the
    whole single view or ray batch, else the central 64x48 crop of every view.
    Returns (sample scene, [(view index in s, the view's pixel indices)] per sample
    view, text)."""
    from paper_2308_14737_gb300 import synth

    if workload == "orbit":
        sub = synth.make_scene([(s.means, s.chol, s.weights)],
                               [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views[:2]], s.poses)
        pick = [(i, np.arange(s.views[i]["W"] * s.views[i]["H"])) for i in range(2)]
        return sub, pick, "2 of the 16 views (320x240, K=100)"
    if workload in ("single", "minibatch"):
        pick = [(i, np.arange(synth.view_entries(v))) for i, v in enumerate(s.views)]
        what = {"single": "the whole view", "minibatch": f"the whole batch of {s.n_pixels} rays"}[workload]
        return s, pick, what
    cw, ch = 64, 48
    sub = synth.crop_views(s, cw, ch)
    pick = []
    yy, xx = np.meshgrid(np.arange(ch), np.arange(cw), indexing="ij")
    for i, v in enumerate(s.views):
        x0, y0 = (v["W"] - cw) // 2, (v["H"] - ch) // 2
        pick.append((i, ((y0 + yy) * v["W"] + (x0 + xx)).reshape(-1)))
    return sub, pick, f"the central 64x48 crop of all {len(s.views)} views"


def sample_upstream(sub, ref, n_flow, normals, seed=7):
    """Random upstream gradients over the sample, masked like the paper's losses:
    depth, normal and flow where the oracle's alpha >= 1e-2, the normal also where
    its blended-normal magnitude |N| >= 0.05 (where the renormalisation is
    well-conditioned)."""
    from paper_2308_14737_gb300 import synth

    gd, ga, gn, gf = synth.upstream_grads(np.random.default_rng(seed), sub.n_pixels, max(n_flow, 1))
    m = (ref["alpha"] >= 1e-2).astype(np.float32)
    gd = gd * m
    gn_b = np.zeros(3 * sub.n_pixels, dtype=np.float32)
    gf_b = np.zeros(2 * max(n_flow, 1) * sub.n_pixels, dtype=np.float32)
    for v in sub.views:
        o, P = v["pix_offset"], synth.view_entries(v)
        nn = ref["saved"][3 * o + 2 * P:3 * o + 3 * P]
        gn_b[3 * o:3 * (o + P)] = (gn[:, o:o + P] * (m[o:o + P] * (nn >= 0.05))).reshape(-1)
        if n_flow:
            gf_b[2 * n_flow * o:2 * n_flow * (o + P)] = (gf[:n_flow, :, o:o + P] * m[o:o + P]).reshape(-1)
    return dict(g_depth=gd, g_alpha=ga, g_normal=gn_b if normals else None, g_flow=gf_b if n_flow else None)


def _gather(full, s, sub, pick, ch):
    """The sample's entries of a batched GPU plane with ``ch`` channels per view,
    in the sample's batched layout."""
    out = np.zeros(ch * sub.n_pixels)
    for (fi, pix), sv in zip(pick, sub.views):
        fv = s.views[fi]
        Pf, Ps, of, os_ = fv["W"] * fv["H"] if fv.get("rays") is None else len(fv["rays"]), len(pix), \
            fv["pix_offset"], sv["pix_offset"]
        for c in range(ch):
            out[ch * os_ + c * Ps:ch * os_ + (c + 1) * Ps] = full[ch * of + c * Pf + pix]
    return out


def _scatter(vals, s, sub, pick, ch):
    """Inverse of _gather: the sample's entries placed into a zero batched plane."""
    out = np.zeros(ch * s.n_pixels, dtype=np.float32)
    for (fi, pix), sv in zip(pick, sub.views):
        fv = s.views[fi]
        Pf, Ps, of, os_ = fv["W"] * fv["H"] if fv.get("rays") is None else len(fv["rays"]), len(pix), \
            fv["pix_offset"], sv["pix_offset"]
        for c in range(ch):
            out[ch * of + c * Pf + pix] = vals[ch * os_ + c * Ps:ch * os_ + (c + 1) * Ps]
    return out


def cpu_baseline(name, s, renderer, dev_scene, want_pose, args):
    """The FP64 oracle (test infrastructure, not tuned) timed on the host cores on a
    bounded sample of the workload (forward, then backward from masked random
    upstream gradients), and the parity of the GPU result on the same sample: the
    timed forward's planes at the sample's pixels, and the gradients of one more
    GPU backward call whose upstream gradients are those of the sample (zero
    elsewhere), against the oracle's."""
    import oracle
    import torch

    oracle.build()
    wl = WORKLOADS[name]
    nf, normals = wl["n_flow"], bool(wl["normals"])
    var = 1 if args.variant == "ac" else 0
    sub, pick, what = oracle_sample(name, s)
    t0 = time.perf_counter()
    ref = oracle.render_scene(sub, n_flow=nf, variant=var)
    t_f = time.perf_counter() - t0
    u = sample_upstream(sub, ref, nf, normals)
    t0 = time.perf_counter()
    refg = oracle.backward_scene(sub, u["g_depth"], u["g_alpha"], u["g_normal"], u["g_flow"], n_flow=nf, variant=var)
    t_b = time.perf_counter() - t0
    out = {"value": sub.n_pairs / (t_f + t_b), "unit": "pairs/s", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": what + ", forward + backward (FP64, OpenMP over pixels)", "pairs": sub.n_pairs,
           "seconds": t_f + t_b, "cpu_model": cpu_model(), "single_thread": oracle_single_thread(name, s, args)}
    # parity of the GPU result on the sample
    torch.cuda.synchronize()
    g = lambda t, ch: _gather(t.cpu().numpy().astype(np.float64), s, sub, pick, ch)
    ra, rd = ref["alpha"], ref["depth"]
    ga, gd = g(renderer.alpha, 1), g(renderer.depth, 1)
    mask = ra >= 1e-2
    tol = lambda r: 1e-4 + 1e-5 * np.abs(r)
    par = {"alpha_max_abs": float(np.max(np.abs(ga - ra))),
           "alpha_within_tol": bool(np.all(np.abs(ga - ra) <= tol(ra)))}
    if var == 0:
        ed = np.abs(gd - rd)[mask]
        par.update(depth_max_abs=float(ed.max()) if ed.size else 0.0,
                   depth_within_tol=bool(np.all(ed <= tol(rd[mask]))))
        if normals:
            gn = g(renderer.normal, 3).reshape(-1)
            en = np.zeros(sub.n_pixels)
            nn = np.zeros(sub.n_pixels)
            for v in sub.views:
                o, P = v["pix_offset"], v["W"] * v["H"] if v.get("rays") is None else len(v["rays"])
                en[o:o + P] = np.abs(gn[3 * o:3 * (o + P)] - ref["normal"][3 * o:3 * (o + P)]).reshape(3, P).max(0)
                nn[o:o + P] = ref["saved"][3 * o + 2 * P:3 * o + 3 * P]
            ratio = (en * np.maximum(nn, 0.05) / 1e-4)[mask]
            par.update(normal_max_abs=float(en[mask].max()) if mask.any() else 0.0,
                       normal_tol_ratio=float(ratio.max()) if ratio.size else 0.0)
        if nf:
            gfl = g(renderer.flow, 2 * nf)
            ef = np.zeros(sub.n_pixels)
            for v in sub.views:
                o, P = v["pix_offset"], v["W"] * v["H"] if v.get("rays") is None else len(v["rays"])
                blk = np.abs(gfl[2 * nf * o:2 * nf * (o + P)] - ref["flow"][2 * nf * o:2 * nf * (o + P)])
                ef[o:o + P] = blk.reshape(2 * nf, P).max(0)
            par["flow_max_abs_px"] = float(ef[mask].max()) if mask.any() else 0.0
    else:
        par["note"] = ("alpha compositing: only the order-independent alpha plane is compared here; depth, normal, "
                       "flow and gradients are compared by the parity tests away from fp32 depth-order ties")
    if var == 0:
        dev = dev_scene[0].device
        T = lambda a: None if a is None else torch.as_tensor(a, device=dev)
        full = dict(g_depth=T(_scatter(u["g_depth"], s, sub, pick, 1)), g_alpha=T(_scatter(u["g_alpha"], s, sub,
                                                                                           pick, 1)),
                    g_normal=T(_scatter(u["g_normal"], s, sub, pick, 3)) if normals else None,
                    g_flow=T(_scatter(u["g_flow"], s, sub, pick, 2 * nf)) if nf else None)
        gg = renderer.backward(*dev_scene, full["g_depth"], full["g_alpha"], full["g_normal"], full["g_flow"],
                               want_pose=want_pose)
        torch.cuda.synchronize()
        for k in ("means", "chol", "weights") + (("poses",) if want_pose else ()):
            a = gg[k].cpu().numpy().astype(np.float64).reshape(refg[k].shape)
            par[f"grad_{k}_max_rel"] = float(np.max(np.abs(a - refg[k])) / max(np.max(np.abs(refg[k])), 1e-300))
        par["grads_within_tol"] = all(v <= 1e-4 for k, v in par.items() if k.startswith("grad_"))
        par["note"] = ("upstream depth/normal/flow gradients masked by the oracle's alpha >= 1e-2, the normal "
                       "gradient also by its |N| >= 0.05; tolerances: planes 1e-4 + 1e-5 |ref| (normal "
                       "1e-4 / max(|N|, 0.05): tol_ratio <= 1), gradients 1e-4 of the tensor's max")
    out["parity"] = par
    return out


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same metric, unit and
    config; each step is a bounded sample of the workload (oracle_sample), forward
    and backward."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    wl = WORKLOADS[args.workload]
    s, _ = scene_and_inputs(workload=args.workload)
    sub, _, what = oracle_sample(args.workload, s)
    nf, normals = wl["n_flow"], bool(wl["normals"])
    var = 1 if args.variant == "ac" else 0

    def step():
        ref = oracle.render_scene(sub, n_flow=nf, variant=var)
        u = sample_upstream(sub, ref, nf, normals)
        oracle.backward_scene(sub, u["g_depth"], u["g_alpha"], u["g_normal"], u["g_flow"], n_flow=nf, variant=var)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = sub.n_pairs / dt
    config = dict(workload_config(s, wl, args.variant), parallelism="replicas" if ws > 1 else "single GPU")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": what + ", forward + backward per step", "pairs_per_step": sub.n_pairs},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fmb", choices=["fmb", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--configs", default="all", choices=["all", "none"],
                    help="all: also measure the other configurations (single, orbit, ragged, recon) into 'configs'")
    ap.add_argument("--variant", default="two-param", choices=["two-param", "ac"],
                    help="weights of Eq. 3: the two-parameter model (Eq. 7) or alpha compositing (Eq. 9-10)")
    ap.add_argument("--points", action="store_true", help="also time the oriented point export (Sec. 6)")
    ap.add_argument("--attribution", action="store_true",
                    help="also time the loss attribution of the splitting criterion (Sec. 8)")
    ap.add_argument("--views", type=int, default=None,
                    help="render only the first N views of the headline workload (a smaller case for profiling)")
    ap.add_argument("--stored", action="store_true",
                    help="also time the stored-intermediate adjoint (always on for --workload recon)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
