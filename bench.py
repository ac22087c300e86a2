"""Benchmark of the Fuzzy Metaballs render path: ray-Gaussian pairs/s for one
forward + backward pass over a batch of views, batched versus plain per-view
launches.

Workload (one step): the object-orbit configuration -- 16 views at 320x240
(f = 320) on a radius-4 ring, K = 100 Gaussians, depth + alpha + normal planes,
flow to the next view, and the full backward (means, Cholesky factors, weights,
poses) from random upstream gradients.  Inputs are seeded synthetic data; the
planes (about 50 MB) fit in L2, so L2 is flushed (256 MiB write) between timed
steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The batched arm's tiles come from the autotuner, run before the timed region; set
FMB_AUTOTUNE_CACHE to a file to reuse a previous run's choice (e.g. when
profiling, so the profiled run launches no tuning candidates).

Prints one JSON line.  Under torchrun (N > 1) every rank renders its own replica
of the batch (weak scaling) and rank 0 prints the aggregate.
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
WORKLOAD = ("object orbit: 16 views 320x240 (f=320) on a radius-4 ring, K=100 Gaussians, depth+alpha+normal "
            "planes, flow to the next view, backward w.r.t. means, Cholesky factors, weights and poses")

# Algorithmic per-pair work of the implemented formulation (FP32-pipe ops and
# MUFU ops; counted from the kernels' arithmetic, loads and control excluded).
FWD_FP32, FWD_MUFU = 58, 4
BWD_FP32, BWD_MUFU = 110, 4
N_SM = 152
LANES_PER_SM = 128


def peak_issue_ginstr(clock_mhz: float) -> float:
    """FP32-pipe / issue-slot peak in G lane-instructions per second."""
    return N_SM * LANES_PER_SM * clock_mhz * 1e6 / 1e9


PROFILE = os.path.join(ROOT, "profiles", "backward_kernel_orbit16x320x240_K100.md")


def csrc_sha256() -> str:
    """Hash of the sources that define the backward kernel."""
    import hashlib

    d = os.path.join(ROOT, "paper_2308_14737_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("fmb_backward.cu", "fmb_internal.cuh", "fmb_f32x2.cuh"):
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic():
    """DRAM bytes (read + write) per launch of the backward kernel from the
    committed ncu summary, or None if the kernel sources changed since the capture."""
    try:
        txt = open(PROFILE).read()
    except OSError:
        return None
    vals = dict(line.split(":", 1) for line in txt.splitlines() if line.startswith(("dram_bytes_per_launch",
                                                                                    "source_sha256")))
    sha = next((v for k, v in vals.items() if k.startswith("source_sha256")), "").strip()
    if not sha or sha.split()[-1] != csrc_sha256():
        return None
    try:
        return int(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def scene_and_inputs(seed=0):
    from paper_2308_14737_gb300 import synth

    s = synth.config1(seed=seed)
    rng = np.random.default_rng(seed + 1)
    gd, ga, gn, gf = synth.upstream_grads(rng, s.n_pixels, 1)
    return s, dict(g_depth=gd, g_alpha=ga, g_normal=gn.reshape(-1), g_flow=gf.reshape(-1))


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

    s, ups = scene_and_inputs()
    pairs = s.n_pairs
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    means, chol, weights, poses = T(s.means), T(s.chol), T(s.weights), T(s.poses)
    gd, ga, gn, gf = (T(ups[k]) for k in ("g_depth", "g_alpha", "g_normal", "g_flow"))
    params = fmb.default_params(n_flow=1, want_normals=1)
    batched = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params, device=dev)
    G = means.shape[0]
    grads = dict(means=torch.empty(G, 3, device=dev), chol=torch.empty(G, 6, device=dev),
                 weights=torch.empty(G, device=dev), poses=torch.empty(len(s.poses), 12, device=dev))
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
        o, P = v["pix_offset"], v["W"] * v["H"]
        mn = m[o:o + P] * (batched.saved[3 * o + 2 * P:3 * o + 3 * P] >= 0.05).float()
        gn[3 * o:3 * (o + P)].view(3, P).mul_(mn)
        gf[2 * o:2 * (o + P)].view(2, P).mul_(m[o:o + P])
    for k, t in (("g_depth", gd), ("g_normal", gn), ("g_flow", gf)):
        ups[k] = t.cpu().numpy()

    # Batched arm: tiles chosen by the autotuner (before the timed region), forward and
    # backward each replayed from a CUDA graph.
    from paper_2308_14737_gb300 import autotune

    tuned_params, tune_timings = autotune.tune(
        s.obj_offsets, s.views, len(s.poses), params, means, chol, weights, poses,
        dict(g_depth=gd, g_alpha=ga, g_normal=gn, g_flow=gf), want_pose=True,
        cache_path=os.environ.get("FMB_AUTOTUNE_CACHE") or
        os.path.join(tempfile.gettempdir(), f"fmb_autotune_{os.getpid()}.json"))
    batched = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), tuned_params, device=dev)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for _ in range(2):
            batched.forward(means, chol, weights, poses)
            batched.backward(means, chol, weights, poses, gd, ga, gn, gf, out=grads)
    torch.cuda.current_stream(dev).wait_stream(side)
    graph_f, graph_b = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph_f):
        batched.forward(means, chol, weights, poses)
    with torch.cuda.graph(graph_b):
        batched.backward(means, chol, weights, poses, gd, ga, gn, gf, out=grads)

    def step(r):
        graph_f.replay()
        graph_b.replay()

    # plain arm: one forward and one backward call per view (default tiles, no graph)
    plain = []
    for v in s.views:
        vv = dict(v, pix_offset=0)  # each single-view renderer owns its own planes
        plain.append((fmb.Renderer(s.obj_offsets, [vv], len(s.poses), params, device=dev), v["pix_offset"],
                      v["W"] * v["H"]))

    # per-view gradient buffers, summed over the views after the calls (as a caller of
    # per-view launches has to)
    pgrads = [{k: torch.empty_like(v) for k, v in grads.items()} for _ in plain]
    psum = {k: torch.empty_like(v) for k, v in grads.items()}

    def plain_step():
        for (r, o, P), g in zip(plain, pgrads):
            r.forward(means, chol, weights, poses)
            r.backward(means, chol, weights, poses, gd[o:o + P], ga[o:o + P], gn[3 * o:3 * (o + P)],
                       gf[2 * o:2 * (o + P)], out=g)
        for k in psum:
            torch.sum(torch.stack([g[k] for g in pgrads]), dim=0, out=psum[k])

    def timed(fn, steps, warmup, split=False):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        evs = []
        for _ in range(steps):
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
        t_b, t_f, t_bw = timed(lambda: step(batched), args.steps, args.warmup, split=True)
    clocks = clk.summary()
    t_p, _, _ = timed(plain_step, max(args.steps // 4, 3), max(args.warmup, 3))
    args.psum = psum
    plain_steps = max(args.steps // 4, 3)
    assert fmb.fmb_read_device_status(batched.ws) == 0

    # max over ranks of the timed region
    ms_step = t_b / args.steps
    if ws > 1:
        import torch.distributed as dist

        x = torch.tensor([ms_step, t_p / plain_steps], device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        ms_step, ms_plain = float(x[0]), float(x[1])
    else:
        ms_plain = t_p / plain_steps
    value = ws * pairs / (ms_step * 1e-3)
    plain_value = ws * pairs / (ms_plain * 1e-3)

    # e2e: through the public API with host buffers (pinned), copies inside the timed region
    e2e = e2e_measure(args, s, ups, params, dev) if rank == 0 else None

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    bwd_ms = t_bw / args.steps
    clock_for_peak = 2070.0
    roofline = {
        "bound": "alu",
        "kernel": "backward_kernel (fmb_render_backward call)",
        "achieved": pairs * (BWD_FP32 + BWD_MUFU) / (bwd_ms * 1e-3) / 1e9,
        "peak": peak_issue_ginstr(clock_for_peak),
        "unit": "Ginstr/s",
        "frac": None,
        "traffic": None,
        "per_pair_ops": {"fwd_fp32": FWD_FP32, "fwd_mufu": FWD_MUFU, "bwd_fp32": BWD_FP32, "bwd_mufu": BWD_MUFU},
        "peak_basis": "152 SMs x 128 FP32 lanes (one warp-instruction issue per SMSP per clock) x 2070 MHz max SM clock",
    }
    roofline["frac"] = roofline["achieved"] / roofline["peak"]
    roofline["traffic"] = profiled_traffic()
    fwd_ms = t_f / args.steps
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "pairs/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded; stands in for the paper's CO3D sequences)",
        "config": {"workload": WORKLOAD, "views": len(s.views), "width": 320, "height": 240, "K": s.K(0),
                   "pairs_per_step": pairs,
                   "launch": "batched: one forward and one backward call for all views, autotuned tiles, "
                             "each pass replayed from a CUDA graph",
                   "tiles": {k: int(getattr(tuned_params, k)) for k in autotune.TUNED_FIELDS},
                   "l2": "flushed between timed steps (256 MiB write, outside the timed events)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "plain": {"value": plain_value, "ms_per_step": ms_plain,
                  "launch": "one forward and one backward call per view"},
        "batched_over_plain": value / plain_value,
        "fwd_ms": fwd_ms,
        "bwd_ms": bwd_ms,
        "frames_per_s": ws * len(s.views) / (ms_step * 1e-3),
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": 5 * args.steps,  # prologue + forward; zeroing + prologue + backward per step
        "e2e": e2e,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s, ups, batched, grads, args)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def e2e_measure(args, s, ups, params, dev):
    """Same metric through the public API with pinned host buffers: the step's
    inputs (scene, poses, upstream gradient planes) are copied host -> device and
    its results (depth, alpha, normal, flow planes and all gradients) device ->
    host inside the timed region."""
    import torch

    from paper_2308_14737_gb300 import fmb

    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).pin_memory()
    h_in = [pin(s.means), pin(s.chol), pin(s.weights), pin(s.poses), pin(ups["g_depth"]), pin(ups["g_alpha"]),
            pin(ups["g_normal"]), pin(ups["g_flow"])]
    d_in = [torch.empty_like(h, device=dev) for h in h_in]
    r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params, device=dev)
    G = s.means.shape[0]
    grads = dict(means=torch.empty(G, 3, device=dev), chol=torch.empty(G, 6, device=dev),
                 weights=torch.empty(G, device=dev), poses=torch.empty(len(s.poses), 12, device=dev))
    outs_d = [r.depth, r.alpha, r.normal, r.flow, grads["means"], grads["chol"], grads["weights"], grads["poses"]]
    outs_h = [torch.empty(o.shape, dtype=o.dtype).pin_memory() for o in outs_d]
    h2d = sum(h.numel() * 4 for h in h_in)
    d2h = sum(o.numel() * 4 for o in outs_d)

    def step():
        for h, d in zip(h_in, d_in):
            d.copy_(h, non_blocking=True)
        m, c, w, p, gd, ga, gn, gf = d_in
        r.forward(m, c, w, p)
        r.backward(m, c, w, p, gd, ga, gn, gf, out=grads)
        for d, h in zip(outs_d, outs_h):
            h.copy_(d, non_blocking=True)

    n = max(args.steps // 4, 5)
    for _ in range(3):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(n):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / n
    return {"value": s.n_pairs / (ms * 1e-3), "unit": "pairs/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms}


def cpu_baseline(s, ups, renderer, grads, args):
    """The FP64 oracle (test infrastructure, not tuned) timed on the host cores on
    one full step of the same workload, and compared with the GPU result on sampled
    pixels of that step."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.render_scene(s, n_flow=1)
    refg = oracle.backward_scene(s, ups["g_depth"], ups["g_alpha"], ups["g_normal"], ups["g_flow"], n_flow=1)
    dt = time.perf_counter() - t0
    out = {"value": s.n_pairs / dt, "unit": "pairs/s", "cores": oracle.max_threads(), "kind": "oracle",
           "sample": "one full step: all 16 views, forward + backward (FP64, OpenMP over pixels)",
           "seconds": dt}
    # parity of the timed GPU step (depth on alpha >= 1e-2, gradients normwise)
    import torch

    torch.cuda.synchronize()
    # the plain arm compares too: its summed per-view gradients must equal the batched ones
    out["plain_vs_batched_grad_max_rel"] = {
        k: float((args.psum[k] - grads[k]).abs().max() / grads[k].abs().max()) for k in grads}
    d = renderer.depth.cpu().numpy().astype(np.float64)
    mask = ref["alpha"] >= 1e-2
    err = {"depth_max_abs": float(np.max(np.abs(d - ref["depth"])[mask]))}
    for k in ("means", "chol", "weights", "poses"):
        g = grads[k].cpu().numpy().astype(np.float64).reshape(refg[k].shape)
        err[f"grad_{k}_max_rel"] = float(np.max(np.abs(g - refg[k])) / np.max(np.abs(refg[k])))
    out["parity"] = err
    out["parity_note"] = ("upstream depth/normal/flow gradients masked by the rendered alpha >= 1e-2, the normal "
                          "gradient also by the rendered |N| >= 0.05")
    return out


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, same metric and unit;
    each step is a bounded sample (2 of the 16 views, forward + backward)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    s, ups = scene_and_inputs()
    from paper_2308_14737_gb300 import synth

    sub = synth.make_scene([(s.means, s.chol, s.weights)],
                           [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views[:2]], s.poses)
    P = sub.n_pixels
    sl = lambda a, c: np.ascontiguousarray(a[:c * P])
    u = dict(g_depth=sl(ups["g_depth"], 1), g_alpha=sl(ups["g_alpha"], 1))
    u["g_normal"] = np.concatenate([ups["g_normal"][3 * v["pix_offset"]:3 * (v["pix_offset"] + v["W"] * v["H"])]
                                    for v in s.views[:2]])
    u["g_flow"] = np.concatenate([ups["g_flow"][2 * v["pix_offset"]:2 * (v["pix_offset"] + v["W"] * v["H"])]
                                  for v in s.views[:2]])

    def step():
        oracle.render_scene(sub, n_flow=1)
        oracle.backward_scene(sub, u["g_depth"], u["g_alpha"], u["g_normal"], u["g_flow"], n_flow=1)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    v = sub.n_pairs / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pairs/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "views": 16, "width": 320, "height": 240, "K": 100,
                       "pairs_per_step": sub.n_pairs, "sample": "2 of the 16 views per step"},
            "cpu_baseline": {"value": v, "unit": "pairs/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "2 of the 16 views (320x240, K=100), forward + backward, per step"},
            "e2e": {"value": v, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fmb", choices=["fmb", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
