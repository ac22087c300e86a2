"""Measures the GPU's FP32-pipe and SFU (MUFU) throughput with the library's probe
kernels (``fmb_probe_alu``): lane-operations per second for scalar FMA, packed
FP32x2 FMA, ex2, rcp and rsqrt."""

from __future__ import annotations

import ctypes

import torch

from . import fmb

KINDS = {0: "ffma", 1: "ffma2", 2: "ex2", 3: "rcp", 4: "rsqrt"}


def measure(iters: int = 4096, blocks_per_sm: int = 8, reps: int = 5, device="cuda") -> dict:
    L = fmb.load_library()
    L.fmb_probe_alu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.fmb_probe_alu.restype = ctypes.c_int
    n_sm = torch.cuda.get_device_properties(device).multi_processor_count
    blocks = n_sm * blocks_per_sm
    out = torch.empty(blocks * 256, dtype=torch.float32, device=device)
    stream = torch.cuda.current_stream(device)
    res = {"sms": n_sm}
    for kind, name in KINDS.items():
        lanes_per_op = 2 if kind == 1 else 1
        ops = blocks * 256 * 8 * iters * lanes_per_op
        best = None
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = L.fmb_probe_alu(kind, blocks, iters, ctypes.c_void_p(out.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))
            e1.record(stream)
            if st != 0:
                raise RuntimeError(f"fmb_probe_alu failed ({st})")
            torch.cuda.synchronize(device)
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        res[name] = ops / (best * 1e-3)  # lane-ops per second
    return res


def sample_clocks(fn, period_ms: int = 100):
    """Runs fn() while nvidia-smi samples the SM clock; returns (fn's result, median
    SM MHz of the samples, max SM MHz, throttle reasons seen)."""
    import os
    import statistics
    import subprocess
    import tempfile

    fd, path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    idx = torch.cuda.current_device()
    with open(path, "w") as fh:
        try:
            proc = subprocess.Popen(["nvidia-smi", "-i", str(idx), f"--query-gpu={fields}",
                                     "--format=csv,noheader,nounits", "-lms", str(period_ms)], stdout=fh,
                                    stderr=subprocess.DEVNULL)
        except OSError:
            proc = None
        try:
            res = fn()
        finally:
            if proc is not None:
                proc.terminate()
                proc.wait(timeout=5)
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        p = [x.strip() for x in line.split(",")]
        try:
            sm.append(float(p[0]))
            smax.append(float(p[1]))
        except (ValueError, IndexError):
            continue
        reasons.update(n for n, v in zip(names, p[2:6]) if v.lower().startswith("active"))
    os.unlink(path)
    return res, (statistics.median(sm) if sm else None), (max(smax) if smax else None), sorted(reasons)


if __name__ == "__main__":  # pragma: no cover
    import json

    # about 6 s in all (0.07 to 0.5 s per launch), long enough for the clock samples
    r, mhz, max_mhz, reasons = sample_clocks(lambda: measure(iters=1 << 20, reps=3))
    out = {"sms": r["sms"], "sm_mhz_median": mhz, "sm_max_mhz": max_mhz, "reasons": reasons}
    for k in KINDS.values():
        out[k + "_tops"] = r[k] / 1e12
        if mhz:
            out[k + "_per_sm_clock"] = r[k] / (r["sms"] * mhz * 1e6)
    print(json.dumps(out))
