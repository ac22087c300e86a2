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


if __name__ == "__main__":  # pragma: no cover
    import json

    r = measure()
    clk = torch.cuda.clock_rate() if hasattr(torch.cuda, "clock_rate") else None
    print(json.dumps({k: (v if k == "sms" else v / 1e12) for k, v in r.items()}))
