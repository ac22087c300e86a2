"""The reference arm of bench.py (the FP64 oracle on the host cores) prints one JSON
line with the contract's keys; it needs no GPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "pairs/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # the same config object as the GPU arm's (both come from bench.workload_config)
    sys.path.insert(0, ROOT)
    import bench

    s, _ = bench.scene_and_inputs(workload=bench.DEFAULT_WORKLOAD)
    want = dict(bench.workload_config(s, bench.WORKLOADS[bench.DEFAULT_WORKLOAD]), parallelism="single GPU")
    assert d["config"] == json.loads(json.dumps(want))
    assert d["config"]["pairs_per_step"] == 8 * 1024 * 768 * 4096


def test_profile_gate_follows_sources_and_compile_flags(monkeypatch):
    """The committed backward ncu summary is used for roofline.traffic only while
    the backward's sources, its compile flags and the launch tiles are the ones it
    was captured with."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2308_14737_gb300 import build

    for src in build.EXTRA_FLAGS:
        assert src in build.SOURCES, src
    tiles = {"bwd_ray_tile": 384, "bwd_threads": 128, "fwd_rays_per_thread": 2, "use_persistent": 0}
    sha = bench.csrc_sha256()
    assert bench.profiled_traffic(tiles) is not None, "profile summary out of date with the sources"
    assert bench.profiled_traffic(dict(tiles, bwd_ray_tile=256)) is None
    monkeypatch.setitem(build.EXTRA_FLAGS, "fmb_backward.cu", [])
    assert bench.csrc_sha256() != sha
    assert bench.profiled_traffic(tiles) is None
