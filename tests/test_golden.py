"""The values the paper prints (tests/golden/paper_values.txt, each with its
citation) against the ones the library, the oracle and the bench use."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def golden():
    vals = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_values.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, citation = line.split(None, 2)
            assert citation, name
            vals[name] = float(value)
    return vals


def test_default_weights_are_the_papers():
    from paper_2308_14737_gb300 import build, fmb

    build.build()
    g = golden()
    p = fmb.default_params()
    assert p.beta1 == pytest.approx(g["beta1"], rel=1e-7) and p.beta2 == pytest.approx(g["beta2"], rel=1e-7)


def test_oracle_weights_are_the_papers():
    import oracle

    g = golden()
    assert oracle.BETA1 == g["beta1"] and oracle.BETA2 == g["beta2"]


def test_bench_context_quotes_the_papers_runtime_table():
    sys.path.insert(0, ROOT)
    import bench

    g = golden()
    assert bench.PAPER_RUNTIME_GAUSSIANS == g["runtime_gaussians"]
    for name, key in (("weighted blending", "weighted_blending"), ("alpha compositing", "alpha_compositing")):
        assert bench.PAPER_RUNTIME_PER_RAY[name]["cpu_us"] == g[f"runtime_{key}_cpu_us"]
        assert bench.PAPER_RUNTIME_PER_RAY[name]["gpu_ns"] == g[f"runtime_{key}_gpu_ns"]
    c = bench.paper_context("ac")
    assert c["gtx1080_ns_per_ray"] == g["runtime_alpha_compositing_gpu_ns"]
    assert c["gtx1080_pairs_per_s"] == pytest.approx(g["runtime_gaussians"] / (g["runtime_alpha_compositing_gpu_ns"] * 1e-9))
