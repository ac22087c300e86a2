"""Fused Adam, the CUDA-graph reconstruction step and the tile autotuner."""

import json

import numpy as np
import pytest
import torch

import oracle
from paper_2308_14737_gb300 import autotune, fmb, synth
from paper_2308_14737_gb300.step import ReconstructionStep

gpu = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_14737_gb300 import build

    build.build()
    fmb.load_library()


def adam_reference(theta, grad, m, v, positive_begin, t, lr, b1, b2, eps):
    """Plain PyTorch fp32 restatement of the update (log-space for the positive tail)."""
    theta, m, v = theta.clone(), m.clone(), v.clone()
    g = grad.clone()
    g[positive_begin:] = g[positive_begin:] * theta[positive_begin:]
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    c1, c2 = 1 - b1 ** t, 1 - b2 ** t
    upd = lr * np.sqrt(c2) / c1 * m / (torch.sqrt(v) + eps * np.sqrt(c2))
    theta[:positive_begin] -= upd[:positive_begin]
    theta[positive_begin:] *= torch.exp(-upd[positive_begin:])
    return theta, m, v


@gpu
def test_adam_matches_reference(lib):
    torch.manual_seed(0)
    n, pb = 1000, 900
    theta = torch.rand(n, device="cuda") + 0.1
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    p = fmb.FmbAdamParams(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    rt, rm, rv = theta.clone(), m.clone(), v.clone()
    for t in range(1, 4):
        grad = torch.randn(n, device="cuda")
        fmb.fmb_adam_step(p, theta, grad, m, v, pb, step)
        rt, rm, rv = adam_reference(rt, grad, rm, rv, pb, t, 1e-2, 0.9, 0.999, 1e-8)
    torch.cuda.synchronize()
    assert int(step.item()) == 3
    torch.testing.assert_close(theta, rt, rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(m, rm, rtol=1e-5, atol=1e-7)
    torch.testing.assert_close(v, rv, rtol=5e-5, atol=0)  # fma vs separate multiply-add
    assert torch.all(theta[pb:] > 0)


def _recon_problem():
    """Targets rendered by the FP64 oracle from a second seed; the model starts from
    the first seed."""
    tgt_scene = synth.reconstruction(seed=1, n_views=4, K=24, W=40, H=30)
    model = synth.reconstruction(seed=0, n_views=4, K=24, W=40, H=30)
    model.poses = tgt_scene.poses.copy()  # same cameras
    ref = oracle.render_scene(tgt_scene, n_flow=1)
    return model, dict(depth=ref["depth"], alpha=ref["alpha"], flow=ref["flow"])


@gpu
def test_graph_replay_matches_eager_and_loss_decreases(lib):
    model, targets = _recon_problem()
    p = fmb.default_params(n_flow=1, want_normals=0, deterministic=1)
    eager = ReconstructionStep(model, targets, params=p)
    graphed = ReconstructionStep(model, targets, params=p)
    losses = []
    for _ in range(2):  # capture() runs 2 eager warm-up steps; the captured step only records
        eager.step()
    graphed.capture(warmup=2)
    for _ in range(25):
        eager.step()
        graphed.replay()
        losses.append(float(eager.loss))
    torch.cuda.synchronize()
    assert torch.equal(eager.theta, graphed.theta)
    assert int(graphed.step_counter.item()) == 27
    assert losses[-1] < 0.8 * losses[0], losses


@gpu
def test_autotune_picks_a_candidate_and_caches(lib, tmp_path):
    s = synth.object_orbit(K=40, n_views=2, W=48, H=32)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    P = s.n_pixels
    ups = dict(g_depth=torch.randn(P, device="cuda"), g_alpha=torch.randn(P, device="cuda"),
               g_normal=torch.randn(3 * P, device="cuda"), g_flow=torch.randn(2 * P, device="cuda"))
    base = fmb.default_params(n_flow=1)
    cache = tmp_path / "tune.json"
    cands = autotune.CANDIDATES[:4]
    best, timings = autotune.tune(s.obj_offsets, s.views, len(s.poses), base, T(s.means), T(s.chol), T(s.weights),
                                  T(s.poses), ups, candidates=cands, reps=1, cache_path=str(cache))
    assert len(timings) == 4
    assert any(all(getattr(best, k) == c.get(k, getattr(base, k)) for k in autotune.TUNED_FIELDS) for c in cands)
    data = json.loads(cache.read_text())
    assert len(data) == 1
    best2, _ = autotune.tune(s.obj_offsets, s.views, len(s.poses), base, T(s.means), T(s.chol), T(s.weights),
                             T(s.poses), ups, candidates=cands, reps=1, cache_path=str(cache))
    assert all(getattr(best, k) == getattr(best2, k) for k in autotune.TUNED_FIELDS)
