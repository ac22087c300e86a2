"""The host-fed pipeline (copies overlapped with neighbouring steps' kernels) gives
each step exactly the results of a plain device-resident call on that step's
inputs: same kernels, same tiles, so the comparison is bitwise."""

import numpy as np
import pytest
import torch

from paper_2308_14737_gb300 import fmb, pipeline, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_14737_gb300 import build

    build.build()
    fmb.load_library()


def _plain(s, params, st):
    """Planes and gradients of one plain device-resident forward + backward."""
    r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params)
    d = {k: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float32, device="cuda") for k, v in st.items()}
    out = r.forward(d["means"], d["chol"], d["weights"], d["poses"])
    g = r.backward(d["means"], d["chol"], d["weights"], d["poses"], d["g_depth"], d["g_alpha"], d["g_normal"],
                   d["g_flow"], want_pose=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in
            dict(depth=out["depth"], alpha=out["alpha"], normal=out["normal"], flow=out["flow"],
                 grad_means=g["means"], grad_chol=g["chol"], grad_weights=g["weights"],
                 grad_poses=g["poses"]).items()}


def _same(got, want, deterministic, what):
    for k, b in want.items():
        a = np.asarray(got[k]).reshape(b.shape)
        if k.startswith("grad") and not deterministic:
            # sums of fp32 atomics (order-dependent): equal up to rounding
            assert np.allclose(a, b, rtol=1e-5, atol=1e-6 * np.abs(b).max()), (what, k)
        else:
            assert np.array_equal(a, b), (what, k)


# variant 1 at K = 100: four keys per lane, so the per-ray sort runs the
# refinement from the neighbouring ray's (or, with keep_order, the forward's) order
@pytest.mark.parametrize("variant,keep_order,deterministic,K", [(0, 0, 0, 60), (0, 0, 1, 60), (1, 0, 1, 60),
                                                                (1, 0, 1, 100), (1, 1, 1, 100), (1, 1, 0, 100)])
def test_host_pipeline_matches_plain_calls(variant, keep_order, deterministic, K):
    s = synth.object_orbit(K=K, n_views=4, W=64, H=48)
    n_flow = 1
    params = fmb.default_params(n_flow=n_flow, variant=variant, keep_order=keep_order, deterministic=deterministic)
    P = s.n_pixels
    rng = np.random.default_rng(3)
    steps = []
    for i in range(5):  # every step has its own inputs (moved means, new upstream planes)
        means = (s.means + 0.01 * i).astype(np.float32)
        ups = synth.upstream_grads(rng, P, n_flow)
        steps.append(dict(means=means, chol=s.chol, weights=s.weights, poses=s.poses, g_depth=ups[0],
                          g_alpha=ups[1], g_normal=ups[2].reshape(-1), g_flow=ups[3].reshape(-1)))
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).pin_memory()
    h_in = [{k: pin(v) for k, v in st.items()} for st in steps]
    want = [_plain(s, params, st) for st in steps]

    pipe = pipeline.HostPipeline(s.obj_offsets, s.views, len(s.poses), params, h_in[0], want_pose=True)
    # each buffer set's captured graph, replayed on the set-up inputs as they are
    for j, sl in enumerate(pipe.slots):
        sl["graph"].replay()
        torch.cuda.synchronize()
        _same({k: v.cpu().numpy() for k, v in pipe.outputs(sl).items()}, want[0], deterministic, f"slot {j}")

    h_out = [pipe.host_outputs() for _ in steps]
    events = [pipe.submit(h_in[i], h_out[i]) for i in range(2)]
    events[0].synchronize()
    for i in range(2, len(steps)):  # a slot is reused only after its previous step is out
        events[i - 2].synchronize()
        events.append(pipe.submit(h_in[i], h_out[i]))
    torch.cuda.synchronize()
    for i in range(len(steps)):
        _same({k: v.numpy() for k, v in h_out[i].items()}, want[i], deterministic, f"step {i}")


@pytest.mark.parametrize("variant,keep_order", [(0, 0), (1, 1)])
def test_fixed_host_buffer_graphs_match_plain_calls(variant, keep_order):
    """The fixed-buffer mode (each buffer set's copies in, render, adjoint and copies
    out captured as one graph) gives each step the plain calls' results on the
    inputs the host buffers held: the buffers are refilled between steps."""
    s = synth.object_orbit(K=100, n_views=4, W=64, H=48)
    params = fmb.default_params(n_flow=1, variant=variant, keep_order=keep_order, deterministic=1)
    P = s.n_pixels
    rng = np.random.default_rng(11)
    steps = []
    for i in range(4):
        ups = synth.upstream_grads(rng, P, 1)
        steps.append(dict(means=(s.means + 0.02 * i).astype(np.float32), chol=s.chol, weights=s.weights,
                          poses=s.poses, g_depth=ups[0], g_alpha=ups[1], g_normal=ups[2].reshape(-1),
                          g_flow=ups[3].reshape(-1)))
    want = [_plain(s, params, st) for st in steps]
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).pin_memory()
    h_in = {k: pin(v) for k, v in steps[0].items()}
    pipe = pipeline.HostPipeline(s.obj_offsets, s.views, len(s.poses), params, h_in, want_pose=True)
    h_outs = [pipe.host_outputs(), pipe.host_outputs()]
    pipe.capture_fixed(h_in, h_outs)
    for i, st in enumerate(steps):
        for k, v in st.items():  # refill the fixed host inputs between steps
            h_in[k].copy_(torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float32).reshape(h_in[k].shape))
        pipe.submit_fixed().synchronize()
        _same({k: v.numpy() for k, v in h_outs[i % 2].items()}, want[i], True, f"step {i}")
