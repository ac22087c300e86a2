"""The forward entry point that allocates nothing, fmb_render_forward_noalloc.

Some callers of this library cannot allocate device memory: a plugin whose host
application owns all device memory and offers no allocator, or code on a path where
cudaMalloc's implicit device synchronisation is not allowed.  For them the forward
render keeps its scratch in a fixed array inside the library.  These tests call it
through the C ABI and check it against fmb_render_forward, which takes a workspace,
on two calls in a row with different batches (the second reuses the scratch the
first one left behind), in both launch modes, both weightings and with and without
colours; check that its status word reads 0 after each call and that the device's
free memory does not change across the calls; and check that a batch too large for
the fixed scratch is rejected before any work is enqueued.
"""

import numpy as np
import pytest
import torch

from paper_2308_14737_gb300 import fmb, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_14737_gb300 import build

    build.build()
    fmb.load_library()


def _dev(scene):
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    return T(scene.means), T(scene.chol), T(scene.weights), T(scene.poses)


def _planes(P, n_flow):
    f = dict(dtype=torch.float32, device="cuda")
    return dict(depth=torch.full((P,), -1.0, **f), alpha=torch.full((P,), -1.0, **f),
                normal=torch.full((3 * P,), -1.0, **f), flow=torch.full((2 * n_flow * P,), -1.0, **f),
                saved=torch.full((3 * P,), -1.0, **f), color=torch.full((3 * P,), -1.0, **f))


def _colours(scene, seed):
    rng = np.random.default_rng(seed)
    return torch.as_tensor(rng.uniform(0.0, 1.0, (scene.means.shape[0], 3)).astype(np.float32), device="cuda")


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("colors", [0, 1])
def test_noalloc_matches_workspace_forward_on_two_calls(persistent, variant, colors):
    scenes = [synth.object_orbit(K=100, n_views=4, W=64, H=48), synth.object_orbit(seed=3, K=30, n_views=2, W=40, H=30)]
    keys = ("depth", "alpha", "normal", "flow", "saved") + (("color",) if colors else ())
    cases = []
    for i, s in enumerate(scenes):
        params = fmb.default_params(n_flow=1, want_normals=1, use_persistent=persistent, variant=variant,
                                    colors=colors)
        means, chol, weights, poses = _dev(s)
        col = _colours(s, i) if colors else None
        ref = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params).forward(means, chol, weights, poses,
                                                                                colors=col)
        out = _planes(s.n_pixels, 1)
        cases.append((s, params, (means, chol, weights, poses), col, ref, out))

    def call(case):
        s, params, (means, chol, weights, poses), col, _, out = case
        fmb.fmb_render_forward_noalloc(params, s.obj_offsets, means, chol, weights, poses, s.views, out["depth"],
                                       out["alpha"], out["normal"], out["flow"], out["saved"], colors=col,
                                       color=out["color"] if colors else None)

    # one untimed call per batch first, so that every kernel the calls launch is
    # loaded before the free device memory is recorded
    for c in cases:
        call(c)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for c in cases:
        for k in c[5]:
            c[5][k].fill_(-1.0)
    torch.cuda.synchronize()
    for c in cases:  # two calls in a row, the second on another batch
        call(c)
        assert fmb.fmb_read_noalloc_status() == 0
        ref, out = c[4], c[5]
        for k in keys:
            a = out[k].cpu().numpy().astype(np.float64)
            b = ref[k].cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(a)), k
            assert np.all(np.abs(a - b) <= 1e-4 + 1e-5 * np.abs(b)), (k, float(np.max(np.abs(a - b))))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_batches_beyond_the_fixed_scratch():
    s = synth.object_orbit(K=5000, n_views=4, W=8, H=8)  # 20000 records x 64 bytes > 1 MiB
    params = fmb.default_params(n_flow=1, want_normals=1)
    means, chol, weights, poses = _dev(s)
    out = _planes(s.n_pixels, 1)
    with pytest.raises(fmb.FmbError) as ei:
        fmb.fmb_render_forward_noalloc(params, s.obj_offsets, means, chol, weights, poses, s.views, out["depth"],
                                       out["alpha"], out["normal"], out["flow"], out["saved"])
    assert ei.value.status == 4 and "static scratch" in str(ei.value)
    torch.cuda.synchronize()
    assert torch.all(out["depth"] == -1.0)  # nothing was enqueued
