"""The differentiable render behind ``torch.autograd.Function`` (``fmb.FmbRender``):
its planes against the FP64 oracle, ``torch.autograd.grad`` of a random linear
functional of the planes against the oracle's analytic adjoint (per tensor,
max |g - g_ref| <= 1e-4 max |g_ref|), with and without pose gradients, two backward
passes of one forward, two renders alive in one graph, and the reconstruction step
(Sec. 4: loss, adjoint, Adam) routed through it at the reconstruction workload's
layout."""

import numpy as np
import pytest
import torch

import oracle
from paper_2308_14737_gb300 import fmb, synth

from gpu_util import compare_forward, compare_grads, many_small_views, masked_upstream, nnorm_batched

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_14737_gb300 import build

    build.build()
    oracle.build()
    fmb.load_library()


def _leaves(scene, pose_grad=True):
    T = lambda a, g: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda").requires_grad_(g)
    return T(scene.means, True), T(scene.chol, True), T(scene.weights, True), T(scene.poses, pose_grad)


def _functional(planes, ups):
    """sum of upstream x plane over the four planes (a random linear functional)."""
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float32, device="cuda")
    depth, alpha, normal, flow = planes[:4]
    f = (T(ups["g_depth"]) * depth).sum() + (T(ups["g_alpha"]) * alpha).sum()
    if normal.numel():
        f = f + (T(ups["g_normal"]) * normal).sum()
    if flow.numel() and ups["g_flow"] is not None:
        f = f + (T(ups["g_flow"]) * flow).sum()
    return f


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("pose_grad", [True, False])
@pytest.mark.parametrize("deterministic", [False, True])
def test_fmbrender_forward_and_gradients_match_oracle(pose_grad, deterministic):
    s = synth.object_orbit(K=60, n_views=3, W=40, H=30)
    params = fmb.default_params(n_flow=1, want_normals=1, deterministic=int(deterministic))
    r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params)
    means, chol, weights, poses = _leaves(s, pose_grad)
    planes = fmb.render(r, means, chol, weights, poses)
    assert all(p.requires_grad for p in planes)
    own = r.forward(means.detach(), chol.detach(), weights.detach(), poses.detach())  # the renderer's own planes
    torch.cuda.synchronize()
    for k, p in zip(("depth", "alpha", "normal", "flow"), planes):
        assert torch.equal(p.detach(), own[k]), k
    ref = oracle.render_scene(s, n_flow=1)
    gpu = dict(depth=_np(planes[0]), alpha=_np(planes[1]), normal=_np(planes[2]), flow=_np(planes[3]),
               saved=_np(own["saved"]))
    compare_forward(s, gpu, ref, 1, True)
    ups = masked_upstream(s, ref["alpha"], 1, seed=5, nnorm_ref=nnorm_batched(s, ref["saved"]))
    leaves = [means, chol, weights] + ([poses] if pose_grad else [])
    grads = torch.autograd.grad(_functional(planes, ups), leaves, retain_graph=True)
    refg = oracle.backward_scene(s, ups["g_depth"], ups["g_alpha"], ups["g_normal"], ups["g_flow"], n_flow=1)
    keys = ("means", "chol", "weights") + (("poses",) if pose_grad else ())
    got = {k: _np(g) for k, g in zip(keys, grads)}
    compare_grads(got, refg, keys=keys)
    # a second backward pass of the same forward recomputes from the saved planes
    grads2 = torch.autograd.grad(_functional(planes, ups), leaves)
    for k, g1, g2 in zip(keys, grads, grads2):
        if deterministic:
            assert torch.equal(g1, g2), k
        else:
            torch.testing.assert_close(g1, g2, rtol=0, atol=1e-6 * float(g1.abs().max()))


def test_fmbrender_over_300_views():
    """A renderer over 300 views of three objects (its passes run as two launches of
    at most 256 views): planes and autograd gradients, pose gradients included,
    against the oracle."""
    s = many_small_views(300)
    params = fmb.default_params(n_flow=1, want_normals=1, deterministic=1)
    r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params)
    means, chol, weights, poses = _leaves(s)
    planes = fmb.render(r, means, chol, weights, poses)
    own = r.forward(means.detach(), chol.detach(), weights.detach(), poses.detach())  # for the saved plane
    ref = oracle.render_scene(s, n_flow=1)
    gpu = dict(depth=_np(planes[0]), alpha=_np(planes[1]), normal=_np(planes[2]), flow=_np(planes[3]),
               saved=_np(own["saved"]))
    compare_forward(s, gpu, ref, 1, True)
    ups = masked_upstream(s, ref["alpha"], 1, seed=6, nnorm_ref=nnorm_batched(s, ref["saved"]))
    keys = ("means", "chol", "weights", "poses")
    grads = torch.autograd.grad(_functional(planes, ups), [means, chol, weights, poses])
    refg = oracle.backward_scene(s, ups["g_depth"], ups["g_alpha"], ups["g_normal"], ups["g_flow"], n_flow=1)
    compare_grads({k: _np(g) for k, g in zip(keys, grads)}, refg, keys=keys)


@pytest.mark.parametrize("variant,keep_order", [(0, 0), (1, 0), (1, 1)])
def test_fmbrender_two_renders_alive_in_one_graph(variant, keep_order):
    """Two calls on one renderer keep their own planes: the gradient of a functional
    of the first render, taken after the second render ran, is the first render's.
    The second render moves the means, so (alpha compositing) its depth orders differ;
    with keep_order the first render's backward finds the second's stored orders in
    the workspace, sorts the rays whose order fails its check afresh and reaches the
    same gradients up to the rounding of the other summation order (bit for bit
    otherwise)."""
    s = synth.object_orbit(K=40, n_views=2, W=32, H=24)
    params = fmb.default_params(n_flow=1, want_normals=1, deterministic=1, variant=variant, keep_order=keep_order)
    r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params)
    means, chol, weights, poses = _leaves(s)
    ref = oracle.render_scene(s, n_flow=1)
    ups = masked_upstream(s, ref["alpha"], 1, seed=9, nnorm_ref=nnorm_batched(s, ref["saved"]))
    alone = torch.autograd.grad(_functional(fmb.render(r, means, chol, weights, poses), ups),
                                [means, chol, weights, poses])
    shift = torch.as_tensor(np.random.default_rng(4).normal(0.0, 0.2, s.means.shape).astype(np.float32),
                            device="cuda")
    pa = fmb.render(r, means, chol, weights, poses)
    # overwrites the renderer's workspace (records, and with keep_order the depth orders)
    pb = fmb.render(r, means + shift, chol, weights * 1.5, poses)
    ga = torch.autograd.grad(_functional(pa, ups), [means, chol, weights, poses])
    for x, y in zip(alone, ga):
        if keep_order:
            # (the upstream here is not masked at near-equal depths, where the
            # gradient is ill-conditioned: the parity tolerance, 1e-4 of the largest)
            assert float((x - y).abs().max()) <= 1e-4 * float(x.abs().max())
        else:
            assert torch.equal(x, y)
    assert not torch.equal(pa[0], pb[0])


def test_fmbrender_with_colours():
    """The colour plane (Eq. 3 with per-Gaussian colours) through autograd: the
    colour gradient equals the library's backward called directly."""
    s = synth.object_orbit(K=30, n_views=2, W=24, H=16)
    params = fmb.default_params(n_flow=1, want_normals=1, colors=1, deterministic=1)
    r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params)
    means, chol, weights, poses = _leaves(s)
    rng = np.random.default_rng(4)
    cols = torch.as_tensor(rng.uniform(0, 1, (s.means.shape[0], 3)).astype(np.float32), device="cuda")
    cols.requires_grad_(True)
    planes = fmb.render(r, means, chol, weights, poses, cols)
    assert len(planes) == 5
    gc = torch.randn_like(planes[4])
    g = torch.autograd.grad((planes[4] * gc).sum(), [means, cols])
    own = r.forward(means.detach(), chol.detach(), weights.detach(), poses.detach(), colors=cols.detach())
    direct = r.backward(means.detach(), chol.detach(), weights.detach(), poses.detach(), None, None, None, None,
                        colors=cols.detach(), g_color=gc)
    torch.cuda.synchronize()
    assert torch.equal(own["color"], planes[4].detach())
    assert torch.equal(g[0], direct["means"]) and torch.equal(g[1], direct["colors"])
