"""Reconstruction iteration (paper Sec. 4): render every view, compare with target
planes, back-propagate through the renderer's adjoint, take one Adam step -- all
captured once in a CUDA graph and replayed.

The render and its adjoint are the library's kernels (``fmb_render_forward`` /
``fmb_render_backward``), the optimiser is its fused Adam (``fmb_adam_step``); the
loss is ordinary PyTorch elementwise code on preallocated buffers (the caller's
choice of loss; here L1 depth and L2 flow weighted by the target mask, plus binary
cross-entropy on alpha with the prediction clipped to [1e-6, 1 - 1e-6] as in
Sec. 4).
"""

from __future__ import annotations

import numpy as np
import torch

from . import fmb


class ReconstructionStep:
    """Holds the flat parameter buffer [means | chol | weights], Adam state, the
    renderer and the loss buffers of one scene layout."""

    def __init__(self, scene, targets: dict, params: fmb.FmbParams | None = None, lr: float = 1e-2,
                 w_depth: float = 1.0, w_alpha: float = 1.0, w_flow: float = 1.0, device="cuda"):
        self.device = torch.device(device)
        self.params = params if params is not None else fmb.default_params(n_flow=1, want_normals=0)
        dev = self.device
        T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
        G = int(scene.means.shape[0])
        self.G = G
        self.theta = torch.cat([T(scene.means).reshape(-1), T(scene.chol).reshape(-1), T(scene.weights)])
        self.grad = torch.zeros_like(self.theta)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.step_counter = torch.zeros(1, dtype=torch.int32, device=dev)
        self.adam = fmb.FmbAdamParams(lr=lr, beta1=0.9, beta2=0.999, eps=1e-8)
        self.poses = T(scene.poses)
        self.renderer = fmb.Renderer(scene.obj_offsets, scene.views, len(scene.poses), self.params, device=dev)
        P = self.renderer.P
        nf = self.params.n_flow
        self.t_depth = T(targets["depth"])
        self.t_alpha = T(targets["alpha"])
        self.t_flow = T(targets["flow"]) if nf else None
        # flow is compared in units of half the shorter image side (Sec. 4)
        scale = np.zeros(2 * nf * P, dtype=np.float32)
        for v in scene.views:
            o, Pv = v["pix_offset"], v["W"] * v["H"]
            scale[2 * nf * o:2 * nf * (o + Pv)] = 2.0 / min(v["W"], v["H"])
        self.flow_scale = T(scale) if nf else None
        self.mask_flow = None
        if nf:
            mf = np.zeros(2 * nf * P, dtype=np.float32)
            ta = np.asarray(targets["alpha"], dtype=np.float32)
            for v in scene.views:
                o, Pv = v["pix_offset"], v["W"] * v["H"]
                mf[2 * nf * o:2 * nf * (o + Pv)] = np.tile(ta[o:o + Pv], 2 * nf)
            self.mask_flow = T(mf)
        self.g_depth = torch.zeros(P, device=dev)
        self.g_alpha = torch.zeros(P, device=dev)
        self.g_flow = torch.zeros(2 * nf * P, device=dev) if nf else None
        self.loss = torch.zeros((), device=dev)
        self.w = (w_depth / P, w_alpha / P, w_flow / P)
        self.graph = None

    def views(self):
        G = self.G
        return self.theta[:3 * G].view(G, 3), self.theta[3 * G:9 * G].view(G, 6), self.theta[9 * G:]

    def _loss_and_upstream(self, out):
        wd, wa, wf = self.w
        d = out["depth"] - self.t_depth
        l_depth = (self.t_alpha * d.abs()).sum()
        torch.mul(torch.sign(d), self.t_alpha * wd, out=self.g_depth)
        a = out["alpha"]
        ac = a.clamp(1e-6, 1.0 - 1e-6)
        l_alpha = -(self.t_alpha * torch.log(ac) + (1.0 - self.t_alpha) * torch.log1p(-ac)).sum()
        inside = ((a > 1e-6) & (a < 1.0 - 1e-6)).float()
        torch.mul((ac - self.t_alpha) / (ac * (1.0 - ac)), inside * wa, out=self.g_alpha)
        loss = wd * l_depth + wa * l_alpha
        if self.g_flow is not None:
            f = (out["flow"] - self.t_flow) * self.flow_scale
            loss = loss + wf * (self.mask_flow * f * f).sum()
            torch.mul(f * self.flow_scale, self.mask_flow * (2.0 * wf), out=self.g_flow)
        self.loss.copy_(loss)

    def step(self):
        """One iteration on the current stream (eager)."""
        means, chol, weights = self.views()
        out = self.renderer.forward(means, chol, weights, self.poses)
        self._loss_and_upstream(out)
        G = self.G
        gd = dict(means=self.grad[:3 * G].view(G, 3), chol=self.grad[3 * G:9 * G].view(G, 6),
                  weights=self.grad[9 * G:], poses=None)
        self.renderer.backward(means, chol, weights, self.poses, self.g_depth, self.g_alpha, None, self.g_flow,
                               want_pose=False, out=gd)
        fmb.fmb_adam_step(self.adam, self.theta, self.grad, self.m, self.v, 9 * G, self.step_counter)

    def capture(self, warmup: int = 2):
        """Runs `warmup` eager steps on a side stream, then records one step in a
        CUDA graph (later steps: ``replay``)."""
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream(self.device).wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self):
        self.graph.replay()
