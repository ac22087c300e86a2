"""Reconstruction iteration (paper Sec. 4): render every view, compare with target
planes, back-propagate through the renderer's adjoint, take one Adam step -- all
captured once in a CUDA graph and replayed.

The render is ``fmb.FmbRender`` (a ``torch.autograd.Function`` over the library's
``fmb_render_forward`` / ``fmb_render_backward`` kernels); the loss is ordinary
PyTorch code on the rendered planes (the caller's choice of loss; here L1 depth and
L2 flow weighted by the target mask, plus binary cross-entropy on alpha with the
prediction clipped to [1e-6, 1 - 1e-6] as in Sec. 4), differentiated by autograd
down to the planes, from where the library's adjoint takes over; the optimiser is
the library's fused Adam (``fmb_adam_step``) over the packed parameters.
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
        # the packed parameters [means | chol | weights], the leaf autograd differentiates to
        self.theta = torch.cat([T(scene.means).reshape(-1), T(scene.chol).reshape(-1), T(scene.weights)])
        self.theta.requires_grad_(True)
        self.grad = torch.zeros_like(self.theta, requires_grad=False)
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
        self.loss = torch.zeros((), device=dev)
        self.w = (w_depth / P, w_alpha / P, w_flow / P)
        self.graph = None

    def views(self):
        """means, chol, weights as differentiable views of the packed parameters."""
        G = self.G
        return self.theta[:3 * G].view(G, 3), self.theta[3 * G:9 * G].view(G, 6), self.theta[9 * G:]

    def loss_of(self, depth, alpha, flow):
        """The Sec. 4 loss of rendered planes (autograd-differentiable)."""
        wd, wa, wf = self.w
        loss = wd * (self.t_alpha * (depth - self.t_depth).abs()).sum()
        ac = alpha.clamp(1e-6, 1.0 - 1e-6)
        loss = loss - wa * (self.t_alpha * torch.log(ac) + (1.0 - self.t_alpha) * torch.log1p(-ac)).sum()
        if self.t_flow is not None:
            f = (flow - self.t_flow) * self.flow_scale
            loss = loss + wf * (self.mask_flow * f * f).sum()
        return loss

    def step(self):
        """One iteration on the current stream (eager): render through FmbRender, the
        loss, its gradient with respect to the packed parameters by autograd (the
        library's adjoint for the render), then the fused Adam step."""
        means, chol, weights = self.views()
        depth, alpha, _, flow = fmb.render(self.renderer, means, chol, weights, self.poses)
        loss = self.loss_of(depth, alpha, flow)
        (g,) = torch.autograd.grad(loss, [self.theta])
        self.grad.copy_(g)
        self.loss.copy_(loss.detach())
        with torch.no_grad():
            fmb.fmb_adam_step(self.adam, self.theta, self.grad, self.m, self.v, 9 * self.G, self.step_counter)

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
