"""Independent float64 PyTorch-CPU restatement of the renderer (test infrastructure).

A second, separately written evaluation of the same equations as ``fmb_oracle.c``
(Sec. 3.1-3.3, Eq. 2, 3, 4, 7, 8, 9, 10, 17; flow of Sec. 5), vectorised over pixels x
Gaussians, whose gradients come from autograd instead of a hand-derived adjoint.
It exists only to cross-check the oracle's analytic adjoint on tiny inputs.  Only
the test suite imports it.
"""

from __future__ import annotations

import torch


def render(means, chol, weights, R, t, target_R, target_t, cam, beta1=21.4, beta2=3.14, eta=1.0, variant=0,
           colors=None):
    """``variant`` 0: two-parameter weights (Eq. 7); 1: alpha compositing (Eq. 9-10,
    transmittance from a (P, K, K) indicator matrix of "j strictly in front of i").
    All tensors float64.  means (K,3), chol (K,6) packed (L00,L10,L11,L20,L21,L22),
    weights (K,), R (3,3) and t (3,) world->camera, target_R (T,3,3), target_t (T,3),
    cam = (W, H, fx, fy, cx, cy).  Returns depth (P,), alpha (P,), normal (P,3) in the
    camera frame, flow (P,T,2), and with ``colors`` (K,3) the blended colour (P,3)."""
    W, H, fx, fy, cx, cy = cam
    K = means.shape[0]
    ys, xs = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                            indexing="ij")
    px = xs.reshape(-1) + 0.5
    py = ys.reshape(-1) + 0.5
    dirs = torch.stack([(px - cx) / fx, (py - cy) / fy, torch.ones_like(px)], dim=1)
    vcam = dirs / dirs.norm(dim=1, keepdim=True)  # (P,3)
    v = vcam @ R  # rows: R^T vcam
    o = -(R.transpose(0, 1) @ t)  # (3,)

    Lm = torch.zeros(K, 3, 3, dtype=torch.float64)
    idx = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    for c, (r_, k_) in enumerate(idx):
        Lm = Lm.index_put((torch.arange(K), torch.full((K,), r_), torch.full((K,), k_)), chol[:, c])
    Prec = Lm @ Lm.transpose(1, 2)  # (K,3,3) = Sigma^-1

    m = means - o  # (K,3)
    Pv = torch.einsum("kab,pb->pka", Prec, v)  # (P,K,3)
    num = torch.einsum("ka,pka->pk", m, Pv)
    den = torch.einsum("pa,pka->pk", v, Pv)
    tt = num / den  # (P,K)
    r = v[:, None, :] * tt[..., None] - m[None]  # (P,K,3)
    g = torch.einsum("kab,pkb->pka", Prec, r)
    q = (r * g).sum(-1)
    d = -0.5 * q + torch.log(weights)[None]
    delta = torch.exp(d)
    if variant == 1:
        front = (tt[:, None, :] < tt[:, :, None]).to(torch.float64)  # [p, i, j] = 1 if t_j < t_i
        trans = torch.exp(-torch.einsum("pij,pj->pi", front, delta))
        wa = trans * -torch.expm1(-delta)
        w = wa / wa.sum(1, keepdim=True)
    else:
        e = beta1 * d - (beta2 / eta) * tt
        w = torch.softmax(e, dim=1)
    depth = (w * tt).sum(1)
    alpha = -torch.expm1(-delta.sum(1))
    n = g / g.norm(dim=-1, keepdim=True)
    N = (w[..., None] * n).sum(1)
    nf = N / N.norm(dim=-1, keepdim=True)
    normal = nf @ R.transpose(0, 1)
    p = o[None] + v * depth[:, None]
    flows = []
    for j in range(target_R.shape[0]):
        X = p @ target_R[j].transpose(0, 1) + target_t[j][None]
        u = fx * X[:, 0] / X[:, 2] + cx - px
        vv = fy * X[:, 1] / X[:, 2] + cy - py
        flows.append(torch.stack([u, vv], dim=1))
    flow = torch.stack(flows, dim=1) if flows else torch.zeros(depth.shape[0], 0, 2, dtype=torch.float64)
    if colors is not None:  # Eq. 3 with per-Gaussian colours: (P, 3)
        return depth, alpha, normal, flow, w @ colors
    return depth, alpha, normal, flow
