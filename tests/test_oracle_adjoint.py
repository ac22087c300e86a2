"""Pins of the oracle's analytic FP64 adjoint.

Two independent checks: central finite differences of the oracle's own forward
(every scalar of means, Cholesky factors, weights, the view pose and a flow-target
pose), and the gradients autograd gives for a separately written float64 PyTorch
restatement of the same equations (``oracle.torch_ref``).
"""

import numpy as np
import pytest
import torch

from paper_2308_14737_gb300 import synth
from oracle import torch_ref

CAM = (5, 4, 5.0, 5.0, 2.5, 2.0)


def tiny_scene(seed, K=3):
    rng = np.random.default_rng(seed)
    mu, chol, lam = synth.random_gaussians(rng, K, "cholesky")
    mu = mu.astype(np.float64) * 0.6
    pose = synth.look_at_pose((0.4, -0.3, -4.0))
    tgt = synth.look_at_pose((1.0, 0.2, -3.9))
    ups = dict(g_depth=rng.standard_normal(20), g_alpha=rng.standard_normal(20),
               g_normal=rng.standard_normal((20, 3)), g_flow=0.1 * rng.standard_normal((20, 1, 2)))
    return mu, chol.astype(np.float64), lam.astype(np.float64), pose, tgt, ups


def loss(o, mu, chol, lam, pose, tgt, ups, variant=0):
    r = o.render_view(mu, chol, lam, pose, tgt[None], CAM, variant=variant)
    return (np.sum(ups["g_depth"] * r["depth"]) + np.sum(ups["g_alpha"] * r["alpha"])
            + np.sum(ups["g_normal"] * r["normal"]) + np.sum(ups["g_flow"] * r["flow"]))


def fd_grad(f, x, h_rel=1e-6):
    g = np.zeros_like(x)
    flat = x.reshape(-1)
    gf = g.reshape(-1)
    for i in range(flat.size):
        h = h_rel * max(1.0, abs(flat[i]))
        old = flat[i]
        flat[i] = old + h
        fp = f()
        flat[i] = old - h
        fm = f()
        flat[i] = old
        gf[i] = (fp - fm) / (2 * h)
    return g


@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_matches_central_differences(oracle_mod, seed, variant):
    """variant 1 (alpha compositing): the hit depths of the tiny scenes are far
    apart, so no finite-difference step crosses a change of depth order."""
    mu, chol, lam, pose, tgt, ups = tiny_scene(seed)
    g = oracle_mod.backward_view(mu, chol, lam, pose, tgt[None], CAM, **ups, variant=variant)
    f = lambda: loss(oracle_mod, mu, chol, lam, pose, tgt, ups, variant)
    checks = [("means", mu, g["means"]), ("chol", chol, g["chol"]), ("weights", lam, g["weights"]),
              ("pose", pose, g["pose"]), ("target", tgt, g["target_poses"][0])]
    for name, x, ga in checks:
        gfd = fd_grad(f, x)
        err = np.max(np.abs(ga - gfd))
        scale = np.max(np.abs(gfd))
        assert err <= 1e-6 * scale, (name, err, scale)


@pytest.mark.parametrize("variant", [0, 1])
def test_adjoint_matches_torch_autograd(oracle_mod, variant):
    for seed in (3, 4):
        mu, chol, lam, pose, tgt, ups = tiny_scene(seed, K=4)
        g = oracle_mod.backward_view(mu, chol, lam, pose, tgt[None], CAM, **ups, variant=variant)
        f = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
        tm, tc, tl = f(mu), f(chol), f(lam)
        tR, tt = f(pose[:9].reshape(3, 3)), f(pose[9:])
        gR, gt = f(tgt[:9].reshape(3, 3)[None]), f(tgt[9:][None])
        d, a, n, fl = torch_ref.render(tm, tc, tl, tR, tt, gR, gt, CAM, variant=variant)
        r = oracle_mod.render_view(mu, chol, lam, pose, tgt[None], CAM, variant=variant)
        np.testing.assert_allclose(d.detach().numpy(), r["depth"], rtol=1e-12)
        np.testing.assert_allclose(a.detach().numpy(), r["alpha"], rtol=1e-12)
        np.testing.assert_allclose(n.detach().numpy(), r["normal"], atol=1e-12)
        np.testing.assert_allclose(fl.detach().numpy(), r["flow"], atol=1e-10)
        L = ((d * torch.tensor(ups["g_depth"])).sum() + (a * torch.tensor(ups["g_alpha"])).sum()
             + (n * torch.tensor(ups["g_normal"])).sum() + (fl * torch.tensor(ups["g_flow"])).sum())
        L.backward()
        for name, tg, og in [("means", tm.grad, g["means"]), ("chol", tc.grad, g["chol"]),
                             ("weights", tl.grad, g["weights"]),
                             ("R", tR.grad.reshape(-1), g["pose"][:9]), ("t", tt.grad, g["pose"][9:]),
                             ("tR", gR.grad.reshape(-1), g["target_poses"][0, :9]),
                             ("tt", gt.grad.reshape(-1), g["target_poses"][0, 9:])]:
            tg = tg.numpy()
            assert np.max(np.abs(tg - og)) <= 1e-10 * max(1.0, np.max(np.abs(tg))), name


def test_twist_gradient_matches_rotation_differences(oracle_mod):
    """The 6-DoF (left twist) pose gradient derived from the free-matrix gradient
    equals central differences of the loss along exp(xi^) [R | t]."""
    from scipy.linalg import expm

    mu, chol, lam, pose, tgt, ups = tiny_scene(7)
    g = oracle_mod.backward_view(mu, chol, lam, pose, tgt[None], CAM, **ups)
    tw = oracle_mod.pose_twist_grad(pose, g["pose"])
    R = pose[:9].reshape(3, 3)
    t = pose[9:]

    def perturbed(xi):
        rho, om = xi[:3], xi[3:]
        S = np.zeros((4, 4))
        S[:3, :3] = [[0, -om[2], om[1]], [om[2], 0, -om[0]], [-om[1], om[0], 0]]
        S[:3, 3] = rho
        T = expm(S) @ np.block([[R, t[:, None]], [np.zeros((1, 3)), np.ones((1, 1))]])
        return np.concatenate([T[:3, :3].reshape(-1), T[:3, 3]])

    h = 1e-6
    fd = np.zeros(6)
    for i in range(6):
        e = np.zeros(6)
        e[i] = h
        fd[i] = (loss(oracle_mod, mu, chol, lam, perturbed(e), tgt, ups)
                 - loss(oracle_mod, mu, chol, lam, perturbed(-e), tgt, ups)) / (2 * h)
    np.testing.assert_allclose(tw, fd, rtol=1e-6, atol=1e-6 * np.max(np.abs(fd)))


def test_scene_backward_sums_views(oracle_mod):
    """The multi-view wrapper adds each view's gradients into the shared object and
    into the right pose rows (own pose and flow target)."""
    s = synth.object_orbit(K=5, n_views=3, W=6, H=5)
    rng = np.random.default_rng(0)
    gd, ga, gn, gf = synth.upstream_grads(rng, s.n_pixels, 1)
    g = oracle_mod.backward_scene(s, gd, ga, gn.reshape(-1), gf.reshape(-1), n_flow=1)
    acc_mu = np.zeros_like(g["means"])
    acc_pose = np.zeros_like(g["poses"])
    for v in s.views:
        o, P = v["pix_offset"], v["W"] * v["H"]
        tgt = v["flow_target"][0]
        r = oracle_mod.backward_view(s.means, s.chol, s.weights, s.poses[v["pose"]], s.poses[[tgt]],
                                     (v["W"], v["H"], v["fx"], v["fy"], v["cx"], v["cy"]),
                                     gd[o:o + P], ga[o:o + P], gn.reshape(-1)[3 * o:3 * o + 3 * P].reshape(3, P).T,
                                     gf.reshape(-1)[2 * o:2 * o + 2 * P].reshape(1, 2, P).transpose(2, 0, 1))
        acc_mu += r["means"]
        acc_pose[v["pose"]] += r["pose"]
        acc_pose[tgt] += r["target_poses"][0]
    np.testing.assert_allclose(g["means"], acc_mu, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g["poses"], acc_pose, rtol=1e-12, atol=1e-12)



@pytest.mark.parametrize("variant", [0, 1])
def test_colour_adjoint_matches_differences_and_autograd(oracle_mod, variant):
    """The colour plane's adjoint: the colours' gradient and the colour term of every
    other gradient, against central differences and the torch restatement."""
    mu, chol, lam, pose, tgt, ups = tiny_scene(11, K=4)
    rng = np.random.default_rng(12)
    col = rng.uniform(0.0, 1.0, (4, 3))
    gcol = rng.standard_normal((20, 3))

    def f():
        r = oracle_mod.render_view(mu, chol, lam, pose, tgt[None], CAM, variant=variant, colors=col)
        return (np.sum(ups["g_depth"] * r["depth"]) + np.sum(ups["g_alpha"] * r["alpha"])
                + np.sum(ups["g_normal"] * r["normal"]) + np.sum(ups["g_flow"] * r["flow"]) + np.sum(gcol * r["color"]))

    g = oracle_mod.backward_view(mu, chol, lam, pose, tgt[None], CAM, **ups, variant=variant, colors=col,
                                 g_color=gcol)
    for name, x, ga in (("colors", col, g["colors"]), ("means", mu, g["means"]), ("chol", chol, g["chol"]),
                        ("weights", lam, g["weights"])):
        gfd = fd_grad(f, x)
        assert np.max(np.abs(ga - gfd)) <= 1e-6 * np.max(np.abs(gfd)), name
    t = lambda a: torch.tensor(a, dtype=torch.float64, requires_grad=True)
    tm, tc, tl, tcol = t(mu), t(chol), t(lam), t(col)
    tR, tt_ = t(pose[:9].reshape(3, 3)), t(pose[9:])
    gR, gt = t(tgt[:9].reshape(3, 3)[None]), t(tgt[9:][None])
    d, a, n, fl, c = torch_ref.render(tm, tc, tl, tR, tt_, gR, gt, CAM, variant=variant, colors=tcol)
    L = ((d * torch.tensor(ups["g_depth"])).sum() + (a * torch.tensor(ups["g_alpha"])).sum()
         + (n * torch.tensor(ups["g_normal"])).sum() + (fl * torch.tensor(ups["g_flow"])).sum()
         + (c * torch.tensor(gcol)).sum())
    L.backward()
    for name, tg, og in (("colors", tcol.grad, g["colors"]), ("means", tm.grad, g["means"]),
                         ("chol", tc.grad, g["chol"]), ("weights", tl.grad, g["weights"])):
        tg = tg.numpy()
        assert np.max(np.abs(tg - og)) <= 1e-10 * max(1.0, np.max(np.abs(tg))), name


def test_package_twist_gradient_matches_oracle(oracle_mod):
    """The package's batched 6-DoF pose gradient (host/torch) against the oracle's,
    which the rotation-difference test above pins."""
    import torch

    from paper_2308_14737_gb300 import fmb

    rng = np.random.default_rng(12)
    poses, grads = [], []
    for _ in range(5):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        poses.append(np.concatenate([q.reshape(-1), rng.normal(size=3)]))
        grads.append(rng.normal(size=12))
    poses, grads = np.array(poses), np.array(grads)
    got = fmb.pose_twist_grad(torch.as_tensor(poses), torch.as_tensor(grads)).numpy()
    for i in range(5):
        assert np.allclose(got[i], oracle_mod.pose_twist_grad(poses[i], grads[i]), rtol=1e-12, atol=1e-12)
