"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these retypes the oracle's formulas: each expected value comes from a
brute-force search, a closed form of a special case, or an invariance the paper
states (sort-free blending, shape scale eta, rigid motion, flow as a reprojection
difference).  A dropped term, a wrong sign or index, or a transposed operand in
``oracle/fmb_oracle.c`` fails at least one of them.
"""

import numpy as np
import pytest

from paper_2308_14737_gb300 import synth

B1, B2 = 21.4, 3.14


def ray_of_pixel(pose, cam, x, y):
    """Pinhole ray through the centre of pixel (x, y): world direction, origin,
    camera-frame direction."""
    W, H, fx, fy, cx, cy = cam
    R = np.asarray(pose[:9], dtype=np.float64).reshape(3, 3)
    t = np.asarray(pose[9:12], dtype=np.float64)
    c = np.array([(x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1.0])
    vc = c / np.linalg.norm(c)
    return R.T @ vc, -R.T @ t, vc


def chol_matrix(c):
    L = np.zeros((3, 3))
    L[0, 0], L[1, 0], L[1, 1], L[2, 0], L[2, 1], L[2, 2] = c
    return L


def golden_min(f, a, b, tol=1e-13):
    g = (np.sqrt(5.0) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    while b - a > tol:
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    return 0.5 * (a + b)


def render1(o, mu, chol, lam, pose, cam, pixels=None, targets=None, **kw):
    return o.render_view(np.atleast_2d(mu), np.atleast_2d(chol), np.atleast_1d(lam), pose, targets, cam,
                         pixels=pixels, **kw)


CAM = (16, 12, 16.0, 16.0, 8.0, 6.0)


def test_max_likelihood_depth_matches_line_search(oracle_mod):
    """t_i (next to Eq. 2) is the maximiser of the density along the ray: compare
    with a brute-force golden-section search of q(t) on K=1 scenes, where D = t_1
    (Eq. 3 with one term) and A = 1 - exp(-lambda exp(-q(t*)/2)) (Eq. 2, 4, 8)."""
    rng = np.random.default_rng(11)
    pose = synth.look_at_pose((0.3, -0.2, -4.0))
    for trial in range(6):
        mu, chol, lam = synth.random_gaussians(rng, 1, "cholesky")
        mu = mu.astype(np.float64)[0]
        L = chol_matrix(chol[0].astype(np.float64))
        P = L @ L.T
        pix = rng.integers(0, CAM[0] * CAM[1], size=5)
        r = render1(oracle_mod, mu, chol[0], lam[0], pose, CAM, pixels=pix)
        for k, p in enumerate(pix):
            v, o, _ = ray_of_pixel(pose, CAM, p % CAM[0], p // CAM[0])

            def q(tt):
                x = o + v * tt - mu
                return float(x @ P @ x)

            ts = np.linspace(0.0, 10.0, 2001)
            t0 = ts[int(np.argmin([q(s) for s in ts]))]
            tstar = golden_min(q, t0 - 0.01, t0 + 0.01)
            assert abs(r["depth"][k] - tstar) < 1e-6, (trial, k, r["depth"][k], tstar)
            assert q(r["depth"][k]) <= min(q(r["depth"][k] + 1e-4), q(r["depth"][k] - 1e-4))
            expect_a = 1.0 - np.exp(-float(lam[0]) * np.exp(-0.5 * q(tstar)))
            assert abs(r["alpha"][k] - expect_a) < 1e-9
            assert abs(r["saved"][k, 1] - float(lam[0]) * np.exp(-0.5 * q(tstar))) < 1e-9


def test_single_gaussian_depth_ignores_betas(oracle_mod):
    """K = 1: the blend of Eq. 3 returns t_1 whatever beta1, beta2, eta are."""
    rng = np.random.default_rng(5)
    mu, chol, lam = synth.random_gaussians(rng, 1, "cholesky")
    pose = synth.look_at_pose((0.0, 1.0, -4.0))
    a = render1(oracle_mod, mu[0], chol[0], lam[0], pose, CAM)
    b = render1(oracle_mod, mu[0], chol[0], lam[0], pose, CAM, beta1=3.0, beta2=-7.0, eta=0.3)
    np.testing.assert_allclose(a["depth"], b["depth"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a["alpha"], b["alpha"], rtol=0, atol=1e-15)


def test_isotropic_gaussian_hit_through_centre(oracle_mod):
    """A ray through the centre of an isotropic Gaussian: depth = |mu - o| (camera
    distance to the centre) and alpha = 1 - exp(-lambda) (q = 0, so delta = lambda).
    The local normal of Eq. 17 is undefined there (0/0), so it is not checked."""
    pose = synth.look_at_pose((1.0, 0.5, -4.0))
    for (x, y, rho, s, lam) in [(3, 2, 3.7, 2.0, 0.8), (8, 6, 4.2, 5.0, 1.3), (15, 0, 2.5, 1.0, 0.5)]:
        v, o, _ = ray_of_pixel(pose, CAM, x, y)
        mu = o + rho * v
        chol = np.array([s, 0, s, 0, 0, s])
        r = render1(oracle_mod, mu, chol, lam, pose, CAM, pixels=[y * CAM[0] + x])
        assert abs(r["depth"][0] - rho) < 1e-12
        assert abs(r["alpha"][0] - (1 - np.exp(-lam))) < 1e-12


def test_isotropic_offcentre_normal_direction(oracle_mod):
    """Eq. 17 for an isotropic Gaussian: Sigma^-1 (v t - mu) is parallel to the
    vector from the centre to the foot of the perpendicular on the ray, and the
    output is that unit vector expressed in the camera frame."""
    pose = synth.look_at_pose((0.5, -1.0, -4.0))
    R = np.asarray(pose[:9]).reshape(3, 3)
    rng = np.random.default_rng(3)
    for _ in range(5):
        x, y = int(rng.integers(0, 16)), int(rng.integers(0, 12))
        v, o, _ = ray_of_pixel(pose, CAM, x, y)
        off = rng.standard_normal(3)
        off -= (off @ v) * v
        off *= 0.3 / np.linalg.norm(off)
        mu = o + 3.5 * v + off  # centre displaced perpendicular to the ray
        s = float(rng.uniform(1, 4))
        r = render1(oracle_mod, mu, [s, 0, s, 0, 0, s], 1.0, pose, CAM, pixels=[y * CAM[0] + x])
        foot = o + 3.5 * v
        n_world = (foot - mu) / np.linalg.norm(foot - mu)
        np.testing.assert_allclose(r["normal"][0], R @ n_world, atol=1e-12)
        assert abs(r["depth"][0] - 3.5) < 1e-12


def test_offcentre_isotropic_normals_blend_closed_form(oracle_mod):
    """Eq. 17 blended by Eq. 3 over K = 2 and K = 3 Gaussians.  Isotropic Gaussian i
    (L = s_i I) with its centre displaced from the ray by eps_i along a unit vector
    e_i perpendicular to the ray, at distance rho_i along it: the hit depth is
    t_i = rho_i, the residual o + v t_i - mu_i = -eps_i e_i, so q_i = s_i^2 eps_i^2
    (Eq. 2), the unit normal is n_i = -e_i (Eq. 17), and the Eq. 7 log-weights are
    beta1 (ln lambda_i - q_i / 2) - beta2 rho_i / eta.  With w_i their normalised
    exponentials (Eq. 3): N = -sum_i w_i e_i, the output normal is R N / |N| in the
    camera frame, the saved magnitude is |N| and the depth is sum_i w_i rho_i.
    Blending Sigma^-1 r instead of the unit n_i, or leaving out the
    renormalisation, or a wrong frame, fails this."""
    pose = synth.look_at_pose((0.7, -0.4, -4.0))
    R = np.asarray(pose[:9], dtype=np.float64).reshape(3, 3)
    x, y = 6, 4
    v, o, _ = ray_of_pixel(pose, CAM, x, y)
    b1 = np.cross(v, [0.0, 1.0, 0.0])
    b1 /= np.linalg.norm(b1)
    b2 = np.cross(v, b1)  # (v, b1, b2) orthonormal
    cases = [  # (angle of e_i in the plane normal to the ray, eps_i, s_i, rho_i, lambda_i) per Gaussian, eta
        ([(0.0, 0.10, 2.0, 3.5, 1.0), (np.pi / 2, 0.12, 1.5, 3.6, 1.0)], 1.0),
        ([(0.3, 0.05, 3.0, 3.4, 1.0), (1.4, 0.20, 1.0, 3.45, 1.02)], 1.0),
        ([(0.0, 0.08, 2.5, 3.5, 1.0), (2.1, 0.10, 2.0, 3.55, 0.95), (4.2, 0.06, 3.5, 3.52, 1.05)], 1.0),
        ([(1.0, 0.15, 1.2, 3.3, 1.0), (2.5, 0.09, 2.2, 3.5, 1.03)], 2.0),
    ]
    for gs, eta in cases:
        e = np.stack([np.cos(a) * b1 + np.sin(a) * b2 for a, *_ in gs])
        eps = np.array([g[1] for g in gs])
        sc = np.array([g[2] for g in gs])
        rho = np.array([g[3] for g in gs])
        lam = np.array([g[4] for g in gs])
        mu = o + rho[:, None] * v + eps[:, None] * e
        chol = np.stack([[s_, 0, s_, 0, 0, s_] for s_ in sc])
        r = oracle_mod.render_view(mu, chol, lam, pose, None, CAM, pixels=[y * CAM[0] + x], eta=eta)
        lw = B1 * (np.log(lam) - 0.5 * sc ** 2 * eps ** 2) - B2 * rho / eta
        w = np.exp(lw - lw.max())
        w /= w.sum()
        assert 0.05 < w.min() and w.max() < 0.95  # a real blend, not one dominant Gaussian
        N = -(w[:, None] * e).sum(0)
        np.testing.assert_allclose(r["normal"][0], R @ (N / np.linalg.norm(N)), atol=1e-12)
        assert abs(r["saved"][0, 2] - np.linalg.norm(N)) < 1e-12
        assert abs(r["depth"][0] - w @ rho) < 1e-12


def test_two_centred_gaussians_blend_closed_form(oracle_mod):
    """Two Gaussians centred on the same ray at distances rho1 < rho2: both have
    q = 0 and t = rho, so Eq. 7 gives w_i = lambda_i^beta1 exp(-beta2 rho_i / eta)
    and Eq. 3 gives D = (rho1 + rho2 s) / (1 + s), s = w2 / w1; Eq. 8 gives
    A = 1 - exp(-(lambda1 + lambda2)); the saved log-normaliser is log(w1 + w2)."""
    pose = synth.look_at_pose((0.0, 0.0, -4.0))
    x, y = 5, 7
    v, o, _ = ray_of_pixel(pose, CAM, x, y)
    for (r1, r2, l1, l2, eta) in [(3.5, 4.5, 1.0, 1.0, 1.0), (3.0, 3.2, 0.9, 1.1, 1.0), (3.9, 4.4, 1.2, 0.7, 2.0)]:
        mu = np.stack([o + r1 * v, o + r2 * v])
        chol = np.array([[3, 0.2, 2, -0.1, 0.3, 4], [1.5, 0, 1.5, 0, 0, 1.5]], dtype=np.float64)
        r = oracle_mod.render_view(mu, chol, np.array([l1, l2]), pose, None, CAM, pixels=[y * CAM[0] + x], eta=eta)
        lw1 = B1 * np.log(l1) - B2 * r1 / eta
        lw2 = B1 * np.log(l2) - B2 * r2 / eta
        s = np.exp(lw2 - lw1)
        assert abs(r["depth"][0] - (r1 + r2 * s) / (1 + s)) < 1e-12
        assert abs(r["alpha"][0] - (1 - np.exp(-(l1 + l2)))) < 1e-12
        assert abs(r["saved"][0, 0] - np.logaddexp(lw1, lw2)) < 1e-12


def test_duplicated_gaussians(oracle_mod):
    """Duplicating every Gaussian leaves the normalised weights of Eq. 3 unchanged
    (depth, normal, flow identical) and doubles sum delta (Eq. 8)."""
    s = synth.single_view(seed=2, K=7, W=16, H=12)
    tp = synth.look_at_pose((0.5, 0.0, -4.0))
    a = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], tp[None], (16, 12, 16.0, 16.0, 8.0, 6.0))
    b = oracle_mod.render_view(np.concatenate([s.means] * 2), np.concatenate([s.chol] * 2),
                               np.concatenate([s.weights] * 2), s.poses[0], tp[None], (16, 12, 16.0, 16.0, 8.0, 6.0))
    np.testing.assert_allclose(b["depth"], a["depth"], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(b["normal"], a["normal"], atol=1e-12)
    np.testing.assert_allclose(b["flow"], a["flow"], atol=1e-10)
    np.testing.assert_allclose(b["saved"][:, 1], 2 * a["saved"][:, 1], rtol=1e-13)
    np.testing.assert_allclose(b["alpha"], 1 - np.exp(-2 * a["saved"][:, 1]), rtol=1e-13, atol=1e-15)


def test_permutation_invariance(oracle_mod):
    """Sort-free blending (Sec. 3): every output is invariant under any reordering
    of the Gaussians."""
    s = synth.single_view(seed=4, K=23, W=20, H=16)
    cam = (20, 16, 20.0, 20.0, 10.0, 8.0)
    tp = synth.look_at_pose((1.0, 0.3, -3.8))[None]
    a = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], tp, cam)
    perm = np.random.default_rng(0).permutation(23)
    b = oracle_mod.render_view(s.means[perm], s.chol[perm], s.weights[perm], s.poses[0], tp, cam)
    for k in ("depth", "alpha", "normal", "flow", "saved"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-12, atol=1e-12, err_msg=k)


def _random_rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _move_pose(pose, Q, s):
    """Pose after the world moves by x' = Q x + s (camera attached to the world)."""
    R = np.asarray(pose[:9], dtype=np.float64).reshape(3, 3)
    t = np.asarray(pose[9:12], dtype=np.float64)
    R2 = R @ Q.T
    return np.concatenate([R2.reshape(-1), t - R2 @ s])


def test_rigid_motion_invariance(oracle_mod):
    """Moving scene and cameras together by one rigid motion changes no output
    (normals are reported in the camera frame, flow is a reprojection)."""
    rng = np.random.default_rng(9)
    s = synth.single_view(seed=6, K=11, W=18, H=14)
    cam = (18, 14, 18.0, 18.0, 9.0, 7.0)
    tp = synth.look_at_pose((-1.0, 0.4, -3.9))
    a = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], tp[None], cam)
    Q = _random_rotation(rng)
    sh = rng.standard_normal(3)
    mu2 = s.means.astype(np.float64) @ Q.T + sh
    chol2 = []
    for c in s.chol.astype(np.float64):
        L = chol_matrix(c)
        L2 = np.linalg.cholesky(Q @ L @ L.T @ Q.T)
        chol2.append([L2[0, 0], L2[1, 0], L2[1, 1], L2[2, 0], L2[2, 1], L2[2, 2]])
    b = oracle_mod.render_view(mu2, np.array(chol2), s.weights, _move_pose(s.poses[0], Q, sh),
                               _move_pose(tp, Q, sh)[None], cam)
    for k in ("depth", "alpha", "normal", "flow", "saved"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-9, atol=1e-9, err_msg=k)


def test_eta_scale_covariance(oracle_mod):
    """Sec. 3.1: eta lets shapes of different scales return identical results.
    Scaling the world by k (means k mu, precision factors L/k, camera translation
    k t) together with eta -> k eta scales depth by k and leaves alpha, normal and
    flow unchanged."""
    s = synth.single_view(seed=8, K=9, W=16, H=12)
    cam = (16, 12, 16.0, 16.0, 8.0, 6.0)
    tp = synth.look_at_pose((0.7, -0.4, -3.9))
    a = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], tp[None], cam, eta=1.0)
    for k in (0.5, 3.0):
        p2 = np.asarray(s.poses[0], dtype=np.float64).copy()
        p2[9:] *= k
        t2 = tp.copy()
        t2[9:] *= k
        b = oracle_mod.render_view(k * s.means.astype(np.float64), s.chol.astype(np.float64) / k, s.weights, p2,
                                   t2[None], cam, eta=k)
        np.testing.assert_allclose(b["depth"], k * a["depth"], rtol=1e-11)
        np.testing.assert_allclose(b["alpha"], a["alpha"], rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(b["normal"], a["normal"], atol=1e-10)
        np.testing.assert_allclose(b["flow"], a["flow"], atol=1e-9)


def test_identical_pose_flow_is_zero(oracle_mod):
    """Flow (Sec. 5) is the change of a pixel's coordinates under the target pose:
    the view's own pose moves nothing."""
    s = synth.single_view(seed=1, K=13, W=24, H=20)
    cam = (24, 20, 24.0, 24.0, 12.0, 10.0)
    r = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], np.stack([s.poses[0]] * 2), cam)
    assert np.max(np.abs(r["flow"])) < 1e-11


def test_flow_of_sideways_translation(oracle_mod):
    """A camera translated by delta along its own x axis sees a point at z-depth Z
    move by -fx delta / Z pixels horizontally and not at all vertically.  The
    z-depth of the rendered point is D times the z component of the unit ray."""
    s = synth.single_view(seed=3, K=10, W=16, H=12)
    cam = (16, 12, 14.0, 14.0, 8.0, 6.0)
    pose = np.asarray(s.poses[0], dtype=np.float64)
    for delta in (0.05, -0.2):
        tp = pose.copy()
        tp[9] -= delta  # camera centre moves by +delta along x_cam
        r = oracle_mod.render_view(s.means, s.chol, s.weights, pose, tp[None], cam)
        for p in range(0, 16 * 12, 7):
            _, _, vc = ray_of_pixel(pose, cam, p % 16, p // 16)
            Z = r["depth"][p] * vc[2]
            assert abs(r["flow"][p, 0, 0] - (-cam[2] * delta / Z)) < 1e-10
            assert abs(r["flow"][p, 0, 1]) < 1e-10


def test_blended_normal_perpendicular_to_ray(oracle_mod):
    """Eq. 17 is evaluated at the maximum-likelihood point t_i, where the density's
    derivative along the ray vanishes: v^T Sigma^-1 (v t_i - mu) = 0.  So every n_i,
    and the blended normal, is perpendicular to the ray, and the blended normal has
    unit length (Sec. 6)."""
    s = synth.single_view(seed=12, K=17, W=16, H=12)
    cam = (16, 12, 16.0, 16.0, 8.0, 6.0)
    r = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], None, cam)
    for p in range(16 * 12):
        _, _, vc = ray_of_pixel(s.poses[0], cam, p % 16, p // 16)
        assert abs(r["normal"][p] @ vc) < 1e-10
        assert abs(np.linalg.norm(r["normal"][p]) - 1.0) < 1e-12


def test_large_beta1_selects_densest_hit(oracle_mod):
    """With beta2 = 0 and a very large beta1, Eq. 7 puts all the weight on the
    Gaussian with the largest d_i, so D tends to that Gaussian's t_i.  The per-
    Gaussian t_i and d_i come from K = 1 renders (D = t_i, sum delta = e^{d_i})."""
    s = synth.single_view(seed=13, K=6, W=8, H=6)
    cam = (8, 6, 8.0, 8.0, 4.0, 3.0)
    singles = [oracle_mod.render_view(s.means[i:i + 1], s.chol[i:i + 1], s.weights[i:i + 1], s.poses[0], None, cam)
               for i in range(6)]
    ts = np.stack([x["depth"] for x in singles], 1)
    ds = np.log(np.stack([x["saved"][:, 1] for x in singles], 1))
    r = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], None, cam, beta1=4000.0, beta2=0.0)
    srt = np.sort(ds, axis=1)
    ok = (srt[:, -1] - srt[:, -2]) > 0.02  # a clear winner (exp(-80) residual weight)
    assert ok.sum() > 10
    rows = np.arange(len(ts))[ok]
    np.testing.assert_allclose(r["depth"][ok], ts[rows, np.argmax(ds, 1)[ok]], atol=1e-9)


# ---------------------------------------------------------------- alpha compositing
# Pins of the zero-parameter variant (Sec. 3.3, Eq. 9-10): w_i = T_i (1 - e^-delta_i),
# T_i = exp(-sum of delta_j strictly in front of i).


def test_ac_single_gaussian(oracle_mod):
    """K = 1: T = 1, so W = 1 - e^-delta and the depth is the hit depth itself; on a
    ray through an isotropic centre delta = lambda and t = |mu - o|."""
    pose = synth.look_at_pose((1.0, 0.5, -4.0))
    for (x, y, rho, s, lam) in [(3, 2, 3.7, 2.0, 0.8), (8, 6, 4.2, 5.0, 1.3)]:
        v, o, _ = ray_of_pixel(pose, CAM, x, y)
        r = render1(oracle_mod, o + rho * v, [s, 0, s, 0, 0, s], lam, pose, CAM, pixels=[y * CAM[0] + x], variant=1)
        assert abs(r["depth"][0] - rho) < 1e-12
        assert abs(r["saved"][0, 0] - (1 - np.exp(-lam))) < 1e-12
        assert abs(r["alpha"][0] - (1 - np.exp(-lam))) < 1e-12


def test_ac_two_centred_gaussians_closed_form(oracle_mod):
    """Two Gaussians centred on one ray at rho1 < rho2 (q = 0, delta_i = lambda_i):
    the front one has T = 1, the back one T = e^-lambda1, so
    w1 = 1 - e^-l1, w2 = e^-l1 (1 - e^-l2), D = (w1 rho1 + w2 rho2) / (w1 + w2),
    and W = w1 + w2 = 1 - e^-(l1 + l2) = alpha.  Listing the back one first changes
    nothing."""
    pose = synth.look_at_pose((0.0, 0.0, -4.0))
    x, y = 5, 7
    v, o, _ = ray_of_pixel(pose, CAM, x, y)
    chol = np.array([[3, 0.2, 2, -0.1, 0.3, 4], [1.5, 0, 1.5, 0, 0, 1.5]], dtype=np.float64)
    for (r1, r2, l1, l2) in [(3.5, 4.5, 1.0, 1.0), (3.0, 3.2, 0.3, 2.1), (3.9, 4.4, 2.5, 0.7)]:
        w1 = 1 - np.exp(-l1)
        w2 = np.exp(-l1) * (1 - np.exp(-l2))
        for order in ((0, 1), (1, 0)):
            mu = np.stack([o + r1 * v, o + r2 * v])[list(order)]
            lam = np.array([l1, l2])[list(order)]
            r = oracle_mod.render_view(mu, chol[list(order)], lam, pose, None, CAM, pixels=[y * CAM[0] + x],
                                       variant=1)
            assert abs(r["depth"][0] - (w1 * r1 + w2 * r2) / (w1 + w2)) < 1e-12
            assert abs(r["saved"][0, 0] - (w1 + w2)) < 1e-12
            assert abs(r["alpha"][0] - (w1 + w2)) < 1e-12


def test_ac_weights_telescope_to_alpha(oracle_mod):
    """With distinct hit depths the transmittances telescope: sum_i w_i =
    1 - exp(-sum delta) = alpha on every pixel (and W <= 1)."""
    s = synth.single_view(seed=5, K=17, W=16, H=12)
    r = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], None, CAM, variant=1)
    np.testing.assert_allclose(r["saved"][:, 0], r["alpha"], rtol=1e-12, atol=1e-15)


def test_ac_ties_do_not_attenuate(oracle_mod):
    """Eq. 10's indicator is strict: an exact duplicate sits at the same depth as
    its twin, so neither attenuates the other -- both get w = 1 - e^-delta, W is
    twice the single-copy W, the depth is unchanged, while alpha = 1 - e^-2 sum delta."""
    pose = synth.look_at_pose((0.0, 0.0, -4.0))
    v, o, _ = ray_of_pixel(pose, CAM, 5, 7)
    mu = o + 3.7 * v
    c = [2.0, 0.1, 1.5, 0.0, 0.2, 2.5]
    one = render1(oracle_mod, mu, c, 0.9, pose, CAM, pixels=[7 * CAM[0] + 5], variant=1)
    two = oracle_mod.render_view(np.stack([mu, mu]), np.array([c, c], dtype=np.float64), np.array([0.9, 0.9]), pose,
                                 None, CAM, pixels=[7 * CAM[0] + 5], variant=1)
    assert abs(two["saved"][0, 0] - 2 * one["saved"][0, 0]) < 1e-13
    assert abs(two["depth"][0] - one["depth"][0]) < 1e-12
    assert abs(two["alpha"][0] - (1 - np.exp(-2 * one["saved"][0, 1]))) < 1e-13


def test_ac_permutation_invariance(oracle_mod):
    """The variant sorts by depth internally: outputs do not depend on the order in
    which the Gaussians are given."""
    s = synth.single_view(seed=6, K=19, W=20, H=16)
    cam = (20, 16, 20.0, 20.0, 10.0, 8.0)
    tp = synth.look_at_pose((1.0, 0.3, -3.8))[None]
    a = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], tp, cam, variant=1)
    perm = np.random.default_rng(1).permutation(19)
    b = oracle_mod.render_view(s.means[perm], s.chol[perm], s.weights[perm], s.poses[0], tp, cam, variant=1)
    for k in ("depth", "alpha", "normal", "flow", "saved"):
        np.testing.assert_allclose(b[k], a[k], rtol=1e-12, atol=1e-12, err_msg=k)


def test_ac_dense_front_gaussian_occludes(oracle_mod):
    """A very dense Gaussian in front (lambda = 60: T of everything behind it is
    e^-60) makes the depth that of the front hit, whatever lies behind."""
    pose = synth.look_at_pose((0.0, 0.0, -4.0))
    v, o, _ = ray_of_pixel(pose, CAM, 4, 4)
    mu = np.stack([o + 4.6 * v, o + 3.1 * v, o + 5.0 * v])
    chol = np.array([[2, 0, 2, 0, 0, 2]] * 3, dtype=np.float64)
    r = oracle_mod.render_view(mu, chol, np.array([3.0, 60.0, 5.0]), pose, None, CAM, pixels=[4 * CAM[0] + 4],
                               variant=1)
    assert abs(r["depth"][0] - 3.1) < 1e-12


# ------------------------------------------------------ oriented point export (Sec. 6)


def test_points_quality_closed_forms(oracle_mod):
    """quality = max_i w_i / sum w: 1 for one Gaussian; for two Gaussians centred on
    one ray, Eq. 7 gives s = w2/w1 = (l2/l1)^beta1 e^(-beta2 (r2 - r1)) and
    quality = max(1, s) / (1 + s), and Eq. 9-10 give w1 = 1 - e^-l1,
    w2 = e^-l1 (1 - e^-l2); exact duplicates under Eq. 7 split the weight: 1/2."""
    pose = synth.look_at_pose((0.0, 0.0, -4.0))
    x, y = 5, 7
    v, o, _ = ray_of_pixel(pose, CAM, x, y)
    pixel = [y * CAM[0] + x]
    one = oracle_mod.points_view(np.atleast_2d(o + 3.7 * v), np.array([[2.0, 0, 2.0, 0, 0, 2.0]]), np.array([0.8]),
                                 pose, CAM, pixels=pixel)
    assert one["quality"][0] == 1.0
    np.testing.assert_allclose(one["points"][0], o + 3.7 * v, atol=1e-12)  # through the centre: p = mu
    chol = np.array([[3, 0.2, 2, -0.1, 0.3, 4], [1.5, 0, 1.5, 0, 0, 1.5]], dtype=np.float64)
    for (r1, r2, l1, l2) in [(3.5, 4.5, 1.0, 1.0), (3.0, 3.2, 0.9, 1.1), (3.9, 4.4, 1.2, 0.7)]:
        mu = np.stack([o + r1 * v, o + r2 * v])
        lam = np.array([l1, l2])
        s = np.exp(B1 * np.log(l2 / l1) - B2 * (r2 - r1))
        q0 = oracle_mod.points_view(mu, chol, lam, pose, CAM, pixels=pixel)["quality"][0]
        assert abs(q0 - max(1.0, s) / (1.0 + s)) < 1e-12
        w1, w2 = 1 - np.exp(-l1), np.exp(-l1) * (1 - np.exp(-l2))
        q1 = oracle_mod.points_view(mu, chol, lam, pose, CAM, pixels=pixel, variant=1)["quality"][0]
        assert abs(q1 - max(w1, w2) / (w1 + w2)) < 1e-12
    dup = oracle_mod.points_view(np.stack([o + 3.7 * v] * 2), chol[[1, 1]], np.array([0.8, 0.8]), pose, CAM,
                                 pixels=pixel)
    assert abs(dup["quality"][0] - 0.5) < 1e-15


def test_points_normal_at_rendered_depth_two_centred(oracle_mod):
    """Two isotropic Gaussians centred on one ray at r1 < r2: the rendered depth lies
    between them, so the normal of each evaluated there points along the ray
    (+v for the front one, -v for the back one) and their blend, turned to face the
    camera, is -v -- whichever of the two weighs more (both cases are run)."""
    pose = synth.look_at_pose((0.3, -0.2, -4.0))
    x, y = 9, 4
    v, o, _ = ray_of_pixel(pose, CAM, x, y)
    for lam in ([1.0, 0.6], [0.6, 1.0]):
        for variant in (0, 1):
            mu = np.stack([o + 3.4 * v, o + 4.1 * v])
            chol = np.array([[2.0, 0, 2.0, 0, 0, 2.0], [1.2, 0, 1.2, 0, 0, 1.2]])
            r = oracle_mod.points_view(mu, chol, np.array(lam), pose, CAM, pixels=[y * CAM[0] + x], variant=variant)
            np.testing.assert_allclose(r["normal_tf"][0], -v, atol=1e-12)


def _plane_gaussian(nrm, centre, eps=1e-6):
    """A Gaussian whose precision is n n^T + eps^2 I: its max-likelihood depth along
    any ray is the ray's intersection with the plane through ``centre`` with normal
    ``nrm`` up to a relative O(eps^2)."""
    P = np.outer(nrm, nrm) + eps ** 2 * np.eye(3)
    L = np.linalg.cholesky(P)
    return centre[None], np.array([[L[0, 0], L[1, 0], L[1, 1], L[2, 0], L[2, 1], L[2, 2]]]), np.array([1.0])


def test_points_screen_normal_of_a_plane(oracle_mod):
    """Eq. 16 on a rendered plane: every pixel's cross-product normal is the plane's
    normal, turned towards the camera (also on the last column and row, whose
    neighbours are taken on the other side), and the points lie on the plane."""
    pose = synth.look_at_pose((0.5, 0.4, -4.0))
    R = np.asarray(pose[:9]).reshape(3, 3)
    cam_dir = R.T @ np.array([0.0, 0.0, 1.0])
    for nrm in (np.array([0.2, -0.3, 1.0]), np.array([0.5, 0.1, -1.0])):
        nrm = nrm / np.linalg.norm(nrm)
        mu, chol, lam = _plane_gaussian(nrm, np.array([0.1, -0.2, 0.3]))
        r = oracle_mod.points_view(mu, chol, lam, pose, CAM)
        want = -np.sign(nrm @ cam_dir) * nrm
        np.testing.assert_allclose(r["normal_screen"], np.broadcast_to(want, r["normal_screen"].shape), atol=1e-8)
        np.testing.assert_allclose((r["points"] - mu[0]) @ nrm, 0.0, atol=1e-9)
    line = oracle_mod.points_view(mu, chol, lam, pose, (7, 1, 7.0, 7.0, 3.5, 0.5))
    assert np.all(line["normal_screen"] == 0.0)  # one row: no vertical neighbour


# ----------------------------------------------- loss attribution (Sec. 8, Eq. 19)


@pytest.mark.parametrize("variant", [0, 1])
def test_attribution_partition_of_unity(oracle_mod, variant):
    """The normalised weights of every ray sum to one over the Gaussians, so the
    attributions sum to the total ray loss; one Gaussian takes all of it; exact
    duplicates (equal weights under Eq. 7, equal depths under Eq. 10's strict
    indicator) take equal shares; reordering the Gaussians reorders the result."""
    s = synth.object_orbit(K=9, n_views=2, W=12, H=10)
    loss = np.random.default_rng(0).uniform(0.0, 2.0, s.n_pixels)
    a = oracle_mod.attribution_scene(s, loss, variant=variant)
    assert abs(a.sum() - loss.sum()) < 1e-9 * loss.sum()
    one = synth.make_scene([(s.means[:1], s.chol[:1], s.weights[:1])],
                           [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views], s.poses)
    assert abs(oracle_mod.attribution_scene(one, loss, variant=variant)[0] - loss.sum()) < 1e-9 * loss.sum()
    dup = synth.make_scene([(np.concatenate([s.means[:3]] * 2), np.concatenate([s.chol[:3]] * 2),
                             np.concatenate([s.weights[:3]] * 2))],
                           [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views], s.poses)
    ad = oracle_mod.attribution_scene(dup, loss, variant=variant)
    np.testing.assert_allclose(ad[:3], ad[3:], rtol=1e-12)
    perm = np.random.default_rng(1).permutation(9)
    sp = synth.make_scene([(s.means[perm], s.chol[perm], s.weights[perm])],
                          [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views], s.poses)
    np.testing.assert_allclose(oracle_mod.attribution_scene(sp, loss, variant=variant), a[perm], rtol=1e-12,
                               atol=1e-15)


def test_attribution_two_centred_closed_form(oracle_mod):
    """One pixel, two Gaussians centred on its ray: under Eq. 7 the shares are
    1/(1+s) and s/(1+s) with s = (l2/l1)^beta1 e^(-beta2 (r2 - r1))."""
    pose = synth.look_at_pose((0.0, 0.0, -4.0))
    v, o, _ = ray_of_pixel(pose, CAM, 5, 7)
    scene = synth.make_scene([(np.stack([o + 3.5 * v, o + 4.0 * v]),
                               np.array([[3, 0.2, 2, -0.1, 0.3, 4], [1.5, 0, 1.5, 0, 0, 1.5]]),
                               np.array([1.0, 1.1]))],
                             [dict(W=CAM[0], H=CAM[1], fx=CAM[2], fy=CAM[3], cx=CAM[4], cy=CAM[5], object=0, pose=0,
                                   rays=np.array([7 * CAM[0] + 5]))], [pose])
    a = oracle_mod.attribution_scene(scene, np.array([2.0]))
    s_ = np.exp(B1 * np.log(1.1 / 1.0) - B2 * 0.5)
    np.testing.assert_allclose(a, 2.0 * np.array([1.0, s_]) / (1.0 + s_), rtol=1e-6)


# ------------------------------------------------------------ per-Gaussian colours


@pytest.mark.parametrize("variant", [0, 1])
def test_colour_blend_closed_forms(oracle_mod, variant):
    """Eq. 3 with colours: one Gaussian gives its own colour; two centred on one ray
    give the depth blend's weights applied to the colours (Eq. 7: 1/(1+s), s/(1+s);
    Eq. 9-10: w1 = 1 - e^-l1, w2 = e^-l1 (1 - e^-l2)); a constant colour blends to
    itself anywhere (weights normalised)."""
    pose = synth.look_at_pose((0.0, 0.0, -4.0))
    x, y = 5, 7
    v, o, _ = ray_of_pixel(pose, CAM, x, y)
    pix = [y * CAM[0] + x]
    c1, c2 = np.array([0.9, 0.2, 0.1]), np.array([0.1, 0.5, 0.8])
    one = oracle_mod.render_view(np.atleast_2d(o + 3.7 * v), np.array([[2.0, 0, 2.0, 0, 0, 2.0]]), np.array([0.8]),
                                 pose, None, CAM, pixels=pix, variant=variant, colors=c1[None])
    np.testing.assert_allclose(one["color"][0], c1, atol=1e-15)
    chol = np.array([[3, 0.2, 2, -0.1, 0.3, 4], [1.5, 0, 1.5, 0, 0, 1.5]], dtype=np.float64)
    r1, r2, l1, l2 = 3.2, 4.1, 0.9, 1.3
    r = oracle_mod.render_view(np.stack([o + r1 * v, o + r2 * v]), chol, np.array([l1, l2]), pose, None, CAM,
                               pixels=pix, variant=variant, colors=np.stack([c1, c2]))
    if variant == 0:
        s_ = np.exp(B1 * np.log(l2 / l1) - B2 * (r2 - r1))
        w1, w2 = 1.0, s_
    else:
        w1, w2 = 1 - np.exp(-l1), np.exp(-l1) * (1 - np.exp(-l2))
    np.testing.assert_allclose(r["color"][0], (w1 * c1 + w2 * c2) / (w1 + w2), atol=1e-12)
    s = synth.single_view(seed=3, K=11, W=10, H=8)
    const = oracle_mod.render_view(s.means, s.chol, s.weights, s.poses[0], None, (10, 8, 10.0, 10.0, 5.0, 4.0),
                                   variant=variant, colors=np.tile([0.3, 0.6, 0.2], (11, 1)))
    hit = const["alpha"] > 1e-6
    np.testing.assert_allclose(const["color"][hit], np.broadcast_to([0.3, 0.6, 0.2], (hit.sum(), 3)), atol=1e-12)
