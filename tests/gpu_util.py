"""Helpers of the GPU parity tests: run the CUDA path through the C ABI and the FP64
oracle on the same seeded scene, and the tolerances they are compared with.

Tolerances (FP32 GPU vs FP64 oracle):
* depth, alpha, saved sum-delta and the saved log2 normaliser: |d| <= 1e-4 + 1e-5 |ref|
  (depth units; log2 units for the normaliser, whose exponents reach several hundred
  at grazing rays, where the relative term carries the fp32 rounding), depth and
  the other geometric planes only where the oracle's alpha >= 1e-2.  The paper's
  own losses weight depth and flow by the object mask (Sec. 4), and on rays that
  miss every Gaussian the fp32 rounding of the whitened residual (about
  |b| 2^-24 per component, with |b| up to ~40) is amplified by beta1 q, so depth
  there is ill-conditioned for any fp32 evaluation.
* flow (pixels): the depth tolerance propagated through the reprojection,
  |dF/dD| (1e-4 + 1e-5 |D|), plus 1e-4 + 1e-5 |F|.
* normal: 1e-4 / max(|N|, 0.05): the blended vector N carries the weights' ~1e-5
  relative error and is divided by |N| when normalised.
* gradients: per tensor, max |g - g_ref| <= 1e-4 max |g_ref|, with the normal
  plane's upstream gradient weighted by |N| >= 0.05 (oracle): N = sum w_i n_i is
  formed from fp32 terms with ~1e-6 absolute error, so a pixel whose per-Gaussian
  normals nearly cancel carries a relative error ~1e-6/|N| in a gradient that
  itself grows like 1/|N| (one-ulp changes of the fp32 inputs move the exact
  gradient by the same order).
"""

from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2308_14737_gb300 import fmb, synth

ALPHA_MASK = 1e-2
NORMAL_MASK = 0.05
LOG2E = 1.4426950408889634


def dev_scene(scene, device="cuda"):
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
    return T(scene.means), T(scene.chol), T(scene.weights), T(scene.poses)


def gpu_forward(scene, params, device="cuda"):
    r = fmb.Renderer(scene.obj_offsets, scene.views, len(scene.poses), params, device=device)
    m, c, w, p = dev_scene(scene, device)
    out = r.forward(m, c, w, p)
    torch.cuda.synchronize()
    assert fmb.fmb_read_device_status(r.ws) == 0
    res = {k: (v.cpu().numpy().astype(np.float64) if v is not None else None) for k, v in out.items()}
    return res, r, (m, c, w, p)


def gpu_backward(r, dev, ups, want_pose=True):
    T = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float32,
                                                          device=dev[0].device)
    g = r.backward(*dev, T(ups["g_depth"]), T(ups["g_alpha"]), T(ups["g_normal"]), T(ups["g_flow"]),
                   want_pose=want_pose)
    torch.cuda.synchronize()
    assert fmb.fmb_read_device_status(r.ws) == 0
    return {k: (v.cpu().numpy().astype(np.float64) if v is not None else None) for k, v in g.items()}


def many_small_views(n_views, seed=11):
    """n_views tiny views (3x7 to 9x5) of three objects (K = 5, 60, 130), each with its
    own sphere pose and forward flow to the next view's pose."""
    rng = np.random.default_rng(seed)
    objs = [synth.random_gaussians(rng, K, "cholesky") for K in (5, 60, 130)]
    sizes = [(3, 7), (8, 6), (9, 5), (4, 4)]
    poses = [synth.look_at_pose(p) for p in synth.sphere_positions(rng, n_views)]
    views = []
    for i in range(n_views):
        W, H = sizes[i % len(sizes)]
        views.append(dict(W=W, H=H, fx=float(2 * max(W, H)), fy=float(2 * max(W, H)), cx=W / 2, cy=H / 2,
                          object=(i * 7) % 3, pose=i, flow_target=((i + 1) % n_views, -1)))
    return synth.make_scene(objs, views, poses)


def view_slices(scene, n_flow):
    for v in scene.views:
        o, P = v["pix_offset"], synth.view_entries(v)
        yield v, o, P


def plane_view(arr, v, n_ch):
    """The (n_ch, P_v) block of view v in a batched plane."""
    o, P = v["pix_offset"], synth.view_entries(v)
    return arr[n_ch * o:n_ch * (o + P)].reshape(n_ch, P)


def flow_sensitivity(scene, v, depth, n_flow, pix):
    """|dF/dD| per pixel and flow slot (pixels per depth unit), central differences
    of the reprojection at the given depths."""
    R = scene.poses[v["pose"]][:9].astype(np.float64).reshape(3, 3)
    t = scene.poses[v["pose"]][9:].astype(np.float64)
    x = pix % v["W"] + 0.5
    y = pix // v["W"] + 0.5
    c = np.stack([(x - v["cx"]) / v["fx"], (y - v["cy"]) / v["fy"], np.ones_like(x)], 1)
    vc = c / np.linalg.norm(c, axis=1, keepdims=True)
    vw = vc @ R
    o = -R.T @ t
    out = np.zeros((n_flow, len(pix)))
    for j in range(n_flow):
        tg = v["flow_target"][j]
        if tg < 0:
            continue
        Rj = scene.poses[tg][:9].astype(np.float64).reshape(3, 3)
        tj = scene.poses[tg][9:].astype(np.float64)

        def proj(D):
            X = (o + vw * D[:, None]) @ Rj.T + tj
            return np.stack([v["fx"] * X[:, 0] / X[:, 2], v["fy"] * X[:, 1] / X[:, 2]], 1)

        h = 1e-4
        out[j] = np.abs((proj(depth + h) - proj(depth - h)) / (2 * h)).max(1)
    return out


def compare_forward(scene, gpu, ref, n_flow, want_normals, pixels_per_view=None, variant=0, ambiguous=None):
    """Asserts forward parity.  ``gpu`` holds full batched planes; ``ref`` holds the
    oracle's planes either batched (pixels_per_view None) or per view dict
    {view index: (pixel indices, oracle view result)}.  Returns max errors.
    variant 1 (alpha compositing): the first saved plane is W = sum of the weights
    on both sides (compared like alpha) instead of the log-normaliser; pixels in
    ``ambiguous`` (see ac_order_ambiguous) are left out of the depth, normal and
    flow comparisons (alpha, sum delta and W do not depend on the order)."""
    stats = dict(depth=0.0, alpha=0.0, normal=0.0, flow=0.0, sdelta=0.0, lse=0.0)
    for vi, v in enumerate(scene.views):
        o, P = v["pix_offset"], synth.view_entries(v)
        if pixels_per_view is None:
            pix = np.arange(P)
            rd = ref["depth"][o:o + P]
            ra = ref["alpha"][o:o + P]
            rn = plane_view(ref["normal"], v, 3)
            rf = plane_view(ref["flow"], v, 2 * n_flow) if n_flow else None
            rs = plane_view(ref["saved"], v, 3)
        else:
            pix, rv = pixels_per_view[vi]
            rd, ra = rv["depth"], rv["alpha"]
            rn = rv["normal"].T
            rs = rv["saved"].T
            rf = None
            if n_flow:
                rf = np.zeros((2 * n_flow, len(pix)))
                k = 0
                for j in range(n_flow):
                    if v["flow_target"][j] >= 0:
                        rf[2 * j:2 * j + 2] = rv["flow"][:, k, :].T
                        k += 1
        gd = gpu["depth"][o:o + P][pix]
        ga = gpu["alpha"][o:o + P][pix]
        gs = plane_view(gpu["saved"], v, 3)[:, pix]
        mask = ra >= ALPHA_MASK
        unique = np.ones(len(pix), dtype=bool)  # pixels whose result does not depend on an fp32 depth order
        if ambiguous is not None:
            unique = ~(ambiguous[o:o + P][pix] if pixels_per_view is None else ambiguous[vi])
            mask = mask & unique
        tol = lambda ref_: 1e-4 + 1e-5 * np.abs(ref_)
        ea = np.abs(ga - ra)
        assert np.all(ea <= tol(ra)), f"view {vi}: alpha err {ea.max()}"
        ed = np.abs(gd - rd)[mask]
        assert np.all(ed <= tol(rd[mask])), f"view {vi}: depth err {ed.max() if ed.size else 0}"
        es = np.abs(gs[1] - rs[1])
        assert np.all(es <= tol(rs[1])), f"view {vi}: sum-delta err {es.max()}"
        if variant == 1:
            el = np.abs(gs[0] - rs[0])
            assert np.all(el <= tol(rs[0])), f"view {vi}: W err {el.max()}"
        else:
            el = np.abs(gs[0] - rs[0] * LOG2E)[mask]
            assert np.all(el <= tol(rs[0][mask] * LOG2E)), f"view {vi}: lse err {el.max()}"
        stats["alpha"] = max(stats["alpha"], float(ea.max()))
        stats["depth"] = max(stats["depth"], float(ed.max()) if ed.size else 0.0)
        stats["sdelta"] = max(stats["sdelta"], float(es.max()))
        stats["lse"] = max(stats["lse"], float(el.max()) if el.size else 0.0)
        if want_normals:
            gn = plane_view(gpu["normal"], v, 3)[:, pix]
            en = np.abs(gn - rn).max(0)
            ntol = 1e-4 / np.maximum(rs[2], 0.05)
            assert np.all((en <= ntol)[mask]), f"view {vi}: normal err {en[mask].max()}"
            stats["normal"] = max(stats["normal"], float(en[mask].max()) if mask.any() else 0.0)
            assert np.all((np.abs(gs[2] - rs[2]) <= 1e-4 + 1e-4 * rs[2])[unique]), f"view {vi}: |N| err"
        if n_flow:
            gf = plane_view(gpu["flow"], v, 2 * n_flow)[:, pix]
            ray_pix = pix if v.get("rays") is None else np.asarray(v["rays"])[pix]  # image pixels of the entries
            sens = flow_sensitivity(scene, v, rd, n_flow, ray_pix)
            for j in range(n_flow):
                for c in range(2):
                    e = np.abs(gf[2 * j + c] - rf[2 * j + c])
                    ftol = sens[j] * tol(rd) + 1e-4 + 1e-5 * np.abs(rf[2 * j + c])
                    assert np.all((e <= ftol)[mask]), f"view {vi}: flow err {e[mask].max()}"
                    stats["flow"] = max(stats["flow"], float(e[mask].max()) if mask.any() else 0.0)
                    if v["flow_target"][j] < 0:
                        assert np.all(gf[2 * j + c] == 0.0)
    return stats


def masked_upstream(scene, alpha_ref, n_flow, seed=1, pixel_mask=None, nnorm_ref=None, exclude=None):
    """Random upstream gradients in the batched layouts; depth, normal and flow are
    zero where the oracle's alpha < 1e-2 (and outside ``pixel_mask`` if given); the
    normal gradient is also zero where the oracle's blended-normal magnitude |N| is
    below 0.05 (``nnorm_ref``, batched per-pixel array), where the renormalised
    normal is ill-conditioned (its gradient grows like 1/|N|)."""
    rng = np.random.default_rng(seed)
    P = scene.n_pixels
    gd, ga, gn, gf = synth.upstream_grads(rng, P, max(n_flow, 1))
    m = (alpha_ref >= ALPHA_MASK).astype(np.float32)
    if exclude is not None:  # order-ambiguous pixels: only the alpha gradient is unique there
        m = m * (~exclude).astype(np.float32)
    if pixel_mask is not None:
        m = m * pixel_mask
        ga = ga * pixel_mask
    mn = m if nnorm_ref is None else m * (nnorm_ref >= NORMAL_MASK).astype(np.float32)
    gd = gd * m
    gn_b = np.zeros(3 * P, dtype=np.float32)
    gf_b = np.zeros(2 * n_flow * P, dtype=np.float32)
    for v in scene.views:
        o, Pv = v["pix_offset"], synth.view_entries(v)
        gn_b[3 * o:3 * (o + Pv)] = (gn[:, o:o + Pv] * mn[o:o + Pv]).reshape(-1)
        if n_flow:
            gf_b[2 * n_flow * o:2 * n_flow * (o + Pv)] = (gf[:n_flow, :, o:o + Pv] * m[o:o + Pv]).reshape(-1)
    return dict(g_depth=gd, g_alpha=ga, g_normal=gn_b, g_flow=gf_b if n_flow else None)


def compare_grads(gpu, ref, keys=("means", "chol", "weights", "poses"), rel=1e-4):
    errs = {}
    for k in keys:
        if gpu.get(k) is None:
            continue
        g = gpu[k].reshape(ref[k].shape)
        scale = np.max(np.abs(ref[k]))
        err = np.max(np.abs(g - ref[k]))
        errs[k] = err / scale if scale > 0 else err
        assert err <= rel * scale, f"gradient {k}: max err {err:.3e} vs scale {scale:.3e}"
    return errs


def ac_order_ambiguous(scene, pix_per_view=None, rel=1e-6, bound=1e-6):
    """Pixels whose alpha-compositing result depends on a depth order that fp32
    cannot resolve.  Eq. 10's indicator makes depth, normal and flow jump where two
    hits swap order; where two significant hits of a pixel are closer in depth
    than ``rel`` x depth (a few fp32 ulps), either order is a correct fp32 answer.
    A pixel is flagged when swapping such a pair could move the normalised weights
    by more than ``bound`` (|dw_i| + |dw_j| over W).  Computed here in FP64 numpy
    from the hit depths and densities (Eq. 2, 4); returns a bool array over the
    batched pixels, or {view: bool array over its sampled pixels}."""
    out = np.zeros(scene.n_pixels, dtype=bool) if pix_per_view is None else {}
    idx = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    for vi, v in enumerate(scene.views):
        sl = scene.object_slice(v["object"])
        K = sl.stop - sl.start
        R = scene.poses[v["pose"]][:9].astype(np.float64).reshape(3, 3)
        t = scene.poses[v["pose"]][9:].astype(np.float64)
        P = synth.view_entries(v)
        if pix_per_view is None:  # every plane entry: the image's pixels, or the view's ray batch
            pix = np.arange(P) if v.get("rays") is None else np.asarray(v["rays"], dtype=np.int64)
        else:
            pix = np.asarray(pix_per_view[vi], dtype=np.int64)
        x = pix % v["W"] + 0.5
        y = pix // v["W"] + 0.5
        c = np.stack([(x - v["cx"]) / v["fx"], (y - v["cy"]) / v["fy"], np.ones(len(pix))], 1)
        vw = (c / np.linalg.norm(c, axis=1, keepdims=True)) @ R
        o = -R.T @ t
        L = np.zeros((K, 3, 3))
        ch = scene.chol[sl].astype(np.float64)
        for k, (a, b) in enumerate(idx):
            L[:, a, b] = ch[:, k]
        Pm = L @ L.transpose(0, 2, 1)
        m = scene.means[sl].astype(np.float64) - o
        Pv = np.einsum("kab,pb->pka", Pm, vw)
        tt = np.einsum("ka,pka->pk", m, Pv) / np.einsum("pa,pka->pk", vw, Pv)
        r = vw[:, None, :] * tt[..., None] - m[None]
        q = np.einsum("pka,kab,pkb->pk", r, Pm, r)
        delta = np.exp(-0.5 * q + np.log(scene.weights[sl].astype(np.float64))[None])
        order = np.argsort(tt, axis=1)
        ts = np.take_along_axis(tt, order, 1)
        ds = np.take_along_axis(delta, order, 1)
        S = np.concatenate([np.zeros((len(pix), 1)), np.cumsum(ds, 1)[:, :-1]], 1)
        w = np.exp(-S) * -np.expm1(-ds)
        Wt = np.maximum(w.sum(1), 1e-300)
        gap = np.diff(ts, axis=1)  # exact ties (duplicates) are exact in fp32 too: not ambiguous
        close = (gap > 0) & (gap <= rel * np.maximum(np.abs(ts[:, 1:]), 1.0))
        dw = (w[:, :-1] * -np.expm1(-ds[:, 1:]) + w[:, 1:] * np.expm1(ds[:, :-1])) / Wt[:, None]
        flag = np.any(close & (dw > bound), axis=1)
        if pix_per_view is None:
            out[v["pix_offset"]:v["pix_offset"] + P] = flag
        else:
            out[vi] = flag
    return out


def nnorm_batched(scene, saved):
    """Per-pixel |N| (channel 2 of the saved planes) in the batched pixel layout."""
    out = np.zeros(scene.n_pixels)
    for v in scene.views:
        o, P = v["pix_offset"], synth.view_entries(v)
        out[o:o + P] = saved[3 * o + 2 * P:3 * o + 3 * P]
    return out


def oracle_forward_sampled(scene, pix_per_view, n_flow, **kw):
    """Oracle forward of the given pixels of each view: {view: (pixels, result)}."""
    out = {}
    for vi, v in enumerate(scene.views):
        sl = scene.object_slice(v["object"])
        used = [j for j in v["flow_target"][:n_flow] if j >= 0]
        tp = scene.poses[used] if used else None
        cam = (v["W"], v["H"], v["fx"], v["fy"], v["cx"], v["cy"])
        pix = np.asarray(pix_per_view[vi], dtype=np.int64)
        out[vi] = (pix, oracle.render_view(scene.means[sl], scene.chol[sl], scene.weights[sl],
                                           scene.poses[v["pose"]], tp, cam, pixels=pix, **kw))
    return out


def oracle_backward_sampled(scene, ups, pix_per_view, n_flow, **kw):
    """Oracle adjoint restricted to the given pixels (exact when the upstream
    gradients vanish elsewhere)."""
    g = dict(means=np.zeros(scene.means.shape), chol=np.zeros(scene.chol.shape),
             weights=np.zeros(scene.weights.shape), poses=np.zeros(scene.poses.shape))
    for vi, v in enumerate(scene.views):
        pix = np.asarray(pix_per_view[vi], dtype=np.int64)
        if len(pix) == 0:
            continue
        sl = scene.object_slice(v["object"])
        slots = [(s, j) for s, j in enumerate(v["flow_target"][:n_flow]) if j >= 0]
        tp = scene.poses[[j for _, j in slots]] if slots else None
        cam = (v["W"], v["H"], v["fx"], v["fy"], v["cx"], v["cy"])
        o, P = v["pix_offset"], v["W"] * v["H"]
        gd = ups["g_depth"][o:o + P][pix]
        ga = ups["g_alpha"][o:o + P][pix]
        gn = ups["g_normal"][3 * o:3 * (o + P)].reshape(3, P)[:, pix].T
        gf = None
        if n_flow and slots:
            blk = ups["g_flow"][2 * n_flow * o:2 * n_flow * (o + P)].reshape(n_flow, 2, P)[:, :, pix]
            gf = np.stack([blk[s].T for s, _ in slots], axis=1)
        r = oracle.backward_view(scene.means[sl], scene.chol[sl], scene.weights[sl], scene.poses[v["pose"]], tp, cam,
                                 gd, ga, gn, gf, pixels=pix, **kw)
        g["means"][sl] += r["means"]
        g["chol"][sl] += r["chol"]
        g["weights"][sl] += r["weights"]
        g["poses"][v["pose"]] += r["pose"]
        for k, (_, j) in enumerate(slots):
            g["poses"][j] += r["target_poses"][k]
    return g


def sample_pixels(scene, n_per_view, seed=0):
    rng = np.random.default_rng(seed)
    out = {}
    for vi, v in enumerate(scene.views):
        P = v["W"] * v["H"]
        k = min(n_per_view, P)
        out[vi] = np.sort(rng.choice(P, size=k, replace=False))
    return out


def pixel_mask_from(scene, pix_per_view):
    m = np.zeros(scene.n_pixels, dtype=np.float32)
    for vi, v in enumerate(scene.views):
        m[v["pix_offset"] + np.asarray(pix_per_view[vi], dtype=np.int64)] = 1.0
    return m


def _view_pairs_fp64(scene, v):
    """FP64 per (pixel, Gaussian) quantities of one whole view: world rays, hit
    depths t, densities delta and the precision matrices (test-side restatement of
    Eq. 2 and Eq. 4, used only to bound how much fp32 rounding can move an output)."""
    idx = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    sl = scene.object_slice(v["object"])
    K = sl.stop - sl.start
    R = scene.poses[v["pose"]][:9].astype(np.float64).reshape(3, 3)
    t = scene.poses[v["pose"]][9:].astype(np.float64)
    P = v["W"] * v["H"]
    pix = np.arange(P)
    x = pix % v["W"] + 0.5
    y = pix // v["W"] + 0.5
    c = np.stack([(x - v["cx"]) / v["fx"], (y - v["cy"]) / v["fy"], np.ones(P)], 1)
    vw = (c / np.linalg.norm(c, axis=1, keepdims=True)) @ R
    o = -R.T @ t
    L = np.zeros((K, 3, 3))
    ch = scene.chol[sl].astype(np.float64)
    for k, (a, b) in enumerate(idx):
        L[:, a, b] = ch[:, k]
    Pm = L @ L.transpose(0, 2, 1)
    m = scene.means[sl].astype(np.float64) - o
    Pv = np.einsum("kab,pb->pka", Pm, vw)
    tt = np.einsum("ka,pka->pk", m, Pv) / np.einsum("pa,pka->pk", vw, Pv)
    r = vw[:, None, :] * tt[..., None] - m[None]
    q = np.einsum("pka,kab,pkb->pk", r, Pm, r)
    d = -0.5 * q + np.log(scene.weights[sl].astype(np.float64))[None]
    return vw, o, m, Pm, Pv, tt, d


def points_tolerances(scene, ref, variant, dD, beta1=21.4, beta2=3.14):
    """Per-pixel tolerances of the point export.  The GPU evaluates the export at
    its own fp32 depth, the oracle at its FP64 depth; ``dD`` (batched) is the depth
    difference to propagate (the parity test passes the measured |D_gpu - D_ref|,
    itself checked against 1e-4 + 1e-5 |D|, plus 1e-6 |D|):
      points         1e-4 + 1e-5 |D| per component (p = o + v D, |v| = 1)
      normal_tf      2 dD max_i(|Sigma_i^-1 v| / |g_i|) / |N| + 1e-4, the rate at
                     which a per-Gaussian normal at depth D turns with D (over
                     Gaussians with weight > 1e-4), through the renormalisation
      normal_screen  4 dD (|d_x| + |d_y|) / |d_x x d_y| + 1e-4, the cross product
                     of two point differences each off by up to 2 dD (dD the largest
                     of the three pixels')
    Returns batched arrays (points, normal_tf, normal_screen) and, for the two
    normals, where their camera-facing sign is not decided at that tolerance
    (|n_ref . v| <= tol: the normal lies within tol of the plane perpendicular to
    the ray -- at the hit depth every Eq. 17 normal lies in that plane, and a
    sharply peaked two-parameter blend renders close to one hit depth)."""
    Pn = scene.n_pixels
    tp, tn, ts = np.zeros(Pn), np.zeros(Pn), np.zeros(Pn)
    amb_n, amb_s = np.zeros(Pn, dtype=bool), np.zeros(Pn, dtype=bool)
    for v in scene.views:
        o_, Pv_ = v["pix_offset"], v["W"] * v["H"]
        vw, o, m, Pm, Pv, tt, d = _view_pairs_fp64(scene, v)
        D = ref["depth"][o_:o_ + Pv_]
        tolD = 1e-4 + 1e-5 * np.abs(D)
        dDv = dD[o_:o_ + Pv_]
        if variant == 1:
            delta = np.exp(d)
            front = (tt[:, None, :] < tt[:, :, None])
            S = np.einsum("pij,pj->pi", front, delta)
            w = np.exp(-S) * -np.expm1(-delta)
        else:
            e = beta1 * d - beta2 * tt
            w = np.exp(e - e.max(1, keepdims=True))
        w = w / np.maximum(w.sum(1, keepdims=True), 1e-300)
        g = np.einsum("kab,pkb->pka", Pm, vw[:, None, :] * D[:, None, None] - m[None])
        gn = np.linalg.norm(g, axis=-1)
        N = np.einsum("pk,pka->pa", w, g / np.maximum(gn, 1e-300)[..., None])
        rate = np.where(w > 1e-4, np.linalg.norm(Pv, axis=-1) / np.maximum(gn, 1e-300), 0.0).max(1)
        tp[o_:o_ + Pv_] = tolD
        tn[o_:o_ + Pv_] = 2 * dDv * rate / np.maximum(np.linalg.norm(N, axis=1), 1e-300) + 1e-4
        pts = plane_view(ref["points"], v, 3).T
        W_, H_ = v["W"], v["H"]
        pix = np.arange(Pv_)
        xx, yy = pix % W_, pix // W_
        nx = yy * W_ + np.where(xx + 1 < W_, xx + 1, xx - 1)
        ny = np.where(yy + 1 < H_, yy + 1, yy - 1) * W_ + xx
        dx, dy = pts - pts[nx], pts - pts[ny]
        cr = np.linalg.norm(np.cross(dx, dy), axis=1)
        tolDn = np.maximum(np.maximum(dDv, dDv[nx]), dDv[ny])
        ts[o_:o_ + Pv_] = 4 * tolDn * (np.linalg.norm(dx, axis=1) + np.linalg.norm(dy, axis=1)) / np.maximum(
            cr, 1e-300) + 1e-4
        amb_n[o_:o_ + Pv_] = np.abs(np.sum(plane_view(ref["normal_tf"], v, 3).T * vw, 1)) <= tn[o_:o_ + Pv_]
        amb_s[o_:o_ + Pv_] = np.abs(np.sum(plane_view(ref["normal_screen"], v, 3).T * vw, 1)) <= ts[o_:o_ + Pv_]
    return tp, tn, ts, amb_n, amb_s
