"""FP64 CPU oracle of the simplified Fuzzy Metaballs renderer (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and it
shares no code with it.  The arithmetic lives in ``fmb_oracle.c`` (plain C, FP64,
OpenMP over pixels); this module compiles it, loads it with ctypes and lays out a
multi-view scene the same way the batched output planes are laid out:

* ``depth``, ``alpha``: one value per pixel, views concatenated (``pix_offset``);
* ``normal``: per view a (3, H*W) block at ``3 * pix_offset`` (camera frame);
* ``flow``: per view a (n_flow, 2, H*W) block at ``2 * n_flow * pix_offset``
  (pixels; a slot whose target pose is -1 is zero);
* a view with ``rays`` (a ray batch: pixel indices) contributes only those
  pixels, in list order, so its blocks have len(rays) entries instead of H*W;
* ``saved``: per view a (3, H*W) block at ``3 * pix_offset`` holding
  (log-sum-exp of e_i in natural log, sum of delta_i, |N|); for the
  alpha-compositing variant the first entry is W = sum of the weights instead.

``variant`` selects the weights of Eq. 3: 0 = two-parameter model (Eq. 7),
1 = alpha compositing (Eq. 9-10, Sec. 3.3).

Parity unpinned: nothing.  Every function here is pinned by
``tests/test_oracle_pins.py`` (closed forms, brute force, invariants) and its
adjoint by ``tests/test_oracle_adjoint.py`` (central finite differences and an
independent float64 PyTorch autograd restatement, ``oracle.torch_ref``).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BETA1 = 21.4  # Sec. 7: beta1 = 21.4, reused from prior experiments
BETA2 = 3.14  # Sec. 7: beta2 = 3.14
ETA = 1.0  # Sec. 3.1 shape scale; no value is given, 1 is the neutral choice

_lib = None


def build(force: bool = False) -> str:
    """Compile ``fmb_oracle.c`` into ``liboracle.so`` (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_longlong)
        common = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, dp,
                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_longlong, lp]
        L.fmbo_forward.argtypes = common + [dp, dp, dp, dp, dp, ctypes.c_int]
        L.fmbo_forward.restype = ctypes.c_int
        L.fmbo_backward.argtypes = common + [dp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        L.fmbo_backward.restype = ctypes.c_int
        cf = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, dp, ctypes.c_int, dp,
              ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_longlong, lp]
        L.fmbo_forward_c.argtypes = cf + [dp, dp, dp, dp, dp, dp, ctypes.c_int]
        L.fmbo_forward_c.restype = ctypes.c_int
        L.fmbo_backward_c.argtypes = cf + [dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, dp, ctypes.c_int]
        L.fmbo_backward_c.restype = ctypes.c_int
        L.fmbo_forward_ac.argtypes = L.fmbo_forward.argtypes
        L.fmbo_forward_ac.restype = ctypes.c_int
        L.fmbo_backward_ac.argtypes = L.fmbo_backward.argtypes
        L.fmbo_backward_ac.restype = ctypes.c_int
        L.fmbo_points.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_longlong, lp,
                                  dp, dp, dp, dp, ctypes.c_int]
        L.fmbo_points.restype = ctypes.c_int
        L.fmbo_attribution.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_longlong, lp,
                                       dp, dp]
        L.fmbo_attribution.restype = ctypes.c_int
        L.fmbo_max_threads.argtypes = []
        L.fmbo_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().fmbo_max_threads())


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def render_view(means, chol, weights, pose, target_poses, cam, beta1=BETA1, beta2=BETA2, eta=ETA,
                pixels=None, n_threads=0, variant=0, colors=None):
    """Forward render of one view.

    ``cam`` = (W, H, fx, fy, cx, cy); ``target_poses`` is a (T, 12) array (T <= 2).
    ``pixels``: optional int64 array of row-major pixel indices (default: all).
    Returns a dict with depth (n,), alpha (n,), normal (n, 3), flow (n, T, 2),
    saved (n, 3)."""
    means, chol, weights, pose = _f64(means), _f64(chol), _f64(weights), _f64(pose)
    tp = _f64(np.zeros((0, 12)) if target_poses is None else np.asarray(target_poses).reshape(-1, 12))
    T = tp.shape[0]
    K = weights.shape[0]
    W, H, fx, fy, cx, cy = cam
    if pixels is None:
        n = int(W) * int(H)
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        n = pix.shape[0]
    out = dict(depth=np.zeros(n), alpha=np.zeros(n), normal=np.zeros((n, 3)),
               flow=np.zeros((n, max(T, 1), 2)), saved=np.zeros((n, 3)))
    pp = pix.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if pix is not None else None
    if colors is not None:
        out["color"] = np.zeros((n, 3))
        rc = lib().fmbo_forward_c(
            int(variant), K, _dp(means), _dp(chol), _dp(weights), _dp(_f64(colors).reshape(K, 3)), _dp(pose), T,
            _dp(tp) if T else None, int(W), int(H), float(fx), float(fy), float(cx), float(cy), float(beta1),
            float(beta2), float(eta), n, pp, _dp(out["depth"]), _dp(out["alpha"]), _dp(out["normal"]),
            _dp(out["flow"]), _dp(out["saved"]), _dp(out["color"]), int(n_threads))
    else:
        fn = lib().fmbo_forward_ac if variant == 1 else lib().fmbo_forward
        rc = fn(
            K, _dp(means), _dp(chol), _dp(weights), _dp(pose), T, _dp(tp) if T else None,
            int(W), int(H), float(fx), float(fy), float(cx), float(cy), float(beta1), float(beta2), float(eta),
            n, pp, _dp(out["depth"]), _dp(out["alpha"]), _dp(out["normal"]), _dp(out["flow"]), _dp(out["saved"]),
            int(n_threads))
    if rc != 0:
        raise ValueError(f"fmbo_forward failed with status {rc}")
    out["flow"] = out["flow"][:, :T, :]
    return out


def backward_view(means, chol, weights, pose, target_poses, cam, g_depth=None, g_alpha=None, g_normal=None,
                  g_flow=None, beta1=BETA1, beta2=BETA2, eta=ETA, pixels=None, n_threads=0, variant=0,
                  colors=None, g_color=None):
    """Analytic FP64 adjoint of one view.  Upstream layouts follow ``render_view``:
    g_depth (n,), g_alpha (n,), g_normal (n, 3), g_flow (n, T, 2).  Returns a dict
    with means (K, 3), chol (K, 6), weights (K,), pose (12,), target_poses (T, 12)."""
    means, chol, weights, pose = _f64(means), _f64(chol), _f64(weights), _f64(pose)
    tp = _f64(np.zeros((0, 12)) if target_poses is None else np.asarray(target_poses).reshape(-1, 12))
    T = tp.shape[0]
    K = weights.shape[0]
    W, H, fx, fy, cx, cy = cam
    if pixels is None:
        n = int(W) * int(H)
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        n = pix.shape[0]
    gd = None if g_depth is None else _f64(g_depth).reshape(n)
    ga = None if g_alpha is None else _f64(g_alpha).reshape(n)
    gn = None if g_normal is None else _f64(g_normal).reshape(n, 3)
    gf = None if (g_flow is None or T == 0) else _f64(g_flow).reshape(n, T, 2)
    out = dict(means=np.zeros((K, 3)), chol=np.zeros((K, 6)), weights=np.zeros(K), pose=np.zeros(12),
               target_poses=np.zeros((max(T, 1), 12)))
    pp = pix.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if pix is not None else None
    if colors is not None:
        out["colors"] = np.zeros((K, 3))
        gc = None if g_color is None else _f64(g_color).reshape(n, 3)
        rc = lib().fmbo_backward_c(
            int(variant), K, _dp(means), _dp(chol), _dp(weights), _dp(_f64(colors).reshape(K, 3)), _dp(pose), T,
            _dp(tp) if T else None, int(W), int(H), float(fx), float(fy), float(cx), float(cy), float(beta1),
            float(beta2), float(eta), n, pp, _dp(gd), _dp(ga), _dp(gn), _dp(gf), _dp(gc), _dp(out["means"]),
            _dp(out["chol"]), _dp(out["weights"]), _dp(out["colors"]), _dp(out["pose"]), _dp(out["target_poses"]),
            int(n_threads))
    else:
        fn = lib().fmbo_backward_ac if variant == 1 else lib().fmbo_backward
        rc = fn(
            K, _dp(means), _dp(chol), _dp(weights), _dp(pose), T, _dp(tp) if T else None,
            int(W), int(H), float(fx), float(fy), float(cx), float(cy), float(beta1), float(beta2), float(eta),
            n, pp, _dp(gd), _dp(ga), _dp(gn), _dp(gf),
            _dp(out["means"]), _dp(out["chol"]), _dp(out["weights"]), _dp(out["pose"]), _dp(out["target_poses"]),
            int(n_threads))
    if rc != 0:
        raise ValueError(f"fmbo_backward failed with status {rc}")
    out["target_poses"] = out["target_poses"][:T]
    return out


def points_view(means, chol, weights, pose, cam, variant=0, beta1=BETA1, beta2=BETA2, eta=ETA, pixels=None,
                n_threads=0):
    """Oriented point export of one view (Sec. 6; see fmbo_points): world-frame
    points (n, 3), normals at the rendered depth (n, 3), screen-space cross-product
    normals of Eq. 16 (n, 3) and the max-weight quality (n,)."""
    means, chol, weights, pose = _f64(means), _f64(chol), _f64(weights), _f64(pose)
    K = weights.shape[0]
    W, H, fx, fy, cx, cy = cam
    if pixels is None:
        n = int(W) * int(H)
        pix = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        n = pix.shape[0]
    out = dict(points=np.zeros((n, 3)), normal_tf=np.zeros((n, 3)), normal_screen=np.zeros((n, 3)),
               quality=np.zeros(n))
    rc = lib().fmbo_points(
        int(variant), K, _dp(means), _dp(chol), _dp(weights), _dp(pose), int(W), int(H), float(fx), float(fy),
        float(cx), float(cy), float(beta1), float(beta2), float(eta), n,
        pix.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if pix is not None else None,
        _dp(out["points"]), _dp(out["normal_tf"]), _dp(out["normal_screen"]), _dp(out["quality"]), int(n_threads))
    if rc != 0:
        raise ValueError(f"fmbo_points failed with status {rc}")
    return out


def points_scene(scene, variant=0, n_threads=0):
    """points_view over every view, in the batched planar layouts: points,
    normal_tf, normal_screen per view a (3, H*W) block at 3 * pix_offset; quality
    one value per pixel."""
    P = scene.n_pixels
    out = dict(points=np.zeros(3 * P), normal_tf=np.zeros(3 * P), normal_screen=np.zeros(3 * P),
               quality=np.zeros(P))
    for v in scene.views:
        sl = scene.object_slice(v["object"])
        r = points_view(scene.means[sl], scene.chol[sl], scene.weights[sl], scene.poses[v["pose"]], _cam(v),
                        variant=variant, n_threads=n_threads)
        o, Pv = v["pix_offset"], v["W"] * v["H"]
        for k in ("points", "normal_tf", "normal_screen"):
            out[k][3 * o:3 * (o + Pv)] = r[k].T.reshape(-1)
        out["quality"][o:o + Pv] = r["quality"]
    return out


def attribution_scene(scene, ray_loss, variant=0, beta1=BETA1, beta2=BETA2, eta=ETA):
    """Loss attribution of Sec. 8 over every view (ray batches included):
    sum over the rendered rays j of ray_loss[j] (batched per-pixel layout) times the
    normalised weight of Gaussian i on ray j.  Returns (sum K,) float64."""
    out = np.zeros(scene.weights.shape[0])
    loss = _f64(ray_loss)
    for v in scene.views:
        sl = scene.object_slice(v["object"])
        o, Pv = v["pix_offset"], _entries(v)
        rays = v.get("rays")
        pix = None if rays is None else np.ascontiguousarray(np.asarray(rays, dtype=np.int64))
        a = np.zeros(sl.stop - sl.start)
        W, H, fx, fy, cx, cy = _cam(v)
        rc = lib().fmbo_attribution(
            int(variant), sl.stop - sl.start, _dp(_f64(scene.means[sl])), _dp(_f64(scene.chol[sl])),
            _dp(_f64(scene.weights[sl])), _dp(_f64(scene.poses[v["pose"]])), int(W), int(H), float(fx), float(fy),
            float(cx), float(cy), float(beta1), float(beta2), float(eta), Pv,
            pix.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if pix is not None else None,
            _dp(np.ascontiguousarray(loss[o:o + Pv])), _dp(a))
        if rc != 0:
            raise ValueError(f"fmbo_attribution failed with status {rc}")
        out[sl] += a
    return out


def _view_targets(scene, v, n_flow):
    """Target pose indices of a view's flow slots (first n_flow entries)."""
    ft = list(v.get("flow_target", (-1, -1)))[:n_flow]
    return ft + [-1] * (n_flow - len(ft))


def _entries(v):
    """Plane entries of a view: its ray batch ("rays"), else W*H."""
    return int(len(v["rays"])) if v.get("rays") is not None else int(v["W"]) * int(v["H"])


def _cam(v):
    return (v["W"], v["H"], v["fx"], v["fy"], v["cx"], v["cy"])


def render_scene(scene, n_flow=1, beta1=BETA1, beta2=BETA2, eta=ETA, n_threads=0, variant=0, colors=None):
    """Forward render of every view of a ``synth.Scene`` into batched planes
    (layouts in the module docstring).  Returns float64 arrays."""
    P = scene.n_pixels
    out = dict(depth=np.zeros(P), alpha=np.zeros(P), normal=np.zeros(3 * P), flow=np.zeros(2 * n_flow * P),
               saved=np.zeros(3 * P))
    if colors is not None:
        out["color"] = np.zeros(3 * P)
    for v in scene.views:
        sl = scene.object_slice(v["object"])
        ft = _view_targets(scene, v, n_flow)
        used = [j for j in ft if j >= 0]
        tp = scene.poses[used] if used else None
        r = render_view(scene.means[sl], scene.chol[sl], scene.weights[sl], scene.poses[v["pose"]], tp, _cam(v),
                        beta1, beta2, eta, pixels=v.get("rays"), n_threads=n_threads, variant=variant,
                        colors=None if colors is None else np.asarray(colors).reshape(-1, 3)[sl])
        Pv = _entries(v)
        o = v["pix_offset"]
        out["depth"][o:o + Pv] = r["depth"]
        out["alpha"][o:o + Pv] = r["alpha"]
        out["normal"][3 * o:3 * o + 3 * Pv] = r["normal"].T.reshape(-1)
        out["saved"][3 * o:3 * o + 3 * Pv] = r["saved"].T.reshape(-1)
        if colors is not None:
            out["color"][3 * o:3 * o + 3 * Pv] = r["color"].T.reshape(-1)
        fl = np.zeros((n_flow, 2, Pv))
        k = 0
        for s, j in enumerate(ft):
            if j >= 0:
                fl[s] = r["flow"][:, k, :].T
                k += 1
        out["flow"][2 * n_flow * o:2 * n_flow * (o + Pv)] = fl.reshape(-1)
    return out


def backward_scene(scene, g_depth, g_alpha, g_normal, g_flow, n_flow=1, beta1=BETA1, beta2=BETA2, eta=ETA,
                   n_threads=0, variant=0, colors=None, g_color=None):
    """Adjoint over every view of a scene with upstream gradients in the batched
    plane layout.  Returns grads for means (sum K, 3), chol (sum K, 6), weights
    (sum K,) and poses (n_poses, 12), float64."""
    g = dict(means=np.zeros(scene.means.shape), chol=np.zeros(scene.chol.shape),
             weights=np.zeros(scene.weights.shape), poses=np.zeros(scene.poses.shape))
    if colors is not None:
        g["colors"] = np.zeros((scene.weights.shape[0], 3))
    for v in scene.views:
        sl = scene.object_slice(v["object"])
        ft = _view_targets(scene, v, n_flow)
        used = [(s, j) for s, j in enumerate(ft) if j >= 0]
        tp = scene.poses[[j for _, j in used]] if used else None
        Pv = _entries(v)
        o = v["pix_offset"]
        gn = None if g_normal is None else np.asarray(g_normal)[3 * o:3 * o + 3 * Pv].reshape(3, Pv).T
        gf = None
        if g_flow is not None and used:
            blk = np.asarray(g_flow)[2 * n_flow * o:2 * n_flow * (o + Pv)].reshape(n_flow, 2, Pv)
            gf = np.stack([blk[s].T for s, _ in used], axis=1)
        r = backward_view(scene.means[sl], scene.chol[sl], scene.weights[sl], scene.poses[v["pose"]], tp, _cam(v),
                          None if g_depth is None else np.asarray(g_depth)[o:o + Pv],
                          None if g_alpha is None else np.asarray(g_alpha)[o:o + Pv],
                          gn, gf, beta1, beta2, eta, pixels=v.get("rays"), n_threads=n_threads, variant=variant,
                          colors=None if colors is None else np.asarray(colors).reshape(-1, 3)[sl],
                          g_color=None if (colors is None or g_color is None)
                          else np.asarray(g_color)[3 * o:3 * o + 3 * Pv].reshape(3, Pv).T)
        g["means"][sl] += r["means"]
        g["chol"][sl] += r["chol"]
        g["weights"][sl] += r["weights"]
        if colors is not None:
            g["colors"][sl] += r["colors"]
        g["poses"][v["pose"]] += r["pose"]
        for k, (_, j) in enumerate(used):
            g["poses"][j] += r["target_poses"][k]
    return g


def pose_twist_grad(pose, grad_pose):
    """Left-twist gradient (rho, omega) of a pose perturbed as exp(xi^) [R | t], from
    the gradient of R (free 3x3, row-major) and t.  Returns a 6-vector."""
    R = np.asarray(pose, dtype=np.float64)[:9].reshape(3, 3)
    t = np.asarray(pose, dtype=np.float64)[9:12]
    gR = np.asarray(grad_pose, dtype=np.float64)[:9].reshape(3, 3)
    gt = np.asarray(grad_pose, dtype=np.float64)[9:12]
    M = gR @ R.T
    om = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]]) + np.cross(t, gt)
    return np.concatenate([gt, om])


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
