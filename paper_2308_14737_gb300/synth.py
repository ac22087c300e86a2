"""Seeded synthetic scenes for the Fuzzy Metaballs render path.

This module only draws random numbers and lays out cameras. It holds none of the
renderer's arithmetic (no ray/Gaussian evaluation, no blending), so both the CUDA
path and the FP64 oracle can take their inputs from it.

Conventions (shared by every consumer):

* A Gaussian is (mean mu in R^3, lower-triangular precision factor L with
  Sigma^-1 = L L^T, weight lambda > 0).  ``chol`` packs L row-major as
  (L00, L10, L11, L20, L21, L22).  The paper parameterises each component by
  mean, "inverse root precision" and weight (Sec. 3.1).
* A pose is 12 floats: R (3x3, row-major) then t, mapping world to camera,
  x_cam = R x_world + t, with OpenCV axes (x right, y down, z forward).
* A view is a pinhole camera (W, H, fx, fy, cx, cy) looking at one object from one
  pose, optionally with up to two flow-target poses (Sec. 5: forward flow to pose
  i+1, backward flow to pose i-1).  ``pix_offset`` is the pixel offset of the
  view's block inside the batched output planes.

The workloads follow the paper's scale: tens of Gaussians per object (Sec. 4 uses
40) and images of a few hundred pixels per side (Sec. 4 fits about 250x130 on
its GPU).  The paper's own datasets (CO3D videos, the 3DGS ficus) are not
available; these seeded scenes stand in for them.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene",
    "look_at_pose",
    "random_gaussians",
    "ring_positions",
    "sphere_positions",
    "make_scene",
    "single_view",
    "object_orbit",
    "ragged_batch",
    "reconstruction",
    "large_k",
    "SCENES",
    "ray_batch",
    "view_entries",
]


@dataclass
class Scene:
    """Flat, batched scene description (all arrays float32 / int64, C-contiguous)."""

    means: np.ndarray  # (sum K, 3)
    chol: np.ndarray  # (sum K, 6)
    weights: np.ndarray  # (sum K,)
    obj_offsets: np.ndarray  # (n_objects + 1,) int64, Gaussian ranges per object
    poses: np.ndarray  # (n_poses, 12)
    views: list  # list of dicts, see module docstring
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_objects(self) -> int:
        return len(self.obj_offsets) - 1

    @property
    def n_pixels(self) -> int:
        """Entries of the batched planes: every view's pixels, or its ray batch."""
        return int(sum(view_entries(v) for v in self.views))

    def K(self, obj: int) -> int:
        return int(self.obj_offsets[obj + 1] - self.obj_offsets[obj])

    @property
    def n_pairs(self) -> int:
        """Ray-Gaussian pairs of one render: sum over views of (rays of the view) x K."""
        return int(sum(view_entries(v) * self.K(v["object"]) for v in self.views))

    def object_slice(self, obj: int) -> slice:
        return slice(int(self.obj_offsets[obj]), int(self.obj_offsets[obj + 1]))


def _normalize(x: np.ndarray) -> np.ndarray:
    return x / np.linalg.norm(x)


def look_at_pose(position, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World-to-camera pose (R row-major, t) of a camera at ``position`` looking at
    ``target``.  OpenCV axes; ``up`` becomes -y_cam.  If the viewing direction is
    within about 8 degrees of ``up`` the up vector switches to +z."""
    p = np.asarray(position, dtype=np.float64)
    z = _normalize(np.asarray(target, dtype=np.float64) - p)
    u = np.asarray(up, dtype=np.float64)
    if abs(float(np.dot(z, _normalize(u)))) > 0.99:
        u = np.array([0.0, 0.0, 1.0])
    x = _normalize(np.cross(z, u))
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    t = -R @ p
    return np.concatenate([R.reshape(-1), t]).astype(np.float64)


def ring_positions(n: int, radius: float = 4.0) -> np.ndarray:
    """``n`` camera centres evenly spaced on the y=0 circle of the given radius."""
    th = 2.0 * np.pi * np.arange(n) / n
    return np.stack([radius * np.cos(th), np.zeros(n), radius * np.sin(th)], axis=1)


def sphere_positions(rng: np.random.Generator, n: int, radius: float = 4.0) -> np.ndarray:
    """``n`` camera centres with isotropic random directions at the given radius."""
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return radius * d


def random_gaussians(rng: np.random.Generator, K: int, kind: str = "cholesky"):
    """Draw K Gaussians.

    ``kind="cholesky"``: means U[-1,1]^3; L with diagonal exp(U[ln 1, ln 10]) and
    strictly-lower entries N(0, 0.5); weights U[0.5, 1.5].

    ``kind="diag"``: means U[-2,2]^3; diagonal precision exp(U[ln 4, ln 100]) so
    L = diag(sqrt(p)); weights U[0.1, 1].
    """
    if kind == "cholesky":
        mu = rng.uniform(-1.0, 1.0, size=(K, 3))
        diag = np.exp(rng.uniform(np.log(1.0), np.log(10.0), size=(K, 3)))
        off = rng.normal(0.0, 0.5, size=(K, 3))
        lam = rng.uniform(0.5, 1.5, size=K)
        chol = np.stack([diag[:, 0], off[:, 0], diag[:, 1], off[:, 1], off[:, 2], diag[:, 2]], axis=1)
    elif kind == "diag":
        mu = rng.uniform(-2.0, 2.0, size=(K, 3))
        prec = np.exp(rng.uniform(np.log(4.0), np.log(100.0), size=(K, 3)))
        s = np.sqrt(prec)
        z = np.zeros(K)
        chol = np.stack([s[:, 0], z, s[:, 1], z, z, s[:, 2]], axis=1)
        lam = rng.uniform(0.1, 1.0, size=K)
    else:
        raise ValueError(kind)
    return mu.astype(np.float32), chol.astype(np.float32), lam.astype(np.float32)


def view_entries(v) -> int:
    """Rays a view renders: the length of its ray batch ("rays"), else W*H."""
    return int(len(v["rays"])) if v.get("rays") is not None else int(v["W"]) * int(v["H"])


def make_scene(objects, views, poses, name="", meta=None) -> Scene:
    """Assemble a Scene from a list of (means, chol, weights) objects, a list of view
    dicts (without ``pix_offset``) and an array of poses."""
    means = np.concatenate([o[0] for o in objects]).astype(np.float32)
    chol = np.concatenate([o[1] for o in objects]).astype(np.float32)
    weights = np.concatenate([o[2] for o in objects]).astype(np.float32)
    offs = np.zeros(len(objects) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([len(o[2]) for o in objects])
    out_views = []
    pix = 0
    for v in views:
        v = dict(v)
        v.setdefault("flow_target", (-1, -1))
        v["flow_target"] = tuple(int(x) for x in v["flow_target"])
        v["pix_offset"] = pix
        pix += view_entries(v)
        out_views.append(v)
    return Scene(
        means=np.ascontiguousarray(means),
        chol=np.ascontiguousarray(chol),
        weights=np.ascontiguousarray(weights),
        obj_offsets=offs,
        poses=np.ascontiguousarray(np.asarray(poses, dtype=np.float32).reshape(-1, 12)),
        views=out_views,
        name=name,
        meta=dict(meta or {}),
    )


def _view(W, H, f, obj, pose, flow_target=(-1, -1)):
    return dict(W=int(W), H=int(H), fx=float(f), fy=float(f), cx=W / 2.0, cy=H / 2.0,
                object=int(obj), pose=int(pose), flow_target=tuple(flow_target))


def single_view(seed: int = 0, K: int = 40, W: int = 64, H: int = 64) -> Scene:
    """Single view, 64x64, f=64, camera at (0,0,-4) looking at the origin, K=40."""
    rng = np.random.default_rng(seed)
    obj = random_gaussians(rng, K, "cholesky")
    pose = look_at_pose((0.0, 0.0, -4.0))
    return make_scene([obj], [_view(W, H, W, 0, 0)], [pose], name="single_view_64x64_K40")


def object_orbit(seed: int = 0, K: int = 100, n_views: int = 16, W: int = 320, H: int = 240) -> Scene:
    """Object orbit: 16 views at 320x240 (f = W) on the y=0 ring of radius 4, K=100,
    forward flow to the next view (the ring wraps)."""
    rng = np.random.default_rng(seed)
    obj = random_gaussians(rng, K, "cholesky")
    poses = [look_at_pose(p) for p in ring_positions(n_views)]
    views = [_view(W, H, W, 0, i, ((i + 1) % n_views, -1)) for i in range(n_views)]
    return make_scene([obj], views, poses, name=f"orbit_{n_views}x{W}x{H}_K{K}")


def ragged_batch(seed: int = 0, n_objects: int = 64, views_per_object: int = 4,
            K_range=(20, 400), sides=(64, 128, 256, 512)) -> Scene:
    """Ragged batch: objects with K ~ U{20..400}, square sides from {64..512},
    4 random sphere views each (f = side); no flow."""
    rng = np.random.default_rng(seed)
    objects, views, poses = [], [], []
    for o in range(n_objects):
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        side = int(rng.choice(sides))
        objects.append(random_gaussians(rng, K, "cholesky"))
        for p in sphere_positions(rng, views_per_object):
            poses.append(look_at_pose(p))
            views.append(_view(side, side, side, o, len(poses) - 1))
    return make_scene(objects, views, poses, name=f"ragged_{n_objects}obj")


def reconstruction(seed: int = 0, n_views: int = 100, K: int = 256, W: int = 640, H: int = 480) -> Scene:
    """Reconstruction step: 100 sphere views at 640x480 (f=640), K=256, flow to the
    next view (i+1) and the previous one (i-1) where they exist."""
    rng = np.random.default_rng(seed)
    obj = random_gaussians(rng, K, "cholesky")
    poses = [look_at_pose(p) for p in sphere_positions(rng, n_views)]
    views = []
    for i in range(n_views):
        ft = (i + 1 if i + 1 < n_views else -1, i - 1 if i > 0 else -1)
        views.append(_view(W, H, W, 0, i, ft))
    return make_scene([obj], views, poses, name=f"recon_{n_views}x{W}x{H}_K{K}")


def large_k(seed: int = 0, K: int = 4096, n_views: int = 8, W: int = 1024, H: int = 768) -> Scene:
    """Large-K stress: K=4096 diagonal-precision Gaussians, 8 sphere views at
    1024x768 (f=1024), forward flow to the next view."""
    rng = np.random.default_rng(seed)
    obj = random_gaussians(rng, K, "diag")
    poses = [look_at_pose(p) for p in sphere_positions(rng, n_views)]
    views = [_view(W, H, W, 0, i, ((i + 1) % n_views, -1)) for i in range(n_views)]
    return make_scene([obj], views, poses, name=f"largeK_{n_views}x{W}x{H}_K{K}")


SCENES = {"single_view": single_view, "object_orbit": object_orbit, "ragged_batch": ragged_batch,
          "reconstruction": reconstruction, "large_k": large_k}


def ray_batch(scene: Scene, n_rays: int, seed: int = 0) -> Scene:
    """A random ray minibatch drawn across all frames (Sec. 4 optimises on batches of
    rays sampled from every frame): ``n_rays`` (view, pixel) pairs uniform over all
    pixels of all views, without repeats, each view keeping its sampled pixel
    indices (sorted) as ``rays``; views that drew no ray are left out."""
    rng = np.random.default_rng(seed)
    sizes = np.array([int(v["W"]) * int(v["H"]) for v in scene.views], dtype=np.int64)
    flat = np.sort(rng.choice(int(sizes.sum()), size=min(int(n_rays), int(sizes.sum())), replace=False))
    starts = np.concatenate([[0], np.cumsum(sizes)])
    views = []
    for i, v in enumerate(scene.views):
        sel = flat[(flat >= starts[i]) & (flat < starts[i + 1])] - starts[i]
        if len(sel):
            nv = {k: val for k, val in v.items() if k != "pix_offset"}
            nv["rays"] = sel.astype(np.int64)
            views.append(nv)
    objs = [(scene.means[scene.object_slice(o)], scene.chol[scene.object_slice(o)],
             scene.weights[scene.object_slice(o)]) for o in range(scene.n_objects)]
    return make_scene(objs, views, scene.poses, name=scene.name + f"_rays{len(flat)}")


def crop_views(scene: Scene, cw: int, ch: int) -> Scene:
    """Same cameras, but each view restricted to its central cw x ch window (the
    principal point is shifted so the pixels are the central ones of the full
    image)."""
    views = []
    for v in scene.views:
        x0 = (v["W"] - cw) // 2
        y0 = (v["H"] - ch) // 2
        nv = dict(v)
        nv.update(W=cw, H=ch, cx=v["cx"] - x0, cy=v["cy"] - y0)
        nv.pop("pix_offset", None)
        views.append(nv)
    objs = [(scene.means[scene.object_slice(o)], scene.chol[scene.object_slice(o)],
             scene.weights[scene.object_slice(o)]) for o in range(scene.n_objects)]
    return make_scene(objs, views, scene.poses, name=scene.name + f"_crop{cw}x{ch}")


def upstream_grads(rng: np.random.Generator, n_pix: int, n_targets: int = 1):
    """Random upstream gradients for the output planes of ``n_pix`` pixels:
    depth (n), alpha (n), normal (3, n), flow (n_targets, 2, n)."""
    gd = rng.standard_normal(n_pix).astype(np.float32)
    ga = rng.standard_normal(n_pix).astype(np.float32)
    gn = rng.standard_normal((3, n_pix)).astype(np.float32)
    gf = (0.01 * rng.standard_normal((n_targets, 2, n_pix))).astype(np.float32)
    return gd, ga, gn, gf
