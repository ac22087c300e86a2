"""Thin Python binding of libfmb (include/fmb.h).

The functions ``fmb_render_forward``, ``fmb_render_backward``,
``fmb_workspace_bytes`` and ``fmb_read_device_status`` marshal torch tensors (device
memory) and numpy arrays (host metadata) into the C ABI and do nothing else: every
step of the render runs in the library's CUDA kernels.  ``Renderer`` and
``FmbRender`` (a ``torch.autograd.Function``) wrap them for PyTorch users.

There is no fallback: if ``libfmb.so`` has not been built, or no CUDA device is
present, the calls raise.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libfmb.so")

FMB_OK = 0
STATUS_NAMES = {0: "FMB_OK", 1: "FMB_ERR_INVALID_ARG", 2: "FMB_ERR_CUDA", 3: "FMB_ERR_TIMEOUT",
                4: "FMB_ERR_WORKSPACE"}


class FmbParams(ctypes.Structure):
    _fields_ = [("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eta", ctypes.c_float),
                ("variant", ctypes.c_int), ("want_normals", ctypes.c_int), ("n_flow", ctypes.c_int),
                ("deterministic", ctypes.c_int), ("use_persistent", ctypes.c_int),
                ("fwd_rays_per_thread", ctypes.c_int), ("fwd_threads", ctypes.c_int),
                ("bwd_ray_tile", ctypes.c_int), ("bwd_threads", ctypes.c_int), ("store_pairs", ctypes.c_int),
                ("colors", ctypes.c_int), ("fwd_ksplit", ctypes.c_int), ("keep_order", ctypes.c_int),
                ("bwd_gblocks", ctypes.c_int)]


class FmbView(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("object", ctypes.c_int), ("pose", ctypes.c_int),
                ("flow_target", ctypes.c_int * 2), ("pix_offset", ctypes.c_longlong), ("rays", ctypes.c_void_p),
                ("n_rays", ctypes.c_int), ("reserved", ctypes.c_int)]


class FmbAdamParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


class FmbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libfmb.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfmb.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, fp, i, sz = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    P = ctypes.POINTER(FmbParams)
    V = ctypes.POINTER(FmbView)
    LL = ctypes.POINTER(ctypes.c_longlong)
    L.fmb_render_forward.argtypes = [P, i, LL, fp, fp, fp, fp, i, fp, i, V, fp, fp, fp, fp, fp, fp, vp, sz, vp]
    L.fmb_render_forward.restype = ctypes.c_int
    L.fmb_render_backward.argtypes = [P, i, LL, fp, fp, fp, fp, i, fp, i, V, fp, fp, fp, fp, fp, fp, fp, fp, fp,
                                      fp, fp, fp, fp, fp, vp, sz, vp]
    L.fmb_render_backward.restype = ctypes.c_int
    L.fmb_render_forward_noalloc.argtypes = [P, i, LL, fp, fp, fp, fp, i, fp, i, V, fp, fp, fp, fp, fp, fp, vp]
    L.fmb_render_forward_noalloc.restype = ctypes.c_int
    L.fmb_read_noalloc_status.argtypes = [ctypes.POINTER(ctypes.c_int), vp]
    L.fmb_read_noalloc_status.restype = ctypes.c_int
    L.fmb_adam_step.argtypes = [ctypes.POINTER(FmbAdamParams), fp, fp, fp, fp, ctypes.c_longlong, ctypes.c_longlong,
                                fp, vp]
    L.fmb_adam_step.restype = ctypes.c_int
    L.fmb_render_points.argtypes = [P, i, LL, fp, fp, fp, i, fp, i, V, fp, fp, fp, fp, fp, fp, vp, sz, vp]
    L.fmb_render_points.restype = ctypes.c_int
    L.fmb_loss_attribution.argtypes = [P, i, LL, fp, fp, fp, i, fp, i, V, fp, fp, fp, vp, sz, vp]
    L.fmb_loss_attribution.restype = ctypes.c_int
    L.fmb_workspace_bytes.argtypes = [P, i, LL, i, V]
    L.fmb_workspace_bytes.restype = sz
    L.fmb_launch_count.argtypes = [P, i, LL, i, V, i, i]
    L.fmb_launch_count.restype = ctypes.c_int
    L.fmb_forward_ksplit.argtypes = [P, i, LL, i, V]
    L.fmb_forward_ksplit.restype = ctypes.c_int
    L.fmb_read_device_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), vp]
    L.fmb_read_device_status.restype = ctypes.c_int
    L.fmb_last_error.argtypes = []
    L.fmb_last_error.restype = ctypes.c_char_p
    L.fmb_version.argtypes = []
    L.fmb_version.restype = ctypes.c_char_p
    L.fmb_default_params.argtypes = [P]
    L.fmb_default_params.restype = None
    _lib = L
    return L


def default_params(**overrides) -> FmbParams:
    p = FmbParams()
    load_library().fmb_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def view_entries(v) -> int:
    """Plane entries of a view dict: the length of its ray batch ("rays"), else W*H."""
    return int(len(v["rays"])) if v.get("rays") is not None else int(v["W"]) * int(v["H"])


def make_views(views, ray_tensors=None) -> ctypes.Array:
    """ctypes array of FmbView from a list of dicts (W, H, fx, fy, cx, cy, object, pose,
    flow_target, pix_offset[, rays]).  A view with "rays" (a ray batch) needs its
    pixel indices as a device int32 tensor in ``ray_tensors[k]``."""
    arr = (FmbView * len(views))()
    for k, v in enumerate(views):
        a = arr[k]
        a.W, a.H = int(v["W"]), int(v["H"])
        a.fx, a.fy, a.cx, a.cy = float(v["fx"]), float(v["fy"]), float(v["cx"]), float(v["cy"])
        a.object, a.pose = int(v["object"]), int(v["pose"])
        ft = tuple(v.get("flow_target", (-1, -1)))
        a.flow_target[0] = int(ft[0]) if len(ft) > 0 else -1
        a.flow_target[1] = int(ft[1]) if len(ft) > 1 else -1
        a.pix_offset = int(v["pix_offset"])
        if v.get("rays") is not None:
            t = None if ray_tensors is None else ray_tensors[k]
            if t is None or not t.is_cuda or t.dtype != torch.int32:
                raise ValueError("a ray batch needs its pixel indices as a device int32 tensor")
            a.rays = t.data_ptr()
            a.n_rays = int(t.numel())
    return arr


def _offsets(obj_offsets):
    o = np.ascontiguousarray(np.asarray(obj_offsets, dtype=np.int64))
    return o, o.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if t.numel() and not t.is_cuda:
            raise ValueError("device tensors expected")
        if t.numel() and not t.is_contiguous():
            raise ValueError("contiguous tensors expected")
        if t.numel() and t.dtype != torch.float32 and t.dtype != torch.uint8:
            raise ValueError(f"float32 tensors expected, got {t.dtype}")
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(int(t))


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _check(status):
    if status != FMB_OK:
        raise FmbError(status, load_library().fmb_last_error().decode())


# The C ABI takes plain pointers and trusts the caller for every buffer's size, so
# the binding checks each tensor against the batch layout before the call: G, the
# Gaussians (the last object offset); P, the plane entries the views address
# (largest pix_offset + entries); the pose count is the poses tensor's size / 12,
# whatever its shape (a flattened [12 n_poses] tensor is as good as [n_poses][12]).

def _extent(o, va) -> tuple[int, int]:
    G = int(o[-1]) if len(o) else 0
    P = 0
    for a in va:
        P = max(P, int(a.pix_offset) + (int(a.n_rays) if a.rays else int(a.W) * int(a.H)))
    return G, P


def _n_poses(poses) -> int:
    n = int(poses.numel()) if isinstance(poses, torch.Tensor) else 0
    if n == 0 or n % 12:
        raise ValueError(f"poses: 12 floats per camera expected, got {n} floats")
    return n // 12


def _need(**sized):
    """sized: name=(tensor or None, elements the call reads or writes)."""
    for name, (t, n) in sized.items():
        if isinstance(t, torch.Tensor) and t.numel() < n:
            raise ValueError(f"{name}: {t.numel()} elements, the batch needs {n}")


# Elements per Gaussian and per plane entry of the named buffers.
_PER_GAUSSIAN = dict(means=3, chol=6, weights=1, colors=3, grad_means=3, grad_chol=6, grad_weights=1,
                     grad_colors=3, attribution=1)
_PER_ENTRY = dict(depth=1, alpha=1, normal=3, color=3, saved=3, g_depth=1, g_alpha=1, g_normal=3, g_color=3,
                  points=3, normal_tf=3, normal_screen=3, quality=1, ray_loss=1)


def _check_scene(o, va, params, means=None, chol=None, weights=None, colors=None, extent=None, **planes):
    """Checks the scene tensors and the named per-Gaussian or per-entry buffers
    (``flow`` and ``g_flow``: 2 n_flow per entry) against the batch layout;
    ``extent``: its (G, P) when the caller has them (else computed from the views)."""
    G, P = extent if extent is not None else _extent(o, va)
    nf = int(params.n_flow)
    sized = dict(means=(means, 3 * G), chol=(chol, 6 * G), weights=(weights, G), colors=(colors, 3 * G))
    for k, t in planes.items():
        if k in ("flow", "g_flow"):
            sized[k] = (t, 2 * nf * P)
        elif k in _PER_GAUSSIAN:
            sized[k] = (t, _PER_GAUSSIAN[k] * G)
        else:
            sized[k] = (t, _PER_ENTRY[k] * P)
    _need(**sized)


def fmb_workspace_bytes(params: FmbParams, obj_offsets, views) -> int:
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n = L.fmb_workspace_bytes(ctypes.byref(params), len(o) - 1, op, len(va), va)
    if n == 0:
        raise FmbError(1, L.fmb_last_error().decode())
    return int(n)


def fmb_forward_ksplit(params: FmbParams, obj_offsets, views) -> int:
    """Gaussian splits the two-parameter forward uses for this batch (1 = unsplit)."""
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n = L.fmb_forward_ksplit(ctypes.byref(params), len(o) - 1, op, len(va), va)
    if n == 0:
        raise FmbError(1, L.fmb_last_error().decode())
    return int(n)


def fmb_launch_count(params: FmbParams, obj_offsets, views, backward: bool, want_pose: bool = True) -> int:
    """Kernel launches of one forward (backward=False) or backward call of this batch."""
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n = L.fmb_launch_count(ctypes.byref(params), len(o) - 1, op, len(va), va, int(bool(backward)), int(want_pose))
    if n < 0:
        raise FmbError(1, L.fmb_last_error().decode())
    return int(n)


def fmb_render_forward(params, obj_offsets, means, chol, weights, poses, views, depth, alpha, normal, flow, saved,
                       workspace, stream=None, colors=None, color=None, extent=None):
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n_poses = _n_poses(poses)
    _check_scene(o, va, params, means, chol, weights, colors, extent, depth=depth, alpha=alpha, normal=normal,
                 flow=flow, color=color, saved=saved)
    _check(L.fmb_render_forward(ctypes.byref(params), len(o) - 1, op, _ptr(means), _ptr(chol), _ptr(weights),
                                _ptr(colors), n_poses, _ptr(poses), len(va), va, _ptr(depth),
                                _ptr(alpha), _ptr(normal), _ptr(flow), _ptr(color), _ptr(saved), _ptr(workspace),
                                workspace.numel(), _stream(stream)))


def fmb_render_forward_noalloc(params, obj_offsets, means, chol, weights, poses, views, depth, alpha, normal, flow,
                               saved, stream=None, colors=None, color=None, extent=None):
    """fmb_render_forward with the library's fixed scratch instead of a workspace
    (for callers that cannot allocate device memory)."""
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n_poses = _n_poses(poses)
    _check_scene(o, va, params, means, chol, weights, colors, extent, depth=depth, alpha=alpha, normal=normal,
                 flow=flow, color=color, saved=saved)
    _check(L.fmb_render_forward_noalloc(ctypes.byref(params), len(o) - 1, op, _ptr(means), _ptr(chol),
                                        _ptr(weights), _ptr(colors), n_poses, _ptr(poses), len(va), va,
                                        _ptr(depth), _ptr(alpha), _ptr(normal), _ptr(flow), _ptr(color), _ptr(saved),
                                        _stream(stream)))


def fmb_read_noalloc_status(stream=None) -> int:
    """Status word of the last allocation-free forward (0 = no device-side error);
    synchronises the stream."""
    L = load_library()
    st = ctypes.c_int(0)
    _check(L.fmb_read_noalloc_status(ctypes.byref(st), _stream(stream)))
    return int(st.value)


def fmb_render_points(params, obj_offsets, means, chol, weights, poses, views, depth, saved, points, normal_tf,
                      normal_screen, quality, workspace, stream=None, extent=None):
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n_poses = _n_poses(poses)
    _check_scene(o, va, params, means, chol, weights, None, extent, depth=depth, saved=saved, points=points,
                 normal_tf=normal_tf, normal_screen=normal_screen, quality=quality)
    _check(L.fmb_render_points(ctypes.byref(params), len(o) - 1, op, _ptr(means), _ptr(chol), _ptr(weights),
                               n_poses, _ptr(poses), len(va), va, _ptr(depth), _ptr(saved), _ptr(points),
                               _ptr(normal_tf), _ptr(normal_screen), _ptr(quality), _ptr(workspace),
                               workspace.numel(), _stream(stream)))


def fmb_loss_attribution(params, obj_offsets, means, chol, weights, poses, views, saved, ray_loss, attribution,
                         workspace, stream=None, extent=None):
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n_poses = _n_poses(poses)
    _check_scene(o, va, params, means, chol, weights, None, extent, saved=saved, ray_loss=ray_loss,
                 attribution=attribution)
    _check(L.fmb_loss_attribution(ctypes.byref(params), len(o) - 1, op, _ptr(means), _ptr(chol), _ptr(weights),
                                  n_poses, _ptr(poses), len(va), va, _ptr(saved), _ptr(ray_loss),
                                  _ptr(attribution), _ptr(workspace), workspace.numel(), _stream(stream)))


def fmb_render_backward(params, obj_offsets, means, chol, weights, poses, views, depth, normal, saved, g_depth,
                        g_alpha, g_normal, g_flow, grad_means, grad_chol, grad_weights, grad_poses, workspace,
                        stream=None, colors=None, color=None, g_color=None, grad_colors=None, extent=None):
    L = load_library()
    o, op = _offsets(obj_offsets)
    va = views if isinstance(views, ctypes.Array) else make_views(views)
    n_poses = _n_poses(poses)
    _check_scene(o, va, params, means, chol, weights, colors, extent, depth=depth, normal=normal, color=color,
                 saved=saved, g_depth=g_depth, g_alpha=g_alpha, g_normal=g_normal, g_flow=g_flow, g_color=g_color,
                 grad_means=grad_means, grad_chol=grad_chol, grad_weights=grad_weights, grad_colors=grad_colors)
    _need(grad_poses=(grad_poses, 12 * n_poses))
    _check(L.fmb_render_backward(ctypes.byref(params), len(o) - 1, op, _ptr(means), _ptr(chol), _ptr(weights),
                                 _ptr(colors), n_poses, _ptr(poses), len(va), va, _ptr(depth),
                                 _ptr(normal), _ptr(color), _ptr(saved), _ptr(g_depth), _ptr(g_alpha),
                                 _ptr(g_normal), _ptr(g_flow), _ptr(g_color), _ptr(grad_means), _ptr(grad_chol),
                                 _ptr(grad_weights), _ptr(grad_colors), _ptr(grad_poses), _ptr(workspace),
                                 workspace.numel(), _stream(stream)))


def fmb_adam_step(adam: FmbAdamParams, param, grad, m, v, positive_begin, step_counter, stream=None):
    """One fused Adam step over the flat buffers (see include/fmb.h)."""
    L = load_library()
    if step_counter.dtype != torch.int32:
        raise ValueError("step_counter must be an int32 device tensor")
    n = int(param.numel())
    _need(grad=(grad, n), m=(m, n), v=(v, n), step_counter=(step_counter, 1))
    _check(L.fmb_adam_step(ctypes.byref(adam), _ptr(param), _ptr(grad), _ptr(m), _ptr(v), int(param.numel()),
                           int(positive_begin), ctypes.c_void_p(step_counter.data_ptr()), _stream(stream)))


def fmb_read_device_status(workspace, stream=None) -> int:
    L = load_library()
    st = ctypes.c_int(0)
    _check(L.fmb_read_device_status(_ptr(workspace), ctypes.byref(st), _stream(stream)))
    return int(st.value)


def alloc_workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """uint8 device buffer of at least nbytes, 256-byte aligned (torch's caching
    allocator returns 512-byte aligned blocks)."""
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    if ws.data_ptr() % 256:
        raise RuntimeError("workspace not 256-byte aligned")
    return ws


class Renderer:
    """Fixed batch layout (objects, views, params) with preallocated planes and
    workspace.  ``forward`` and ``backward`` enqueue the C ABI calls on the current
    stream; the caller's tensors are read in place."""

    def __init__(self, obj_offsets, views, n_poses, params: FmbParams | None = None, device="cuda"):
        self.params = params if params is not None else default_params()
        self.obj_offsets = np.ascontiguousarray(np.asarray(obj_offsets, dtype=np.int64))
        self.views = [dict(v) for v in views]
        self.rays = [None if v.get("rays") is None else
                     torch.as_tensor(np.asarray(v["rays"], dtype=np.int32), device=device).contiguous()
                     for v in self.views]  # kept alive: the views point at them
        self.c_views = make_views(self.views, self.rays)
        self.n_poses = int(n_poses)
        self.P = max(int(v["pix_offset"]) + view_entries(v) for v in self.views) if self.views else 0
        self.G = int(self.obj_offsets[-1])
        self.device = device
        self.ws = alloc_workspace(fmb_workspace_bytes(self.params, self.obj_offsets, self.c_views), device)
        planes = self.new_planes()
        self.depth, self.alpha, self.normal = planes["depth"], planes["alpha"], planes["normal"]
        self.flow, self.saved, self.color = planes["flow"], planes["saved"], planes["color"]

    def new_planes(self) -> dict:
        """Freshly allocated output planes of this batch layout (depth, alpha, normal,
        flow, color, saved; None for the planes the params do not produce)."""
        nf = self.params.n_flow
        f32 = dict(dtype=torch.float32, device=self.device)
        return dict(depth=torch.empty(self.P, **f32), alpha=torch.empty(self.P, **f32),
                    normal=torch.empty(3 * self.P, **f32) if self.params.want_normals else None,
                    flow=torch.empty(2 * nf * self.P, **f32) if nf > 0 else None,
                    color=torch.empty(3 * self.P, **f32) if self.params.colors else None,
                    saved=torch.empty(3 * self.P, **f32))

    def forward(self, means, chol, weights, poses, stream=None, colors=None, out=None):
        """colors: [G][3] device tensor when params.colors (the colour plane is then
        returned as "color").  out: planes to render into (``new_planes()``); by
        default the renderer's own, which the next call overwrites."""
        if out is None:
            out = dict(depth=self.depth, alpha=self.alpha, normal=self.normal, flow=self.flow, saved=self.saved,
                       color=self.color)
        fmb_render_forward(self.params, self.obj_offsets, means, chol, weights, poses, self.c_views, out["depth"],
                           out["alpha"], out["normal"], out["flow"], out["saved"], self.ws, stream, colors=colors,
                           color=out["color"], extent=(self.G, self.P))
        return out

    def points(self, means, chol, weights, poses, stream=None):
        """Oriented point export (Sec. 6) of the last forward call's depth: world
        points, normals at the rendered depth, screen-space normals (Eq. 16), each
        a planar [3][P_v] block per view, and the max-weight quality [P]."""
        f32 = dict(dtype=torch.float32, device=self.depth.device)
        out = dict(points=torch.empty(3 * self.P, **f32), normal_tf=torch.empty(3 * self.P, **f32),
                   normal_screen=torch.empty(3 * self.P, **f32), quality=torch.empty(self.P, **f32))
        fmb_render_points(self.params, self.obj_offsets, means, chol, weights, poses, self.c_views, self.depth,
                          self.saved, out["points"], out["normal_tf"], out["normal_screen"], out["quality"], self.ws,
                          stream, extent=(self.G, self.P))
        return out

    def attribution(self, means, chol, weights, poses, ray_loss, out=None, stream=None):
        """Sec. 8 loss attribution of the batch's rays (after a forward call of the
        same batch): per Gaussian, the sum of ray_loss times its normalised weight."""
        if out is None:
            out = torch.empty(self.G, dtype=torch.float32, device=means.device)
        fmb_loss_attribution(self.params, self.obj_offsets, means, chol, weights, poses, self.c_views, self.saved,
                             ray_loss, out, self.ws, stream, extent=(self.G, self.P))
        return out

    def backward(self, means, chol, weights, poses, g_depth, g_alpha, g_normal, g_flow, want_pose=True,
                 out=None, stream=None, colors=None, g_color=None, planes=None):
        """Gradients of the forward call whose planes are ``planes`` (default: the
        renderer's own, i.e. its last forward call into them)."""
        G = self.G
        pl = planes if planes is not None else dict(depth=self.depth, normal=self.normal, saved=self.saved,
                                                    color=self.color)
        if out is None:
            f32 = dict(dtype=torch.float32, device=means.device)
            out = dict(means=torch.empty(G, 3, **f32), chol=torch.empty(G, 6, **f32), weights=torch.empty(G, **f32),
                       poses=torch.empty(_n_poses(poses), 12, **f32) if want_pose else None)
            if self.params.colors:
                out["colors"] = torch.empty(G, 3, **f32)
        fmb_render_backward(self.params, self.obj_offsets, means, chol, weights, poses, self.c_views, pl["depth"],
                            pl["normal"], pl["saved"], g_depth, g_alpha, g_normal, g_flow, out["means"], out["chol"],
                            out["weights"], out["poses"], self.ws, stream, colors=colors, color=pl["color"],
                            g_color=g_color, grad_colors=out.get("colors"), extent=(self.G, self.P))
        return out


class FmbRender(torch.autograd.Function):
    """Differentiable render: (means, chol, weights, poses[, colors]) -> (depth,
    alpha, normal, flow[, color]) planes, with the library's adjoint
    (``fmb_render_backward``) as the backward.

    Every call renders into freshly allocated planes (``Renderer.new_planes``), so
    several calls on one renderer may be alive in one autograd graph; the saved
    per-pixel normalisers of each call stay with its graph node.  Planes the
    renderer's params do not produce are returned as empty tensors.  Pose gradients
    are computed only when ``poses`` requires a gradient.  The backward may run
    more than once (``retain_graph``): each run recomputes from the saved planes.
    Inside ``torch.cuda.graph`` the planes come from the graph's memory pool.  With
    ``keep_order`` (alpha compositing) the depth order lives in the renderer's
    workspace, which the last forward wrote: an earlier render's backward finds that
    order instead of its own, and every ray whose stored order fails the check against
    its own recomputed depths is sorted afresh, so the gradients are that render's (to
    the rounding of the other summation order), only slower."""

    @staticmethod
    def forward(ctx, renderer: Renderer, means, chol, weights, poses, colors=None):
        out = renderer.forward(means, chol, weights, poses, colors=colors, out=renderer.new_planes())
        empty = lambda t: t if t is not None else torch.zeros(0, device=means.device)
        res = (out["depth"], out["alpha"], empty(out["normal"]), empty(out["flow"]))
        if renderer.params.colors:
            res = res + (out["color"],)
        ctx.renderer = renderer
        ctx.saved_plane = out["saved"]  # not an output: nothing else holds it
        ctx.has_colors = colors is not None
        ctx.save_for_backward(means, chol, weights, poses, colors, out["depth"], out["normal"], out["color"])
        return res

    @staticmethod
    def backward(ctx, g_depth, g_alpha, g_normal, g_flow, g_color=None):
        r: Renderer = ctx.renderer
        means, chol, weights, poses, colors, depth, normal, color = ctx.saved_tensors
        c = lambda g: None if g is None or g.numel() == 0 else g.contiguous()
        want_pose = bool(ctx.needs_input_grad[4])
        out = r.backward(means, chol, weights, poses, c(g_depth), c(g_alpha), c(g_normal), c(g_flow),
                         want_pose=want_pose, colors=colors, g_color=c(g_color),
                         planes=dict(depth=depth, normal=normal, saved=ctx.saved_plane, color=color))
        return (None, out["means"], out["chol"], out["weights"], out["poses"] if want_pose else None,
                out.get("colors") if ctx.has_colors else None)


def render(renderer: Renderer, means, chol, weights, poses, colors=None):
    """Differentiable render through ``FmbRender``: a tuple (depth, alpha, normal,
    flow) of planes in the batched layouts of ``fmb_render_forward`` (plus the
    colour plane when the renderer's params have colours)."""
    return FmbRender.apply(renderer, means, chol, weights, poses, colors)


def pose_twist_grad(poses, grad_poses):
    """6-DoF pose gradients from the library's free-matrix ones: for each pose [R | t]
    perturbed on the left as exp(xi^) [R | t], xi = (rho, omega), the gradient with
    respect to (rho, omega) is (t_bar, vee(R_bar R^T - (R_bar R^T)^T) + t x t_bar).
    poses, grad_poses: [n][12] (R row-major, then t); returns [n][6]."""
    P = torch.as_tensor(poses).reshape(-1, 12)
    G = torch.as_tensor(grad_poses).reshape(-1, 12).to(P.dtype)
    R, t = P[:, :9].reshape(-1, 3, 3), P[:, 9:]
    gR, gt = G[:, :9].reshape(-1, 3, 3), G[:, 9:]
    M = gR @ R.transpose(1, 2)
    om = torch.stack([M[:, 2, 1] - M[:, 1, 2], M[:, 0, 2] - M[:, 2, 0], M[:, 1, 0] - M[:, 0, 1]], dim=1)
    return torch.cat([gt, om + torch.linalg.cross(t, gt, dim=1)], dim=1)
