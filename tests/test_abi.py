"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/fmb.h declares, its structs match the binding's layout, and host
validation rejects bad arguments before anything touches a device."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2308_14737_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fmb():
    from paper_2308_14737_gb300 import build

    build.build()
    from paper_2308_14737_gb300 import fmb as m

    m.load_library()
    return m


def header_functions():
    src = open(os.path.join(ROOT, "include", "fmb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmb_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_function(fmb):
    names = header_functions()
    assert "fmb_render_forward" in names and "fmb_render_backward" in names
    lib = fmb.load_library()
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layouts(fmb):
    assert ctypes.sizeof(fmb.FmbView) == 64
    assert fmb.FmbView.pix_offset.offset == 40
    assert fmb.FmbView.rays.offset == 48 and fmb.FmbView.n_rays.offset == 56
    assert ctypes.sizeof(fmb.FmbParams) == 68
    assert fmb.FmbParams.store_pairs.offset == 48 and fmb.FmbParams.colors.offset == 52
    assert fmb.FmbParams.keep_order.offset == 60 and fmb.FmbParams.bwd_gblocks.offset == 64


def test_default_params_and_version(fmb):
    p = fmb.default_params()
    assert abs(p.beta1 - 21.4) < 1e-6 and abs(p.beta2 - 3.14) < 1e-6 and p.eta == 1.0
    assert p.want_normals == 1 and p.n_flow == 1 and p.deterministic == 0
    assert b"sm_103a" in fmb.load_library().fmb_version()


def test_workspace_bytes(fmb):
    s = synth.object_orbit(K=10, n_views=3, W=8, H=6)
    p = fmb.default_params()
    n = fmb.fmb_workspace_bytes(p, s.obj_offsets, s.views)
    assert n >= 256 + 48 * 30 and n % 256 == 0
    p.deterministic = 1
    assert fmb.fmb_workspace_bytes(p, s.obj_offsets, s.views) > n


def test_workspace_bytes_stored_pairs(fmb):
    """store_pairs adds three per-pair arrays of sum_v P_v x (K rounded up to a
    multiple of 4) floats each (the stride rounded up to 64 floats)."""
    for K in (10, 11, 12, 13):
        s = synth.object_orbit(K=K, n_views=3, W=8, H=6)
        p = fmb.default_params()
        n0 = fmb.fmb_workspace_bytes(p, s.obj_offsets, s.views)
        p.store_pairs = 1
        n1 = fmb.fmb_workspace_bytes(p, s.obj_offsets, s.views)
        Kp = (K + 3) // 4 * 4
        stride = (3 * 48 * Kp + 63) // 64 * 64
        assert n1 - n0 == 3 * 4 * stride


class _Fake:
    """Stand-in for a device buffer: only its address is used, and validation
    fails before any address is dereferenced."""

    def __init__(self, n=1 << 20):
        self.buf = (ctypes.c_ubyte * 512)()
        self.n = n

    def numel(self):
        return self.n

    def data_ptr(self):
        a = ctypes.addressof(self.buf)
        return (a + 255) // 256 * 256


def _call_fwd(fmb, params, offs, views, n_poses=1, **override):
    L = fmb.load_library()
    f = _Fake()
    va = fmb.make_views(views)
    o = np.asarray(offs, dtype=np.int64)
    args = dict(means=f, chol=f, weights=f, colors=f, poses=f, depth=f, alpha=f, normal=f, flow=f, color=f, saved=f,
                ws=f)
    args.update(override)
    P = lambda k: None if args[k] is None else ctypes.c_void_p(args[k].data_ptr())
    ws = args["ws"]
    return L.fmb_render_forward(ctypes.byref(params), len(o) - 1, o.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                P("means"), P("chol"), P("weights"), P("colors"), n_poses, P("poses"), len(va), va,
                                P("depth"), P("alpha"), P("normal"), P("flow"), P("color"), P("saved"),
                                None if ws is None else ctypes.c_void_p(ws.data_ptr()), 0 if ws is None else ws.n,
                                None), L.fmb_last_error().decode()


def _view(**kw):
    v = dict(W=4, H=3, fx=4.0, fy=4.0, cx=2.0, cy=1.5, object=0, pose=0, flow_target=(-1, -1), pix_offset=0)
    v.update(kw)
    return v


@pytest.mark.parametrize("bad,msg", [
    (dict(W=0), "W and H"),
    (dict(fx=0.0), "fx, fy"),
    (dict(object=1), "object out of range"),
    (dict(pose=3), "pose out of range"),
    (dict(flow_target=(5, -1)), "flow_target"),
    (dict(pix_offset=-1), "pix_offset"),
])
def test_forward_rejects_bad_views(fmb, bad, msg):
    st, err = _call_fwd(fmb, fmb.default_params(), [0, 5], [_view(**bad)])
    assert st == 1 and msg in err


def test_forward_rejects_bad_params(fmb):
    for k, v, msg in [("eta", 0.0, "eta"), ("variant", 3, "variant"), ("n_flow", 3, "n_flow"),
                      ("fwd_rays_per_thread", 3, "fwd_rays_per_thread"), ("bwd_threads", 100, "bwd_threads"),
                      ("bwd_threads", 192, "bwd_threads"), ("bwd_ray_tile", 16, "bwd_ray_tile"),
                      ("store_pairs", 2, "store_pairs"), ("fwd_ksplit", 9, "fwd_ksplit"),
                      ("fwd_ksplit", -1, "fwd_ksplit"), ("bwd_gblocks", 65, "bwd_gblocks"),
                      ("bwd_gblocks", -1, "bwd_gblocks")]:
        p = fmb.default_params()
        setattr(p, k, v)
        st, err = _call_fwd(fmb, p, [0, 5], [_view()])
        assert st == 1 and msg in err, (k, err)


def test_gaussian_block_hint_sizes_the_partials(fmb):
    """bwd_gblocks raises the backward's Gaussian blocks per ray tile: in
    deterministic mode each (tile, block) has a partial slot in the workspace, so the
    workspace grows with the block count; 0 and 1 keep the automatic blocking."""
    s = synth.object_orbit(K=40, n_views=2, W=16, H=16)
    sizes = {}
    for g in (0, 1, 2, 4, 64):
        p = fmb.default_params(deterministic=1, bwd_threads=128, bwd_ray_tile=128, bwd_gblocks=g)
        sizes[g] = fmb.fmb_workspace_bytes(p, s.obj_offsets, s.views)
    assert sizes[0] == sizes[1] < sizes[2] < sizes[4] < sizes[64]


def test_stored_pairs_needs_two_rays_per_thread_and_a_workspace(fmb):
    p = fmb.default_params(store_pairs=1, fwd_rays_per_thread=4)
    st, err = _call_fwd(fmb, p, [0, 5], [_view()])
    assert st == 1 and "store_pairs" in err
    L = fmb.load_library()
    f = _Fake()
    fp = ctypes.c_void_p(f.data_ptr())
    va = fmb.make_views([_view()])
    o = np.asarray([0, 5], dtype=np.int64)
    p = fmb.default_params(store_pairs=1)
    st = L.fmb_render_forward_noalloc(ctypes.byref(p), 1, o.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), fp,
                                      fp, fp, fp, 1, fp, 1, va, fp, fp, fp, fp, fp, fp, None)
    assert st == 1 and "store_pairs" in L.fmb_last_error().decode()


def test_alpha_compositing_limits(fmb):
    """variant 1 takes at most 256 Gaussians per object and no stored pairs."""
    p = fmb.default_params(variant=1)
    st, err = _call_fwd(fmb, p, [0, 257], [_view()])
    assert st == 1 and "256" in err
    assert fmb.fmb_workspace_bytes(p, [0, 256], [_view()]) > 0  # 256 is accepted (no launch here)
    p = fmb.default_params(variant=1, store_pairs=1)
    st, err = _call_fwd(fmb, p, [0, 5], [_view()])
    assert st == 1 and "store_pairs" in err
    p = fmb.default_params(variant=2)
    st, err = _call_fwd(fmb, p, [0, 5], [_view()])
    assert st == 1 and "variant" in err


def test_colour_mode_needs_its_buffers(fmb):
    p = fmb.default_params(colors=1)
    st, err = _call_fwd(fmb, p, [0, 5], [_view()], colors=None)
    assert st == 1 and "colors" in err
    st, err = _call_fwd(fmb, fmb.default_params(colors=1, store_pairs=1), [0, 5], [_view()])
    assert st == 1 and "store_pairs" in err
    st, err = _call_fwd(fmb, fmb.default_params(colors=2), [0, 5], [_view()])
    assert st == 1 and "colors" in err


def test_forward_rejects_bad_scene_and_buffers(fmb):
    p = fmb.default_params()
    assert _call_fwd(fmb, p, [0, 0], [_view()])[0] == 1  # empty object
    assert _call_fwd(fmb, p, [1, 5], [_view()])[0] == 1  # offsets must start at 0
    st, err = _call_fwd(fmb, p, [0, 5], [_view(), _view(pix_offset=6)])
    assert st == 1 and "overlap" in err
    st, err = _call_fwd(fmb, p, [0, 5], [_view()], normal=None)
    assert st == 1 and "normal" in err
    st, err = _call_fwd(fmb, p, [0, 5], [_view()], flow=None)
    assert st == 1 and "flow" in err
    st, err = _call_fwd(fmb, p, [0, 5], [_view()], ws=None)
    assert st == 4
    small = _Fake(n=16)
    st, err = _call_fwd(fmb, p, [0, 5], [_view()], ws=small)
    assert st == 4 and "too small" in err


def test_backward_rejects_missing_outputs(fmb):
    L = fmb.load_library()
    f = _Fake()
    p = fmb.default_params()
    va = fmb.make_views([_view()])
    o = np.asarray([0, 5], dtype=np.int64)
    fp = ctypes.c_void_p(f.data_ptr())
    st = L.fmb_render_backward(ctypes.byref(p), 1, o.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), fp, fp, fp,
                               fp, 1, fp, 1, va, fp, fp, fp, fp, fp, fp, fp, fp, fp, None, fp, fp, fp, None, fp,
                               1 << 20, None)
    assert st == 1 and "grad_means" in L.fmb_last_error().decode()


def test_forward_split_query(fmb):
    """The split count the planner takes (no GPU needed): unsplit by default for a
    full 320x240 orbit, forced when asked, never with colours or stored pairs, and
    the workspace grows by 32 bytes per ray and split."""
    s = synth.object_orbit(K=100, n_views=2, W=32, H=24)
    p = fmb.default_params()
    assert fmb.fmb_forward_ksplit(p, s.obj_offsets, s.views) == 1
    base = fmb.fmb_workspace_bytes(p, s.obj_offsets, s.views)
    p3 = fmb.default_params(fwd_ksplit=3)
    assert fmb.fmb_forward_ksplit(p3, s.obj_offsets, s.views) == 3
    grown = fmb.fmb_workspace_bytes(p3, s.obj_offsets, s.views)
    assert grown - base >= 32 * 3 * s.n_pixels
    assert fmb.fmb_forward_ksplit(fmb.default_params(fwd_ksplit=3, colors=1), s.obj_offsets, s.views) == 1
    assert fmb.fmb_forward_ksplit(fmb.default_params(fwd_ksplit=3, store_pairs=1), s.obj_offsets, s.views) == 1


def test_noalloc_status_reader_rejects_a_null_pointer(fmb):
    """fmb_read_noalloc_status validates its argument on the host before touching a device."""
    L = fmb.load_library()
    assert L.fmb_read_noalloc_status(None, None) == 1
    assert "h_status" in L.fmb_last_error().decode()


def test_launch_count_follows_the_batch_split(fmb):
    """Launches per call: prologue + kernel per launch batch; views beyond one
    batch's capacity (64 views, or 256 for the two-parameter render and adjoint of a
    call with more than 64) add batches; deterministic mode adds the reductions."""
    s = synth.object_orbit(K=10, n_views=3, W=8, H=6)
    p = fmb.default_params()
    assert fmb.fmb_launch_count(p, s.obj_offsets, s.views, backward=False) == 2
    assert fmb.fmb_launch_count(p, s.obj_offsets, s.views, backward=True) == 2
    pd = fmb.default_params(deterministic=1)
    assert fmb.fmb_launch_count(pd, s.obj_offsets, s.views, backward=True, want_pose=True) == 4
    assert fmb.fmb_launch_count(pd, s.obj_offsets, s.views, backward=True, want_pose=False) == 3
    # the two-parameter render and adjoint take up to 256 views per launch once a call
    # has more than 64; alpha compositing keeps 64 per launch
    for n_views, batches in ((64, 1), (65, 1), (200, 1), (256, 1), (300, 2)):
        many = synth.object_orbit(K=10, n_views=n_views, W=4, H=4)
        assert fmb.fmb_launch_count(p, many.obj_offsets, many.views, backward=False) == 2 * batches, n_views
        assert fmb.fmb_launch_count(p, many.obj_offsets, many.views, backward=True) == 2 * batches, n_views
        pa = fmb.default_params(variant=1)
        ac_batches = (n_views + 63) // 64
        assert fmb.fmb_launch_count(pa, many.obj_offsets, many.views, backward=False) == 2 * ac_batches, n_views
    p.fwd_ksplit = 2
    assert fmb.fmb_launch_count(p, s.obj_offsets, s.views, backward=False) == 3


def test_keep_order_workspace_and_validation(fmb):
    """keep_order (alpha compositing) adds 32 M bytes per plane entry to the
    workspace (M = 4 for objects of at most 128 Gaussians), is rejected for the
    two-parameter model and by the allocation-free forward."""
    views = [_view(W=10, H=7)]
    p1 = fmb.default_params(variant=1)
    pk = fmb.default_params(variant=1, keep_order=1)
    extra = fmb.fmb_workspace_bytes(pk, [0, 100], views) - fmb.fmb_workspace_bytes(p1, [0, 100], views)
    assert 70 * 32 * 4 <= extra < 70 * 32 * 4 + 256
    st, err = _call_fwd(fmb, fmb.default_params(keep_order=1), [0, 5], [_view()])
    assert st == 1 and "keep_order" in err
    L = fmb.load_library()
    f = _Fake()
    fp = ctypes.c_void_p(f.data_ptr())
    o = np.asarray([0, 5], dtype=np.int64)
    st = L.fmb_render_forward_noalloc(ctypes.byref(pk), 1, o.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)), fp,
                                      fp, fp, fp, 1, fp, 1, fmb.make_views([_view()]), fp, fp, fp, fp, fp, fp, None)
    assert st == 1 and "keep_order" in L.fmb_last_error().decode()


def _host_call_args(s, fmb, n_flow=1):
    """Host tensors of the right sizes for fmb_render_forward / backward on scene s
    (the binding checks sizes before it requires device memory)."""
    import torch

    G, P = int(s.obj_offsets[-1]), int(s.n_pixels)
    z = lambda n: torch.zeros(n, dtype=torch.float32)
    fwd = dict(means=z(3 * G), chol=z(6 * G), weights=z(G), poses=torch.as_tensor(s.poses, dtype=torch.float32),
               depth=z(P), alpha=z(P), normal=z(3 * P), flow=z(2 * n_flow * P), saved=z(3 * P))
    bwd = dict(g_depth=z(P), g_alpha=z(P), g_normal=z(3 * P), g_flow=z(2 * n_flow * P), grad_means=z(3 * G),
               grad_chol=z(6 * G), grad_weights=z(G), grad_poses=z(12 * len(s.poses)))
    return fwd, bwd


def _call_backward(fmb, s, p, f, b):
    ws = None  # no device: the size checks run before any pointer is taken
    fmb.fmb_render_backward(p, s.obj_offsets, f["means"], f["chol"], f["weights"], f["poses"], s.views,
                            f["depth"], f["normal"], f["saved"], b["g_depth"], b["g_alpha"], b["g_normal"],
                            b["g_flow"], b["grad_means"], b["grad_chol"], b["grad_weights"], b["grad_poses"], ws)


@pytest.mark.parametrize("short", ["means", "chol", "weights", "depth", "normal", "saved", "g_depth", "g_alpha",
                                   "g_normal", "g_flow", "grad_means", "grad_chol", "grad_weights", "grad_poses"])
def test_binding_rejects_short_buffers(fmb, short):
    # The C ABI takes plain pointers; the binding checks every tensor's size against
    # the batch layout (G Gaussians, P plane entries, n_poses = poses' size / 12).
    s = synth.object_orbit(K=10, n_views=3, W=8, H=6)
    p = fmb.default_params(n_flow=1)
    f, b = _host_call_args(s, fmb)
    d = f if short in f else b
    d[short] = d[short][:-1]
    with pytest.raises(ValueError, match=short):
        _call_backward(fmb, s, p, f, b)


def test_binding_pose_count_from_size(fmb):
    # a flattened [12 n_poses] poses tensor is n_poses cameras (its first dimension
    # is not the count): it passes the size checks, and so does a grad_poses of
    # exactly 12 n_poses floats; a size that is not a multiple of 12 is refused
    s = synth.object_orbit(K=10, n_views=3, W=8, H=6)
    p = fmb.default_params(n_flow=1)
    f, b = _host_call_args(s, fmb)
    f["poses"] = f["poses"].reshape(-1)
    with pytest.raises(ValueError, match="device tensors expected"):  # past the size checks
        _call_backward(fmb, s, p, f, b)
    f["poses"] = f["poses"][:-1]
    with pytest.raises(ValueError, match="12 floats per camera"):
        _call_backward(fmb, s, p, f, b)


def test_binding_forward_checks_planes(fmb):
    s = synth.object_orbit(K=10, n_views=3, W=8, H=6)
    p = fmb.default_params(n_flow=1)
    f, _ = _host_call_args(s, fmb)
    for k in ("depth", "alpha", "normal", "flow", "saved"):
        g = dict(f)
        g[k] = g[k][:-1]
        with pytest.raises(ValueError, match=k):
            fmb.fmb_render_forward(p, s.obj_offsets, g["means"], g["chol"], g["weights"], g["poses"], s.views,
                                   g["depth"], g["alpha"], g["normal"], g["flow"], g["saved"], None)


def test_adam_binding_rejects_short_state(fmb):
    import torch

    adam = fmb.FmbAdamParams(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    z = lambda n: torch.zeros(n, dtype=torch.float32)
    step = torch.zeros(1, dtype=torch.int32)
    for short in ("grad", "m", "v"):
        bufs = dict(param=z(10), grad=z(10), m=z(10), v=z(10))
        bufs[short] = z(9)
        with pytest.raises(ValueError, match=short):
            fmb.fmb_adam_step(adam, bufs["param"], bufs["grad"], bufs["m"], bufs["v"], 0, step)
