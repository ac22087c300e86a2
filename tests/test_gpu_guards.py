"""No call writes outside the buffers it is given.  Every output (planes, gradients,
point export, attribution, the Adam step's state) is cut out of a larger buffer whose guard zones on both
sides hold a NaN bit pattern; after forward, backward, point export and loss
attribution the guards must be unchanged and the results bitwise those of the same
calls on plainly allocated buffers (deterministic mode).  The inputs are passed
flattened ([3G], [6G], [G], [12 n_poses]): the binding takes the counts from the
batch layout and the poses' size, not from a tensor's first dimension."""

import numpy as np
import pytest
import torch

from paper_2308_14737_gb300 import fmb, synth

pytestmark = pytest.mark.gpu

GUARD = 4096  # floats on each side
SENTINEL = 0x7F8DEAD1  # a NaN bit pattern no kernel writes


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_14737_gb300 import build

    build.build()
    fmb.load_library()


class Arena:
    """Guarded device buffers: ``take(n)`` returns an n-float view with GUARD floats
    of sentinel before and after it."""

    def __init__(self):
        self.bufs = []

    def take(self, n):
        raw = torch.full((n + 2 * GUARD,), SENTINEL, dtype=torch.int32, device="cuda")
        self.bufs.append((raw, n))
        return raw[GUARD:GUARD + n].view(torch.float32)

    def intact(self):
        torch.cuda.synchronize()
        bad = []
        for i, (raw, n) in enumerate(self.bufs):
            lo = raw[:GUARD].cpu().numpy()
            hi = raw[GUARD + n:].cpu().numpy()
            if (lo != SENTINEL).any() or (hi != SENTINEL).any():
                bad.append(i)
        return bad


def _scene(variant):
    if variant == 1:
        return synth.object_orbit(K=100, n_views=3, W=40, H=32)  # 4 keys per lane: the refinement path
    return synth.object_orbit(K=60, n_views=4, W=48, H=40)


@pytest.mark.parametrize("variant,keep_order,deterministic", [(0, 0, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1),
                                                               (1, 1, 0)])
def test_outputs_stay_inside_their_buffers(variant, keep_order, deterministic):
    s = _scene(variant)
    nf = 1
    params = fmb.default_params(n_flow=nf, variant=variant, keep_order=keep_order, deterministic=deterministic)
    G, P, NP = int(s.obj_offsets[-1]), s.n_pixels, len(s.poses)
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a).reshape(-1), dtype=torch.float32, device="cuda")
    m, c, w, po = T(s.means), T(s.chol), T(s.weights), T(s.poses)  # flattened on purpose
    rng = np.random.default_rng(5)
    gd, ga, gn, gf = (T(u) for u in synth.upstream_grads(rng, P, nf))
    r = fmb.Renderer(s.obj_offsets, s.views, NP, params)

    # plainly allocated reference (the renderer's own planes, which points() and
    # attribution() read)
    ref_planes = r.forward(m, c, w, po)
    ref_grads = r.backward(m, c, w, po, gd, ga, gn, gf, want_pose=True)
    ref_points = r.points(m, c, w, po)
    ray_loss = torch.rand(P, device="cuda")
    ref_attr = r.attribution(m, c, w, po, ray_loss)
    torch.cuda.synchronize()

    A = Arena()
    planes = dict(depth=A.take(P), alpha=A.take(P), normal=A.take(3 * P), flow=A.take(2 * nf * P), color=None,
                  saved=A.take(3 * P))
    grads = dict(means=A.take(3 * G).view(G, 3), chol=A.take(6 * G).view(G, 6), weights=A.take(G),
                 poses=A.take(12 * NP).view(NP, 12))
    r.forward(m, c, w, po, out=planes)
    r.backward(m, c, w, po, gd, ga, gn, gf, want_pose=True, out=grads, planes=planes)
    pts = dict(points=A.take(3 * P), normal_tf=A.take(3 * P), normal_screen=A.take(3 * P), quality=A.take(P))
    fmb.fmb_render_points(params, s.obj_offsets, m, c, w, po, r.c_views, planes["depth"], planes["saved"],
                          pts["points"], pts["normal_tf"], pts["normal_screen"], pts["quality"], r.ws)
    attr = A.take(G)
    fmb.fmb_loss_attribution(params, s.obj_offsets, m, c, w, po, r.c_views, planes["saved"], ray_loss, attr, r.ws)
    assert A.intact() == []
    assert fmb.fmb_read_device_status(r.ws) == 0

    for k in ("depth", "alpha", "normal", "flow", "saved"):
        assert torch.equal(planes[k], ref_planes[k]), k
    for k in ("means", "chol", "weights", "poses"):
        a, b = grads[k].reshape(-1), ref_grads[k].reshape(-1)
        if deterministic:
            assert torch.equal(a, b), k
        else:  # fp32 atomics: equal up to the order of the additions
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * float(b.abs().max())), k
    for k in ("points", "normal_tf", "normal_screen", "quality"):
        assert torch.equal(pts[k], ref_points[k]), k
    assert torch.allclose(attr, ref_attr, rtol=1e-5, atol=1e-6 * float(ref_attr.abs().max()))


def test_adam_step_stays_inside_its_buffers():
    n, pos = 3 * 1000 + 37, 3000  # the last 37 entries are updated in log space
    A = Arena()
    rng = np.random.default_rng(2)
    vals = {k: torch.as_tensor(rng.uniform(0.1, 1.0, n).astype(np.float32), device="cuda")
            for k in ("param", "grad", "m", "v")}
    ref = {k: v.clone() for k, v in vals.items()}
    got = {}
    for k, v in vals.items():
        got[k] = A.take(n)
        got[k].copy_(v)
    step_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
    step_raw = torch.full((2 * GUARD + 1,), SENTINEL, dtype=torch.int32, device="cuda")
    step_got = step_raw[GUARD:GUARD + 1]
    step_got.zero_()
    adam = fmb.FmbAdamParams(lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8)
    for _ in range(3):
        fmb.fmb_adam_step(adam, ref["param"], ref["grad"], ref["m"], ref["v"], pos, step_ref)
        fmb.fmb_adam_step(adam, got["param"], got["grad"], got["m"], got["v"], pos, step_got)
    assert A.intact() == []
    lo, hi = step_raw[:GUARD].cpu().numpy(), step_raw[GUARD + 1:].cpu().numpy()
    assert (lo == SENTINEL).all() and (hi == SENTINEL).all()
    assert int(step_got.item()) == 3 and int(step_ref.item()) == 3
    for k in ("param", "m", "v"):
        assert torch.equal(got[k], ref[k]), k
