"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Small cases are compared on every pixel and every gradient
entry; the full-size workloads run in the launch configuration the benchmark
uses and are compared on sampled pixels (forward) and on the exact gradient of
sampled pixels (backward: the upstream gradients vanish outside the sample, so
the oracle needs only those pixels)."""

import numpy as np
import pytest
import torch

import oracle
from paper_2308_14737_gb300 import fmb, synth

from gpu_util import (ac_order_ambiguous, compare_forward, compare_grads, dev_scene, gpu_backward, gpu_forward,
                      masked_upstream,
                      plane_view, points_tolerances,
                      nnorm_batched, many_small_views,
                      oracle_backward_sampled, oracle_forward_sampled, pixel_mask_from, sample_pixels)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_14737_gb300 import build

    build.build()
    oracle.build()
    fmb.load_library()


def _full_check(scene, n_flow, normals=True, deterministic=False, want_pose=True, seed=1, **pk):
    variant = pk.get("variant", 0)
    params = fmb.default_params(n_flow=n_flow, want_normals=int(normals), deterministic=int(deterministic), **pk)
    gpu, r, dev = gpu_forward(scene, params)
    ref = oracle.render_scene(scene, n_flow=n_flow, variant=variant)
    amb = ac_order_ambiguous(scene) if variant == 1 else None
    stats = compare_forward(scene, gpu, ref, n_flow, normals, variant=variant, ambiguous=amb)
    ups = masked_upstream(scene, ref["alpha"], n_flow, seed=seed, nnorm_ref=nnorm_batched(scene, ref["saved"]),
                          exclude=amb)
    if not normals:
        ups["g_normal"] = np.zeros_like(ups["g_normal"])
    g = gpu_backward(r, dev, ups, want_pose=want_pose)
    refg = oracle.backward_scene(scene, ups["g_depth"], ups["g_alpha"], ups["g_normal"] if normals else None,
                                 ups["g_flow"], n_flow=n_flow, variant=variant)
    errs = compare_grads(g, refg, keys=("means", "chol", "weights") + (("poses",) if want_pose else ()))
    return stats, errs, g


def test_single_view_64x64_K40():
    s = synth.single_view()
    _full_check(s, n_flow=0)


def test_orbit_small_with_flow_and_pose():
    s = synth.object_orbit(K=100, n_views=4, W=64, H=48)
    _full_check(s, n_flow=1)


def test_two_flow_slots_with_missing_targets():
    s = synth.reconstruction(n_views=3, K=37, W=40, H=30)
    _full_check(s, n_flow=2)


def test_normals_off():
    s = synth.object_orbit(K=30, n_views=2, W=33, H=17)
    _full_check(s, n_flow=1, normals=False)


@pytest.mark.parametrize("ksplit", [2, 3, 8])
def test_gaussian_split_forward(ksplit):
    """Forward with each object's Gaussians split over ksplit CTAs per ray tile and the
    per-ray partial sums merged: planes and (through the saved normalisers) gradients
    against the oracle, including objects with fewer Gaussians than splits (those
    views stay unsplit in the same launch, and the merge must leave them alone)."""
    _full_check(synth.object_orbit(K=100, n_views=3, W=48, H=40), n_flow=1, fwd_ksplit=ksplit)
    _full_check(_ragged_scene(), n_flow=1, fwd_ksplit=ksplit)
    _full_check(synth.reconstruction(n_views=3, K=37, W=40, H=30), n_flow=2, normals=False, fwd_ksplit=ksplit)


def test_gaussian_split_forward_ray_batch_and_auto():
    """The automatic choice against the unsplit forward (a 6000-ray minibatch at
    K = 256 is split, also over 80 views in one 256-view launch; a single 64x64 view
    at K = 40 is not): the same planes up to the rounding of the merge."""
    from paper_2308_14737_gb300 import synth as sy

    # the 80-view batch runs its render in one 256-view launch (and the merge with it)
    big = sy.ray_batch(sy.reconstruction(n_views=80, K=256, W=80, H=60), 8000, seed=3)
    for scene, nf, nrm in ((sy.ray_batch(sy.reconstruction(n_views=20, K=256, W=160, H=120), 6000, seed=2), 2, 0),
                           (big, 2, 0), (sy.single_view(), 0, 1)):
        outs = []
        for ks in (1, 0):
            params = fmb.default_params(n_flow=nf, want_normals=nrm, fwd_ksplit=ks)
            gpu, r, dev = gpu_forward(scene, params)
            outs.append(gpu)
            if ks == 0:
                assert fmb.fmb_forward_ksplit(params, scene.obj_offsets, r.c_views) == (6 if nf == 2 else 1)
            if scene is big:  # prologue, forward (and merge) as one launch each for the 80 views
                assert fmb.fmb_launch_count(params, scene.obj_offsets, r.c_views, backward=False) == 2 + (ks == 0)
        for k in ("depth", "alpha"):
            assert np.allclose(outs[0][k], outs[1][k], rtol=1e-5, atol=1e-6), k
        sv0, sv1 = outs[0]["saved"], outs[1]["saved"]
        assert np.allclose(sv0, sv1, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("normals,n_flow,deterministic", [(True, 1, False), (False, 2, False), (True, 0, True),
                                                         (False, 0, True)])
def test_backward_without_pose_gradients(normals, n_flow, deterministic):
    """No pose gradient requested: the kernel specialisation that accumulates the
    lower triangle of sum v abar^T together with sum gbar u^T gives the oracle's
    Gaussian gradients, and those of the run that also returns pose gradients."""
    s = (synth.object_orbit(K=100, n_views=3, W=48, H=40) if n_flow < 2 else
         synth.reconstruction(n_views=3, K=37, W=40, H=30))
    _, _, g1 = _full_check(s, n_flow=n_flow, normals=normals, deterministic=deterministic, want_pose=False)
    _, _, g2 = _full_check(s, n_flow=n_flow, normals=normals, deterministic=deterministic, want_pose=True)
    assert g1["poses"] is None
    for k in ("means", "chol", "weights"):
        assert np.allclose(g1[k], g2[k], rtol=1e-5, atol=1e-6 * np.abs(g2[k]).max()), k


@pytest.mark.parametrize("rpt", [1, 2, 4])
def test_rays_per_thread_variants(rpt):
    s = synth.object_orbit(K=45, n_views=2, W=37, H=29)
    _full_check(s, n_flow=1, fwd_rays_per_thread=rpt)


def _ragged_scene(seed=7):
    rng = np.random.default_rng(seed)
    objs, views, poses = [], [], []
    sizes = [(1, 1), (3, 5), (33, 17), (65, 9), (16, 16)]
    for o, K in enumerate([1, 2, 31, 33, 300]):
        objs.append(synth.random_gaussians(rng, K, "cholesky"))
        for W, H in sizes[o:o + 2]:
            poses.append(synth.look_at_pose(synth.sphere_positions(rng, 1)[0]))
            views.append(dict(W=W, H=H, fx=float(max(W, H)), fy=float(max(W, H)), cx=W / 2, cy=H / 2, object=o,
                              pose=len(poses) - 1, flow_target=(len(poses) % 3, -1)))
    return synth.make_scene(objs, views, poses)


def test_ragged_objects_and_edge_sizes():
    """K in {1, 2, 31, 33, 300} (300 crosses the 256-record staging chunk), images
    from 1x1 to 65x9, several objects and views in one launch."""
    _full_check(_ragged_scene(), n_flow=1)


@pytest.mark.parametrize("deterministic", [False, True])
def test_persistent_launch(deterministic):
    """Persistent mode: resident CTAs pop (view, tile) items, most expensive first."""
    _full_check(_ragged_scene(), n_flow=1, use_persistent=1, deterministic=deterministic)
    _full_check(synth.object_orbit(K=100, n_views=5, W=64, H=48), n_flow=1, use_persistent=1,
                deterministic=deterministic)


def test_persistent_matches_grid_launch_bitwise():
    """Work items compute the same thing in either launch mode: forward planes and
    the deterministic backward agree bit for bit."""
    s = synth.ragged_batch(n_objects=6, views_per_object=2, sides=(32, 48, 64))
    rng = np.random.default_rng(0)
    res = []
    for pers in (0, 1):
        p = fmb.default_params(n_flow=0, use_persistent=pers, deterministic=1)
        gpu, r, dev = gpu_forward(s, p)
        gd, ga, gn, _ = synth.upstream_grads(np.random.default_rng(5), s.n_pixels, 1)
        g = gpu_backward(r, dev, dict(g_depth=gd, g_alpha=ga, g_normal=gn.reshape(-1), g_flow=None))
        res.append((gpu, g))
    for k in ("depth", "alpha", "normal", "saved"):
        assert np.array_equal(res[0][0][k], res[1][0][k]), k
    for k in ("means", "chol", "weights", "poses"):
        assert np.array_equal(res[0][1][k], res[1][1][k]), k


def test_deterministic_mode_is_bitwise_reproducible():
    s = synth.object_orbit(K=100, n_views=3, W=48, H=40)
    _, _, g1 = _full_check(s, n_flow=1, deterministic=True)
    _, _, g2 = _full_check(s, n_flow=1, deterministic=True)
    for k in g1:
        assert np.array_equal(g1[k], g2[k]), k
    _, _, ga = _full_check(s, n_flow=1, deterministic=False)
    for k in g1:
        np.testing.assert_allclose(g1[k], ga[k], rtol=0, atol=1e-5 * np.abs(g1[k]).max())


@pytest.mark.parametrize("ray_tile,threads", [(32, 64), (128, 128), (512, 96), (1024, 160), (320, 160), (450, 160), (33, 32)])
def test_backward_tilings(ray_tile, threads):
    s = synth.object_orbit(K=70, n_views=2, W=50, H=31)
    _full_check(s, n_flow=1, bwd_ray_tile=ray_tile, bwd_threads=threads)


@pytest.mark.parametrize("gblocks,deterministic", [(2, False), (4, True), (8, False), (64, True)])
def test_backward_gaussian_block_hint(gblocks, deterministic):
    """bwd_gblocks raises each object's Gaussian blocks to at least that many (K = 37
    in 2, 4, 8 blocks; K = 5 in one block per Gaussian, 128 ray subgroups of one
    thread; two uniform blocks run as 2-CTA clusters), in a ragged two-object batch
    and in a ray minibatch, against the oracle."""
    rng = np.random.default_rng(21)
    objs = [synth.random_gaussians(rng, K, "cholesky") for K in (37, 5)]
    poses = [synth.look_at_pose(p) for p in synth.sphere_positions(rng, 4)]
    views = [dict(W=W, H=H, fx=float(W), fy=float(W), cx=W / 2, cy=H / 2, object=o, pose=i,
                  flow_target=((i + 1) % 4, -1)) for i, (W, H, o) in enumerate(((40, 30, 0), (17, 9, 1), (33, 33, 0),
                                                                                (8, 8, 1)))]
    s = synth.make_scene(objs, views, poses)
    _full_check(s, n_flow=1, deterministic=deterministic, bwd_gblocks=gblocks, bwd_threads=128, bwd_ray_tile=128)
    _full_check(synth.object_orbit(K=60, n_views=3, W=32, H=24), n_flow=1, deterministic=deterministic,
                bwd_gblocks=gblocks, bwd_threads=128, bwd_ray_tile=256)
    mb = synth.ray_batch(synth.reconstruction(n_views=6, K=64, W=40, H=30), 900, seed=4)
    _full_check(mb, n_flow=2, normals=False, deterministic=deterministic, bwd_gblocks=gblocks, bwd_threads=128,
                bwd_ray_tile=256)


def test_gaussian_blocks_over_128():
    """K = 300 splits into several Gaussian blocks per CTA; K = 129 leaves a block
    with one Gaussian."""
    for K in (129, 300):
        s = synth.object_orbit(K=K, n_views=2, W=24, H=20)
        _full_check(s, n_flow=1, deterministic=(K == 300))


@pytest.mark.parametrize("deterministic", [False, True])
def test_cluster_backward(deterministic):
    """K = 100 at 128 backward threads runs as two Gaussian blocks, which grid mode
    launches as 2-CTA clusters sharing the per-ray records (each CTA builds half
    of them); persistent mode runs the same blocks as single CTAs.  Both match the
    oracle, and each other up to the order of the fp32 sums."""
    s = synth.object_orbit(K=100, n_views=4, W=64, H=48)
    res = []
    for pers in (0, 1):
        _, _, g = _full_check(s, n_flow=1, deterministic=deterministic, bwd_threads=128, bwd_ray_tile=384,
                              use_persistent=pers)
        res.append(g)
    for k in res[0]:
        np.testing.assert_allclose(res[0][k], res[1][k], rtol=0, atol=2e-5 * np.abs(res[1][k]).max(), err_msg=k)
    if deterministic:
        _, _, g2 = _full_check(s, n_flow=1, deterministic=True, bwd_threads=128, bwd_ray_tile=384)
        for k in g2:
            assert np.array_equal(res[0][k], g2[k]), k


@pytest.mark.parametrize("deterministic", [False, True])
def test_more_than_64_views_in_one_launch(deterministic):
    """A two-parameter call with more than 64 views runs each pass as one launch over a
    256-view table: 70 orbit views at K = 100 and 128 backward threads (two Gaussian
    blocks, so grid mode launches 2-CTA clusters), in atomic and deterministic mode,
    against the oracle."""
    s = synth.object_orbit(K=100, n_views=70, W=24, H=16)
    p = fmb.default_params(n_flow=1, deterministic=int(deterministic), bwd_threads=128, bwd_ray_tile=384)
    assert fmb.fmb_launch_count(p, s.obj_offsets, s.views, backward=False) == 2
    assert fmb.fmb_launch_count(p, s.obj_offsets, s.views, backward=True, want_pose=True) == (4 if deterministic else 2)
    _full_check(s, n_flow=1, deterministic=deterministic, bwd_threads=128, bwd_ray_tile=384)


@pytest.mark.parametrize("deterministic", [False, True])
@pytest.mark.parametrize("variant", [0, 1])
def test_more_than_256_views_in_one_call(variant, deterministic):
    """300 views of three objects in one call: the two-parameter passes run as two
    launches (256 + 44 views; this small batch also takes the automatic Gaussian split
    of the forward, so each forward launch has its merge), alpha compositing as five of
    at most 64; forward planes and gradients against the oracle in atomic and
    deterministic mode."""
    s = many_small_views(300)
    p = fmb.default_params(n_flow=1, variant=variant, deterministic=int(deterministic))
    batches = 2 if variant == 0 else 5
    merge = variant == 0 and fmb.fmb_forward_ksplit(p, s.obj_offsets, s.views) > 1
    assert fmb.fmb_launch_count(p, s.obj_offsets, s.views, backward=False) == (3 if merge else 2) * batches
    if not deterministic:
        assert fmb.fmb_launch_count(p, s.obj_offsets, s.views, backward=True, want_pose=True) == 2 * batches
    _full_check(s, n_flow=1, deterministic=deterministic, variant=variant)


def test_permutation_invariance():
    s = synth.object_orbit(K=60, n_views=2, W=40, H=30)
    p = fmb.default_params(n_flow=1)
    a, _, _ = gpu_forward(s, p)
    perm = np.random.default_rng(3).permutation(60)
    s2 = synth.make_scene([(s.means[perm], s.chol[perm], s.weights[perm])],
                          [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views], s.poses)
    b, _, _ = gpu_forward(s2, p)
    mask = a["alpha"] >= 1e-2
    assert np.all(np.abs(a["depth"] - b["depth"])[mask] <= 1e-4 + 1e-5 * np.abs(a["depth"][mask]))
    assert np.all(np.abs(a["alpha"] - b["alpha"]) <= 1e-5)


def _sampled_full_size(scene, n_flow, n_per_view, seed=0, deterministic=False, persistent=False, normals=True,
                       want_pose=True, **pk):
    params = fmb.default_params(n_flow=n_flow, deterministic=int(deterministic), use_persistent=int(persistent),
                                want_normals=int(normals), **pk)
    gpu, r, dev = gpu_forward(scene, params)
    pix = sample_pixels(scene, n_per_view, seed)
    ref = oracle_forward_sampled(scene, pix, n_flow)
    stats = compare_forward(scene, gpu, None, n_flow, normals, pixels_per_view=ref)
    alpha_ref = np.zeros(scene.n_pixels)
    nn_ref = np.zeros(scene.n_pixels)
    for vi, v in enumerate(scene.views):
        alpha_ref[v["pix_offset"] + ref[vi][0]] = ref[vi][1]["alpha"]
        nn_ref[v["pix_offset"] + ref[vi][0]] = ref[vi][1]["saved"][:, 2]
    ups = masked_upstream(scene, alpha_ref, n_flow, seed=seed + 1, pixel_mask=pixel_mask_from(scene, pix),
                          nnorm_ref=nn_ref)
    if not normals:
        ups["g_normal"] = np.zeros_like(ups["g_normal"])
    g = gpu_backward(r, dev, dict(ups, g_normal=ups["g_normal"] if normals else None), want_pose=want_pose)
    refg = oracle_backward_sampled(scene, ups, pix, n_flow)
    errs = compare_grads(g, refg, keys=("means", "chol", "weights") + (("poses",) if want_pose else ()))
    return stats, errs


def test_orbit_full_size_16x320x240_K100_sampled():
    _sampled_full_size(synth.object_orbit(), n_flow=1, n_per_view=400)


def test_orbit_full_size_benchmark_tiles_sampled():
    """The benchmark's tuned tiles (128 backward threads, 384-ray tiles: two
    Gaussian blocks per tile, launched as 2-CTA clusters)."""
    _sampled_full_size(synth.object_orbit(), n_flow=1, n_per_view=200, seed=3, bwd_threads=128, bwd_ray_tile=384,
                       fwd_rays_per_thread=2)


def test_orbit_full_size_dense_gradients():
    """Every pixel of the 16-view 320x240 K=100 orbit contributes to the gradients
    (the benchmark's workload and launch configuration)."""
    s = synth.object_orbit()
    params = fmb.default_params(n_flow=1)
    gpu, r, dev = gpu_forward(s, params)
    ref = oracle.render_scene(s, n_flow=1)
    ups = masked_upstream(s, ref["alpha"], 1, seed=2, nnorm_ref=nnorm_batched(s, ref["saved"]))
    g = gpu_backward(r, dev, ups)
    refg = oracle.backward_scene(s, ups["g_depth"], ups["g_alpha"], ups["g_normal"], ups["g_flow"], n_flow=1)
    compare_grads(g, refg)


def test_orbit_unmasked_normal_gradient_within_bound():
    """Gradients on the 16-view orbit with the normal plane's upstream gradient NOT
    masked by |N| >= 0.05 (only by the paper's object mask, alpha >= 1e-2), against
    a bound computed per gradient entry.  A pixel p whose per-Gaussian normals nearly
    cancel contributes c_p = J_p^T Nbar_p with Nbar_p = (I - n n^T) nbar_f / |N_p|:
    an error dN_p of the forward's blended vector N_p moves n = N/|N| and 1/|N| by at
    most dN_p/|N_p| each, and (I - n n^T) by 2 dN_p/|N_p|, so c_p moves by at most
    |c_p| (4 dN_p/|N_p| + e), e = 1e-4 for the per-pair terms.  dN_p is the measured
    forward error at that pixel (GPU against oracle, both |N| n_f), c_p the oracle's
    gradient of that pixel alone.  The bound is the masked tolerance, 1e-4 of the
    tensor's largest entry (it covers every pixel with |N| >= 0.05, as the masked
    tests show), plus the sum of those terms over the pixels with |N| < 0.05."""
    s = synth.object_orbit()
    params = fmb.default_params(n_flow=1)
    gpu, r, dev = gpu_forward(s, params)
    ref = oracle.render_scene(s, n_flow=1)
    ups = masked_upstream(s, ref["alpha"], 1, seed=2)  # object mask only
    g = gpu_backward(r, dev, ups)
    refg = oracle.backward_scene(s, ups["g_depth"], ups["g_alpha"], ups["g_normal"], ups["g_flow"], n_flow=1)
    nn = nnorm_batched(s, ref["saved"])
    small = np.nonzero((ref["alpha"] >= 1e-2) & (nn < 0.05))[0]
    bound = {k: np.full(refg[k].shape, 1e-4 * np.max(np.abs(refg[k]))) for k in refg}
    for vi, v in enumerate(s.views):
        o, P = v["pix_offset"], v["W"] * v["H"]
        Ng = plane_view(gpu["normal"], v, 3) * plane_view(gpu["saved"], v, 3)[2]
        Nr = plane_view(ref["normal"], v, 3) * plane_view(ref["saved"], v, 3)[2]
        dN = np.linalg.norm(Ng - Nr, axis=0)
        for p in small[(small >= o) & (small < o + P)] - o:
            c = oracle_backward_sampled(s, ups, {vj: ([p] if vj == vi else []) for vj in range(len(s.views))}, 1)
            f = 4.0 * dN[p] / max(nn[o + p], 1e-30) + 1e-4
            for k in bound:
                bound[k] += f * np.abs(c[k])
    report = {}
    for k in ("means", "chol", "weights", "poses"):
        err = np.abs(g[k].reshape(refg[k].shape) - refg[k])
        scale = np.max(np.abs(refg[k]))
        report[k] = (float(err.max() / scale), float(bound[k].max() / scale))
        assert np.all(err <= bound[k]), (k, report[k])
    print(f"unmasked normal-gradient errors (max err / max |g|, max bound / max |g|), {len(small)} pixels with "
          f"|N| < 0.05: {report}")


def test_large_K4096_8x1024x768_sampled():
    _sampled_full_size(synth.large_k(), n_flow=1, n_per_view=48)


def test_ragged_batch_64_objects_sampled():
    _sampled_full_size(synth.ragged_batch(), n_flow=0, n_per_view=64, deterministic=True)


def test_ragged_batch_64_objects_persistent_sampled():
    _sampled_full_size(synth.ragged_batch(), n_flow=0, n_per_view=48, persistent=True)


@pytest.mark.parametrize("deterministic,ray_tile", [(False, 256), (True, 384)])
def test_reconstruction_full_size_100x640x480_K256_sampled(deterministic, ray_tile):
    """The reconstruction workload at full size: 100 sphere views 640x480, K=256,
    flow to the next and the previous view, depth + alpha (no normal plane), no pose
    gradients, in the tiles its benchmark tunes to (128 backward threads, so one
    block of all 256 Gaussians per ray tile; the no-pose adjoint), in both
    reduction modes."""
    _sampled_full_size(synth.reconstruction(), n_flow=2, n_per_view=40, seed=5, deterministic=deterministic,
                       normals=False, want_pose=False, bwd_threads=128, bwd_ray_tile=ray_tile,
                       fwd_rays_per_thread=2)


def test_reconstruction_stored_intermediate_full_size_sampled():
    """The stored-intermediate adjoint at the reconstruction workload's view size
    and K (10 of its 640x480 views: 12 bytes per pair, 9.4 GB of stored values)."""
    _sampled_full_size(synth.reconstruction(n_views=10), n_flow=2, n_per_view=60, seed=6, normals=False,
                       want_pose=False, bwd_threads=128, bwd_ray_tile=384, fwd_rays_per_thread=2, store_pairs=1)


def test_device_status_is_clear_and_outputs_finite():
    s = synth.object_orbit(K=20, n_views=2, W=16, H=12)
    gpu, r, _ = gpu_forward(s, fmb.default_params())
    for k in ("depth", "alpha", "normal", "flow", "saved"):
        assert np.all(np.isfinite(gpu[k])), k
    assert fmb.fmb_read_device_status(r.ws) == 0


@pytest.mark.parametrize("deterministic", [False, True])
def test_stored_intermediate_adjoint(deterministic):
    """store_pairs = 1: the forward keeps every pair's t, log2 weight and density
    and the backward reads them; same tolerances against the oracle, and the
    gradients agree with the recomputing adjoint (only the rounding of the log2
    weight's last add differs).  Odd K (the rows are padded to even) included."""
    for scene, nf in ((synth.object_orbit(K=101, n_views=3, W=40, H=30), 1), (_ragged_scene(), 1),
                      (synth.single_view(), 0)):
        _, _, gs = _full_check(scene, n_flow=nf, store_pairs=1, deterministic=deterministic,
                               normals=(nf == 1))
        _, _, gr = _full_check(scene, n_flow=nf, deterministic=deterministic, normals=(nf == 1))
        for k in gs:
            np.testing.assert_allclose(gs[k], gr[k], rtol=0, atol=2e-5 * np.abs(gr[k]).max())
    # Gaussian blocks that would start at an odd index (K = 37 in 8 blocks of 5, or 2 of
    # 19) are rounded up to even sizes in this mode, whose loads take two Gaussians
    s37 = synth.object_orbit(K=37, n_views=2, W=24, H=20)
    for g in (2, 8):
        _full_check(s37, n_flow=1, store_pairs=1, deterministic=deterministic, bwd_gblocks=g, bwd_threads=128,
                    bwd_ray_tile=128)


def test_stored_intermediate_adjoint_full_size_sampled():
    s = synth.object_orbit()
    params = fmb.default_params(n_flow=1, store_pairs=1)
    gpu, r, dev = gpu_forward(s, params)
    pix = sample_pixels(s, 200, 3)
    ref = oracle_forward_sampled(s, pix, 1)
    compare_forward(s, gpu, None, 1, True, pixels_per_view=ref)
    alpha_ref = np.zeros(s.n_pixels)
    nn_ref = np.zeros(s.n_pixels)
    for vi, v in enumerate(s.views):
        alpha_ref[v["pix_offset"] + ref[vi][0]] = ref[vi][1]["alpha"]
        nn_ref[v["pix_offset"] + ref[vi][0]] = ref[vi][1]["saved"][:, 2]
    ups = masked_upstream(s, alpha_ref, 1, seed=4, pixel_mask=pixel_mask_from(s, pix), nnorm_ref=nn_ref)
    g = gpu_backward(r, dev, ups)
    compare_grads(g, oracle_backward_sampled(s, ups, pix, 1))


# ---------------------------------------------- alpha-compositing variant (Sec. 3.3)

def _ac_ragged_scene(seed=8):
    """K in {1, 2, 31, 33, 64, 65, 129, 256} (every sort width: 64, 128 and 256
    keys per ray), images from 1x1 to 65x9, several objects in one launch."""
    rng = np.random.default_rng(seed)
    objs, views, poses = [], [], []
    sizes = [(1, 1), (3, 5), (33, 17), (65, 9), (16, 16), (20, 7), (9, 31), (12, 12)]
    for o, K in enumerate([1, 2, 31, 33, 64, 65, 129, 256]):
        objs.append(synth.random_gaussians(rng, K, "cholesky"))
        W, H = sizes[o]
        poses.append(synth.look_at_pose(synth.sphere_positions(rng, 1)[0]))
        views.append(dict(W=W, H=H, fx=float(max(W, H)), fy=float(max(W, H)), cx=W / 2, cy=H / 2, object=o,
                          pose=len(poses) - 1, flow_target=((len(poses) + 2) % 8, -1)))
    while len(poses) < 8:
        poses.append(synth.look_at_pose(synth.sphere_positions(rng, 1)[0]))
    return synth.make_scene(objs, views, poses)


@pytest.mark.parametrize("deterministic", [False, True])
def test_alpha_compositing_parity(deterministic):
    """variant 1 against the oracle's literal Eq. 9-10: forward planes and every
    gradient, on each sort width, with and without normals and flow."""
    _full_check(synth.single_view(), n_flow=0, normals=False, variant=1, deterministic=deterministic)
    _full_check(synth.object_orbit(K=100, n_views=3, W=48, H=40), n_flow=1, variant=1, deterministic=deterministic)
    _full_check(synth.reconstruction(n_views=3, K=37, W=40, H=30), n_flow=2, variant=1, deterministic=deterministic)
    _full_check(_ac_ragged_scene(), n_flow=1, variant=1, deterministic=deterministic)


@pytest.mark.parametrize("deterministic", [False, True])
def test_alpha_compositing_keep_order(deterministic):
    """keep_order = 1: the backward walks each ray's depth order as the forward kept
    it, four threads per ray, instead of sorting again.  Same tolerances against the
    oracle, and within 1e-5 of the largest entry of the re-sorting adjoint (the
    summation order differs), over objects of 1 to 256 Gaussians (every sort width;
    objects below 8 Gaussians take the re-sorting path inside the same launch)."""
    for scene, nf in ((synth.object_orbit(K=100, n_views=3, W=40, H=30), 1), (_ac_ragged_scene(), 1)):
        _, _, gk = _full_check(scene, n_flow=nf, variant=1, keep_order=1, deterministic=deterministic)
        _, _, g0 = _full_check(scene, n_flow=nf, variant=1, deterministic=deterministic)
        for k in gk:
            np.testing.assert_allclose(gk[k], g0[k], rtol=0, atol=1e-5 * np.abs(g0[k]).max())
    # without the normal plane, two flow slots, with and without pose gradients
    scene = synth.reconstruction(n_views=3, K=37, W=40, H=30)
    for want_pose in (True, False):
        _full_check(scene, n_flow=2, normals=False, want_pose=want_pose, variant=1, keep_order=1,
                    deterministic=deterministic)


@pytest.mark.parametrize("deterministic", [False, True])
def test_alpha_compositing_keep_order_stale_orders(deterministic):
    """The workspace holds another render's depth orders when the backward runs (a
    second forward of the same layout from other cameras, into planes of its own):
    every ray whose stored order is not strictly increasing in its own recomputed
    depths is sorted again, so the gradients still match the oracle; and a stale
    order gives the same gradients, to rounding, as the ray's own."""
    s = synth.object_orbit(K=100, n_views=3, W=40, H=30)
    params = fmb.default_params(n_flow=1, variant=1, keep_order=1, deterministic=int(deterministic))
    gpu, r, dev = gpu_forward(s, params)
    ref = oracle.render_scene(s, n_flow=1, variant=1)
    amb = ac_order_ambiguous(s)
    ups = masked_upstream(s, ref["alpha"], 1, seed=2, nnorm_ref=nnorm_batched(s, ref["saved"]), exclude=amb)
    own = gpu_backward(r, dev, ups)
    for shift in (1, 0):  # other views' cameras; the same cameras with the means moved slightly
        poses = torch.roll(dev[3].reshape(len(s.poses), 12), shift, 0).contiguous().reshape(dev[3].shape)
        means = dev[0] if shift else dev[0] + 1e-3
        r.forward(means, dev[1], dev[2], poses, out=r.new_planes())
        torch.cuda.synchronize()
        g = gpu_backward(r, dev, ups)
        refg = oracle.backward_scene(s, ups["g_depth"], ups["g_alpha"], ups["g_normal"], ups["g_flow"], n_flow=1,
                                     variant=1)
        compare_grads(g, refg)
        for k in own:
            np.testing.assert_allclose(g[k], own[k], rtol=0, atol=1e-5 * np.abs(own[k]).max())


def test_alpha_compositing_persistent():
    _full_check(_ac_ragged_scene(), n_flow=1, variant=1, use_persistent=1)


@pytest.mark.parametrize("keep_order", [0, 1])
def test_alpha_compositing_equal_depth_ties(keep_order):
    """Exact duplicates hit at bitwise-equal depths on the GPU too, so the strict
    indicator of Eq. 10 leaves them unattenuated by each other, as in the oracle
    (with keep_order the rays with equal depths take the run-aware sorting path)."""
    s = synth.object_orbit(K=50, n_views=2, W=32, H=24)
    s2 = synth.make_scene([(np.concatenate([s.means] * 2), np.concatenate([s.chol] * 2),
                            np.concatenate([s.weights] * 2))],
                          [{k: v for k, v in vv.items() if k != "pix_offset"} for vv in s.views], s.poses)
    _full_check(s2, n_flow=1, variant=1, keep_order=keep_order)


@pytest.mark.parametrize("keep_order", [0, 1])
def test_alpha_compositing_full_size_sampled(keep_order):
    """The 16-view 320x240 K=100 orbit, sampled pixels, forward and backward."""
    s = synth.object_orbit()
    params = fmb.default_params(n_flow=1, variant=1, keep_order=keep_order)
    gpu, r, dev = gpu_forward(s, params)
    pix = sample_pixels(s, 150, 5)
    ref = oracle_forward_sampled(s, pix, 1, variant=1)
    amb = ac_order_ambiguous(s, pix)
    compare_forward(s, gpu, None, 1, True, pixels_per_view=ref, variant=1, ambiguous=amb)
    alpha_ref = np.zeros(s.n_pixels)
    nn_ref = np.zeros(s.n_pixels)
    amb_b = np.zeros(s.n_pixels, dtype=bool)
    for vi, v in enumerate(s.views):
        alpha_ref[v["pix_offset"] + ref[vi][0]] = ref[vi][1]["alpha"]
        nn_ref[v["pix_offset"] + ref[vi][0]] = ref[vi][1]["saved"][:, 2]
        amb_b[v["pix_offset"] + ref[vi][0]] = amb[vi]
    ups = masked_upstream(s, alpha_ref, 1, seed=6, pixel_mask=pixel_mask_from(s, pix), nnorm_ref=nn_ref,
                          exclude=amb_b)
    g = gpu_backward(r, dev, ups)
    compare_grads(g, oracle_backward_sampled(s, ups, pix, 1, variant=1))


# ---------------------------------------------------- oriented point export (Sec. 6)

@pytest.mark.parametrize("variant", [0, 1])
def test_points_export_parity(variant):
    """fmb_render_points against the oracle: points, normals at the rendered depth,
    Eq. 16 screen-space normals and the max-weight quality, with the tolerances the
    fp32 depth error propagates to (gpu_util.points_tolerances), where the oracle's
    alpha >= 1e-2 (at the pixel and, for Eq. 16, its two neighbours) and the depth
    order is unambiguous in fp32."""
    for scene, nf in ((synth.object_orbit(K=100, n_views=3, W=48, H=40), 1), (synth.single_view(), 0)):
        params = fmb.default_params(n_flow=nf, variant=variant)
        gpu, r, dev = gpu_forward(scene, params)
        pts = {k: v.cpu().numpy().astype(np.float64) for k, v in r.points(*dev).items()}
        torch.cuda.synchronize()
        ref = oracle.points_scene(scene, variant=variant)
        fr = oracle.render_scene(scene, n_flow=0, variant=variant)
        ref["depth"] = fr["depth"]
        dD = np.abs(gpu["depth"] - fr["depth"]) + 1e-6 * np.abs(fr["depth"])
        tp, tn, ts, amb_n, amb_s = points_tolerances(scene, ref, variant, dD)
        ok = fr["alpha"] >= 1e-2
        if variant == 1:
            ok &= ~ac_order_ambiguous(scene)
        for v in scene.views:
            o, P = v["pix_offset"], v["W"] * v["H"]
            W_, H_ = v["W"], v["H"]
            pix = np.arange(P)
            xx, yy = pix % W_, pix // W_
            nx = yy * W_ + np.where(xx + 1 < W_, xx + 1, xx - 1)
            ny = np.where(yy + 1 < H_, yy + 1, yy - 1) * W_ + xx
            okv = ok[o:o + P]
            okn = okv & okv[nx] & okv[ny]
            for key, tol, msk, amb in (("points", tp, okv, None), ("normal_tf", tn, okv, amb_n),
                                       ("normal_screen", ts, okn, amb_s)):
                g_, r_ = plane_view(pts[key], v, 3), plane_view(ref[key], v, 3)
                e = np.abs(g_ - r_).max(0)
                if amb is not None:  # facing sign undecided at the tolerance: compare up to sign
                    e = np.where(amb[o:o + P], np.minimum(e, np.abs(g_ + r_).max(0)), e)
                assert np.all((e <= tol[o:o + P])[msk]), (key, float(e[msk].max()))
            eq = np.abs(pts["quality"][o:o + P] - ref["quality"][o:o + P])
            assert np.all((eq <= 1e-4)[okv]), ("quality", float(eq[okv].max()))



@pytest.mark.parametrize("variant", [0, 1])
def test_points_export_full_size_sampled(variant):
    """The 16-view 320x240 orbit at full size, in the bench's configuration: the
    exported points and the max-weight quality at 200 sampled pixels per view
    against the oracle (points within the depth tolerance plus the measured depth
    difference, quality within 1e-4), where the oracle's alpha >= 1e-2 and the
    depth order is unambiguous in fp32.  The normals are compared on every pixel of
    the small cases above."""
    s = synth.object_orbit()
    params = fmb.default_params(n_flow=1, variant=variant)
    gpu, r, dev = gpu_forward(s, params)
    pts = {k: v.cpu().numpy().astype(np.float64) for k, v in r.points(*dev).items()}
    samp = sample_pixels(s, 200, seed=5)
    amb = ac_order_ambiguous(s, samp) if variant == 1 else None
    n_checked = 0
    for vi, v in enumerate(s.views):
        sl = s.object_slice(v["object"])
        cam = (v["W"], v["H"], v["fx"], v["fy"], v["cx"], v["cy"])
        pix = samp[vi]
        ref = oracle.points_view(s.means[sl], s.chol[sl], s.weights[sl], s.poses[v["pose"]], cam,
                                 variant=variant, pixels=pix)
        fr = oracle.render_view(s.means[sl], s.chol[sl], s.weights[sl], s.poses[v["pose"]], None, cam,
                                pixels=pix, variant=variant)
        o, P = v["pix_offset"], v["W"] * v["H"]
        ok = fr["alpha"] >= 1e-2
        if amb is not None:
            ok &= ~amb[vi]
        D = fr["depth"]
        dD = np.abs(gpu["depth"][o + pix] - D)
        assert np.all((dD <= 1e-4 + 1e-5 * np.abs(D))[ok])
        g_pts = pts["points"][3 * o:3 * (o + P)].reshape(3, P)[:, pix].T
        e = np.abs(g_pts - ref["points"]).max(1)
        assert np.all((e <= 1e-4 + 1e-5 * np.abs(D) + dD)[ok]), float(e[ok].max())
        eq = np.abs(pts["quality"][o + pix] - ref["quality"])
        assert np.all((eq <= 1e-4)[ok]), float(eq[ok].max())
        n_checked += int(ok.sum())
    assert n_checked > 1000


# ------------------------------------------------ ray minibatches across frames (Sec. 4)

@pytest.mark.parametrize("variant", [0, 1])
def test_ray_batch_parity(variant):
    """Views that render only a list of pixels (random minibatch across all frames):
    forward planes hold the listed rays in order and the gradients are the sums over
    those rays alone -- against the oracle on the same pixel lists."""
    base = synth.object_orbit(K=100, n_views=6, W=48, H=40)
    s = synth.ray_batch(base, 3000, seed=2)
    assert s.n_pixels == 3000 and all(v.get("rays") is not None for v in s.views)
    _full_check(s, n_flow=1, variant=variant)
    _full_check(s, n_flow=1, variant=variant, deterministic=True)
    if variant == 0:
        _full_check(s, n_flow=1, use_persistent=1)
        _full_check(s, n_flow=1, store_pairs=1)
    else:  # the adjoint walking the forward's stored orders, four threads per ray
        _full_check(s, n_flow=1, variant=1, keep_order=1)
        _full_check(s, n_flow=1, variant=1, keep_order=1, deterministic=True, use_persistent=1)


def test_ray_batch_matches_full_render():
    """A ray batch renders exactly the listed pixels of the full image: bitwise the
    same depth, alpha, normal and flow values."""
    base = synth.object_orbit(K=60, n_views=2, W=40, H=30)
    s = synth.ray_batch(base, 700, seed=3)
    p = fmb.default_params(n_flow=1)
    full, _, _ = gpu_forward(base, p)
    part, _, _ = gpu_forward(s, p)
    for v in s.views:
        bv = next(b for b in base.views if b["pose"] == v["pose"])
        rays = np.asarray(v["rays"])
        for key, ch in (("depth", 1), ("alpha", 1), ("normal", 3), ("flow", 2)):
            a = plane_view(part[key], v, ch)
            b = plane_view(full[key], bv, ch)[:, rays]
            assert np.array_equal(a, b), key



# --------------------------------------------------- loss attribution (Sec. 8, Eq. 19)

@pytest.mark.parametrize("variant", [0, 1])
def test_loss_attribution_parity(variant):
    """Per-Gaussian sums of ray loss x normalised weight against the oracle, on a ray
    batch across frames (the paper's ~5 % sample), on whole images, and for K above
    one 256-Gaussian block (two-parameter only); relative to the total loss."""
    cases = [synth.ray_batch(synth.object_orbit(K=100, n_views=8, W=48, H=40), 800, seed=4),
             synth.object_orbit(K=37, n_views=2, W=30, H=20), _ac_ragged_scene()]
    if variant == 0:
        cases.append(synth.object_orbit(K=300, n_views=2, W=24, H=20))
    for s in cases:
        params = fmb.default_params(n_flow=0, variant=variant)
        gpu, r, dev = gpu_forward(s, params)
        loss = np.random.default_rng(7).uniform(0.0, 1.0, s.n_pixels).astype(np.float32)
        loss[::5] = 0.0  # skipped rays
        a = r.attribution(*dev, torch.as_tensor(loss, device="cuda")).cpu().numpy().astype(np.float64)
        ref = oracle.attribution_scene(s, loss, variant=variant)
        assert np.max(np.abs(a - ref)) <= 1e-5 * loss.sum(), float(np.max(np.abs(a - ref)) / loss.sum())
        assert abs(a.sum() - loss.astype(np.float64).sum()) <= 1e-4 * loss.sum()


@pytest.mark.parametrize("variant", [0, 1])
def test_loss_attribution_full_size(variant):
    """The 16-view 320x240 orbit at full size in the bench's configuration: the
    normalised weights of a ray sum to one (the softmax of Eq. 3 on every ray; the
    alpha-compositing weights w / W wherever W > 0, i.e. alpha > 0), so the
    attribution adds up to the loss of those rays; no entry is negative; a zero loss
    attributes nothing."""
    s = synth.object_orbit()
    params = fmb.default_params(n_flow=1, variant=variant)
    gpu, r, dev = gpu_forward(s, params)
    loss = np.random.default_rng(11).uniform(0.0, 1.0, s.n_pixels).astype(np.float32)
    loss[::7] = 0.0
    a = r.attribution(*dev, torch.as_tensor(loss, device="cuda")).cpu().numpy().astype(np.float64)
    covered = gpu["alpha"].reshape(-1) > 0.0 if variant == 1 else np.ones(s.n_pixels, dtype=bool)
    want = float(loss.astype(np.float64)[covered].sum())
    assert np.all(a >= 0.0)
    assert abs(a.sum() - want) <= 1e-4 * want, (a.sum(), want)
    z = r.attribution(*dev, torch.zeros(s.n_pixels, device="cuda")).cpu().numpy()
    assert np.all(z == 0.0)


# ------------------------------------------------------------ per-Gaussian colours

@pytest.mark.parametrize("variant,deterministic,keep_order", [(0, False, 0), (0, True, 0), (1, False, 0), (1, True, 0),
                                                           (1, True, 1)])
def test_colour_parity(variant, deterministic, keep_order):
    """Colour mode: the colour plane (Eq. 3 with per-Gaussian RGB) and every gradient,
    colours' included, against the oracle; the other planes and gradients are those
    of the colour-free render."""
    for s, nf in ((synth.object_orbit(K=100, n_views=3, W=40, H=30), 1), (synth.single_view(), 0)):
        rng = np.random.default_rng(9)
        colors = rng.uniform(0.0, 1.0, (s.means.shape[0], 3)).astype(np.float32)
        params = fmb.default_params(n_flow=nf, variant=variant, colors=1, deterministic=int(deterministic),
                                    keep_order=keep_order)
        r = fmb.Renderer(s.obj_offsets, s.views, len(s.poses), params)
        dev = dev_scene(s)
        cdev = torch.as_tensor(colors, device="cuda")
        out = r.forward(*dev, colors=cdev)
        torch.cuda.synchronize()
        gpu = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items() if v is not None}
        ref = oracle.render_scene(s, n_flow=nf, variant=variant, colors=colors)
        amb = ac_order_ambiguous(s) if variant == 1 else None
        compare_forward(s, gpu, ref, nf, True, variant=variant, ambiguous=amb)
        ok = ref["alpha"] >= 1e-2
        if amb is not None:
            ok &= ~amb
        for v in s.views:
            o, P = v["pix_offset"], synth.view_entries(v)
            e = np.abs(plane_view(gpu["color"], v, 3) - plane_view(ref["color"], v, 3)).max(0)
            assert np.all((e <= 1e-4)[ok[o:o + P]]), float(e[ok[o:o + P]].max())
        ups = masked_upstream(s, ref["alpha"], nf, seed=3, nnorm_ref=nnorm_batched(s, ref["saved"]), exclude=amb)
        gcol = np.random.default_rng(10).standard_normal(3 * s.n_pixels).astype(np.float32)
        for v in s.views:  # colour gradient only where the colour is unique (alpha >= 1e-2, order resolved)
            o, P = v["pix_offset"], synth.view_entries(v)
            gcol[3 * o:3 * (o + P)] *= np.tile(ok[o:o + P], 3)
        T = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32,
                                                              device="cuda")
        g = r.backward(*dev, T(ups["g_depth"]), T(ups["g_alpha"]), T(ups["g_normal"]), T(ups["g_flow"]),
                       colors=cdev, g_color=T(gcol))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items() if v is not None}
        refg = oracle.backward_scene(s, ups["g_depth"], ups["g_alpha"], ups["g_normal"], ups["g_flow"], n_flow=nf,
                                     variant=variant, colors=colors, g_color=gcol)
        compare_grads(g, refg, keys=("means", "chol", "weights", "poses", "colors"))
