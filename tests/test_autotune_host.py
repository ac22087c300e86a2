"""Host-side logic of the autotuner (no GPU needed)."""

from paper_2308_14737_gb300 import autotune, fmb, synth


def test_layout_key_groups_by_shape_class():
    from paper_2308_14737_gb300 import build

    build.build()
    p = fmb.default_params(n_flow=1)
    a = synth.object_orbit(K=100, n_views=16, W=320, H=240)
    b = synth.object_orbit(seed=5, K=110, n_views=16, W=320, H=240)  # same log2 buckets
    c = synth.object_orbit(K=400, n_views=16, W=320, H=240)
    ka = autotune.layout_key(a.obj_offsets, a.views, p, True)
    assert ka == autotune.layout_key(b.obj_offsets, b.views, p, True)
    assert ka != autotune.layout_key(c.obj_offsets, c.views, p, True)
    assert ka != autotune.layout_key(a.obj_offsets, a.views, p, False)


def test_apply_sets_only_tuned_fields():
    from paper_2308_14737_gb300 import build

    build.build()
    p = fmb.default_params(n_flow=2, want_normals=0)
    q = autotune.apply(p, dict(fwd_rays_per_thread=4, bwd_threads=128, bwd_ray_tile=256, use_persistent=1))
    assert (q.fwd_rays_per_thread, q.bwd_threads, q.bwd_ray_tile, q.use_persistent) == (4, 128, 256, 1)
    assert (q.n_flow, q.want_normals) == (2, 0) and abs(q.beta1 - 21.4) < 1e-6
    assert p.fwd_rays_per_thread == 0  # the input is not modified


def test_small_batches_get_short_tile_candidates():
    """A batch with fewer rays than two waves of 256-ray tiles also tries the short
    tiles; a full-size batch keeps the standard list."""
    small = synth.single_view()  # one 64 x 64 view
    big = synth.object_orbit()   # 16 views of 320 x 240
    cs = autotune.candidates_for(small.views, 152)
    cb = autotune.candidates_for(big.views, 152)
    assert cb == autotune.CANDIDATES
    assert cs == autotune.CANDIDATES + autotune.SMALL_CANDIDATES
    for c in autotune.SMALL_CANDIDATES:
        assert c["bwd_ray_tile"] % 32 == 0 and 32 <= c["bwd_threads"] <= 160 and c["bwd_threads"] % 32 == 0
        assert c["fwd_rays_per_thread"] in (1, 2, 4)
        # a Gaussian split runs only with packed (even) rays per thread
        assert c.get("fwd_ksplit", 0) in (0, 2, 4) and (c.get("fwd_ksplit", 0) == 0 or c["fwd_rays_per_thread"] == 2)
        assert 0 <= c.get("bwd_gblocks", 0) <= 64
    # the Gaussian-block hint is among the small-batch candidates, and a tuned field
    assert {c.get("bwd_gblocks", 0) for c in autotune.SMALL_CANDIDATES} == {0, 2, 4}
    assert "bwd_gblocks" in autotune.TUNED_FIELDS
    p = autotune.apply(fmb.default_params(), dict(bwd_gblocks=4, bwd_threads=128))
    assert p.bwd_gblocks == 4 and p.bwd_threads == 128
