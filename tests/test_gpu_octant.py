"""Box tests specialised to a warp's direction octant (vsr_trace octant 1).

A warp whose rays all point into one octant runs a traversal compiled for
that octant, whose slab test reads each axis's entry and exit plane directly
instead of ordering the two planes with min/max; other warps run the generic
test.  Both give every box test the same outcome, so:

- hits and COUNT counters equal the oracle's for every intersector and query,
  on frames with warps of one octant (camera rays in row order, shadow rays
  toward one light) and warps that mix octants (the camera rays shuffled,
  diffuse rays);
- on the full-size billboard forest the records are bit-identical to the
  generic kernel's in the benchmark's launch configuration;
- after a vertex update whose refit leaves a box non-finite or inverted, the
  scene falls back to the generic test, and results stay identical;
- the parameter is refused where it does not apply.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = ["none", "default", "alpha_tex", "proc_alpha", "count"]


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    return vsr


@pytest.fixture(scope="module")
def small(V):
    sc, rays = scenes.small_quads()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    yield sc, rays, blob, s
    s.close()


def _same_as_oracle(hits, ref, st, label):
    got = hits.cpu().numpy().view(np.uint32)
    want = O.hits_raw(ref).view(np.uint32)
    bad = np.any(got != want, axis=1) & (st[:, 3] == 0)
    assert not bad.any(), f"{label}: {int(bad.sum())} rays differ"


def _octants_per_warp(rays):
    """Number of distinct direction octants among each run of 32 rays."""
    sign = np.signbit(rays[:, 4:7]).astype(np.int64)
    code = sign[:, 0] | (sign[:, 1] << 1) | (sign[:, 2] << 2)
    pad = (-len(code)) % 32
    code = np.concatenate([code, np.full(pad, code[-1])]).reshape(-1, 32)
    return np.array([len(np.unique(w)) for w in code])


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", KINDS)
def test_octant_matches_oracle(V, small, kind, query):
    sc, rays, blob, s = small
    # the camera frame in row order: every warp is one row segment of one
    # image quadrant, so one octant; shuffled, almost every warp mixes octants
    shuffled = rays[np.random.default_rng(5).permutation(len(rays))]
    assert np.all(_octants_per_warp(rays) == 1)
    assert (_octants_per_warp(shuffled) > 1).mean() > 0.9
    for label, rr in (("frame", rays), ("shuffled", shuffled)):
        ref, st = O.trace_bvh(sc, blob, rr, kind, query)
        d = torch.from_numpy(np.ascontiguousarray(rr)).cuda()
        for c in (dict(block_size=128), dict(block_size=64, image_width=256),
                  dict(block_size=256, image_width=37)):
            p = V.trace_params(octant=1, **c)
            hits, cnt = V.trace(s, d, kind, query, counters=(kind == "count"), params=p)
            _same_as_oracle(hits, ref, st, f"octant {label} {kind}/{query}/{c}")
            if kind == "count":
                assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])
    assert V.vsr_get_device_error(s) == 0


def test_octant_shadow_and_diffuse_rays(V, small):
    """Shadow rays toward one light (every warp one octant) and diffuse rays
    (octants mixed in almost every warp), any hit and closest hit."""
    sc, rays, blob, s = small
    href, _ = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest")
    sh = O.shadow_rays(rays, O.hits_raw(href), scenes.light_dir_f32(), scenes.shadow_eps(sc))
    diff = scenes.diffuse_rays(np.random.default_rng(11), sc, 40_000)
    assert (_octants_per_warp(diff) > 1).mean() > 0.9
    for label, rr in (("shadow", sh), ("diffuse", diff)):
        d = torch.from_numpy(np.ascontiguousarray(rr)).cuda()
        for kind, q in (("alpha_tex", "any"), ("proc_alpha", "closest"), ("count", "any")):
            ref, st = O.trace_bvh(sc, blob, rr, kind, q)
            hits, cnt = V.trace(s, d, kind, q, counters=(kind == "count"),
                                params=V.trace_params(octant=1))
            _same_as_oracle(hits, ref, st, f"{label} {kind}/{q}")
            if kind == "count":
                assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])


def test_octant_in_coherence_order(V, small):
    """Coherence order (the rays sorted by origin cell and direction inside
    the launch) with the octant test: warps of sorted, shuffled camera rays
    and of diffuse rays give the oracle's records."""
    sc, rays, blob, s = small
    shuffled = rays[np.random.default_rng(9).permutation(len(rays))]
    diff = scenes.diffuse_rays(np.random.default_rng(12), sc, 30_000)
    for rr in (shuffled, diff):
        d = torch.from_numpy(np.ascontiguousarray(rr)).cuda()
        for kind, q in (("alpha_tex", "closest"), ("count", "any")):
            ref, st = O.trace_bvh(sc, blob, rr, kind, q)
            hits, cnt = V.trace(s, d, kind, q, counters=(kind == "count"),
                                params=V.trace_params(ray_order=1, octant=1))
            _same_as_oracle(hits, ref, st, f"ordered {kind}/{q}")
            if kind == "count":
                assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])


@pytest.mark.parametrize("n", [1, 31, 33, 4097])
def test_octant_ragged_and_clip(V, small, n):
    sc, rays, blob, s = small
    sub = rays[::-1][:n].copy()
    ref, st = O.trace_bvh(sc, blob, sub, "alpha_tex", "closest")
    hits, _ = V.trace(s, torch.from_numpy(sub).cuda(), "alpha_tex", "closest",
                      params=V.trace_params(octant=1, block_size=96))
    _same_as_oracle(hits, ref, st, f"n={n}")
    lo, hi = (0.2, 0.1, 0.0), (0.8, 0.7, 0.9)
    ref, st = O.trace_bvh(sc, blob, sub, "clip", "any", clip_lo=lo, clip_hi=hi)
    hits, _ = V.trace(s, torch.from_numpy(sub).cuda(), "clip", "any",
                      params=V.trace_params(octant=1), clip_lo=lo, clip_hi=hi)
    _same_as_oracle(hits, ref, st, f"clip n={n}")


def test_octant_edge_case_rays(V, small):
    sc, rays, blob, s = small
    inf, nan = np.inf, np.nan
    special = np.array([
        [0.5, 0.5, -1, 0, 0, 0, 1, inf],        # axis-parallel
        [0.5, 0.5, -1, 0, 0, 0, 1, -1],         # inactive (tmax < tmin)
        [0.5, 0.5, -1, 0, 0, 0, 0, inf],        # zero direction
        [0.5, 0.5, -1, 0, nan, 0, 1, inf],      # NaN direction component
        [-1e30, 0.5, 0.5, 0, 1, 0, 0, inf],     # far origin
        [0.5, 0.5, 0.5, 0, -0.0, 0.0, 1, inf],  # signed zeros
        [0.5, 0.5, 0.5, 0, 1e-30, -1e-30, 1, inf],
    ], np.float32)
    # each ray alone in its warp (one octant), then all in one warp (mixed)
    for rr in (np.repeat(special, 32, axis=0), special):
        d = torch.from_numpy(np.ascontiguousarray(rr)).cuda()
        for kind, q in (("default", "closest"), ("alpha_tex", "any"), ("count", "closest")):
            ref, st = O.trace_bvh(sc, blob, rr, kind, q)
            hits, cnt = V.trace(s, d, kind, q, counters=(kind == "count"),
                                params=V.trace_params(octant=1))
            _same_as_oracle(hits, ref, st, f"special {kind}/{q}")
            if kind == "count":
                assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])


def test_octant_after_refit(V):
    """Vertex updates: moved vertices (boxes still ordered) trace identically
    with and without the octant test; vertices set to NaN make the refit
    leave inverted boxes, the scene drops to the generic test, and results
    are still identical."""
    sc, rays = scenes.small_quads(seed=scenes.SEED_BASE + 46)
    s = V.scene_from_inputs(sc, sc.bvh())
    d = torch.from_numpy(rays).cuda()
    try:
        rng = np.random.default_rng(3)
        moved = sc.verts + rng.normal(0, 0.01, sc.verts.shape).astype(np.float32)
        bad = moved.copy()
        bad[sc.idx[:300].ravel()] = np.nan
        for verts in (moved, bad):
            V.vsr_scene_update(s, torch.from_numpy(np.ascontiguousarray(verts)).cuda())
            for kind, q in (("default", "closest"), ("count", "any"), ("alpha_tex", "closest")):
                cnt = kind == "count"
                h0, c0 = V.trace(s, d, kind, q, counters=cnt, params=V.trace_params())
                h1, c1 = V.trace(s, d, kind, q, counters=cnt, params=V.trace_params(octant=1))
                assert torch.equal(h0.view(torch.int32), h1.view(torch.int32)), (kind, q)
                if cnt:
                    assert torch.equal(c0, c1)
        assert V.vsr_get_device_error(s) == 0
    finally:
        s.close()


def test_octant_forest_full_size(V):
    """The full billboard forest frame in the benchmark's launch layout
    (4x8 pixel tiles): primary closest hits and shadow any hits with the
    alpha texture are bit-identical to the generic kernel's, and a seeded
    sample of the primary rays equals the oracle's."""
    import bench
    sc, rays = scenes.billboard_forest()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    try:
        d = torch.from_numpy(rays).cuda()
        p0 = bench.default_params(V)
        p1 = bench.default_params(V)
        p1.octant = 1
        h0, _ = V.trace(s, d, "alpha_tex", "closest", params=p0)
        h1, _ = V.trace(s, d, "alpha_tex", "closest", params=p1)
        assert torch.equal(h0.view(torch.int32), h1.view(torch.int32))
        sh = torch.empty_like(d)
        V.vsr_make_shadow_rays(d, h0, scenes.light_dir_f32(), scenes.shadow_eps(sc), sh)
        s0, _ = V.trace(s, sh, "alpha_tex", "any", params=p0)
        s1, _ = V.trace(s, sh, "alpha_tex", "any", params=p1)
        assert torch.equal(s0.view(torch.int32), s1.view(torch.int32))
        # the other intersectors of the bench's octant comparison, both passes
        for kind in ("default", "proc_alpha", "count"):
            cnt = kind == "count"
            for q, rr in (("closest", d), ("any", sh)):
                g0, c0 = V.trace(s, rr, kind, q, counters=cnt, params=p0)
                g1, c1 = V.trace(s, rr, kind, q, counters=cnt, params=p1)
                assert torch.equal(g0.view(torch.int32), g1.view(torch.int32)), (kind, q)
                if cnt:
                    assert torch.equal(c0, c1)
        sel = np.sort(np.random.default_rng(8).choice(len(rays), 5000, replace=False))
        ref, st = O.trace_bvh(sc, blob, rays[sel], "alpha_tex", "closest")
        _same_as_oracle(h1[torch.from_numpy(sel).cuda()], ref, st, "forest sample")
        assert V.vsr_get_device_error(s) == 0
    finally:
        s.close()


def test_octant_tuned_and_rejected(V, small):
    sc, rays, blob, s = small
    d = torch.from_numpy(rays).cuda()
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    for bad in (dict(octant=2), dict(octant=1, persistent=1), dict(octant=1, lockstep=1),
                dict(octant=1, stack_regs=2), dict(octant=1, reg_cap_blocks=4)):
        with pytest.raises(V.VsrError, match="octant"):
            V.vsr_trace(s, d, V.intersector("default"), "closest", hits, None,
                        V.trace_params(**bad))
    with pytest.raises(V.VsrError, match="octant"):
        V.vsr_trace(s, d, V.intersector("default", "dynamic"), "closest", hits, None,
                    V.trace_params(octant=1))
    multi = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="octant"):
        V.vsr_trace_multi(s, d, V.intersector("default"), 1, multi, None,
                          V.trace_params(octant=1))
    # the tuner's choice, whatever it is, gives the oracle's records
    ref, st = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest")
    tp = V.vsr_trace_tune(s, d, V.intersector("alpha_tex"), "closest", hits, image_width=256)
    assert V.params_dict(tp)["octant"] in (0, 1)
    got, _ = V.trace(s, d, "alpha_tex", "closest", params=tp)
    _same_as_oracle(got, ref, st, "tuned")


def test_octant_render_and_path(V, small):
    """The render (trace kernels + shading) and the path tracer take the
    parameter too: images, hit records and path radiance are identical with
    and without it."""
    sc, rays, blob, s = small
    d = torch.from_numpy(rays).cuda()
    n = len(rays)
    shade = V.shade_params(scenes.light_dir_f32())
    out = {}
    for oc in (0, 1):
        p = V.trace_params(image_width=256, octant=oc)
        img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        hits = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        V.vsr_render(s, d, V.intersector("alpha_tex"), shade, img, hits, p)
        dirs = torch.from_numpy(scenes.path_dirs(n, 2)).cuda()
        rad = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        pp = V.path_params(2, scenes.shadow_eps(sc))
        V.vsr_path_trace(s, d, V.intersector("alpha_tex"), pp, dirs, rad, None, p)
        torch.cuda.synchronize()
        out[oc] = (img, hits, rad)
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    assert V.vsr_get_device_error(s) == 0
