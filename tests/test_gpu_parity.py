"""GPU traversal vs the CPU oracle, through the C ABI (needs a GB300).

Bar: primitive ids, hit distances, barycentrics and counts are bit-identical
to the oracle's while-while traversal in the same fixed order (both sides use
FP32 with the same rounding order).  Rays the oracle flags as near ties
(within 1e-6 of a triangle edge in barycentric terms, or of an alpha decision
boundary) may differ in primitive id and are reported; every other ray must
match exactly, and t must in any case agree within 1e-5 relative when the ids
agree.
"""
import ctypes
import math
import os

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


def _cudart():
    import ctypes.util
    import glob
    cands = [ctypes.util.find_library("cudart"), "/usr/local/cuda/lib64/libcudart.so"]
    cands += glob.glob(os.path.join(os.path.dirname(torch.__file__), "..", "nvidia", "*",
                                    "lib", "libcudart.so*"))
    for c in cands:
        if not c:
            continue
        try:
            lib = ctypes.CDLL(c)
        except OSError:
            continue
        lib.cudaMalloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t]
        lib.cudaFree.argtypes = [ctypes.c_void_p]
        return lib
    return None


def _to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def compare(gpu_hits, ref_hits, ref_stats=None, label=""):
    """Bitwise comparison; returns the number of near-tie rays that differ."""
    g = gpu_hits.cpu().numpy()
    gb = g.view(np.uint32)
    ref = O.hits_raw(ref_hits).view(np.uint32)
    diff = np.any(gb != ref, axis=1)
    ties = np.zeros(len(g), bool) if ref_stats is None else ref_stats[:, 3] != 0
    bad = diff & ~ties
    if bad.any():
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{label}: {int(bad.sum())} rays differ, first {i}: gpu "
                             f"{g[i].tolist()} prim {gb[i,3]:#x} vs oracle "
                             f"{ref.view(np.float32)[i].tolist()} prim {ref[i,3]:#x}")
    same_prim = gb[:, 3] == ref[:, 3]
    hit = same_prim & (ref[:, 3] != O.NONE)
    t_g, t_r = g[hit, 0].astype(np.float64), ref.view(np.float32)[hit, 0].astype(np.float64)
    assert np.all(np.abs(t_g - t_r) <= 1e-5 * np.maximum(1.0, np.abs(t_r))), label
    return int((diff & ties).sum())


@pytest.fixture(scope="module")
def small(V):
    sc, rays = scenes.small_quads()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    yield sc, rays, blob, s
    s.close()


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("dispatch", ["static", "dynamic"])
@pytest.mark.parametrize("kind", KINDS)
def test_small_all_intersectors(V, small, kind, query, dispatch):
    sc, rays, blob, s = small
    ref, st = O.trace_bvh(sc, blob, rays, kind, query, cutoff_u8=128)
    hits, cnt = V.trace(s, _to_dev(rays), kind, query, dispatch, counters=(kind == "count"))
    compare(hits, ref, st, f"{kind}/{query}/{dispatch}")
    if kind == "count":
        assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", ["default", "alpha_tex", "proc_alpha"])
def test_stats_variant_counts(V, small, kind, query):
    sc, rays, blob, s = small
    ref, st = O.trace_bvh(sc, blob, rays, kind, query)
    r = _to_dev(rays)
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    stats = torch.empty((len(rays), 4), dtype=torch.int32, device="cuda")
    V.vsr_trace_stats(s, r, V.intersector(kind), query, hits, stats)
    compare(hits, ref, st, "stats")
    got = stats.cpu().numpy().view(np.uint32)
    assert np.array_equal(got[:, :3], st[:, :3])
    # texture look-ups: every triangle of this scene is textured, so the
    # alpha intersectors look up once per consultation and the others never
    want = st[:, 2] if kind in ("alpha_tex", "proc_alpha") else np.zeros_like(st[:, 2])
    assert np.array_equal(got[:, 3], want)


@pytest.mark.parametrize("block,refill", [(32, 1), (128, 16), (256, 32), (64, 24)])
@pytest.mark.parametrize("query", ["closest", "any"])
def test_persistent_refill(V, small, block, refill, query):
    sc, rays, blob, s = small
    ref, st = O.trace_bvh(sc, blob, rays, "alpha_tex", query)
    p = V.trace_params(block_size=block, persistent=1, refill_threshold=refill)
    hits, _ = V.trace(s, _to_dev(rays), "alpha_tex", query, params=p)
    compare(hits, ref, st, "persistent")
    ref_c, st_c = O.trace_bvh(sc, blob, rays, "count", query)
    hits_c, cnt = V.trace(s, _to_dev(rays), "count", query, counters=True, params=p)
    compare(hits_c, ref_c, st_c, "persistent count")
    assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st_c[:, :2])


@pytest.mark.parametrize("n", [0, 1, 31, 33, 127, 129, 4097, 65536 + 17])
@pytest.mark.parametrize("persistent", [0, 1])
def test_ragged_sizes(V, small, n, persistent):
    sc, rays, blob, s = small
    sel = np.resize(rays[::-1], (n, 8)) if n else np.zeros((0, 8), np.float32)
    p = V.trace_params(block_size=96, persistent=persistent, refill_threshold=20)
    if n == 0:
        r = torch.zeros((0, 8), dtype=torch.float32, device="cuda")
        hits = torch.zeros((0, 4), dtype=torch.float32, device="cuda")
        V.vsr_trace(s, r, V.intersector("alpha_tex"), "closest", hits, None, p)
        return
    ref, st = O.trace_bvh(sc, blob, sel, "alpha_tex", "closest")
    hits, _ = V.trace(s, _to_dev(sel), "alpha_tex", "closest", params=p)
    compare(hits, ref, st, f"n={n}")


@pytest.mark.parametrize("width", [1, 3, 4, 5, 37, 256, 1000])
@pytest.mark.parametrize("n", [1, 31, 33, 4097, 65536])
def test_image_width_tiles(V, small, width, n):
    """Pixel-tile thread mapping: every ray traced exactly once, results
    identical to buffer order (and so to the oracle) for static, dynamic and
    persistent launches, COUNT counters included, at ragged sizes and widths
    that leave partial tiles and a partial last row."""
    sc, rays, blob, s = small
    sel = _to_dev(np.resize(rays, (n, 8)))
    for disp, pers, kind, q in [("static", 0, "alpha_tex", "closest"),
                                ("static", 0, "count", "any"),
                                ("dynamic", 0, "proc_alpha", "closest"),
                                ("static", 1, "alpha_tex", "any"),
                                ("static", 1, "count", "closest")]:
        cnt = kind == "count"
        base = V.trace_params(block_size=96, persistent=pers)
        tiled = V.trace_params(block_size=96, persistent=pers, image_width=width)
        h0, c0 = V.trace(s, sel, kind, q, disp, counters=cnt, params=base)
        h1 = torch.full_like(h0, float("nan"))
        c1 = torch.full_like(c0, -1) if cnt else None
        V.vsr_trace(s, sel, V.intersector(kind, disp), q, h1, c1, tiled)
        torch.cuda.synchronize()
        assert torch.equal(h0.view(torch.int32), h1.view(torch.int32)), (disp, pers, kind, q)
        if cnt:
            assert torch.equal(c0, c1)
    if n == 65536:
        ref, st = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest")
        p = V.trace_params(image_width=width)
        hits, _ = V.trace(s, sel, "alpha_tex", "closest", params=p)
        compare(hits, ref, st, f"width={width}")
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("leaf,bins,cost", [(1, 32, 1.0), (2, 8, 1.0), (8, 128, 1.0),
                                            (4, 32, 0.0), (4, 32, 4.0)])
def test_other_build_parameters(V, small, leaf, bins, cost):
    """Trees of other shapes (leaf sizes 1..8, 8..128 bins, traversal costs
    0..4): closest and any hits and counts still match the oracle's traversal
    of the same tree, and closest hits equal the default tree's."""
    from paper_1912_12786_gb300.inputs import _lib
    sc, rays, blob0, s0 = small
    blob = _lib.bvh_build(sc.verts, sc.idx, leaf_max=leaf, bins=bins, traversal_cost=cost)
    s = V.scene_from_inputs(sc, blob)
    try:
        d = _to_dev(rays)
        for q in ("closest", "any"):
            ref, st = O.trace_bvh(sc, blob, rays, "count", q)
            hits, cnt = V.trace(s, d, "count", q, counters=True)
            compare(hits, ref, st, f"leaf={leaf} bins={bins} cost={cost} {q}")
            ok = st[:, 3] == 0
            assert np.array_equal(cnt.cpu().numpy().view(np.uint32)[ok], st[ok, :2])
        h0, _ = V.trace(s0, d, "alpha_tex", "closest")
        h1, _ = V.trace(s, d, "alpha_tex", "closest")
        assert torch.equal(h0.view(torch.int32), h1.view(torch.int32))
        assert V.vsr_get_device_error(s) == 0
    finally:
        s.close()


def test_shadow_rays_and_any_hit(V, small):
    sc, rays, blob, s = small
    href, _ = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest")
    light = scenes.light_dir_f32()
    eps = scenes.shadow_eps(sc)
    sref = O.shadow_rays(rays, O.hits_raw(href), light, eps)
    out = torch.empty((len(rays), 8), dtype=torch.float32, device="cuda")
    V.vsr_make_shadow_rays(_to_dev(rays), _to_dev(O.hits_raw(href)), light, eps, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), sref.view(np.uint32))
    for kind in ("alpha_tex", "default", "proc_alpha"):
        ref, st = O.trace_bvh(sc, blob, sref, kind, "any")
        hits, _ = V.trace(s, _to_dev(sref), kind, "any")
        compare(hits, ref, st, f"shadow {kind}")


def test_edge_case_rays(V, small):
    sc, rays, blob, s = small
    inf, nan = np.inf, np.nan
    special = np.array([
        [0.5, 0.5, -1, 0, 0, 0, 1, inf],        # axis-parallel
        [0.5, 0.5, -1, 0, 0, 0, 1, -1],         # inactive (tmax < tmin)
        [0.5, 0.5, -1, 2, 0, 0, 1, 1],          # empty interval
        [0.5, 0.5, -1, 0, 0, 0, 0, inf],        # zero direction
        [0.5, 0.5, -1, 0, nan, 0, 1, inf],      # NaN direction component
        [0.5, 0.5, -1, 0, 0, 0, -1, inf],       # pointing away
        [-1e30, 0.5, 0.5, 0, 1, 0, 0, inf],     # far origin
        [0.5, 0.5, 0.5, 0, 1, 1, 1, inf],       # origin inside the scene
        [0.5, 0.5, 0.5, 0, -0.0, 0.0, 1, inf],  # signed zeros
    ], np.float32)
    for kind in ("default", "alpha_tex", "count"):
        for q in ("closest", "any"):
            ref, st = O.trace_bvh(sc, blob, special, kind, q)
            hits, cnt = V.trace(s, _to_dev(special), kind, q, counters=(kind == "count"))
            compare(hits, ref, st, f"special {kind}/{q}")
            if kind == "count":
                assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])


def test_empty_and_single_triangle_scenes(V):
    e = scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32),
                     np.zeros((0, 3, 2), np.float32), np.zeros(0, np.uint32), [])
    rays = scenes.pinhole_rays((0, 0, -1), (0, 0, 0), (0, 1, 0), 60, 8, 8)
    s = V.scene_from_inputs(e, e.bvh())
    hits, cnt = V.trace(s, _to_dev(rays), "count", "closest", counters=True)
    h = hits.cpu().numpy()
    assert np.all(h[:, 3].view(np.uint32) == O.NONE) and np.all(np.isinf(h[:, 0]))
    assert np.all(cnt.cpu().numpy() == 0)
    v = np.array([[-1, -1, 0], [1, -1, 0], [0, 1, 0]], np.float32)
    one = scenes.Scene("one", v, np.array([[0, 1, 2]], np.uint32), np.zeros((1, 3, 2), np.float32),
                       np.array([scenes.NONE], np.uint32), [])
    blob = one.bvh()
    s1 = V.scene_from_inputs(one, blob)
    for kind in ("alpha_tex", "proc_alpha", "count"):
        ref, st = O.trace_bvh(one, blob, rays, kind, "closest")
        hits, _ = V.trace(s1, _to_dev(rays), kind, "closest", counters=(kind == "count"))
        compare(hits, ref, st, f"single {kind}")


def test_invalid_arguments_rejected_before_launch(V, small):
    sc, rays, blob, s = small
    r = _to_dev(rays)
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    isect = V.intersector("alpha_tex")
    host = np.zeros((len(rays), 8), np.float32)
    L = V.lib()
    st = L.vsr_trace(s.handle, host.ctypes.data, len(rays), ctypes.byref(isect), 0,
                     hits.data_ptr(), None, None, None)
    assert st == V.VSR_ERR_ARG and "device memory" in V.vsr_last_error()
    # A buffer from cudaMalloc that is too small for n hits is rejected.  (The
    # check sees whole allocations, so it is made with a raw allocation rather
    # than a tensor carved from the caching allocator's larger blocks.)
    rt = _cudart()
    if rt is not None:
        raw = ctypes.c_void_p()
        assert rt.cudaMalloc(ctypes.byref(raw), ctypes.c_size_t(256)) == 0
        try:
            st = L.vsr_trace(s.handle, r.data_ptr(), len(rays), ctypes.byref(isect), 0,
                             raw.value, None, None, None)
            assert st == V.VSR_ERR_ARG and "smaller" in V.vsr_last_error()
        finally:
            rt.cudaFree(raw)
    cnt = torch.empty((len(rays), 2), dtype=torch.int32, device="cuda")
    with pytest.raises(V.VsrError, match="COUNT"):
        V.vsr_trace(s, r, isect, "closest", hits, cnt)
    with pytest.raises(V.VsrError, match="block_size"):
        V.vsr_trace(s, r, isect, "closest", hits, None, V.trace_params(block_size=100))
    with pytest.raises(V.VsrError, match="refill"):
        V.vsr_trace(s, r, isect, "closest", hits, None, V.trace_params(refill_threshold=0))
    bad = V.intersector("alpha_tex")
    bad.kind = 9
    with pytest.raises(V.VsrError, match="kind"):
        V.vsr_trace(s, r, bad, "closest", hits)
    s2 = V.vsr_scene_create_indexed(sc.verts, sc.idx, sc.uvs, sc.geom_id, sc.textures)
    with pytest.raises(V.VsrError, match="VSR_ERR_STATE"):
        V.vsr_trace(s2, r, isect, "closest", hits)
    corrupt = blob.copy()
    corrupt[100] ^= 1
    with pytest.raises(V.VsrError, match="VSR_ERR_BLOB"):
        V.vsr_bvh_load(s2, corrupt)
    other = scenes.small_quads(seed=5, n_quads=10)[0].bvh()
    with pytest.raises(V.VsrError, match="different number"):
        V.vsr_bvh_load(s2, other)
    with pytest.raises(V.VsrError, match="geom_id"):
        V.vsr_scene_create_indexed(sc.verts, sc.idx, sc.uvs, sc.geom_id + 3, sc.textures)
    with pytest.raises(V.VsrError, match="vertex index"):
        V.vsr_scene_create_indexed(sc.verts[:10], sc.idx, sc.uvs, sc.geom_id, sc.textures)
    s2.close()


# --------------------------------------------------------------------------
# full-size billboard forest, in the benchmark's launch configuration


@pytest.fixture(scope="module")
def forest(V):
    sc, rays = scenes.billboard_forest()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    yield sc, rays, blob, s
    s.close()


def test_forest_full_size_sampled(V, forest):
    """2,073,600 primary closest-hit rays and the shadow any-hit pass, both
    with the alpha-texture intersector; a seeded sample of rays is compared
    with the oracle one by one."""
    import bench
    sc, rays, blob, s = forest
    p = bench.default_params(V)
    hits, _ = V.trace(s, _to_dev(rays), "alpha_tex", "closest", params=p)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    sel = np.sort(rng.choice(len(rays), 20000, replace=False))
    ref, st = O.trace_bvh(sc, blob, rays[sel], "alpha_tex", "closest")
    ties = compare(hits[torch.from_numpy(sel).cuda()], ref, st, "forest primary")
    assert ties <= 2
    # shadow rays built by the oracle from its own primary hits
    light, eps = scenes.light_dir_f32(), scenes.shadow_eps(sc)
    sref = O.shadow_rays(rays[sel], O.hits_raw(ref), light, eps)
    sh_ref, sh_st = O.trace_bvh(sc, blob, sref, "alpha_tex", "any")
    sh, _ = V.trace(s, _to_dev(sref), "alpha_tex", "any", params=p)
    compare(sh, sh_ref, sh_st, "forest shadow")
    # properties of the full launch
    h = hits.cpu().numpy()
    prim = h[:, 3].view(np.uint32)
    ok = prim != O.NONE
    assert ok.mean() > 0.9
    assert np.all(prim[ok] < sc.ntri) and np.all(h[ok, 0] > 0) and np.all(np.isinf(h[~ok, 0]))
    assert np.all((h[ok, 1] >= 0) & (h[ok, 2] >= 0) & (h[ok, 1] + h[ok, 2] <= 1.0000001))
    assert V.vsr_get_device_error(s) == 0


def test_forest_invariants_full_size(V, forest):
    """Invariants that hold at any size: default == none == count hits,
    static == dynamic, persistent == one-ray-per-thread, any-hit boolean ==
    closest-hit boolean."""
    sc, rays, blob, s = forest
    r = _to_dev(rays)
    base, _ = V.trace(s, r, "default", "closest")
    for kind, disp in (("none", "static"), ("count", "static"), ("default", "dynamic"),
                       ("count", "dynamic")):
        h, _ = V.trace(s, r, kind, "closest", disp, counters=(kind == "count"))
        assert torch.equal(h.view(torch.int32), base.view(torch.int32)), (kind, disp)
    for kind in ("alpha_tex", "proc_alpha"):
        a, _ = V.trace(s, r, kind, "closest")
        b, _ = V.trace(s, r, kind, "closest", "dynamic")
        c, _ = V.trace(s, r, kind, "closest", params=V.trace_params(persistent=1))
        assert torch.equal(a.view(torch.int32), b.view(torch.int32)), kind
        assert torch.equal(a.view(torch.int32), c.view(torch.int32)), kind
        an, _ = V.trace(s, r, kind, "any")
        assert torch.equal(V.prim_ids(an) != V.MISS, V.prim_ids(a) != V.MISS), kind
