"""Pins of the CPU oracle to facts fixed outside it (no GPU).

Each test ties the oracle to something it does not compute itself: values
worked out by hand (tests/golden/worked_examples.json), an FP64 linear solve of
the ray/triangle system, closed-form coverage of the alpha patterns, a
brute-force FP64 closest-hit search, a structural enumeration of the BVH nodes
a ray must reach, and the invariants the paper's design implies (the default
intersector forwards intersect unchanged, Section 3.1; bvh_costs returns the
default result, Section 4).
"""
import json
import math
import os
import struct

import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes, bvh_validate, bvh_build

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _ray(o, d, tmin=0.0, tmax=math.inf):
    return np.array([*o, tmin, *d, tmax], np.float32)


# --------------------------------------------------------------------------
# worked examples


def test_triangle_worked_examples():
    g = json.load(open(GOLDEN))
    v0, v1, v2 = (np.array(v, np.float32) for v in g["triangle"])
    for c in g["triangle_cases"]:
        code, t, u, v = O.intersect_triangle(_ray(c["o"], c["d"]), v0, v1, v2)
        assert code == c["code"], c["name"]
        if code != -1:
            expect = tuple(float(np.float32(c[k])) for k in ("t", "u", "v"))
            assert (t, u, v) == expect, c["name"]


def test_box_worked_examples():
    g = json.load(open(GOLDEN))
    lo, hi = g["box"]["lo"], g["box"]["hi"]
    for c in g["box_cases"]:
        tf = math.inf if c["t_far"] == "inf" else c["t_far"]
        got = O.intersect_aabb(_ray(c["o"], c["d"], tmin=c["tmin"]), lo, hi, tf)
        assert got == c["hit"], c["name"]


def test_triangle_against_fp64_solve():
    """t, u, v agree with the FP64 solution of [-d, e1, e2](t,u,v) = o - v0,
    with u weighting v1 and v weighting v2 (hit point = w0 v0 + u v1 + v v2)."""
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(3000):
        V = rng.uniform(-1, 1, (3, 3)).astype(np.float32)
        o = rng.uniform(-3, 3, 3).astype(np.float32)
        target = (rng.dirichlet([1, 1, 1]) @ V.astype(np.float64))
        d = (target - o).astype(np.float32)
        code, t, u, v = O.intersect_triangle(_ray(o, d), V[0], V[1], V[2])
        V64 = V.astype(np.float64)
        M = np.stack([-d.astype(np.float64), V64[1] - V64[0], V64[2] - V64[0]], 1)
        if abs(np.linalg.det(M)) < 1e-3:
            continue
        tuv = np.linalg.solve(M, o.astype(np.float64) - V64[0])
        assert code in (0, 1)
        np.testing.assert_allclose([t, u, v], tuv, rtol=2e-4, atol=2e-4)
        w = (1 - tuv[1] - tuv[2], tuv[1], tuv[2])
        if min(w) > 1e-4:
            assert code == 1
        checked += 1
    assert checked > 2000


def test_box_against_fp64_slabs():
    """Slab test agrees with an FP64 interval computation away from ties."""
    rng = np.random.default_rng(12)
    agree = 0
    for _ in range(4000):
        lo = rng.uniform(-1, 0.5, 3)
        hi = lo + rng.uniform(0.01, 1.0, 3)
        o = rng.uniform(-3, 3, 3)
        d = rng.normal(size=3)
        d[rng.uniform(size=3) < 0.1] = 0.0
        tmin = float(rng.uniform(0, 1))
        tfar = float(rng.choice([math.inf, rng.uniform(0, 5)]))
        lo32, hi32, o32, d32 = (np.asarray(x, np.float32) for x in (lo, hi, o, d))
        tn, tf, margin = tmin, tfar, math.inf
        ok = True
        for a in range(3):
            if d32[a] == 0:
                if not (lo32[a] < o32[a] < hi32[a]):
                    ok = False
                margin = min(margin, abs(o32[a] - lo32[a]), abs(o32[a] - hi32[a]))
                continue
            t0 = (float(lo32[a]) - float(o32[a])) / float(d32[a])
            t1 = (float(hi32[a]) - float(o32[a])) / float(d32[a])
            tn = max(tn, min(t0, t1))
            tf = min(tf, max(t0, t1))
        exact = ok and tn <= tf
        if margin < 1e-4 or (math.isfinite(tf) and abs(tf - tn) < 1e-4):
            continue
        got = O.intersect_aabb(_ray(o32, d32, tmin=tmin), lo32, hi32, tfar)
        assert got == exact
        agree += 1
    assert agree > 3000


# --------------------------------------------------------------------------
# hand-built BVH with hand-traced counts (bvh_costs, Section 4)


def _fnv(b: bytes) -> int:
    h = 1469598103934665603
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def make_blob(nodes, order, max_depth, leaf_max=4):
    payload = b"".join(struct.pack("<3fI3fI", *n[0], n[1], *n[2], n[3]) for n in nodes)
    payload += struct.pack(f"<{len(order)}I", *order)
    nleaves = sum(1 for n in nodes[2:] if n[3] >> 2) + (1 if nodes[0][3] >> 2 else 0)
    hdr = struct.pack("<8s8I3Q", b"VSRBVH01", 1, 64, len(nodes), len(order), max_depth,
                      leaf_max, nleaves, 0, len(payload), _fnv(payload), 0)
    return np.frombuffer(hdr + payload, np.uint8).copy()


def two_tri_scene():
    verts = np.array([[-1, -1, 1], [1, -1, 1], [0, 1, 1],
                      [-1, -1, 3], [1, -1, 3], [0, 1, 3]], np.float32)
    idx = np.array([[0, 1, 2], [3, 4, 5]], np.uint32)
    uvs = np.zeros((2, 3, 2), np.float32)
    sc = scenes.Scene("two", verts, idx, uvs, np.zeros(2, np.uint32),
                      [scenes.Texture("u8", 1, 1, np.full((1, 1), 255, np.uint8))])
    nodes = [([-1, -1, 1], 2, [1, 1, 3], 2),          # root: inner, split on z
             ([0, 0, 0], 0, [0, 0, 0], 0),            # padding
             ([-1, -1, 1], 0, [1, 1, 1], 1 << 2),     # leaf: slot 0 (prim 0)
             ([-1, -1, 3], 1, [1, 1, 3], 1 << 2)]     # leaf: slot 1 (prim 1)
    return sc, make_blob(nodes, [0, 1], 1)


def test_hand_bvh_is_valid():
    _, blob = two_tri_scene()
    assert bvh_validate(blob) == ""


@pytest.mark.parametrize("case", [
    # (origin, direction, query, prim, t, boxes, tris)
    ((0, 0, 0), (0, 0, 1), "closest", 0, 1.0, 3, 2),   # near leaf first, far leaf popped
    ((0, 0, 4), (0, 0, -1), "closest", 1, 1.0, 3, 2),  # sign bit: right child first
    ((0, 0, 0), (0, 0, 1), "any", 0, 1.0, 3, 1),       # any-hit stops at first accept
    ((0, 0, 4), (0, 0, -1), "any", 1, 1.0, 3, 1),
    ((5, 5, 0), (0, 0, 1), "closest", None, None, 1, 0),  # root missed
    ((0, 0, 2), (0, 0, 1), "closest", 1, 1.0, 3, 1),   # only the far leaf's box is hit
    ((0.9, -0.9, 0), (0, 0, 1), "closest", 0, 1.0, 3, 2),
])
def test_hand_traced_counts(case):
    o, d, q, prim, t, boxes, tris = case
    sc, blob = two_tri_scene()
    h, st = O.trace_bvh(sc, blob, _ray(o, d)[None], "count", q, nthreads=1)
    assert (int(st[0, 0]), int(st[0, 1])) == (boxes, tris)
    if prim is None:
        assert h["prim"][0] == O.NONE and math.isinf(h["t"][0])
    else:
        assert h["prim"][0] == prim and h["t"][0] == t


# --------------------------------------------------------------------------
# closed-form coverage of the alpha patterns (Section 4 use cases)


def _quad_hits(tex, kind, n, **kw):
    sc = scenes.quad_grid_scene(tex)
    rays = scenes.orthographic_rays((0, 0), (1, 1), -1.0, n)
    blob = sc.bvh()
    h, _ = O.trace_bvh(sc, blob, rays, kind, "closest", **kw)
    return h, rays


def test_texture_orientation():
    """u selects the column, v the row; 8-bit alpha compared with the cutoff."""
    a = np.zeros((2, 4), np.uint8)
    a[0, 0:2] = 255            # row 0 (v < 0.5), columns 0-1 (u < 0.5)
    h, rays = _quad_hits(scenes.Texture("u8", 4, 2, a), "alpha_tex", 64, cutoff_u8=128)
    acc = h["prim"] != O.NONE
    expect = (rays[:, 0] < 0.5) & (rays[:, 1] < 0.5)
    assert np.array_equal(acc, expect)


def test_alpha_cutoff_is_inclusive_and_rgba_channel():
    tex = np.zeros((1, 1, 4), np.uint8)
    tex[0, 0] = (0, 0, 0, 128)
    for cut, expect in ((128, True), (129, False)):
        h, _ = _quad_hits(scenes.Texture("rgba8", 1, 1, tex), "alpha_tex", 8, cutoff_u8=cut)
        assert bool((h["prim"] != O.NONE).all()) == expect
    f = np.zeros((1, 1, 4), np.float32)
    f[0, 0] = (1.0, 1.0, 1.0, 0.3)
    for cut, expect in ((0.3, True), (0.30001, False)):
        h, _ = _quad_hits(scenes.Texture("rgba32f", 1, 1, f), "alpha_tex", 8, cutoff_f=cut)
        assert bool((h["prim"] != O.NONE).all()) == expect


def test_disc_alpha_coverage():
    """Accepted fraction on the unit quad = texel coverage of the disc
    (about pi * 0.4^2), within the grid discretisation."""
    tex = scenes.disc_alpha_u8(256, 0.4)
    h, _ = _quad_hits(tex, "alpha_tex", 1024, cutoff_u8=128)
    frac = float((h["prim"] != O.NONE).mean())
    texel_cov = float((tex.texels == 255).mean())
    assert abs(frac - texel_cov) < 0.004
    assert abs(frac - math.pi * 0.16) < 0.006


def test_procedural_alpha_coverage_and_pointwise():
    """sin(40u) sin(40v) > 0 covers p^2 + (1-p)^2 with p = 1 - 3 pi / 20."""
    tex = scenes.disc_alpha_u8(4, 0.4)  # texture only supplies geom id 0
    h, rays = _quad_hits(tex, "proc_alpha", 2048, freq=40.0)
    p = 1 - 3 * math.pi / 20
    frac = float((h["prim"] != O.NONE).mean())
    assert abs(frac - (p * p + (1 - p) ** 2)) < 0.005
    h2, rays2 = _quad_hits(tex, "proc_alpha", 256, freq=40.0)
    x = rays2[:, 0].astype(np.float64)
    y = rays2[:, 1].astype(np.float64)
    prod = np.sin(40 * x) * np.sin(40 * y)
    clear = np.abs(prod) > 1e-3
    assert np.array_equal((h2["prim"] != O.NONE)[clear], (prod > 0)[clear])


# --------------------------------------------------------------------------
# closest-hit = nearest accepted candidate, checked by an FP64 brute force


def _fp64_closest(V, idx, rays):
    o = rays[:, 0:3].astype(np.float64)
    d = rays[:, 4:7].astype(np.float64)
    A = V[idx[:, 0]].astype(np.float64)
    e1 = V[idx[:, 1]].astype(np.float64) - A
    e2 = V[idx[:, 2]].astype(np.float64) - A
    p = np.cross(d[:, None, :], e2[None])
    det = np.einsum("tk,rtk->rt", e1, p)
    s = o[:, None, :] - A[None]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.einsum("rtk,rtk->rt", s, p) / det
        q = np.cross(s, e1[None])
        v = np.einsum("rk,rtk->rt", d, q) / det
        t = np.einsum("tk,rtk->rt", e2, q) / det
    ok = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > rays[:, 3:4]) & (t < rays[:, 7:8])
    tt = np.where(ok, t, np.inf)
    best = tt.argmin(1)
    hit = np.isfinite(tt.min(1))
    srt = np.sort(tt, 1)
    with np.errstate(invalid="ignore"):
        gap = (srt[:, 1] - srt[:, 0]) / np.maximum(1.0, np.abs(srt[:, 0]))
    m = np.minimum(np.minimum(u, v), 1 - u - v)
    edge_tie = np.any((np.abs(m) < 1e-5) & (t > 0), 1)
    return np.where(hit, best, O.NONE).astype(np.uint32), hit, (gap < 1e-5) | edge_tie


def test_closest_hit_matches_fp64_bruteforce():
    rng = np.random.default_rng(13)
    corners = scenes.random_quads(rng, 48, 0.0, 1.0, 0.1, 0.4)
    verts, idx, uvs = scenes._quads_to_tris(corners)
    sc = scenes.Scene("tiny", verts, idx, uvs, np.zeros(len(idx), np.uint32),
                      [scenes.disc_alpha_u8(8, 0.4)])
    rays = scenes.pinhole_rays((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 50, 64, 64)
    ref, hit, tie = _fp64_closest(verts, idx, rays)
    hl, _ = O.trace_list(sc, rays, "default", "closest")
    hb, _ = O.trace_bvh(sc, sc.bvh(), rays, "default", "closest")
    clear = ~tie
    assert clear.sum() > 3500 and hit.sum() > 1000
    assert np.array_equal(hl["prim"][clear], ref[clear])
    assert np.array_equal(hb["prim"][clear], ref[clear])


# --------------------------------------------------------------------------
# BVH traversal == brute force; invariants of the intersector design


@pytest.fixture(scope="module")
def small():
    sc, rays = scenes.small_quads()
    return sc, rays, sc.bvh()


@pytest.mark.parametrize("kind", ["default", "alpha_tex", "proc_alpha"])
def test_bvh_equals_bruteforce_closest(small, kind):
    sc, rays, blob = small
    hb, _ = O.trace_bvh(sc, blob, rays, kind, "closest")
    hl, _ = O.trace_list(sc, rays, kind, "closest")
    for k in ("prim", "t", "u", "v"):
        assert np.array_equal(hb[k], hl[k]), k


@pytest.mark.parametrize("kind", ["default", "alpha_tex", "proc_alpha", "count"])
def test_any_hit_boolean_equals_closest(small, kind):
    sc, rays, blob = small
    hc, _ = O.trace_bvh(sc, blob, rays, kind, "closest")
    ha, _ = O.trace_bvh(sc, blob, rays, kind, "any")
    assert np.array_equal(hc["prim"] != O.NONE, ha["prim"] != O.NONE)
    # an any-hit record is a real accepted candidate: never nearer than the closest
    both = ha["prim"] != O.NONE
    assert np.all(ha["t"][both] >= hc["t"][both])


def test_default_equals_none_and_count(small):
    """Default intersector forwards intersect unchanged (Section 3.1); bvh_costs
    returns the default result (Section 4)."""
    sc, rays, blob = small
    for q in ("closest", "any"):
        hn, sn = O.trace_bvh(sc, blob, rays, "none", q)
        hd, sd = O.trace_bvh(sc, blob, rays, "default", q)
        hc, sc_ = O.trace_bvh(sc, blob, rays, "count", q)
        for k in ("prim", "t", "u", "v"):
            assert np.array_equal(hn[k], hd[k]) and np.array_equal(hd[k], hc[k])
        assert np.array_equal(sd[:, :2], sc_[:, :2])


def test_alpha_extremes(small):
    sc, rays, blob = small
    full = scenes.Scene(sc.name, sc.verts, sc.idx, sc.uvs, sc.geom_id,
                        [scenes.Texture("u8", 256, 256, np.full((256, 256), 255, np.uint8))])
    empty = scenes.Scene(sc.name, sc.verts, sc.idx, sc.uvs, sc.geom_id,
                         [scenes.Texture("u8", 256, 256, np.zeros((256, 256), np.uint8))])
    hd, _ = O.trace_bvh(sc, blob, rays, "default", "closest")
    hf, _ = O.trace_bvh(full, blob, rays, "alpha_tex", "closest", cutoff_u8=128)
    he, _ = O.trace_bvh(empty, blob, rays, "alpha_tex", "closest", cutoff_u8=128)
    for k in ("prim", "t"):
        assert np.array_equal(hd[k], hf[k])
    assert np.all(he["prim"] == O.NONE)


def test_count_structural_enumeration(small):
    """Any-hit with every candidate rejected visits exactly the nodes whose box
    and all ancestor boxes the ray hits: boxes = 1 + 2 * inner nodes reached,
    tris = triangles in reached leaves."""
    sc, rays, blob = small
    empty = scenes.Scene(sc.name, sc.verts, sc.idx, sc.uvs, sc.geom_id,
                         [scenes.Texture("u8", 1, 1, np.zeros((1, 1), np.uint8))])
    sel = rays[::331]
    _, st = O.trace_bvh(empty, blob, sel, "alpha_tex", "any", cutoff_u8=1)
    nn = struct.unpack_from("<I", blob.tobytes(), 16)[0]
    nodes = np.frombuffer(blob.tobytes(), np.uint8, 32 * nn, 64)
    f = nodes.view(np.float32).reshape(nn, 8)
    u = nodes.view(np.uint32).reshape(nn, 8)
    for r, s in zip(sel, st):
        boxes, tris = 1, 0
        todo = [0] if O.intersect_aabb(r, f[0, 0:3], f[0, 4:7], r[7]) else []
        while todo:
            n = todo.pop()
            cnt = u[n, 7] >> 2
            if cnt:
                tris += int(cnt)
                continue
            boxes += 2
            for c in (u[n, 3], u[n, 3] + 1):
                if O.intersect_aabb(r, f[c, 0:3], f[c, 4:7], r[7]):
                    todo.append(int(c))
        assert (int(s[0]), int(s[1])) == (boxes, tris)


def test_edge_near_tie_flagged():
    sc, blob = two_tri_scene()
    _, st = O.trace_bvh(sc, blob, _ray((0.0, -1.0, 0), (0, 0, 1))[None], "default", "closest")
    assert st[0, 3] & O.TIE_EDGE


def test_shadow_ray_origin_is_hit_point():
    prim = np.array([[0.5, 0.25, -1.0, 0.0, 0.0, 0.5, 2.0, np.inf]], np.float32)
    hit = np.array([[0.5, 0.1, 0.2, 0.0]], np.float32)
    hit[0, 3] = np.array([7], np.uint32).view(np.float32)[0]
    miss = np.array([[np.inf, 0, 0, 0]], np.float32)
    miss[0, 3] = np.array([O.NONE], np.uint32).view(np.float32)[0]
    l = np.array([0, 1, 0], np.float32)
    s = O.shadow_rays(np.concatenate([prim, prim]), np.concatenate([hit, miss]), l, 1e-3)
    assert s[0, 0:3].tolist() == [0.5, 0.5, 0.0] and s[0, 4:7].tolist() == [0, 1, 0]
    assert s[0, 3] == np.float32(1e-3) and np.isinf(s[0, 7])
    assert s[1, 7] == -1.0 and s[1, 3] == 0.0


# --------------------------------------------------------------------------
# blob structure


def test_blob_valid_and_leaves_contain_triangles(small):
    sc, _, blob = small
    assert bvh_validate(blob) == ""
    b = blob.tobytes()
    nn, npr = struct.unpack_from("<II", b, 16)
    f = np.frombuffer(b, np.float32, 8 * nn, 64).reshape(nn, 8)
    u = np.frombuffer(b, np.uint32, 8 * nn, 64).reshape(nn, 8)
    order = np.frombuffer(b, np.uint32, npr, 64 + 32 * nn)
    assert np.array_equal(np.sort(order), np.arange(npr))
    tri = sc.verts[sc.idx]  # [T,3,3]
    for n in range(nn):
        cnt = u[n, 7] >> 2
        if n == 1 or cnt == 0:
            continue
        prims = order[u[n, 3]:u[n, 3] + cnt]
        assert np.all(tri[prims].min(1) >= f[n, 0:3]) and np.all(tri[prims].max(1) <= f[n, 4:7])


def test_blob_corruptions_rejected(small):
    _, _, blob = small
    bad = blob.copy()
    bad[0] ^= 1
    assert "magic" in bvh_validate(bad)
    assert bvh_validate(blob[:-4]) != ""
    bad = blob.copy()
    bad[200] ^= 0x40
    assert "checksum" in bvh_validate(bad)
    assert bvh_validate(blob[:10]) != ""


def test_children_must_follow_their_parent():
    """The GPU traversal bounds its descent by the node index, so the
    validator rejects an inner node whose children sit at a lower index; the
    same tree laid out top-down is accepted."""
    def leaf(first):
        return ([-1, -1, 0], first, [1, 1, 3], 1 << 2)

    def inner(left):
        return ([-1, -1, 0], left, [1, 1, 3], 2)   # count 0, split on z

    pad = ([0, 0, 0], 0, [0, 0, 0], 0)
    back = [inner(4), pad, leaf(0), leaf(1), inner(2), leaf(2)]
    down = [inner(2), pad, inner(4), leaf(2), leaf(0), leaf(1)]
    assert "follow their parent" in bvh_validate(make_blob(back, [0, 1, 2], 2))
    assert bvh_validate(make_blob(down, [0, 1, 2], 2)) == ""


def test_empty_and_single_triangle_blobs():
    b0 = bvh_build(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32))
    assert bvh_validate(b0) == ""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    b1 = bvh_build(v, np.array([[0, 1, 2]], np.uint32))
    assert bvh_validate(b1) == ""
    sc = scenes.Scene("one", v, np.array([[0, 1, 2]], np.uint32), np.zeros((1, 3, 2), np.float32),
                      np.zeros(1, np.uint32), [scenes.disc_alpha_u8(4)])
    h, st = O.trace_bvh(sc, b1, _ray((0.25, 0.25, -1), (0, 0, 1))[None], "count", "closest")
    assert h["prim"][0] == 0 and h["t"][0] == 1.0 and tuple(st[0, :2]) == (1, 1)
    e = scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32),
                     np.zeros((0, 3, 2), np.float32), np.zeros(0, np.uint32), [])
    h, st = O.trace_bvh(e, b0, _ray((0, 0, 0), (0, 0, 1))[None], "count", "closest")
    assert h["prim"][0] == O.NONE and tuple(st[0, :2]) == (0, 0)


def test_ao_rays_cosine_sampling_about_the_face_normal():
    """Ambient-occlusion rays (4 per pixel): each leaves from the primary hit
    point (within 1e-5 of o + t d in FP64), along a
    unit vector on the side of the face that the primary ray came from; its
    cosine to that normal is sqrt(1 - xi1) (cosine-weighted sampling), and two
    samples of one pixel are turned about the normal by 2 pi (xi2' - xi2) in a
    right-handed tangent frame.  A miss gives inactive rays (tmax < tmin)."""
    rng = np.random.default_rng(21)
    m, spp = 1500, 4
    tri = rng.uniform(-1, 1, (m, 3, 3)).astype(np.float32)
    sc = scenes.Scene("tris", tri.reshape(-1, 3), np.arange(3 * m, dtype=np.uint32).reshape(m, 3),
                      np.zeros((m, 3, 2), np.float32), np.full(m, O.NONE, np.uint32), [])
    rays = np.zeros((m, 8), np.float32)
    rays[:, 0:3] = rng.uniform(-3, 3, (m, 3))
    d = rng.standard_normal((m, 3))
    rays[:, 4:7] = d / np.linalg.norm(d, axis=1, keepdims=True)
    rays[:, 7] = np.inf
    hits = np.zeros((m, 4), np.float32)
    hits[:, 0] = rng.uniform(0.1, 5, m)
    prim = np.arange(m, dtype=np.uint32)
    prim[::7] = O.NONE
    hits[:, 3] = prim.view(np.float32)
    xi = rng.uniform(0, 1, (m * spp, 2)).astype(np.float32)
    out = O.ao_rays(sc, rays, hits, spp, xi, 0.5, 1e-3).reshape(m, spp, 8)
    miss = prim == O.NONE
    assert np.all(out[miss][..., 7] < out[miss][..., 3])
    h = ~miss
    o, dd = rays[h, 0:3].astype(np.float64), rays[h, 4:7].astype(np.float64)
    t = hits[h, 0].astype(np.float64)
    q = out[h]
    want_o = np.broadcast_to((o + t[:, None] * dd)[:, None, :], q[:, :, 0:3].shape)
    np.testing.assert_allclose(q[:, :, 0:3], want_o, rtol=0, atol=1e-5)
    assert np.all(q[:, :, 3] == np.float32(1e-3)) and np.all(q[:, :, 7] == np.float32(0.5))
    tr = tri[h].astype(np.float64)
    n = np.cross(tr[:, 1] - tr[:, 0], tr[:, 2] - tr[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[np.einsum("ij,ij->i", n, dd) > 0] *= -1
    w = q[:, :, 4:7].astype(np.float64)
    assert np.allclose(np.linalg.norm(w, axis=2), 1.0, atol=1e-6)
    x = xi.reshape(m, spp, 2)[h].astype(np.float64)
    cos = np.einsum("ikj,ij->ik", w, n)
    np.testing.assert_allclose(cos, np.sqrt(1 - x[:, :, 0]), rtol=0, atol=2e-6)
    p = w - cos[:, :, None] * n[:, None, :]
    sin_ok = np.sqrt(x[:, 0, 0]) > 1e-2
    for k in range(1, spp):
        ok = sin_ok & (np.sqrt(x[:, k, 0]) > 1e-2)
        a, b = p[ok, 0], p[ok, k]
        ang = np.arctan2(np.einsum("ij,ij->i", np.cross(a, b), n[ok]), np.einsum("ij,ij->i", a, b))
        want = 2 * np.pi * (x[ok, k, 1] - x[ok, 0, 1])
        diff = np.angle(np.exp(1j * (ang - want)))
        assert np.abs(diff).max() < 1e-3, np.abs(diff).max()
