"""Pins of the oracle's multi-hit query (no GPU).

The multi-hit query returns the first N accepted hits of a ray in ascending
(t, prim) order, the order closest-hit uses to break ties, with miss records
after them.  The answer does not depend on the traversal order, so the BVH
traversal (an N-entry buffer whose last entry bounds the search) is pinned
exactly by the plain definition over the list (every candidate tested,
accepted ones sorted, first N kept), by the closest-hit query at N = 1, by
hand-traced cases on a two-leaf BVH and by a stack of parallel planes at
known depths.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes
from test_oracle_pins import _ray, two_tri_scene


@pytest.fixture(scope="module")
def small():
    sc, rays = scenes.small_quads()
    return sc, rays, sc.bvh()


def _eq(a, b, label=""):
    for k in ("prim", "t", "u", "v"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), (label, k)


@pytest.mark.parametrize("kind", ["none", "default", "alpha_tex", "proc_alpha", "count"])
def test_one_hit_is_the_closest_hit(small, kind):
    sc, rays, blob = small
    hm, sm = O.trace_multi(sc, rays, 1, kind, blob)
    hc, scl = O.trace_bvh(sc, blob, rays, kind, "closest")
    _eq({k: v[:, 0] for k, v in hm.items()}, hc, kind)
    assert np.array_equal(sm, scl)


@pytest.mark.parametrize("nh", [2, 5, 16])
@pytest.mark.parametrize("kind", ["default", "alpha_tex", "proc_alpha"])
def test_bvh_equals_sorted_bruteforce(small, kind, nh):
    sc, rays, blob = small
    sel = rays[::5]
    hb, _ = O.trace_multi(sc, sel, nh, kind, blob)
    hl, _ = O.trace_multi(sc, sel, nh, kind)
    _eq(hb, hl, f"{kind} nh={nh}")
    assert (hl["prim"] != O.NONE).sum(1).max() >= 2  # the scene has depth


def test_invariants(small):
    sc, rays, blob = small
    h16, _ = O.trace_multi(sc, rays, 16, "alpha_tex", blob)
    h4, _ = O.trace_multi(sc, rays, 4, "alpha_tex", blob)
    hc, _ = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest")
    hit = h16["prim"] != O.NONE
    # hits first, misses after; ascending (t, prim); no primitive twice
    assert np.all(hit[:, :-1] >= hit[:, 1:])
    t, p = h16["t"], h16["prim"].astype(np.int64)
    both = hit[:, 1:]
    later = (t[:, 1:] > t[:, :-1]) | ((t[:, 1:] == t[:, :-1]) & (p[:, 1:] > p[:, :-1]))
    assert np.all(later[both])
    for row in range(0, len(rays), 97):
        q = p[row][hit[row]]
        assert len(np.unique(q)) == len(q)
    assert np.all(np.isinf(t[~hit]) & (h16["u"][~hit] == 0) & (h16["v"][~hit] == 0))
    # shorter buffers are prefixes; the first entry is the closest hit
    _eq({k: v[:, :4] for k, v in h16.items()}, h4, "prefix")
    _eq({k: v[:, 0] for k, v in h16.items()}, hc, "first")
    # an all-255 alpha mask is the default intersector; all-0 accepts nothing
    full = scenes.Scene(sc.name, sc.verts, sc.idx, sc.uvs, sc.geom_id,
                        [scenes.Texture("u8", 256, 256, np.full((256, 256), 255, np.uint8))])
    empty = scenes.Scene(sc.name, sc.verts, sc.idx, sc.uvs, sc.geom_id,
                         [scenes.Texture("u8", 256, 256, np.zeros((256, 256), np.uint8))])
    hd, _ = O.trace_multi(sc, rays, 8, "default", blob)
    hf, _ = O.trace_multi(full, rays, 8, "alpha_tex", blob)
    he, _ = O.trace_multi(empty, rays, 8, "alpha_tex", blob)
    _eq(hd, hf, "alpha 255")
    assert np.all(he["prim"] == O.NONE)


@pytest.mark.parametrize("case", [
    # (origin, direction, nh, prims, ts, boxes, tris)
    ((0, 0, 0), (0, 0, 1), 2, [0, 1], [1.0, 3.0], 3, 2),
    ((0, 0, 4), (0, 0, -1), 2, [1, 0], [1.0, 3.0], 3, 2),
    ((0, 0, 0), (0, 0, 1), 3, [0, 1, O.NONE], [1.0, 3.0, np.inf], 3, 2),
    ((0, 0, 2), (0, 0, 1), 2, [1, O.NONE], [1.0, np.inf], 3, 1),
    ((5, 5, 0), (0, 0, 1), 2, [O.NONE, O.NONE], [np.inf, np.inf], 1, 0),
])
def test_hand_traced_two_leaves(case):
    """Two triangles at z = 1 and z = 3 in two leaves under one root: along
    +z both are reported nearest first; from z = 4 along -z the order flips;
    spare entries are misses; counts follow the traversal by hand."""
    o, d, nh, prims, ts, boxes, tris = case
    sc, blob = two_tri_scene()
    h, st = O.trace_multi(sc, _ray(o, d)[None], nh, "count", blob, nthreads=1)
    assert list(h["prim"][0]) == [np.uint32(x) for x in prims]
    assert list(h["t"][0]) == ts
    assert (int(st[0, 0]), int(st[0, 1])) == (boxes, tris)


def test_plane_stack_depths():
    """Five unit squares at z = 1..5 (two triangles each) seen along +z from
    z = 0: every ray reports the five depths in order, one triangle per
    square, then misses; with the alpha intersector the square whose mask is
    all zero drops out and the others move up."""
    quads = [np.array([[0, 0, z], [1, 0, z], [1, 1, z], [0, 1, z]], np.float32)
             for z in range(1, 6)]
    verts = np.concatenate(quads)
    idx = np.concatenate([np.array([[0, 1, 2], [0, 2, 3]], np.uint32) + 4 * k for k in range(5)])
    uvs = np.tile(np.array([[[0, 0], [1, 0], [1, 1]], [[0, 0], [1, 1], [0, 1]]], np.float32),
                  (5, 1, 1))
    geom = np.full(10, O.NONE, np.uint32)
    geom[4:6] = 0  # the square at z = 3
    sc = scenes.Scene("stack", verts, idx, uvs, geom,
                      [scenes.Texture("u8", 4, 4, np.zeros((4, 4), np.uint8))])
    rng = np.random.default_rng(3)
    xy = rng.uniform(0.02, 0.98, (256, 2))
    xy = xy[np.abs(xy[:, 0] - xy[:, 1]) > 1e-3]  # off the shared diagonal
    rays = np.zeros((len(xy), 8), np.float32)
    rays[:, 0:2] = xy
    rays[:, 6] = 1.0
    rays[:, 7] = np.inf
    blob = sc.bvh()
    for kind, depths in (("default", [1, 2, 3, 4, 5]), ("alpha_tex", [1, 2, 4, 5])):
        h, _ = O.trace_multi(sc, rays, 8, kind, blob)
        m = len(depths)
        np.testing.assert_allclose(h["t"][:, :m], np.tile(depths, (len(rays), 1)), rtol=1e-6)
        assert np.all(h["prim"][:, m:] == O.NONE)
        assert np.array_equal(h["prim"][:, :m] // 2, np.tile(np.array(depths) - 1, (len(rays), 1)))
        hl, _ = O.trace_multi(sc, rays, 8, kind)
        _eq(h, hl, kind)
