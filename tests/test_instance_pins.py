"""Pins of the oracle's instanced queries (no GPU).

Instancing (Section 3.2): BVHs act as primitives of a list or of a top-level
BVH, and the intersector is passed on to each BVH's own traversal.  Pinned
by: one unmoved instance is the mesh itself; a signed axis permutation is
exact in float32, so the instance equals the mesh traced with the permuted
rays; the linear list equals the top-level BVH for closest-hit (the answer
does not depend on the order); any-hit finds a hit exactly when closest-hit
does; an FP64 brute force over all instances agrees away from near ties; ties
between coincident instances go to the lower id.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes
from test_oracle_pins import two_tri_scene

KINDS = ["none", "default", "alpha_tex", "proc_alpha", "count"]


@pytest.fixture(scope="module")
def small():
    sc, rays = scenes.small_quads()
    return sc, rays, sc.bvh()


@pytest.fixture(scope="module")
def inst():
    return scenes.instanced_small()


def _trace(I, rays, kind="default", query="closest", top=True, **kw):
    return O.trace_instances(list(zip(I.meshes, I.blobs)), I.inst_mesh, I.w2o, rays, kind, query,
                             I.top if top else None, **kw)


def _eq(a, b, label=""):
    for k in ("prim", "t", "u", "v"):
        assert np.array_equal(a[k].view(np.uint32), b[k].view(np.uint32)), (label, k)


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", KINDS)
def test_one_unmoved_instance_is_the_mesh(small, kind, query):
    sc, rays, blob = small
    I = scenes.make_instance_set("one", [sc], [0], [np.hstack([np.eye(3), np.zeros((3, 1))])])
    h, ids, st = _trace(I, rays, kind, query)
    hm, sm = O.trace_bvh(sc, blob, rays, kind, query)
    _eq(h, hm, kind)
    hit = hm["prim"] != O.NONE
    assert np.all(ids[hit] == 0) and np.all(ids[~hit] == O.NONE)
    extra = st[:, 0].astype(np.int64) - sm[:, 0]
    assert np.all((extra == 0) | (extra == 1)) and np.array_equal(st[:, 1], sm[:, 1])


def test_signed_axis_permutation_is_exact(small):
    """W = a signed permutation: the object-space ray is (P o, P d) exactly,
    so the instance answers as the mesh does for the permuted rays."""
    sc, rays, blob = small
    P = np.array([[0, 0, -1], [1, 0, 0], [0, -1, 0]], np.float64)  # world -> object
    o2w = np.hstack([P.T, np.zeros((3, 1))])
    I = scenes.make_instance_set("perm", [sc], [0], [o2w])
    assert np.array_equal(I.w2o[0].reshape(3, 4)[:, :3], P.astype(np.float32))
    world = rays.copy()
    world[:, 0:3] = rays[:, 0:3] @ P  # P^T o: object origin o maps to world P^T o
    world[:, 4:7] = rays[:, 4:7] @ P
    for kind in ("default", "alpha_tex"):
        h, ids, _ = _trace(I, world, kind)
        hm, _ = O.trace_bvh(sc, blob, rays, kind, "closest")
        _eq(h, hm, kind)


@pytest.mark.parametrize("kind", ["default", "alpha_tex", "proc_alpha"])
def test_list_equals_top_level_bvh(inst, kind):
    I, rays = inst
    h, ids, _ = _trace(I, rays, kind)
    hl, idl, _ = _trace(I, rays, kind, top=False)
    _eq(h, hl, kind)
    assert np.array_equal(ids, idl)
    assert len(np.unique(ids[ids != O.NONE])) >= 4  # several instances are visible


@pytest.mark.parametrize("kind", KINDS)
def test_any_hit_boolean_equals_closest(inst, kind):
    I, rays = inst
    hc, _, _ = _trace(I, rays, kind)
    ha, ida, _ = _trace(I, rays, kind, "any")
    assert np.array_equal(hc["prim"] != O.NONE, ha["prim"] != O.NONE)
    assert np.all(ha["t"] >= hc["t"])


def test_fp64_bruteforce(inst):
    """Closest hit over every triangle of every instance in float64 (rays
    mapped by the float64 inverse of the placement)."""
    I, rays = inst
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(len(rays), 3000, replace=False))
    h, ids, st = _trace(I, rays[sel], "default")
    best_t = np.full(len(sel), np.inf)
    best = np.full((len(sel), 2), -1, np.int64)
    o = rays[sel, 0:3].astype(np.float64)
    d = rays[sel, 4:7].astype(np.float64)
    for i, (m, a) in enumerate(zip(I.inst_mesh, I.o2w)):
        inv = np.linalg.inv(np.vstack([a, [0, 0, 0, 1]]))[:3]
        oo = o @ inv[:, :3].T + inv[:, 3]
        dd = d @ inv[:, :3].T
        sc = I.meshes[m]
        tri = sc.verts[sc.idx].astype(np.float64)
        v0, e1, e2 = tri[:, 0], tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]
        for r in range(len(sel)):
            p = np.cross(dd[r], e2)
            det = np.einsum("ij,ij->i", e1, p)
            with np.errstate(divide="ignore", invalid="ignore"):
                s = oo[r] - v0
                u = np.einsum("ij,ij->i", s, p) / det
                q = np.cross(s, e1)
                v = (q @ dd[r]) / det
                t = np.einsum("ij,ij->i", e2, q) / det
            ok = (det != 0) & (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
            if ok.any():
                k = np.argmin(np.where(ok, t, np.inf))
                if t[k] < best_t[r]:
                    best_t[r], best[r] = t[k], (i, k)
    hit = np.isfinite(best_t)
    near = st[:, 3] != 0
    assert np.array_equal(h["prim"] != O.NONE, hit | (near & (h["prim"] != O.NONE)))
    agree = hit & ~near
    assert np.array_equal(ids[agree], best[agree, 0].astype(np.uint32))
    assert np.array_equal(h["prim"][agree], best[agree, 1].astype(np.uint32))
    np.testing.assert_allclose(h["t"][agree], best_t[agree], rtol=1e-5)
    assert agree.sum() > 1000


def test_coincident_instances_tie_to_the_lower_id():
    sc, blob = two_tri_scene()
    ident = np.hstack([np.eye(3), np.zeros((3, 1))])
    moved = np.hstack([np.eye(3), np.array([[10.0], [0.0], [0.0]])])
    I = scenes.make_instance_set("two", [sc], [0, 0, 0], [moved, ident, ident])
    rays = np.array([[0, 0, 0, 0, 0, 0, 1, np.inf], [10, 0, 0, 0, 0, 0, 1, np.inf],
                     [0, 0, 4, 0, 0, 0, -1, np.inf]], np.float32)
    for top in (True, False):
        h, ids, _ = _trace(I, rays, "default", top=top)
        assert list(ids) == [1, 0, 1]
        assert list(h["prim"]) == [0, 0, 1] and list(h["t"]) == [1.0, 1.0, 1.0]
