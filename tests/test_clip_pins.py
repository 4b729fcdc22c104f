"""Pins of the oracle's clip-box intersector (no GPU).

The clip box intercepts both calls to intersect (Section 3.2): a node box
that does not overlap the clip box counts as missed, and a candidate is
accepted iff its hit point fmaf(t, d, o) lies in the closed box.  The answer
is the nearest hit inside the box, whatever the culling, so the BVH traversal
(which culls) is pinned by the brute force (which never does) and by the
unclipped hit list filtered by position; a box around everything reduces to
the default intersector and culls nothing; a box off the scene culls at the
root.  Rays whose hit point lies within 1e-6 of a clip face are near ties.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

BOXES = [((0.2, 0.1, 0.0), (0.7, 0.6, 1.0)), ((-1.0, 0.4, 0.35), (2.0, 2.0, 0.6)),
         ((0.45, -1.0, -1.0), (2.0, 2.0, 2.0))]


@pytest.fixture(scope="module")
def small():
    sc, rays = scenes.small_quads()
    return sc, rays, sc.bvh()


def _eq(a, b, ok, label=""):
    for k in ("prim", "t", "u", "v"):
        assert np.array_equal(a[k].view(np.uint32)[ok], b[k].view(np.uint32)[ok]), (label, k)


@pytest.mark.parametrize("box", BOXES)
def test_culling_traversal_equals_bruteforce(small, box):
    sc, rays, blob = small
    kw = dict(clip_lo=box[0], clip_hi=box[1])
    hb, sb = O.trace_bvh(sc, blob, rays, "clip", "closest", **kw)
    hl, sl = O.trace_list(sc, rays, "clip", "closest", **kw)
    ok = (sb[:, 3] == 0) & (sl[:, 3] == 0)
    _eq(hb, hl, ok, str(box))
    assert ok.mean() > 0.99 and (hb["prim"] != O.NONE).sum() > 1000
    # culling only removes work
    hd, sd = O.trace_bvh(sc, blob, rays, "default", "closest")
    assert sb[:, 0].sum() < sd[:, 0].sum()
    mb, _ = O.trace_multi(sc, rays[::7], 6, "clip", blob, **kw)
    ml, _ = O.trace_multi(sc, rays[::7], 6, "clip", None, **kw)
    _eq(mb, ml, np.ones(len(mb["prim"]), bool), "multi")


def test_nearest_hit_inside_the_box(small):
    """From the sorted list of every accepted default hit, the first whose
    hit point lies in the box is the clip intersector's answer."""
    sc, rays, blob = small
    lo, hi = np.array(BOXES[0][0]), np.array(BOXES[0][1])
    sel = rays[::3]
    hc, sc_ = O.trace_bvh(sc, blob, sel, "clip", "closest", clip_lo=lo, clip_hi=hi)
    hm, _ = O.trace_multi(sc, sel, 16, "default")
    o, d = sel[:, None, 0:3].astype(np.float64), sel[:, None, 4:7].astype(np.float64)
    p = o + hm["t"][:, :, None].astype(np.float64) * d
    inside = np.all((p >= lo) & (p <= hi), axis=2) & (hm["prim"] != O.NONE)
    full = hm["prim"][:, -1] != O.NONE
    first = np.where(inside.any(1), inside.argmax(1), -1)
    decided = ((first >= 0) | ~full) & (sc_[:, 3] == 0)
    want = np.where(first >= 0, hm["prim"][np.arange(len(sel)), np.maximum(first, 0)], O.NONE)
    assert np.array_equal(hc["prim"][decided], want[decided].astype(np.uint32))
    assert decided.mean() > 0.99


def test_box_around_everything_is_default(small):
    sc, rays, blob = small
    for q in ("closest", "any"):
        hc, stc = O.trace_bvh(sc, blob, rays, "clip", q, clip_lo=(-10, -10, -10),
                              clip_hi=(10, 10, 10))
        hd, std = O.trace_bvh(sc, blob, rays, "default", q)
        _eq(hc, hd, np.ones(len(rays), bool), q)
        assert np.array_equal(stc[:, :2], std[:, :2])


def test_box_off_the_scene_culls_at_the_root(small):
    sc, rays, blob = small
    h, st = O.trace_bvh(sc, blob, rays, "clip", "closest", clip_lo=(5, 5, 5), clip_hi=(6, 6, 6))
    assert np.all(h["prim"] == O.NONE) and np.all(st[:, 0] == 1) and np.all(st[:, 1] == 0)
