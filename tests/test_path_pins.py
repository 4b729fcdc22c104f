"""Pins of the oracle's path tracer (no GPU).

A diffuse path tracer on the closest-hit query with the intersector: a
miss returns throughput x sky, a hit multiplies the throughput by the
albedo and bounces along a given local direction in the face's tangent
frame, and a path whose bounces are spent returns 0.  Pinned by closed forms
(zero bounces: sky for a miss, 0 for a hit; a lit plane seen from above
returns albedo x sky exactly; a closed box returns 0), by the local direction
(0, 0, 1), which must leave along the face normal, and by the alpha mask of
all 255, which must equal the default intersector.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

SKY = np.array([0.7, 0.8, 1.0], np.float32)


def _plane(z=0.0, size=4.0):
    c = np.array([[[-size, -size, z], [size, -size, z], [size, size, z], [-size, size, z]]])
    v, i, uv = scenes._quads_to_tris(c)
    return scenes.Scene("plane", v, i, uv, np.full(2, O.NONE, np.uint32), [])


def _down_rays(n, rng, z=2.0):
    r = np.zeros((n, 8), np.float32)
    r[:, 0:2] = rng.uniform(-1, 1, (n, 2))
    r[:, 2] = z
    d = np.stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n), -np.ones(n)], 1)
    r[:, 4:7] = d / np.linalg.norm(d, axis=1, keepdims=True)
    r[:, 7] = np.inf
    return r


def test_zero_bounces_is_sky_or_black():
    sc, rays = scenes.small_quads()
    blob = sc.bvh()
    rad, _ = O.path_trace(sc, blob, rays, 0, np.zeros((0, 3)), 1e-4, SKY)
    h, _ = O.trace_bvh(sc, blob, rays, "default", "closest")
    miss = h["prim"] == O.NONE
    assert np.array_equal(rad[miss], np.tile(SKY, (miss.sum(), 1)))
    assert np.all(rad[~miss] == 0)


@pytest.mark.parametrize("bounces", [1, 3])
def test_plane_from_above_is_albedo_times_sky(bounces):
    sc = _plane()
    rng = np.random.default_rng(4)
    rays = _down_rays(500, rng)
    dirs = scenes.path_dirs(len(rays), bounces, seed=9)
    untex = np.array([0.5, 0.25, 0.8], np.float32)
    rad, _ = O.path_trace(sc, sc.bvh(), rays, bounces, dirs, 1e-4, SKY, untex)
    assert np.array_equal(rad, np.tile(untex * SKY, (len(rays), 1)))


def test_straight_up_bounce_leaves_along_the_normal():
    """Local direction (0, 0, 1) is the turned face normal: from a plane at
    z = 0 seen from above the bounce goes straight up and escapes, even with
    a second plane beside the path; with the plane above it instead, the
    bounce hits it and the path ends black after one bounce."""
    lower = _plane(0.0)
    rng = np.random.default_rng(5)
    rays = _down_rays(200, rng)
    up = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (len(rays), 1))
    rad, _ = O.path_trace(lower, lower.bvh(), rays, 1, up, 1e-4, SKY)
    assert np.allclose(rad, 0.8 * SKY)
    c = np.array([[[-4, -4, 0], [4, -4, 0], [4, 4, 0], [-4, 4, 0]],
                  [[-4, -4, 5], [4, -4, 5], [4, 4, 5], [-4, 4, 5]]], np.float64)
    v, i, uv = scenes._quads_to_tris(c)
    two = scenes.Scene("two", v, i, uv, np.full(4, O.NONE, np.uint32), [])
    rays[:, 2] = 2.0
    rad, _ = O.path_trace(two, two.bvh(), rays, 1, up, 1e-4, SKY)
    assert np.all(rad == 0)


def test_closed_box_is_black():
    lo, hi = -1.0, 1.0
    faces = np.array([[[lo, lo, lo], [hi, lo, lo], [hi, hi, lo], [lo, hi, lo]],
                      [[lo, lo, hi], [hi, lo, hi], [hi, hi, hi], [lo, hi, hi]],
                      [[lo, lo, lo], [hi, lo, lo], [hi, lo, hi], [lo, lo, hi]],
                      [[lo, hi, lo], [hi, hi, lo], [hi, hi, hi], [lo, hi, hi]],
                      [[lo, lo, lo], [lo, hi, lo], [lo, hi, hi], [lo, lo, hi]],
                      [[hi, lo, lo], [hi, hi, lo], [hi, hi, hi], [hi, lo, hi]]], np.float64)
    v, i, uv = scenes._quads_to_tris(faces)
    box = scenes.Scene("box", v, i, uv, np.full(12, O.NONE, np.uint32), [])
    rng = np.random.default_rng(6)
    rays = np.zeros((300, 8), np.float32)
    d = rng.standard_normal((300, 3))
    rays[:, 4:7] = d / np.linalg.norm(d, axis=1, keepdims=True)
    rays[:, 7] = np.inf
    for bounces in (0, 2, 5):
        rad, _ = O.path_trace(box, box.bvh(), rays, bounces, scenes.path_dirs(300, bounces),
                              1e-4, SKY)
        assert np.all(rad == 0)


def test_alpha_255_is_default():
    sc, rays = scenes.small_quads()
    blob = sc.bvh()
    full = scenes.Scene(sc.name, sc.verts, sc.idx, sc.uvs, sc.geom_id,
                        [scenes.Texture("u8", 256, 256, np.full((256, 256), 255, np.uint8))])
    dirs = scenes.path_dirs(len(rays), 3)
    a, fa = O.path_trace(sc, blob, rays, 3, dirs, 1e-4, SKY, kind="default")
    b, fb = O.path_trace(full, blob, rays, 3, dirs, 1e-4, SKY, kind="alpha_tex")
    assert np.array_equal(a, b)
    assert (a.sum(1) > 0).mean() > 0.2  # many paths escape to the sky


def test_bounce_frame_against_fp64():
    """On random triangles and rays, the bounce leaves from fmaf(t, d, o), its
    direction agrees within 1e-6 with the same construction in float64 (face
    normal turned against d, Duff et al. frame, l.x t1 + l.y t2 + l.z n), is
    a unit vector to float32 accuracy and lies in the turned normal's
    hemisphere; the frame is orthonormal."""
    rng = np.random.default_rng(12)
    m = 4000
    tri = rng.uniform(-1, 1, (m, 3, 3)).astype(np.float32)
    verts = tri.reshape(-1, 3)
    idx = np.arange(3 * m, dtype=np.uint32).reshape(m, 3)
    sc = scenes.Scene("tris", verts, idx, np.zeros((m, 3, 2), np.float32),
                      np.full(m, O.NONE, np.uint32), [])
    rays = np.zeros((m, 8), np.float32)
    rays[:, 0:3] = rng.uniform(-3, 3, (m, 3))
    d = rng.standard_normal((m, 3))
    rays[:, 4:7] = d / np.linalg.norm(d, axis=1, keepdims=True)
    rays[:, 7] = np.inf
    hits = np.zeros((m, 4), np.float32)
    hits[:, 0] = rng.uniform(0.1, 5, m)
    hits[:, 3] = np.arange(m, dtype=np.uint32).view(np.float32)
    loc = scenes.path_dirs(m, 1, seed=13)
    out = O.bounce(sc, rays, hits, loc, 1e-3)
    t = hits[:, 0].astype(np.float64)
    o, dd = rays[:, 0:3].astype(np.float64), rays[:, 4:7].astype(np.float64)
    np.testing.assert_allclose(out[:, 0:3], o + t[:, None] * dd, rtol=0, atol=1e-5)
    assert np.all(out[:, 3] == np.float32(1e-3)) and np.all(np.isinf(out[:, 7]))
    e1 = tri[:, 1].astype(np.float64) - tri[:, 0]
    e2 = tri[:, 2].astype(np.float64) - tri[:, 0]
    n = np.cross(e1, e2)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    n[np.einsum("ij,ij->i", n, dd) > 0] *= -1
    s = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (s + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    t1 = np.stack([1 + s * n[:, 0] ** 2 * a, s * b, -s * n[:, 0]], 1)
    t2 = np.stack([b, s + n[:, 1] ** 2 * a, -n[:, 1]], 1)
    frame = np.stack([t1, t2, n], 1)
    assert np.allclose(np.einsum("kij,kmj->kim", frame, frame), np.eye(3), atol=1e-12)
    l = loc.astype(np.float64)
    want = l[:, 0:1] * t1 + l[:, 1:2] * t2 + l[:, 2:3] * n
    np.testing.assert_allclose(out[:, 4:7], want, rtol=0, atol=1e-6)
    assert np.allclose(np.linalg.norm(out[:, 4:7], axis=1), 1.0, atol=1e-6)
    assert np.all(np.einsum("ij,ij->i", out[:, 4:7], n) >= -1e-7)
