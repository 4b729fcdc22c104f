"""Pins of the FP64 shading reference (oracle/adjoint.py), no GPU.

The reference gradient is autograd of a plainly written FP64 forward; these
tests tie that forward and its gradient to values worked out by hand and to
central finite differences of the loss (h = 1e-3).
"""
import math

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes


def _tri_scene(v2=(0, 1, 0), v1=(1, 0, 0), tex=None):
    verts = np.array([[0, 0, 0], v1, v2], np.float32)
    idx = np.array([[0, 1, 2]], np.uint32)
    uvs = np.array([[[0, 0], [1, 0], [0, 1]]], np.float32)
    if tex is None:
        tex = np.zeros((1, 1, 4), np.float32)
        tex[0, 0] = (0.2, 0.5, 0.8, 1.0)
    return scenes.Scene("tri", verts, idx, uvs, np.zeros(1, np.uint32),
                        [scenes.Texture("rgba32f", tex.shape[1], tex.shape[0], tex)])


def _ortho(points):
    r = np.zeros((len(points), 8), np.float32)
    r[:, 0:2] = points
    r[:, 2] = -1
    r[:, 6] = 1
    r[:, 7] = np.inf
    return r


def test_normal_path_closed_form():
    """Tilting v2 out of the plane: n_f = (0, z2, -1)/sqrt(1 + z2^2), so with
    L = (0, 0.6, -0.8) the shading factor is (0.6 z2 + 0.8)/sqrt(1 + z2^2),
    whose slope at z2 = 0 is 0.6; barycentrics are unchanged.  With target 0,
    dL/dz2 = N * 2 * 0.8 * 0.6 * |a|^2 and dL/dT = N * 2 * 0.8^2 * a."""
    sc = _tri_scene()
    pts = np.array([[0.1, 0.1], [0.3, 0.2], [0.05, 0.6], [0.4, 0.4]], np.float32)
    rays = _ortho(pts)
    prims = np.zeros(len(pts), np.uint32)
    fs = A.FrozenShading(sc, rays, prims, light=(0.0, 0.6, -0.8))
    a = sc.textures[0].texels[0, 0, :3].astype(np.float64)
    img = fs.image(A._t(sc.verts), A._t(sc.textures[0].texels)).numpy()
    np.testing.assert_allclose(img, np.tile(0.8 * a, (4, 1)), rtol=1e-12)
    L, gv, gt, _ = fs.loss_grad(sc.verts, sc.textures[0].texels, np.zeros((4, 3)))
    n = len(pts)
    assert math.isclose(gv[2, 2], n * 2 * 0.8 * 0.6 * float(a @ a), rel_tol=1e-9)
    np.testing.assert_allclose(gt[0, 0, :3], n * 2 * 0.8 * 0.8 * a, rtol=1e-9)
    assert gt[0, 0, 3] == 0.0


def test_texcoord_path_closed_form():
    """Stretching v1 = (A, 0, 0): u = x / A, the 2x1 texture gives
    albedo = (1 - fx) T0 + fx T1 with fx = 2u - 0.5, so
    dL/dA = 2 * albedo . (2 (T1 - T0)) * (-x / A^2) for one pixel, L = (0,0,-1)."""
    tex = np.zeros((1, 2, 4), np.float32)
    tex[0, 0] = (0.1, 0.2, 0.3, 1)
    tex[0, 1] = (0.9, 0.4, 0.0, 1)
    sc = _tri_scene(tex=tex)
    x, y = 0.4, 0.1
    rays = _ortho(np.array([[x, y]], np.float32))
    fs = A.FrozenShading(sc, rays, np.zeros(1, np.uint32), light=(0.0, 0.0, -1.0))
    T0, T1 = tex[0, 0, :3].astype(np.float64), tex[0, 1, :3].astype(np.float64)
    fx = 2 * x - 0.5
    alb = (1 - fx) * T0 + fx * T1
    img = fs.image(A._t(sc.verts), A._t(tex)).numpy()[0]
    np.testing.assert_allclose(img, alb, rtol=1e-7)
    _, gv, gt, _ = fs.loss_grad(sc.verts, tex, np.zeros((1, 3)))
    want = 2 * float(alb @ (2 * (T1 - T0))) * (-x / 1.0)
    assert math.isclose(gv[1, 0], want, rel_tol=1e-6)
    np.testing.assert_allclose(gt[0, 0, :3], 2 * alb * (1 - fx), rtol=1e-6)
    np.testing.assert_allclose(gt[0, 1, :3], 2 * alb * fx, rtol=1e-6)


def test_miss_pixels_are_background_and_carry_no_gradient():
    sc = _tri_scene()
    rays = _ortho(np.array([[0.9, 0.9], [0.1, 0.1]], np.float32))
    prims = np.array([O.NONE, 0], np.uint32)
    fs = A.FrozenShading(sc, rays, prims, light=(0, 0, -1), background=(0.3, 0.3, 0.3))
    img = fs.image(A._t(sc.verts), A._t(sc.textures[0].texels)).numpy()
    assert img[0].tolist() == [0.3, 0.3, 0.3]


@pytest.fixture(scope="module")
def small_sphere():
    sc, rays, tv, tt = scenes.displaced_icosphere(freq=12, res=96, tex_size=64)
    blob = sc.bvh()
    h, _ = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest", cutoff_f=0.3)
    light = scenes.light_dir_f32().astype(np.float64)
    fs = A.FrozenShading(sc, rays, h["prim"], light)
    # target rendered from the perturbed parameters at the same visibility
    target = fs.image(A._t(tv), A._t(tt)).numpy()
    return sc, rays, fs, target


def test_gradient_matches_central_differences(small_sphere):
    sc, rays, fs, target = small_sphere
    verts, tex = sc.verts, sc.textures[0].texels
    _, gv, gt, _ = fs.loss_grad(verts, tex, target)
    rng = np.random.default_rng(3)
    used = np.unique(fs.idx)
    ks = rng.choice(used, 120, replace=False)
    # central differences converge as h^2: 1e-3 relative at h = 1e-3 (the
    # gradient tolerance), and 100x tighter at h = 1e-4
    for h, tol in ((1e-3, 1e-3), (1e-4, 2e-5)):
        ref, fd = [], []
        for k in ks:
            for ax in range(3):
                val, kink = fs.fd_vertex(verts, tex, target, int(k), ax, h=h)
                if kink:  # stencil crosses a bilinear cell or shading kink
                    continue
                fd.append(val)
                ref.append(gv[k, ax])
        ref, fd = np.array(ref), np.array(fd)
        assert len(ref) > 200
        assert np.linalg.norm(fd - ref) <= tol * np.linalg.norm(ref), h
    # texels: the loss is quadratic in them, so central differences are exact
    tj = rng.integers(0, tex.shape[0], 300)
    ti = rng.integers(0, tex.shape[1], 300)
    tc = rng.integers(0, 3, 300)
    fdt = np.array([fs.fd_texel(verts, tex, target, j, i, c) for j, i, c in zip(tj, ti, tc)])
    reft = gt[tj, ti, tc]
    assert np.linalg.norm(reft) > 0
    np.testing.assert_allclose(fdt, reft, rtol=1e-6, atol=1e-9 * np.abs(reft).max())


def test_ao_shading_closed_form():
    """c = albedo * visibility; with a 1x1 texture a and target 0,
    dL/dT = sum over pixels of 2 * a * vis^2; untextured pixels have albedo 1."""
    sc = _tri_scene()
    pts = np.array([[0.1, 0.1], [0.3, 0.2], [0.05, 0.6]], np.float32)
    rays = _ortho(pts)
    vis = np.array([0.25, 1.0, 0.5])
    fa = A.FrozenAO(sc, rays, np.zeros(3, np.uint32), vis)
    a = sc.textures[0].texels[0, 0, :3].astype(np.float64)
    img = fa.image(A._t(sc.verts), A._t(sc.textures[0].texels)).numpy()
    np.testing.assert_allclose(img, vis[:, None] * a[None], rtol=1e-12)
    _, _, gt, _ = fa.loss_grad(sc.verts, sc.textures[0].texels, np.zeros((3, 3)))
    np.testing.assert_allclose(gt[0, 0, :3], 2 * a * float((vis ** 2).sum()), rtol=1e-12)


def test_ao_bary_option_matches_the_solved_uv():
    """On a well-conditioned triangle the oracle's FP32 (u, v) agree with the
    FP64 ray-plane solution to float32 rounding, so FrozenAO gives the same
    image and texel gradients with and without `bary` (to ~1e-6 relative),
    and differs from them when the barycentrics are shifted by half a texel."""
    rng = np.random.default_rng(5)
    tex = rng.uniform(0, 1, (16, 16, 4)).astype(np.float32)
    sc = _tri_scene(tex=tex)
    pts = rng.uniform(0.02, 0.45, (64, 2)).astype(np.float32)
    rays = _ortho(pts)
    hits, _ = O.trace_list(sc, rays, "default", "closest")
    assert np.all(hits["prim"] == 0)
    bary = np.stack([hits["u"], hits["v"]], 1)
    vis = rng.choice([0.25, 0.5, 1.0], len(pts))
    target = np.zeros((len(pts), 3))
    fa = A.FrozenAO(sc, rays, hits["prim"], vis)
    fb = A.FrozenAO(sc, rays, hits["prim"], vis, bary=bary)
    ia = fa.image(A._t(sc.verts), A._t(tex)).numpy()
    ib = fb.image(A._t(sc.verts), A._t(tex)).numpy()
    np.testing.assert_allclose(ib, ia, rtol=1e-5, atol=1e-6)
    _, _, ga, _ = fa.loss_grad(sc.verts, tex, target)
    _, _, gb, _ = fb.loss_grad(sc.verts, tex, target)
    assert np.linalg.norm(gb - ga) <= 1e-5 * np.linalg.norm(ga)
    for k in range(8):
        j, i, c = rng.integers(0, 16), rng.integers(0, 16), rng.integers(0, 3)
        assert np.array_equal(fb.pixels_of_texel(sc.verts, j, i),
                              fa.pixels_of_texel(sc.verts, j, i))
        assert math.isclose(fb.fd_texel(sc.verts, tex, target, j, i, c), gb[j, i, c],
                            rel_tol=1e-7, abs_tol=1e-12)
    shifted = A.FrozenAO(sc, rays, hits["prim"], vis, bary=bary + np.float32(0.5 / 16))
    assert np.abs(shifted.image(A._t(sc.verts), A._t(tex)).numpy() - ia).max() > 1e-2
