"""Seeded synthetic scenes, textures and camera rays.

These generators are the only code shared by the GPU path and the oracle.  They
produce plain arrays (geometry, per-corner texture coordinates, texture ids,
texels, rays); none of the traversal, intersection or intersector arithmetic
lives here.  The workloads stand in for the paper's Fig. 1 use cases
(billboards with alpha masks, procedural alpha, heat maps), whose scenes are
not published.

Layouts:
  verts    float32 [V, 3]
  idx      uint32  [T, 3]      vertex indices per triangle
  uvs      float32 [T, 3, 2]   texture coordinate of corner k of triangle p
  geom_id  uint32  [T]         texture index, 0xFFFFFFFF = untextured/opaque
  rays     float32 [N, 8]      (ox, oy, oz, tmin, dx, dy, dz, tmax)
Textures: fmt "u8" ([H, W] alpha), "rgba8" ([H, W, 4] uint8) or "rgba32f"
([H, W, 4] float32); row j covers v in [j/H, (j+1)/H), column i covers u in
[i/W, (i+1)/W).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import _lib

NONE = 0xFFFFFFFF
SEED_BASE = 0x191212786


@dataclass
class Texture:
    fmt: str
    w: int
    h: int
    texels: np.ndarray


@dataclass
class Scene:
    name: str
    verts: np.ndarray
    idx: np.ndarray
    uvs: np.ndarray
    geom_id: np.ndarray
    textures: list = field(default_factory=list)
    meta: dict = field(default_factory=dict)

    @property
    def ntri(self) -> int:
        return int(self.idx.shape[0])

    def extent(self) -> float:
        if self.verts.shape[0] == 0:
            return 1.0
        lo = self.verts.min(axis=0).astype(np.float64)
        hi = self.verts.max(axis=0).astype(np.float64)
        return float(np.linalg.norm(hi - lo))

    def bvh(self, leaf_max: int = 4, bins: int = 32) -> np.ndarray:
        return _lib.bvh_build(self.verts, self.idx, leaf_max=leaf_max, bins=bins)


# ---------------------------------------------------------------------------
# cameras


def pinhole_rays(eye, target, up, fovy_deg: float, width: int, height: int,
                 tmin: float = 0.0, tmax: float = math.inf) -> np.ndarray:
    """Pixel-centre rays of a pinhole camera, row-major from the top row;
    directions normalised in float64 and rounded to float32."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(np.asarray(up, np.float64), f)
    r /= np.linalg.norm(r)
    u = np.cross(f, r)
    th = math.tan(math.radians(fovy_deg) * 0.5)
    aspect = width / height
    sx = (2.0 * (np.arange(width) + 0.5) / width - 1.0) * th * aspect
    sy = (1.0 - 2.0 * (np.arange(height) + 0.5) / height) * th
    d = f[None, None, :] + sx[None, :, None] * r[None, None, :] + sy[:, None, None] * u[None, None, :]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    rays = np.empty((height * width, 8), np.float32)
    rays[:, 0:3] = eye.astype(np.float32)
    rays[:, 3] = np.float32(tmin)
    rays[:, 4:7] = d.reshape(-1, 3).astype(np.float32)
    rays[:, 7] = np.float32(tmax)
    return rays


def orthographic_rays(lo_xy, hi_xy, z: float, n: int) -> np.ndarray:
    """n x n rays along +z through cell centres of [lo, hi]^2 at depth z."""
    xs = lo_xy[0] + (np.arange(n) + 0.5) / n * (hi_xy[0] - lo_xy[0])
    ys = lo_xy[1] + (np.arange(n) + 0.5) / n * (hi_xy[1] - lo_xy[1])
    X, Y = np.meshgrid(xs, ys)
    rays = np.zeros((n * n, 8), np.float32)
    rays[:, 0] = X.ravel()
    rays[:, 1] = Y.ravel()
    rays[:, 2] = z
    rays[:, 3] = 0.0
    rays[:, 6] = 1.0
    rays[:, 7] = np.inf
    return rays


# ---------------------------------------------------------------------------
# textures


def disc_alpha_u8(size: int = 256, radius: float = 0.4) -> Texture:
    """8-bit alpha: 255 where the texel centre lies within `radius` of the
    UV centre (0.5, 0.5), else 0."""
    c = (np.arange(size) + 0.5) / size
    X, Y = np.meshgrid(c, c)
    a = np.where((X - 0.5) ** 2 + (Y - 0.5) ** 2 <= radius * radius, 255, 0).astype(np.uint8)
    return Texture("u8", size, size, a)


def value_noise(rng: np.random.Generator, w: int, h: int, base: int = 16,
                octaves: int = 3) -> np.ndarray:
    """Lattice value noise (smoothstep-interpolated), base lattice plus
    `octaves` finer octaves with halving amplitude, normalised to [0, 1]."""
    out = np.zeros((h, w), np.float64)
    amp, total = 1.0, 0.0
    for o in range(octaves + 1):
        L = base * (2 ** o)
        lat = rng.uniform(0.0, 1.0, (L + 1, L + 1))
        x = (np.arange(w) + 0.5) / w * L
        y = (np.arange(h) + 0.5) / h * L
        i0 = np.minimum(np.floor(x).astype(np.int64), L - 1)
        j0 = np.minimum(np.floor(y).astype(np.int64), L - 1)
        fx = x - i0
        fy = y - j0
        fx = fx * fx * (3 - 2 * fx)
        fy = fy * fy * (3 - 2 * fy)
        a = lat[j0[:, None], i0[None, :]]
        b = lat[j0[:, None], i0[None, :] + 1]
        c = lat[j0[:, None] + 1, i0[None, :]]
        d = lat[j0[:, None] + 1, i0[None, :] + 1]
        top = a + (b - a) * fx[None, :]
        bot = c + (d - c) * fx[None, :]
        out += amp * (top + (bot - top) * fy[:, None])
        total += amp
        amp *= 0.5
    return out / total


def foliage_rgba8(rng: np.random.Generator, size: int = 1024, coverage: float = 0.45) -> Texture:
    """RGBA8 foliage: alpha 255 where value noise exceeds its (1-coverage)
    quantile, green-ramp colour from a second noise field."""
    n = value_noise(rng, size, size)
    thr = np.quantile(n, 1.0 - coverage)
    col = value_noise(rng, size, size)
    tex = np.empty((size, size, 4), np.uint8)
    tex[..., 0] = np.clip(30 + 70 * col, 0, 255).astype(np.uint8)
    tex[..., 1] = np.clip(90 + 150 * col, 0, 255).astype(np.uint8)
    tex[..., 2] = np.clip(20 + 50 * col, 0, 255).astype(np.uint8)
    tex[..., 3] = np.where(n > thr, 255, 0).astype(np.uint8)
    return Texture("rgba8", size, size, tex)


# ---------------------------------------------------------------------------
# geometry helpers

_QUAD_UV = np.array([[[0, 0], [1, 0], [1, 1]], [[0, 0], [1, 1], [0, 1]]], np.float32)


def _quads_to_tris(corners: np.ndarray):
    """corners [Q,4,3] (counter-clockwise, UV (0,0),(1,0),(1,1),(0,1)) ->
    verts [4Q,3], idx [2Q,3], uvs [2Q,3,2]."""
    q = corners.shape[0]
    verts = corners.reshape(-1, 3).astype(np.float32)
    base = (np.arange(q, dtype=np.uint32) * 4)[:, None]
    idx = np.empty((q, 2, 3), np.uint32)
    idx[:, 0, :] = base + np.array([0, 1, 2], np.uint32)
    idx[:, 1, :] = base + np.array([0, 2, 3], np.uint32)
    uvs = np.broadcast_to(_QUAD_UV, (q, 2, 3, 2)).reshape(-1, 3, 2).copy()
    return verts, idx.reshape(-1, 3), uvs


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform rotations on SO(3) from normalised Gaussian quaternions."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def random_quads(rng: np.random.Generator, n_quads: int, lo: float, hi: float,
                 side_lo: float, side_hi: float) -> np.ndarray:
    """Squares with centres U[lo,hi]^3, side U[side_lo,side_hi], uniform
    orientation.  Returns corners [Q,4,3] float64."""
    centres = rng.uniform(lo, hi, (n_quads, 3))
    side = rng.uniform(side_lo, side_hi, n_quads)
    R = _random_rotations(rng, n_quads)
    local = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0.5, 0.5, 0], [-0.5, 0.5, 0]])
    pts = np.einsum("qij,kj->qki", R, local) * side[:, None, None]
    return centres[:, None, :] + pts


# ---------------------------------------------------------------------------
# workloads


def small_quads(seed: int = SEED_BASE + 0, n_quads: int = 2048, res: int = 256):
    """2,048 random quads (4,096 triangles) in the unit cube with one 256x256
    u8 disc alpha texture, and res x res pinhole primary rays from
    (0.5, 0.5, -1) towards the cube centre (fovy 60 degrees)."""
    rng = np.random.default_rng(seed)
    corners = random_quads(rng, n_quads, 0.0, 1.0, 0.02, 0.1)
    verts, idx, uvs = _quads_to_tris(corners)
    geom = np.zeros(idx.shape[0], np.uint32)
    scene = Scene("small_quads", verts, idx, uvs, geom, [disc_alpha_u8(256, 0.4)],
                  {"n_quads": n_quads})
    rays = pinhole_rays((0.5, 0.5, -1.0), (0.5, 0.5, 0.5), (0, 1, 0), 60.0, res, res)
    return scene, rays


def billboard_forest(seed: int = SEED_BASE + 1, n_quads: int = 500_000,
                     width: int = 1920, height: int = 1080, tex_size: int = 1024,
                     extent: float = 100.0):
    """Vertical alpha-masked billboards scattered over an extent x extent
    ground plane with Poisson-disc spacing (r = 0.1 at the full size), height
    U[0.5, 3], width height*U[0.5, 1], yaw U[0, 2 pi); two opaque ground
    triangles first; texture id = quad index mod 4 over four RGBA8 foliage
    textures (about 45 % opaque).  Camera at (50, 1.7, -2) looking at
    (50, 1, 50) scaled with the extent, fovy 60 degrees."""
    rng = np.random.default_rng(seed)
    # Poisson-disc radius keeps the full-size density (500k per 100x100).
    r = 0.1 * math.sqrt((extent * extent / 1e4) / (n_quads / 5e5))
    pts = _lib.poisson_disc(extent, extent, r, n_quads, seed).astype(np.float64)
    q = pts.shape[0]
    h = rng.uniform(0.5, 3.0, q)
    w = h * rng.uniform(0.5, 1.0, q)
    yaw = rng.uniform(0.0, 2 * math.pi, q)
    ax = np.stack([np.cos(yaw), np.zeros(q), np.sin(yaw)], 1) * (0.5 * w)[:, None]
    base = np.stack([pts[:, 0], np.zeros(q), pts[:, 1]], 1)
    up = np.zeros((q, 3))
    up[:, 1] = h
    corners = np.stack([base - ax, base + ax, base + ax + up, base - ax + up], 1)
    ground = np.array([[[0, 0, 0], [extent, 0, 0], [extent, 0, extent], [0, 0, extent]]], np.float64)
    verts, idx, uvs = _quads_to_tris(np.concatenate([ground, corners], 0))
    geom = np.empty(idx.shape[0], np.uint32)
    geom[:2] = NONE
    geom[2:] = (np.arange(q, dtype=np.uint32) % 4).repeat(2)
    texs = [foliage_rgba8(np.random.default_rng(seed * 7 + k), tex_size) for k in range(4)]
    s = extent / 100.0
    scene = Scene("billboard_forest", verts, idx, uvs, geom, texs,
                  {"n_quads": q, "poisson_r": r})
    rays = pinhole_rays((50 * s, 1.7, -2 * s), (50 * s, 1.0, 50 * s), (0, 1, 0), 60.0,
                        width, height)
    return scene, rays


# ---------------------------------------------------------------------------
# instancing workloads: meshes placed by affine maps, a top-level BVH over
# the instances' world boxes


@dataclass
class InstanceSet:
    name: str
    meshes: list          # Scene per mesh
    blobs: list           # BVH blob per mesh
    inst_mesh: np.ndarray  # uint32 [m]
    o2w: np.ndarray       # float64 [m, 3, 4] object-to-world placement
    w2o: np.ndarray       # float32 [m, 12] world-to-object map the traversal applies
    boxes: np.ndarray     # float32 [m, 6] world boxes (lo.xyz, hi.xyz)
    top: np.ndarray       # BVH blob over the boxes (primitive i = instance i)


def _place(rot, scale, trans):
    """Object-to-world map x -> scale * rot @ x + trans as a 3 x 4 matrix."""
    m = np.zeros((3, 4))
    m[:, :3] = scale * np.asarray(rot, np.float64)
    m[:, 3] = trans
    return m


def _rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def make_instance_set(name, meshes, inst_mesh, o2w) -> InstanceSet:
    """Inverse maps (float64, rounded to float32) and world boxes: the mesh's
    box corners mapped to world space, padded by 1e-5 of the box size (the
    traversal applies the float32 inverse) and rounded outward to float32."""
    inst_mesh = np.asarray(inst_mesh, np.uint32)
    o2w = np.asarray(o2w, np.float64).reshape(-1, 3, 4)
    blobs = [m.bvh() for m in meshes]
    w2o = np.zeros((len(o2w), 12), np.float32)
    boxes = np.zeros((len(o2w), 6), np.float32)
    obox = []
    for m in meshes:
        v = m.verts[np.asarray(m.idx).reshape(-1)].astype(np.float64)
        obox.append((v.min(0), v.max(0)))
    for i, (mid, a) in enumerate(zip(inst_mesh, o2w)):
        inv = np.linalg.inv(np.vstack([a, [0, 0, 0, 1]]))[:3]
        w2o[i] = inv.reshape(-1).astype(np.float32)
        lo, hi = obox[mid]
        corners = np.array([[x, y, z] for x in (lo[0], hi[0]) for y in (lo[1], hi[1])
                            for z in (lo[2], hi[2])])
        wc = corners @ a[:, :3].T + a[:, 3]
        wlo, whi = wc.min(0), wc.max(0)
        pad = 1e-5 * max(float(np.linalg.norm(whi - wlo)), 1.0)
        boxes[i, :3] = np.nextafter((wlo - pad).astype(np.float32), np.float32(-np.inf))
        boxes[i, 3:] = np.nextafter((whi + pad).astype(np.float32), np.float32(np.inf))
    return InstanceSet(name, list(meshes), blobs, inst_mesh, o2w, w2o, boxes,
                       _lib.bvh_build_boxes(boxes))


def instanced_small(seed: int = SEED_BASE + 7, n_inst: int = 7):
    """The small quad scene and a unit quad (u8 disc alpha) placed n_inst
    times by random rotations (uniform on SO(3)), scales U[0.5, 1.5] and
    translations around (0.5, 0.5, 0.5); instance 0 is the small scene
    unmoved.  Rays: the small scene's 256 x 256 camera."""
    rng = np.random.default_rng(seed)
    quads, rays = small_quads()
    unit = quad_grid_scene(disc_alpha_u8(256, 0.4))
    o2w = [_place(np.eye(3), 1.0, np.zeros(3))]
    mesh = [0]
    for k in range(1, n_inst):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        scale = rng.uniform(0.5, 1.5)
        centre = np.array([0.5, 0.5, 0.5]) + rng.uniform(-0.7, 0.7, 3)
        m = k % 2
        ocentre = np.array([0.5, 0.5, 0.5]) if m == 0 else np.array([0.5, 0.5, 0.0])
        o2w.append(_place(rot, scale, centre - scale * rot @ ocentre))
        mesh.append(m)
    return make_instance_set("instanced_small", [quads, unit], mesh, o2w), rays


def instanced_forest(seed: int = SEED_BASE + 6, grid: int = 8, extent: float = 100.0,
                     width: int = 1920, height: int = 1080, tex_size: int = 1024):
    """The billboard forest built by instancing: one tile of extent/grid
    squared with 500,000/grid^2 billboards (the forest's density and
    textures, without ground) placed grid x grid times, each turned about its
    vertical axis by U[0, 2 pi), plus the 100 x 100 ground as a mesh of its
    own (instance 0, unmoved).  The same camera and frame as the forest."""
    rng = np.random.default_rng(seed)
    cell = extent / grid
    tile, _ = billboard_forest(seed=seed, n_quads=int(500_000 / grid ** 2), extent=cell,
                               width=8, height=8, tex_size=tex_size)
    tile = Scene("forest_tile", tile.verts, tile.idx[2:], tile.uvs[2:], tile.geom_id[2:],
                 tile.textures, tile.meta)
    g = np.array([[[0, 0, 0], [extent, 0, 0], [extent, 0, extent], [0, 0, extent]]], np.float64)
    gv, gi, guv = _quads_to_tris(g)
    ground = Scene("ground", gv, gi, guv, np.full(2, NONE, np.uint32), [])
    o2w = [_place(np.eye(3), 1.0, np.zeros(3))]
    mesh = [1]
    tc = np.array([0.5 * cell, 0.0, 0.5 * cell])
    for a in range(grid):
        for b in range(grid):
            rot = _rot_y(rng.uniform(0.0, 2 * math.pi))
            centre = np.array([(a + 0.5) * cell, 0.0, (b + 0.5) * cell])
            o2w.append(_place(rot, 1.0, centre - rot @ tc))
            mesh.append(0)
    inst = make_instance_set("instanced_forest", [tile, ground], mesh, o2w)
    s = extent / 100.0
    rays = pinhole_rays((50 * s, 1.7, -2 * s), (50 * s, 1.0, 50 * s), (0, 1, 0), 60.0,
                        width, height)
    return inst, rays


LIGHT_DIR = np.array([0.3, 1.0, 0.2], np.float64) / np.linalg.norm([0.3, 1.0, 0.2])


def light_dir_f32() -> np.ndarray:
    return LIGHT_DIR.astype(np.float32)


def shadow_eps(scene: Scene) -> float:
    """Offset of secondary-ray origins: 1e-4 of the scene's bounding diagonal."""
    return float(np.float32(1e-4 * scene.extent()))


def quad_grid_scene(texture: Texture, geom: int = 0) -> Scene:
    """One quad spanning [0,1]^2 at z = 0 with UVs equal to (x, y)."""
    corners = np.array([[[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]]], np.float64)
    verts, idx, uvs = _quads_to_tris(corners)
    return Scene("unit_quad", verts, idx, uvs, np.full(2, geom, np.uint32), [texture])


# ---------------------------------------------------------------------------
# differentiation workload


def _icosahedron():
    t = (1.0 + 5 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def geodesic_sphere(freq: int):
    """Unit geodesic sphere: every icosahedron edge split into `freq` parts
    (20 freq^2 triangles, 10 freq^2 + 2 vertices).  Shared vertices are merged
    exactly through their integer barycentric keys."""
    base, faces = _icosahedron()
    keys, pts = {}, []
    tris = []

    def vid(a, b, c, wa, wb, wc):
        key = tuple(sorted((x, w) for x, w in ((a, wa), (b, wb), (c, wc)) if w))
        k = keys.get(key)
        if k is None:
            k = len(pts)
            keys[key] = k
            p = sum(base[x] * w for x, w in key) / freq
            pts.append(p / np.linalg.norm(p))
        return k

    for a, b, c in faces:
        grid = {}
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                grid[i, j] = vid(a, b, c, freq - i - j, i, j)
        for i in range(freq):
            for j in range(freq - i):
                tris.append((grid[i, j], grid[i + 1, j], grid[i, j + 1]))
                if i + j < freq - 1:
                    tris.append((grid[i + 1, j], grid[i + 1, j + 1], grid[i, j + 1]))
    return np.array(pts), np.array(tris, np.int64)


def _spherical_uvs(verts: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """Equirectangular per-corner texture coordinates; triangles across the
    seam get u shifted by one on their small-u corners, and pole corners take
    the mean u of the other two corners."""
    p = verts[idx]  # [T,3,3]
    r = np.linalg.norm(p, axis=-1)
    u = 0.5 + np.arctan2(p[..., 2], p[..., 0]) / (2 * np.pi)
    v = 0.5 - np.arcsin(np.clip(p[..., 1] / r, -1, 1)) / np.pi
    seam = (u.max(1) - u.min(1)) > 0.5
    u[seam] = np.where(u[seam] < 0.5, u[seam] + 1.0, u[seam])
    pole = np.abs(p[..., 1] / r) > 1 - 1e-9
    for k in range(3):
        m = pole[:, k]
        others = [x for x in range(3) if x != k]
        u[m, k] = u[m][:, others].mean(1)
    return np.stack([u, v], -1).astype(np.float32)


def _vertex_neighbours(n: int, idx: np.ndarray):
    e = np.concatenate([idx[:, [0, 1]], idx[:, [1, 2]], idx[:, [2, 0]]])
    e = np.concatenate([e, e[:, ::-1]])
    e = np.unique(e, axis=0)
    return e


def displaced_icosphere(seed: int = SEED_BASE + 2, freq: int = 57, res: int = 512,
                        tex_size: int = 512, alpha_cut: float = 0.3):
    """Displaced geodesic sphere (freq 57: 64,980 triangles, 32,492 vertices),
    radius 1 plus 0.05 N(0,1) per vertex smoothed by three uniform-Laplacian
    passes, along the normal.  RGBA32F albedo: smooth value-noise colour and
    alpha from uniform noise (the intersector keeps alpha >= alpha_cut).
    res x res primary rays from (0, 0, 3) toward the origin, fovy 45 degrees.
    Also returns target parameters: vertices + 0.01 N(0,1), colour texels +
    0.01 N(0,1) (alpha unchanged)."""
    rng = np.random.default_rng(seed)
    pts, idx = geodesic_sphere(freq)
    disp = 0.05 * rng.standard_normal(len(pts))
    e = _vertex_neighbours(len(pts), idx)
    deg = np.bincount(e[:, 0], minlength=len(pts)).astype(np.float64)
    for _ in range(3):
        acc = np.zeros(len(pts))
        np.add.at(acc, e[:, 0], disp[e[:, 1]])
        disp = 0.5 * disp + 0.5 * acc / deg
    verts = (pts * (1.0 + disp)[:, None]).astype(np.float32)
    uvs = _spherical_uvs(pts, idx)
    tex = np.empty((tex_size, tex_size, 4), np.float32)
    for c in range(3):
        tex[..., c] = value_noise(rng, tex_size, tex_size, base=8, octaves=2)
    tex[..., 3] = rng.uniform(0.0, 1.0, (tex_size, tex_size))
    geom = np.zeros(len(idx), np.uint32)
    scene = Scene("displaced_icosphere", verts, idx.astype(np.uint32), uvs, geom,
                  [Texture("rgba32f", tex_size, tex_size, tex)],
                  {"freq": freq, "alpha_cut": alpha_cut})
    rays = pinhole_rays((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0, 1, 0), 45.0, res, res)
    target_verts = (verts + 0.01 * rng.standard_normal(verts.shape)).astype(np.float32)
    target_tex = tex.copy()
    target_tex[..., :3] += (0.01 * rng.standard_normal((tex_size, tex_size, 3))).astype(np.float32)
    return scene, rays, target_verts, target_tex


# ---------------------------------------------------------------------------
# batching workload


def camera_rays_random(rng: np.random.Generator, n: int, eye=(0.5, 0.5, -1.0),
                       target=(0.5, 0.5, 0.5), up=(0, 1, 0), fovy_deg: float = 60.0,
                       aspect: float = 1.0) -> np.ndarray:
    """n pinhole rays through uniformly random image-plane positions."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(np.asarray(up, np.float64), f)
    r /= np.linalg.norm(r)
    u = np.cross(f, r)
    th = math.tan(math.radians(fovy_deg) * 0.5)
    sx = rng.uniform(-1, 1, n) * th * aspect
    sy = rng.uniform(-1, 1, n) * th
    d = f[None] + sx[:, None] * r[None] + sy[:, None] * u[None]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rays = np.empty((n, 8), np.float32)
    rays[:, 0:3] = eye.astype(np.float32)
    rays[:, 3] = 0.0
    rays[:, 4:7] = d.astype(np.float32)
    rays[:, 7] = np.inf
    return rays


def diffuse_rays(rng: np.random.Generator, scene: Scene, n: int) -> np.ndarray:
    """n rays leaving uniformly chosen points of uniformly chosen triangles in
    cosine-distributed directions about a random side of the face normal;
    interval (1e-4 of the scene diagonal, +inf)."""
    tri = rng.integers(0, scene.ntri, n)
    v = scene.verts.astype(np.float64)[scene.idx[tri]]  # [n,3,3]
    e1, e2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    a, b = rng.uniform(size=n), rng.uniform(size=n)
    sa = np.sqrt(a)
    p = v[:, 0] + (sa * (1 - b))[:, None] * e1 + (sa * b)[:, None] * e2
    nrm = np.cross(e1, e2)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm *= np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)[:, None]
    helper = np.where(np.abs(nrm[:, :1]) > 0.9, np.array([[0, 1, 0]]), np.array([[1, 0, 0]]))
    t1 = np.cross(helper, nrm)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    xi1, xi2 = rng.uniform(size=n), rng.uniform(size=n)
    rr, phi = np.sqrt(xi1), 2 * np.pi * xi2
    d = (rr * np.cos(phi))[:, None] * t1 + (rr * np.sin(phi))[:, None] * t2 \
        + np.sqrt(1 - xi1)[:, None] * nrm
    rays = np.empty((n, 8), np.float32)
    rays[:, 0:3] = p.astype(np.float32)
    rays[:, 3] = np.float32(1e-4 * scene.extent())
    rays[:, 4:7] = d.astype(np.float32)
    rays[:, 7] = np.inf
    return rays


def batch_scenes(seed: int = SEED_BASE + 3, n_scenes: int = 256, tri_range=(1_000, 200_000),
                 ray_range=(1_000, 1_000_000), tex_size: int = 256):
    """Independent scenes for the batched launch: triangle counts log-uniform
    in tri_range (rounded to even: random quads as in small_quads), each with
    its own u8 disc alpha of radius U[0.25, 0.45]; ray counts log-uniform in
    ray_range, half pinhole primary rays from (0.5, 0.5, -1) and half diffuse
    rays from random surface points.  Returns a list of (scene, rays)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_scenes):
        ntri = int(np.exp(rng.uniform(np.log(tri_range[0]), np.log(tri_range[1]))))
        nq = max(1, ntri // 2)
        nrays = int(np.exp(rng.uniform(np.log(ray_range[0]), np.log(ray_range[1]))))
        corners = random_quads(rng, nq, 0.0, 1.0, 0.02, 0.1)
        verts, idx, uvs = _quads_to_tris(corners)
        tex = disc_alpha_u8(tex_size, float(rng.uniform(0.25, 0.45)))
        sc = Scene(f"batch_{k}", verts, idx, uvs, np.zeros(len(idx), np.uint32), [tex])
        half = nrays // 2
        rays = np.concatenate([camera_rays_random(rng, half), diffuse_rays(rng, sc, nrays - half)])
        out.append((sc, rays))
    return out


def build_bvhs(scene_list, threads: int | None = None):
    """BVH blobs for many scenes, built concurrently (the builder releases the
    interpreter lock)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or len(os.sched_getaffinity(0))
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda s: s.bvh(), scene_list))


# ---------------------------------------------------------------------------
# large incoherent workload


def heightfield(n_cells: int, extent: float, amplitude: float, rng: np.random.Generator):
    """n_cells x n_cells grid over [0, extent]^2 (two triangles per cell) with
    height amplitude * value noise; returns verts, idx, uvs."""
    h = amplitude * value_noise(rng, n_cells + 1, n_cells + 1, base=8, octaves=3)
    xs = np.linspace(0.0, extent, n_cells + 1)
    X, Z = np.meshgrid(xs, xs)
    verts = np.stack([X, h, Z], -1).reshape(-1, 3).astype(np.float32)
    i = np.arange(n_cells)
    a = (i[:, None] * (n_cells + 1) + i[None, :]).ravel()
    b, c, d = a + 1, a + n_cells + 1, a + n_cells + 2
    idx = np.empty((len(a), 2, 3), np.uint32)
    idx[:, 0] = np.stack([a, b, d], 1)
    idx[:, 1] = np.stack([a, d, c], 1)
    uv = verts[:, [0, 2]] / extent
    idx = idx.reshape(-1, 3)
    return verts, idx, uv[idx].astype(np.float32)


def large_incoherent(seed: int = SEED_BASE + 4, n_quads: int = 7_000_000, ground_cells: int = 1000,
                     width: int = 1920, height: int = 1080, tex_size: int = 1024):
    """7 M random quads (14 M triangles, side U[0.005, 0.05], uniform
    orientation, UVs over [0, 1]^2, textured) in [0, 10]^3 plus a 1000 x 1000
    cell heightfield (2 M opaque triangles, height 0.5 * value noise) over
    [0, 10]^2: 16 M triangles.  One RGBA32F tex_size^2 colour texture (value
    noise, alpha 1).  Primary rays from (5, 8, -5) toward (5, 2, 5), fovy 60
    degrees."""
    rng = np.random.default_rng(seed)
    corners = random_quads(rng, n_quads, 0.0, 10.0, 0.005, 0.05)
    qv, qi, quv = _quads_to_tris(corners)
    del corners
    gv, gi, guv = heightfield(ground_cells, 10.0, 0.5, rng)
    verts = np.concatenate([qv, gv])
    idx = np.concatenate([qi, gi + np.uint32(len(qv))])
    uvs = np.concatenate([quv, guv])
    geom = np.full(len(idx), NONE, np.uint32)
    geom[: len(qi)] = 0
    tex = np.empty((tex_size, tex_size, 4), np.float32)
    for c in range(3):
        tex[..., c] = value_noise(rng, tex_size, tex_size, base=16, octaves=3)
    tex[..., 3] = 1.0
    scene = Scene("large_incoherent", verts, idx, uvs, geom,
                  [Texture("rgba32f", tex_size, tex_size, tex)], {"n_quads": n_quads})
    rays = pinhole_rays((5.0, 8.0, -5.0), (5.0, 2.0, 5.0), (0, 1, 0), 60.0, width, height)
    return scene, rays


def path_dirs(n_paths: int, bounces: int, seed: int = SEED_BASE + 8) -> np.ndarray:
    """Cosine-distributed unit directions in a local frame (z up) for the
    diffuse bounces of path tracing, float32 [n_paths * bounces, 3] (path i's
    bounce k at row i * bounces + k); drawn in float64 and rounded."""
    rng = np.random.default_rng(seed)
    x1 = rng.uniform(0.0, 1.0, n_paths * bounces)
    x2 = rng.uniform(0.0, 1.0, n_paths * bounces)
    r = np.sqrt(x1)
    d = np.stack([r * np.cos(2 * np.pi * x2), r * np.sin(2 * np.pi * x2), np.sqrt(1.0 - x1)], 1)
    return d.astype(np.float32)


def ao_random(n_rays: int, spp: int, seed: int = SEED_BASE + 5) -> np.ndarray:
    """Uniform random numbers in [0, 1) for ambient-occlusion sampling,
    float32 [n_rays * spp, 2]; passed to both the GPU and the oracle."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, (n_rays * spp, 2)).astype(np.float32)
