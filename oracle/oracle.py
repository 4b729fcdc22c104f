"""Python access to the CPU oracle (``vsr_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  It shares no
code with the GPU library: it takes the seeded scene arrays, the rays and the
serialised BVH blob as plain numpy inputs.

Every function cites the part of the paper it follows (Zellmann, "Adding Custom
Intersectors to the C++ Ray Tracing Template Library Visionaray"):

* ``trace_list``  -- closest-hit / any-hit query over a linear primitive list,
  the intersector replacing ``intersect`` inside the loop (Section 3.2, the
  paragraph on linear lists; query definitions Section 3.1).
* ``trace_bvh``   -- the same queries through the while-while BVH traversal
  with both ``intersect`` calls replaced by the intersector (Section 3.2).
* ``trace_multi`` -- the multi-hit query (the third visibility query of the
  library the paper extends, Section 3.1): the first N accepted hits in
  ascending (t, prim) order, over the list as the plain definition (collect,
  sort, keep N) or through the BVH traversal with an N-entry buffer.
* ``trace_instances`` -- instancing (Section 3.2: BVHs as compound primitives
  of a list or of a top-level BVH, the intersector passed on to each BVH's
  own intersect), rays taken to object space by a world-to-object map.
* ``path_trace`` -- a diffuse path tracer on the closest-hit query with the
  intersector (a workload; FP32 with the bounce construction's operation
  order fixed so that every bounce is reproducible).
* intersector kinds follow Section 3.1 (default forwarding), Section 4
  (alpha-mask listing, procedural alpha, ``bvh_costs``) and Section 3.2 (an
  intersector that also replaces intersect(ray, aabb): the clip box).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vsr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NONE = 0xFFFFFFFF
ISECT = {"none": 0, "default": 1, "alpha_tex": 2, "proc_alpha": 3, "count": 4, "clip": 5}
QUERY = {"closest": 0, "any": 1}
TEX_FMT = {"u8": 0, "rgba8": 1, "rgba32f": 2}
TIE_EDGE, TIE_ALPHA, TIE_CLIP = 1, 2, 4


class _Texture(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("w", ctypes.c_uint32), ("h", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("texels", ctypes.c_void_p)]


class _Scene(ctypes.Structure):
    _fields_ = [("verts", ctypes.c_void_p), ("nverts", ctypes.c_uint64),
                ("idx", ctypes.c_void_p), ("uvs", ctypes.c_void_p),
                ("geom_id", ctypes.c_void_p), ("ntri", ctypes.c_uint32),
                ("ntex", ctypes.c_uint32), ("tex", ctypes.c_void_p)]


class _Isect(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("cutoff_u8", ctypes.c_uint32),
                ("cutoff_f", ctypes.c_float), ("freq", ctypes.c_float),
                ("clip_lo", ctypes.c_float * 3), ("clip_hi", ctypes.c_float * 3)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_trace_list.argtypes = [P, P, ctypes.c_int, P, ctypes.c_uint64, P, P, ctypes.c_int]
        lib.orc_trace_bvh.argtypes = [P, P, ctypes.c_uint64, P, ctypes.c_int, P,
                                      ctypes.c_uint64, P, P, ctypes.c_int]
        lib.orc_trace_multi.argtypes = [P, P, ctypes.c_uint64, P, ctypes.c_uint32, P,
                                        ctypes.c_uint64, P, P, ctypes.c_int]
        lib.orc_trace_instances.argtypes = [P, P, P, ctypes.c_uint32, P, P, ctypes.c_uint32, P,
                                            ctypes.c_uint64, P, ctypes.c_int, P, ctypes.c_uint64,
                                            P, P, P, ctypes.c_int]
        lib.orc_path_trace.argtypes = [P, P, ctypes.c_uint64, P, P, ctypes.c_uint64,
                                       ctypes.c_uint32, P, ctypes.c_float, P, P, P, P,
                                       ctypes.c_int]
        lib.orc_bounce.argtypes = [P, P, P, P, ctypes.c_uint64, ctypes.c_float, P]
        lib.orc_bounce.restype = None
        lib.orc_intersect_triangle.argtypes = [P, P, P, P, P]
        lib.orc_intersect_aabb.argtypes = [P, P, P, ctypes.c_float]
        lib.orc_shadow_rays.argtypes = [P, P, ctypes.c_uint64, P, ctypes.c_float, P]
        lib.orc_shadow_rays.restype = None
        lib.orc_ao_rays.argtypes = [P, P, P, ctypes.c_uint64, ctypes.c_uint32, P, ctypes.c_float,
                                    ctypes.c_float, P]
        lib.orc_ao_rays.restype = None
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class _SceneHandle:
    """Keeps the ctypes view of a scene and the arrays it points to alive."""

    def __init__(self, scene):
        self.verts = np.ascontiguousarray(scene.verts, np.float32)
        self.idx = np.ascontiguousarray(scene.idx, np.uint32)
        self.uvs = np.ascontiguousarray(scene.uvs, np.float32)
        self.geom_id = np.ascontiguousarray(scene.geom_id, np.uint32)
        self.texels = [np.ascontiguousarray(t.texels) for t in scene.textures]
        ntex = len(scene.textures)
        self.tex = (_Texture * max(ntex, 1))()
        for k, t in enumerate(scene.textures):
            self.tex[k] = _Texture(TEX_FMT[t.fmt], t.w, t.h, 0, _ptr(self.texels[k]))
        self.c = _Scene(_ptr(self.verts), self.verts.shape[0], _ptr(self.idx),
                        _ptr(self.uvs), _ptr(self.geom_id), self.idx.shape[0], ntex,
                        ctypes.addressof(self.tex))


def _isect(kind: str, cutoff_u8: int = 128, cutoff_f: float = 0.01, freq: float = 40.0,
           clip_lo=(0.0, 0.0, 0.0), clip_hi=(0.0, 0.0, 0.0)):
    return _Isect(ISECT[kind], cutoff_u8, cutoff_f, freq, (ctypes.c_float * 3)(*clip_lo),
                  (ctypes.c_float * 3)(*clip_hi))


def _run(fn, scene, rays, kind, query, nthreads, extra, **kw):
    lib = _load()
    sh = _SceneHandle(scene)
    rays = np.ascontiguousarray(rays, np.float32).reshape(-1, 8)
    n = rays.shape[0]
    hits = np.zeros((n, 4), np.float32)
    stats = np.zeros((n, 4), np.uint32)
    isect = _isect(kind, **kw)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    if fn == "list":
        rc = lib.orc_trace_list(ctypes.byref(sh.c), ctypes.byref(isect), QUERY[query],
                                _ptr(rays), n, _ptr(hits), _ptr(stats), nthreads)
    else:
        blob = extra
        rc = lib.orc_trace_bvh(ctypes.byref(sh.c), _ptr(blob), blob.nbytes,
                               ctypes.byref(isect), QUERY[query], _ptr(rays), n,
                               _ptr(hits), _ptr(stats), nthreads)
    if rc != 0:
        raise ValueError(f"oracle rejected its inputs (code {rc})")
    return split_hits(hits), stats


def split_hits(hits: np.ndarray):
    """(t, u, v, prim) views of an [n,4] float32 hit array."""
    t = hits[:, 0].copy()
    u = hits[:, 1].copy()
    v = hits[:, 2].copy()
    prim = hits[:, 3].copy().view(np.uint32)
    return {"t": t, "u": u, "v": v, "prim": prim}


def trace_list(scene, rays, kind="default", query="closest", nthreads=None, **kw):
    """Brute-force query over all triangles (no BVH).  Returns (hits, stats)."""
    return _run("list", scene, rays, kind, query, nthreads, None, **kw)


def trace_bvh(scene, blob: np.ndarray, rays, kind="default", query="closest",
              nthreads=None, **kw):
    """While-while BVH query over ``blob``.  Returns (hits, stats) where stats
    columns are (box tests, triangle tests, intersector calls, near-tie flags)."""
    blob = np.frombuffer(blob, np.uint8) if not isinstance(blob, np.ndarray) else blob
    return _run("bvh", scene, rays, kind, query, nthreads, np.ascontiguousarray(blob), **kw)


def trace_multi(scene, rays, nh: int, kind="default", blob=None, nthreads=None, **kw):
    """Multi-hit query: the first ``nh`` accepted hits of each ray in
    ascending (t, prim) order, misses after them.  ``blob`` None: sorted brute
    force over every triangle; otherwise the BVH traversal.  Returns (hits,
    stats): hits is a dict of [n, nh] arrays (t, u, v, prim); stats as in
    trace_bvh (for the brute force: triangle tests and consultations)."""
    lib = _load()
    sh = _SceneHandle(scene)
    rays = np.ascontiguousarray(rays, np.float32).reshape(-1, 8)
    n = rays.shape[0]
    hits = np.zeros((n * nh, 4), np.float32)
    stats = np.zeros((n, 4), np.uint32)
    isect = _isect(kind, **kw)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    if blob is not None:
        blob = np.frombuffer(blob, np.uint8) if not isinstance(blob, np.ndarray) else blob
        blob = np.ascontiguousarray(blob)
    rc = lib.orc_trace_multi(ctypes.byref(sh.c), None if blob is None else _ptr(blob),
                             0 if blob is None else blob.nbytes, ctypes.byref(isect), nh,
                             _ptr(rays), n, _ptr(hits), _ptr(stats), nthreads)
    if rc != 0:
        raise ValueError(f"oracle rejected its inputs (code {rc})")
    h = split_hits(hits)
    return {k: v.reshape(n, nh) for k, v in h.items()}, stats


def trace_instances(meshes, inst_mesh, w2o, rays, kind="default", query="closest",
                    top_blob=None, nthreads=None, **kw):
    """Closest-hit / any-hit over instances.  meshes: list of (scene, blob);
    inst_mesh uint32 [m]; w2o float32 [m, 12] world-to-object maps (row-major
    3 x 4); top_blob None: the instances as a linear list, else the top-level
    BVH over them.  Returns (hits, inst_ids, stats)."""
    lib = _load()
    handles = [_SceneHandle(sc) for sc, _ in meshes]
    blobs = [np.ascontiguousarray(np.frombuffer(b, np.uint8) if not isinstance(b, np.ndarray)
                                  else b) for _, b in meshes]
    nm = len(meshes)
    scene_ptrs = (ctypes.c_void_p * max(nm, 1))(*[ctypes.addressof(h.c) for h in handles])
    blob_ptrs = (ctypes.c_void_p * max(nm, 1))(*[_ptr(b) for b in blobs])
    blob_sizes = (ctypes.c_uint64 * max(nm, 1))(*[b.nbytes for b in blobs])
    im = np.ascontiguousarray(inst_mesh, np.uint32).reshape(-1)
    w = np.ascontiguousarray(w2o, np.float32).reshape(-1, 12)
    assert w.shape[0] == im.shape[0]
    rays = np.ascontiguousarray(rays, np.float32).reshape(-1, 8)
    n = rays.shape[0]
    hits = np.zeros((n, 4), np.float32)
    ids = np.zeros(n, np.uint32)
    stats = np.zeros((n, 4), np.uint32)
    isect = _isect(kind, **kw)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    top = None
    if top_blob is not None:
        top = np.ascontiguousarray(np.frombuffer(top_blob, np.uint8)
                                   if not isinstance(top_blob, np.ndarray) else top_blob)
    rc = lib.orc_trace_instances(scene_ptrs, blob_ptrs, blob_sizes, nm,
                                 _ptr(im) if im.size else None, _ptr(w) if w.size else None,
                                 im.shape[0], None if top is None else _ptr(top),
                                 0 if top is None else top.nbytes, ctypes.byref(isect),
                                 QUERY[query], _ptr(rays), n, _ptr(hits), _ptr(ids), _ptr(stats),
                                 nthreads)
    if rc != 0:
        raise ValueError(f"oracle rejected its inputs (code {rc})")
    return split_hits(hits), ids, stats


def path_trace(scene, blob, rays, bounces: int, dirs, eps: float, sky=(1.0, 1.0, 1.0),
               untex=(0.8, 0.8, 0.8), kind="default", nthreads=None, **kw):
    """Diffuse path tracing with the intersector (FP32, fixed operation order):
    returns (radiance float32 [n, 3], near-tie flags uint32 [n]).  dirs:
    float32 [n * bounces, 3] local unit directions, path i's bounce k at
    row i * bounces + k."""
    lib = _load()
    sh = _SceneHandle(scene)
    rays = np.ascontiguousarray(rays, np.float32).reshape(-1, 8)
    n = rays.shape[0]
    d = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
    assert d.shape[0] == n * bounces
    b = np.ascontiguousarray(np.frombuffer(blob, np.uint8) if not isinstance(blob, np.ndarray)
                             else blob)
    sk = np.ascontiguousarray(sky, np.float32)
    ut = np.ascontiguousarray(untex, np.float32)
    rad = np.zeros((n, 3), np.float32)
    flags = np.zeros(n, np.uint32)
    isect = _isect(kind, **kw)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    rc = lib.orc_path_trace(ctypes.byref(sh.c), _ptr(b), b.nbytes, ctypes.byref(isect), _ptr(rays),
                            n, bounces, _ptr(d) if d.size else None, float(eps), _ptr(sk),
                            _ptr(ut), _ptr(rad), _ptr(flags), nthreads)
    if rc != 0:
        raise ValueError(f"oracle rejected its inputs (code {rc})")
    return rad, flags


def bounce(scene, rays, hits_raw, dirs, eps):
    """The path tracer's next segment for each (ray, hit, local direction)."""
    lib = _load()
    sh = _SceneHandle(scene)
    r = np.ascontiguousarray(rays, np.float32).reshape(-1, 8)
    h = np.ascontiguousarray(hits_raw, np.float32).reshape(-1, 4)
    d = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
    assert r.shape[0] == h.shape[0] == d.shape[0]
    out = np.zeros_like(r)
    lib.orc_bounce(ctypes.byref(sh.c), _ptr(r), _ptr(h), _ptr(d), r.shape[0], float(eps), _ptr(out))
    return out


def intersect_triangle(ray, v0, v1, v2):
    """intersect(ray, basic_triangle<3,float>): returns (code, t, u, v) with
    code 1 hit, 0 miss, -1 parallel."""
    lib = _load()
    r = np.ascontiguousarray(ray, np.float32)
    a, b, c = (np.ascontiguousarray(x, np.float32) for x in (v0, v1, v2))
    out = np.zeros(3, np.float32)
    code = lib.orc_intersect_triangle(_ptr(r), _ptr(a), _ptr(b), _ptr(c), _ptr(out))
    return code, float(out[0]), float(out[1]), float(out[2])


def intersect_aabb(ray, lo, hi, t_far=np.inf):
    lib = _load()
    r = np.ascontiguousarray(ray, np.float32)
    l = np.ascontiguousarray(lo, np.float32)
    h = np.ascontiguousarray(hi, np.float32)
    return bool(lib.orc_intersect_aabb(_ptr(r), _ptr(l), _ptr(h), float(t_far)))


def shadow_rays(prim_rays, prim_hits_raw, light, eps):
    """Shadow rays from primary hit points toward a directional light."""
    lib = _load()
    r = np.ascontiguousarray(prim_rays, np.float32).reshape(-1, 8)
    h = np.ascontiguousarray(prim_hits_raw, np.float32).reshape(-1, 4)
    l = np.ascontiguousarray(light, np.float32)
    out = np.zeros_like(r)
    lib.orc_shadow_rays(_ptr(r), _ptr(h), r.shape[0], _ptr(l), float(eps), _ptr(out))
    return out


def ao_rays(scene, prim_rays, prim_hits_raw, spp, xi, tmax, eps):
    """Ambient-occlusion rays from primary hits (spp per pixel, FP64 frame)."""
    lib = _load()
    sh = _SceneHandle(scene)
    r = np.ascontiguousarray(prim_rays, np.float32).reshape(-1, 8)
    h = np.ascontiguousarray(prim_hits_raw, np.float32).reshape(-1, 4)
    x = np.ascontiguousarray(xi, np.float32).reshape(-1, 2)
    assert x.shape[0] == r.shape[0] * spp
    out = np.zeros((r.shape[0] * spp, 8), np.float32)
    lib.orc_ao_rays(ctypes.byref(sh.c), _ptr(r), _ptr(h), r.shape[0], spp, _ptr(x),
                    float(tmax), float(eps), _ptr(out))
    return out


def hits_raw(h: dict) -> np.ndarray:
    """Pack a hit dict back into the [n,4] float32 record layout."""
    out = np.zeros((h["t"].shape[0], 4), np.float32)
    out[:, 0] = h["t"]
    out[:, 1] = h["u"]
    out[:, 2] = h["v"]
    out[:, 3] = h["prim"].view(np.float32)
    return out
