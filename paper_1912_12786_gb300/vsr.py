"""Thin ctypes binding of the GPU library (names as in ``include/vsr.h``).

Argument marshalling only: every step of the traversal runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch provides device
memory and streams).  There is no CPU fallback: if ``libvsr.so`` has not been
built, loading fails with an error.

Tensor layouts:
  rays      float32 [n, 8]  (ox, oy, oz, tmin, dx, dy, dz, tmax)
  hits      float32 [n, 4]  (t, u, v, prim id bits); ``prim_ids(hits)`` gives
            the uint32 ids as int64 (miss = 0xFFFFFFFF)
  counters  int32   [n, 2]  (box tests, triangle tests) for the COUNT intersector
  stats     int32   [n, 4]  (box tests, triangle tests, intersector calls,
            texture look-ups)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

VSR_OK, VSR_ERR_ARG, VSR_ERR_CUDA, VSR_ERR_OOM, VSR_ERR_BLOB, VSR_ERR_STACK, \
    VSR_ERR_TIMEOUT, VSR_ERR_STATE = range(8)
STATUS_NAMES = ["VSR_OK", "VSR_ERR_ARG", "VSR_ERR_CUDA", "VSR_ERR_OOM", "VSR_ERR_BLOB",
                "VSR_ERR_STACK", "VSR_ERR_TIMEOUT", "VSR_ERR_STATE"]
MISS = 0xFFFFFFFF
NO_TEXTURE = 0xFFFFFFFF
ISECT = {"none": 0, "default": 1, "alpha_tex": 2, "proc_alpha": 3, "count": 4, "clip": 5}
DISPATCH = {"static": 0, "dynamic": 1}
QUERY = {"closest": 0, "any": 1}
TEX_FMT = {"u8": 0, "rgba8": 1, "rgba32f": 2}
# device error word bits (vsr_get_device_error)
DEVERR_STACK, DEVERR_STEPS, DEVERR_ALIGN, DEVERR_HIT, DEVERR_TIMEOUT = 1, 2, 4, 8, 16


class VsrError(RuntimeError):
    """A non-OK status from the library; ``status`` is the vsr_status code and
    the message is vsr_last_error() at the time of the call."""
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class vsr_texture_desc(ctypes.Structure):
    """One texture (C layout of vsr_texture_desc): format, size, host texels."""
    _fields_ = [("fmt", ctypes.c_int32), ("w", ctypes.c_uint32), ("h", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("texels", ctypes.c_void_p)]


class vsr_intersector(ctypes.Structure):
    """The custom intersector (C layout of vsr_intersector): kind, static or
    dynamic dispatch, alpha cutoffs, procedural frequency, clip box."""
    _fields_ = [("kind", ctypes.c_int32), ("dispatch", ctypes.c_int32),
                ("alpha_cutoff_u8", ctypes.c_uint32), ("alpha_cutoff_f", ctypes.c_float),
                ("proc_freq", ctypes.c_float), ("clip_lo", ctypes.c_float * 3),
                ("clip_hi", ctypes.c_float * 3)]


class vsr_trace_params(ctypes.Structure):
    """Launch configuration (C layout of vsr_trace_params)."""
    _fields_ = [("block_size", ctypes.c_uint32), ("persistent", ctypes.c_uint32),
                ("refill_threshold", ctypes.c_uint32), ("blocks_per_sm", ctypes.c_uint32),
                ("image_width", ctypes.c_uint32), ("stack_regs", ctypes.c_uint32),
                ("watchdog_iterations", ctypes.c_uint32), ("watchdog_ms", ctypes.c_uint32),
                ("reg_cap_blocks", ctypes.c_uint32), ("ray_order", ctypes.c_uint32),
                ("lockstep", ctypes.c_uint32), ("octant", ctypes.c_uint32)]


class vsr_path_params(ctypes.Structure):
    """Path-tracing parameters (C layout of vsr_path_params)."""
    _fields_ = [("bounces", ctypes.c_uint32), ("eps", ctypes.c_float),
                ("sky", ctypes.c_float * 3), ("untextured", ctypes.c_float * 3)]


def path_params(bounces=3, eps=1e-4, sky=(1.0, 1.0, 1.0), untextured=(0.8, 0.8, 0.8)):
    """vsr_path_params: bounces after the first segment, the interval start of
    every bounce segment, the sky radiance and the albedo of untextured hits."""
    return vsr_path_params(bounces, eps, (ctypes.c_float * 3)(*sky),
                           (ctypes.c_float * 3)(*untextured))


class vsr_shade_params(ctypes.Structure):
    """Diffuse shading parameters (C layout of vsr_shade_params)."""
    _fields_ = [("light", ctypes.c_float * 3), ("background", ctypes.c_float * 3),
                ("grad_tex", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


_lib = None
P = ctypes.c_void_p
_SIGS = {
    "vsr_version": ([], ctypes.c_int32),
    "vsr_last_error": ([], ctypes.c_char_p),
    "vsr_scene_create_indexed": ([P, ctypes.c_uint32, P, P, P, ctypes.c_uint32, P,
                                  ctypes.c_uint32, ctypes.POINTER(P)], ctypes.c_int),
    "vsr_scene_create": ([P, P, P, ctypes.c_uint32, P, ctypes.c_uint32, ctypes.POINTER(P)],
                         ctypes.c_int),
    "vsr_scene_destroy": ([P], ctypes.c_int),
    "vsr_bvh_load": ([P, P, ctypes.c_size_t], ctypes.c_int),
    "vsr_trace": ([P, P, ctypes.c_uint64, P, ctypes.c_int32, P, P, P, P], ctypes.c_int),
    "vsr_trace_tune": ([P, P, ctypes.c_uint64, P, ctypes.c_int32, ctypes.c_uint32, P, P, P],
                       ctypes.c_int),
    "vsr_trace_tuned_params": ([P, P, ctypes.c_int32, P], ctypes.c_int),
    "vsr_trace_stats": ([P, P, ctypes.c_uint64, P, ctypes.c_int32, P, P, P], ctypes.c_int),
    "vsr_trace_multi": ([P, P, ctypes.c_uint64, P, ctypes.c_uint32, P, P, P, P], ctypes.c_int),
    "vsr_instances_create": ([P, ctypes.c_uint32, P, P, ctypes.c_uint32, P, ctypes.c_size_t,
                              ctypes.POINTER(P)], ctypes.c_int),
    "vsr_instances_destroy": ([P], ctypes.c_int),
    "vsr_trace_instances": ([P, P, ctypes.c_uint64, P, ctypes.c_int32, P, P, P, P, P],
                            ctypes.c_int),
    "vsr_instances_device_error": ([P, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "vsr_path_trace": ([P, P, ctypes.c_uint64, P, P, P, P, P, P, P], ctypes.c_int),
    "vsr_trace_persistent_noalloc": ([P, P, ctypes.c_uint64, P, ctypes.c_int32, P, P, P, P],
                                     ctypes.c_int),
    "vsr_batch_create": ([P, P, P, P, ctypes.c_uint32, P, ctypes.c_int32, P, ctypes.POINTER(P)],
                         ctypes.c_int),
    "vsr_batch_launch": ([P, P], ctypes.c_int),
    "vsr_batch_params": ([P, P], ctypes.c_int),
    "vsr_batch_destroy": ([P], ctypes.c_int),
    "vsr_trace_batch": ([P, P, P, P, ctypes.c_uint32, P, ctypes.c_int32, P, P], ctypes.c_int),
    "vsr_render": ([P, P, ctypes.c_uint64, P, P, P, P, P, P], ctypes.c_int),
    "vsr_trace_backward": ([P, P, ctypes.c_uint64, P, P, P, P, P, P, P], ctypes.c_int),
    "vsr_render_backward_hits": ([P, P, P, ctypes.c_uint64, P, P, P, P, P], ctypes.c_int),
    "vsr_render_ao": ([P, P, ctypes.c_uint64, P, ctypes.c_uint32, P, ctypes.c_float,
                       ctypes.c_float, P, P, P, P, P], ctypes.c_int),
    "vsr_render_ao_backward": ([P, P, P, ctypes.c_uint64, P, P, P, P], ctypes.c_int),
    "vsr_scene_update": ([P, P, ctypes.c_uint32, P, P], ctypes.c_int),
    "vsr_make_ao_rays": ([P, P, P, ctypes.c_uint64, ctypes.c_uint32, P, ctypes.c_float,
                          ctypes.c_float, P, P], ctypes.c_int),
    "vsr_make_shadow_rays": ([P, P, ctypes.c_uint64, P, ctypes.c_float, P, P], ctypes.c_int),
    "vsr_get_device_error": ([P, ctypes.POINTER(ctypes.c_uint32)], ctypes.c_int),
    "vsr_read_probe": ([P, ctypes.c_uint64, ctypes.c_uint32, P], ctypes.c_int),
    "vsr_read_probe_l1": ([P, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                           P], ctypes.c_int),
    "vsr_bvh_build": ([P, ctypes.c_uint64, P, ctypes.c_uint32, P, ctypes.POINTER(P),
                       ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "vsr_bvh_free": ([P], None),
    "vsr_bvh_validate": ([P, ctypes.c_size_t], ctypes.c_int),
    "vsr_bvh_last_error": ([], ctypes.c_char_p),
}


def lib_path() -> str:
    """Path of the in-tree libvsr.so."""
    return _build.LIB


def lib():
    """Load libvsr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"GPU library not built: {path} is missing "
                               "(run __graft_entry__.build())")
        L = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status: int):
    if status != VSR_OK:
        raise VsrError(status, lib().vsr_last_error().decode())


def vsr_last_error() -> str:
    """Message of the last failure on the calling thread ("" if none)."""
    return lib().vsr_last_error().decode()


def vsr_version() -> int:
    """Library version, e.g. 100 for 0.1.0."""
    return lib().vsr_version()


def intersector(kind="default", dispatch="static", cutoff_u8=128, cutoff_f=0.01,
                freq=40.0, clip_lo=(0.0, 0.0, 0.0), clip_hi=(0.0, 0.0, 0.0)) -> vsr_intersector:
    """vsr_intersector by name: kind in ISECT, dispatch in DISPATCH; the
    cutoffs apply to u8/RGBA8 and to float alpha, ``freq`` to procedural alpha,
    ``clip_lo``/``clip_hi`` to the clip box."""
    return vsr_intersector(ISECT[kind], DISPATCH[dispatch], cutoff_u8, cutoff_f, freq,
                           (ctypes.c_float * 3)(*clip_lo), (ctypes.c_float * 3)(*clip_hi))


def trace_params(block_size=128, persistent=0, refill_threshold=16, blocks_per_sm=0,
                 image_width=0, stack_regs=0, watchdog_iterations=0, watchdog_ms=0,
                 reg_cap_blocks=0, ray_order=0, lockstep=0, octant=0):
    """vsr_trace_params with the library's defaults; ``image_width`` > 0 maps
    each warp to a 4 x 8 pixel tile of a row-major image of that width;
    ``stack_regs`` stack entries are kept in registers; the watchdog fields
    bound persistent loops (0 iterations: no limit; 0 ms: 60 s);
    ``reg_cap_blocks`` selects a register budget (measurement); ``ray_order``
    1 traces in coherence order; ``lockstep`` 1 runs each warp's traversal
    in lock step; ``octant`` 1 gives warps whose rays share a direction
    octant a box test compiled for it."""
    return vsr_trace_params(block_size, persistent, refill_threshold, blocks_per_sm, image_width,
                            stack_regs, watchdog_iterations, watchdog_ms, reg_cap_blocks,
                            ray_order, lockstep, octant)


def params_dict(p: vsr_trace_params) -> dict:
    """The fields of a vsr_trace_params as a dict."""
    return {name: int(getattr(p, name)) for name, _ in vsr_trace_params._fields_}


class Scene:
    """Owns a ``vsr_scene*``; destroyed with the object or ``close()``."""

    def __init__(self, handle: int, ntri: int):
        self.handle = handle
        self.ntri = ntri

    def close(self):
        if self.handle:
            lib().vsr_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tex_array(textures):
    keep = []
    arr = (vsr_texture_desc * max(len(textures), 1))()
    for k, t in enumerate(textures):
        tx = np.ascontiguousarray(t.texels)
        keep.append(tx)
        arr[k] = vsr_texture_desc(TEX_FMT[t.fmt], t.w, t.h, 0, tx.ctypes.data)
    return arr, keep


def vsr_scene_create_indexed(verts, idx, uvs, geom_id, textures) -> Scene:
    """Copy indexed host geometry, texture coordinates and textures to the
    current CUDA device."""
    v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
    i = np.ascontiguousarray(idx, np.uint32).reshape(-1, 3)
    uv = np.ascontiguousarray(uvs, np.float32).reshape(-1, 3, 2)
    g = np.ascontiguousarray(geom_id, np.uint32).reshape(-1)
    tarr, keep = _tex_array(textures)
    out = P()
    st = lib().vsr_scene_create_indexed(v.ctypes.data, v.shape[0], i.ctypes.data, uv.ctypes.data,
                                        g.ctypes.data, i.shape[0], tarr, len(textures),
                                        ctypes.byref(out))
    del keep
    _check(st)
    return Scene(out.value, i.shape[0])


def vsr_scene_create(verts_xyz, uvs, geom_id, textures) -> Scene:
    """Copy non-indexed host triangles (float32 [m, 9]), per-corner texture
    coordinates and textures to the current CUDA device."""
    v = np.ascontiguousarray(verts_xyz, np.float32).reshape(-1, 9)
    uv = np.ascontiguousarray(uvs, np.float32).reshape(-1, 3, 2)
    g = np.ascontiguousarray(geom_id, np.uint32).reshape(-1)
    tarr, keep = _tex_array(textures)
    out = P()
    st = lib().vsr_scene_create(v.ctypes.data, uv.ctypes.data, g.ctypes.data, v.shape[0], tarr,
                                len(textures), ctypes.byref(out))
    del keep
    _check(st)
    return Scene(out.value, v.shape[0])


def vsr_scene_destroy(scene: Scene):
    """Free the scene's device memory."""
    scene.close()


def vsr_bvh_load(scene: Scene, blob: np.ndarray):
    """Validate a BVH blob (uint8) and convert it to the device layout."""
    b = np.ascontiguousarray(blob, np.uint8)
    _check(lib().vsr_bvh_load(scene.handle, b.ctypes.data if b.size else None, b.size))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


def vsr_trace_multi(scene: Scene, rays, isect: vsr_intersector, max_hits: int, hits,
                    counters=None, params: vsr_trace_params | None = None, stream=None):
    """First ``max_hits`` accepted hits per ray, nearest first, into ``hits``
    (cuda float32 [n * max_hits, 4] or [n, max_hits, 4])."""
    n = int(rays.shape[0])
    _check(lib().vsr_trace_multi(scene.handle, _ptr(rays), n, ctypes.byref(isect), int(max_hits),
                                 _ptr(hits), _ptr(counters),
                                 ctypes.byref(params) if params else None, _stream(stream)))


class Instances:
    """Owns a ``vsr_instances*`` and keeps its meshes alive."""

    def __init__(self, handle: int, meshes):
        self.handle = handle
        self.meshes = list(meshes)

    def close(self):
        if self.handle:
            lib().vsr_instances_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vsr_instances_create(meshes, inst_mesh, world_to_object, top_blob) -> Instances:
    """Instance set over ``meshes`` (Scene objects with BVHs): inst_mesh uint32
    [m], world_to_object float32 [m, 12], top_blob over the instances' boxes."""
    im = np.ascontiguousarray(inst_mesh, np.uint32).reshape(-1)
    w = np.ascontiguousarray(world_to_object, np.float32).reshape(-1, 12)
    tb = np.ascontiguousarray(top_blob, np.uint8)
    arr = (P * len(meshes))(*[m.handle for m in meshes])
    out = P()
    _check(lib().vsr_instances_create(arr, len(meshes), im.ctypes.data if im.size else None,
                                      w.ctypes.data if w.size else None, im.shape[0],
                                      tb.ctypes.data, tb.nbytes, ctypes.byref(out)))
    return Instances(out.value, meshes)


def vsr_trace_instances(inst: Instances, rays, isect: vsr_intersector, query, hits,
                        inst_ids=None, counters=None, params: vsr_trace_params | None = None,
                        stream=None):
    """Trace ``rays`` through an instance set into ``hits`` [n,4] (and the
    instance ids [n])."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    _check(lib().vsr_trace_instances(inst.handle, _ptr(rays), int(rays.shape[0]),
                                     ctypes.byref(isect), q, _ptr(hits), _ptr(inst_ids),
                                     _ptr(counters), ctypes.byref(params) if params else None,
                                     _stream(stream)))


def vsr_instances_device_error(inst: Instances) -> int:
    """Read and clear the instance set's device error word (synchronous)."""
    w = ctypes.c_uint32()
    _check(lib().vsr_instances_device_error(inst.handle, ctypes.byref(w)))
    return int(w.value)


def vsr_path_trace(scene: Scene, rays, isect: vsr_intersector, path: vsr_path_params, dirs,
                   radiance, segments=None, params: vsr_trace_params | None = None, stream=None):
    """Diffuse path tracing of ``rays`` (cuda float32 [n,8]) into radiance [n,3];
    dirs float32 [n * bounces, 3] local unit directions."""
    _check(lib().vsr_path_trace(scene.handle, _ptr(rays), int(rays.shape[0]), ctypes.byref(isect),
                                ctypes.byref(path), _ptr(dirs), _ptr(radiance), _ptr(segments),
                                ctypes.byref(params) if params else None, _stream(stream)))


def vsr_trace(scene: Scene, rays, isect: vsr_intersector, query, hits, counters=None,
              params: vsr_trace_params | None = None, stream=None):
    """Trace ``rays`` (cuda float32 [n,8]) into ``hits`` (cuda float32 [n,4])."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    n = int(rays.shape[0])
    _check(lib().vsr_trace(scene.handle, _ptr(rays), n, ctypes.byref(isect), q, _ptr(hits),
                           _ptr(counters), ctypes.byref(params) if params else None,
                           _stream(stream)))


def vsr_trace_tune(scene: Scene, rays, isect: vsr_intersector, query, hits, image_width=0,
                   stream=None) -> vsr_trace_params:
    """Time launch configurations on ``rays`` (synchronous; ``hits`` is
    overwritten) and keep the fastest in the scene for vsr_trace calls with
    params None; returns it."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    out = vsr_trace_params()
    _check(lib().vsr_trace_tune(scene.handle, _ptr(rays), int(rays.shape[0]), ctypes.byref(isect),
                                q, int(image_width), _ptr(hits), ctypes.byref(out),
                                _stream(stream)))
    return out


def vsr_trace_tuned_params(scene: Scene, isect: vsr_intersector, query):
    """The configuration vsr_trace uses with params None for this scene,
    intersector and query, or None if none was tuned yet."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    out = vsr_trace_params()
    st = lib().vsr_trace_tuned_params(scene.handle, ctypes.byref(isect), q, ctypes.byref(out))
    if st == VSR_ERR_STATE:
        return None
    _check(st)
    return out


def vsr_trace_persistent_noalloc(scene: Scene, rays, isect: vsr_intersector, query, hits,
                                 counters=None, params: vsr_trace_params | None = None,
                                 stream=None, n=None):
    """Persistent trace whose ray counter lives in the library's static device
    array (no allocation by the library).  Calls that overlap on the GPU race."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    count = int(rays.shape[0]) if n is None else int(n)
    _check(lib().vsr_trace_persistent_noalloc(
        scene.handle, _ptr(rays), count, ctypes.byref(isect), q, _ptr(hits), _ptr(counters),
        ctypes.byref(params) if params else None, _stream(stream)))


def vsr_trace_stats(scene: Scene, rays, isect: vsr_intersector, query, hits, stats,
                    stream=None):
    """Trace as vsr_trace and write per-ray (box tests, triangle tests,
    intersector calls, texture fetches) into ``stats`` (int32 [n, 4])."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    _check(lib().vsr_trace_stats(scene.handle, _ptr(rays), int(rays.shape[0]),
                                 ctypes.byref(isect), q, _ptr(hits), _ptr(stats),
                                 _stream(stream)))


class Batch:
    """Owns a ``vsr_batch*`` (see vsr_batch_create)."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle:
            lib().vsr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_arrays(scenes, rays, hits):
    nb = len(scenes)
    sc = (P * nb)(*[s.handle for s in scenes])
    rp = (P * nb)(*[_ptr(r) for r in rays])
    hp = (P * nb)(*[_ptr(h) for h in hits])
    ns = (ctypes.c_uint64 * nb)(*[int(r.shape[0]) for r in rays])
    return nb, sc, rp, hp, ns


def vsr_batch_create(scenes, rays, hits, isect: vsr_intersector, query,
                     params: vsr_trace_params | None = None) -> Batch:
    """Prepare one persistent launch over many scenes (lists of equal length)."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    nb, sc, rp, hp, ns = _batch_arrays(scenes, rays, hits)
    out = P()
    _check(lib().vsr_batch_create(sc, rp, ns, hp, nb, ctypes.byref(isect), q,
                                  ctypes.byref(params) if params else None, ctypes.byref(out)))
    return Batch(out.value, (scenes, rays, hits))


def vsr_batch_launch(batch: Batch, stream=None):
    """Replay the batch's launch on ``stream``."""
    _check(lib().vsr_batch_launch(batch.handle, _stream(stream)))


def vsr_batch_params(batch: Batch) -> vsr_trace_params:
    """The launch configuration the batch was tuned to."""
    p = vsr_trace_params()
    _check(lib().vsr_batch_params(batch.handle, ctypes.byref(p)))
    return p


def vsr_batch_destroy(batch: Batch):
    """Free the batch (its scenes and buffers stay the caller's)."""
    batch.close()


def vsr_trace_batch(scenes, rays, hits, isect: vsr_intersector, query,
                    params: vsr_trace_params | None = None, stream=None):
    """Trace many scenes' ray batches in one persistent launch (untuned)."""
    q = QUERY[query] if isinstance(query, str) else int(query)
    nb, sc, rp, hp, ns = _batch_arrays(scenes, rays, hits)
    _check(lib().vsr_trace_batch(sc, rp, ns, hp, nb, ctypes.byref(isect), q,
                                 ctypes.byref(params) if params else None, _stream(stream)))


def shade_params(light, background=(0.0, 0.0, 0.0), grad_tex=0) -> vsr_shade_params:
    """vsr_shade_params: directional light, background colour and the texture
    whose texels receive gradients."""
    return vsr_shade_params((ctypes.c_float * 3)(*[float(x) for x in light]),
                            (ctypes.c_float * 3)(*[float(x) for x in background]),
                            grad_tex, 0)


def vsr_render(scene: Scene, rays, isect: vsr_intersector, shade: vsr_shade_params, image,
               hits=None, params: vsr_trace_params | None = None, stream=None):
    """Closest-hit trace plus diffuse textured shading into image (float32 [n,3])."""
    _check(lib().vsr_render(scene.handle, _ptr(rays), int(rays.shape[0]), ctypes.byref(isect),
                            ctypes.byref(shade), _ptr(image), _ptr(hits),
                            ctypes.byref(params) if params else None, _stream(stream)))


def vsr_trace_backward(scene: Scene, rays, isect: vsr_intersector, shade: vsr_shade_params,
                       dL_dimage, grad_verts, grad_texels=None,
                       params: vsr_trace_params | None = None, stream=None):
    """Accumulate dL/dverts and dL/dtexels (texture shade.grad_tex) at fixed visibility."""
    _check(lib().vsr_trace_backward(scene.handle, _ptr(rays), int(rays.shape[0]),
                                    ctypes.byref(isect), ctypes.byref(shade), _ptr(dL_dimage),
                                    _ptr(grad_verts), _ptr(grad_texels),
                                    ctypes.byref(params) if params else None, _stream(stream)))


def vsr_render_backward_hits(scene: Scene, rays, hits, shade: vsr_shade_params, dL_dimage,
                             grad_verts, grad_texels=None, stream=None):
    """The adjoint of vsr_render from its saved hit records [n,4] (no
    re-trace): accumulates dL/dverts and dL/dtexels like vsr_trace_backward."""
    _check(lib().vsr_render_backward_hits(scene.handle, _ptr(rays), _ptr(hits),
                                          int(rays.shape[0]), ctypes.byref(shade),
                                          _ptr(dL_dimage), _ptr(grad_verts), _ptr(grad_texels),
                                          _stream(stream)))


def vsr_render_ao(scene: Scene, rays, isect: vsr_intersector, spp: int, xi, ao_tmax: float,
                  eps: float, shade: vsr_shade_params, image, hits, occlusion, stream=None):
    """albedo(uv) * (1 - occluded fraction of spp AO rays) into image [n,3];
    the primary hits [n,4] and occluded fractions [n] are written too."""
    _check(lib().vsr_render_ao(scene.handle, _ptr(rays), int(rays.shape[0]), ctypes.byref(isect),
                               spp, _ptr(xi), float(ao_tmax), float(eps), ctypes.byref(shade),
                               _ptr(image), _ptr(hits), _ptr(occlusion), _stream(stream)))


def vsr_render_ao_backward(scene: Scene, hits, occlusion, shade: vsr_shade_params, dL_dimage,
                           grad_texels, stream=None):
    """Accumulate dL/dtexels of shade.grad_tex for vsr_render_ao from its saved
    hits and occlusion (fixed visibility)."""
    _check(lib().vsr_render_ao_backward(scene.handle, _ptr(hits), _ptr(occlusion),
                                        int(hits.shape[0]), ctypes.byref(shade),
                                        _ptr(dL_dimage), _ptr(grad_texels), _stream(stream)))


def vsr_scene_update(scene: Scene, verts=None, tex_index=0, texels=None, stream=None):
    """Replace vertex positions and/or one texture's texels (device tensors)."""
    _check(lib().vsr_scene_update(scene.handle, _ptr(verts), tex_index, _ptr(texels),
                                  _stream(stream)))


def vsr_make_ao_rays(scene: Scene, prim_rays, prim_hits, spp: int, xi, tmax: float, eps: float,
                     out, stream=None):
    """Ambient-occlusion rays (spp per primary ray) into out (float32 [n*spp, 8])."""
    _check(lib().vsr_make_ao_rays(scene.handle, _ptr(prim_rays), _ptr(prim_hits),
                                  int(prim_rays.shape[0]), spp, _ptr(xi), float(tmax),
                                  float(eps), _ptr(out), _stream(stream)))


def vsr_make_shadow_rays(prim_rays, prim_hits, light, eps: float, out, stream=None):
    """Rays from the primary hit points toward the directional light into
    ``out`` (float32 [n, 8]); misses give inactive rays."""
    l = (ctypes.c_float * 3)(*[float(x) for x in light])
    _check(lib().vsr_make_shadow_rays(_ptr(prim_rays), _ptr(prim_hits), int(prim_rays.shape[0]),
                                      l, float(eps), _ptr(out), _stream(stream)))


def vsr_read_probe(buf, reps: int = 1, stream=None):
    """One launch reading all of ``buf`` (a 16-byte aligned cuda tensor whose
    size is a multiple of 16 bytes) ``reps`` times with L2-cached loads."""
    nbytes = int(buf.numel() * buf.element_size())
    _check(lib().vsr_read_probe(_ptr(buf), nbytes, int(reps), _stream(stream)))


def vsr_read_probe_l1(buf, reps: int = 1, stream=None) -> int:
    """One launch in which every block reads all of ``buf`` (at most 64 KB)
    ``reps`` times through L1; returns the bytes the launch reads."""
    nbytes = int(buf.numel() * buf.element_size())
    out = ctypes.c_uint64()
    _check(lib().vsr_read_probe_l1(_ptr(buf), nbytes, int(reps), ctypes.byref(out),
                                   _stream(stream)))
    return int(out.value)


def vsr_get_device_error(scene: Scene) -> int:
    """Read and clear the scene's device error word (synchronous)."""
    w = ctypes.c_uint32()
    _check(lib().vsr_get_device_error(scene.handle, ctypes.byref(w)))
    return int(w.value)


# ---------------------------------------------------------------- helpers


def prim_ids(hits):
    """uint32 primitive ids of a float32 [n,4] hit tensor, as int64."""
    import torch
    return hits.contiguous().view(torch.int32)[:, 3].to(torch.int64) & 0xFFFFFFFF


def scene_from_inputs(sc, blob: np.ndarray) -> Scene:
    """Upload a generated scene (``inputs.scenes.Scene``) and its BVH blob."""
    s = vsr_scene_create_indexed(sc.verts, sc.idx, sc.uvs, sc.geom_id, sc.textures)
    vsr_bvh_load(s, blob)
    return s


def trace(scene: Scene, rays, kind="default", query="closest", dispatch="static",
          counters=False, params=None, stream=None, **kw):
    """Allocate hits (and counters for COUNT) and trace; returns (hits, counters)."""
    import torch
    n = rays.shape[0]
    hits = torch.empty((n, 4), dtype=torch.float32, device=rays.device)
    cnt = torch.empty((n, 2), dtype=torch.int32, device=rays.device) if counters else None
    vsr_trace(scene, rays, intersector(kind, dispatch, **kw), query, hits, cnt, params, stream)
    return hits, cnt
