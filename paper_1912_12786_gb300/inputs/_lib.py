"""Build and load the host-only input library (BVH builder, Poisson disc).

The library is compiled from ``bvh_build.cpp`` with g++ on first use.  It
contains no ray arithmetic; it produces the BVH blob and point sets that both
the GPU path and the oracle consume as data.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(os.path.dirname(_HERE))
_SRC = os.path.join(_HERE, "bvh_build.cpp")
_HDR = os.path.join(_ROOT, "include", "vsr_bvh.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libvsr_inputs.so")
_lock = threading.Lock()
_lib = None


class BuildParams(ctypes.Structure):
    _fields_ = [("leaf_max", ctypes.c_uint32), ("bins", ctypes.c_uint32),
                ("traversal_cost", ctypes.c_float)]


def build(force: bool = False) -> str:
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-I", os.path.join(_ROOT, "include"), _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L.vsr_bvh_build.argtypes = [P, ctypes.c_uint64, P, ctypes.c_uint32, P,
                                    ctypes.POINTER(ctypes.c_void_p),
                                    ctypes.POINTER(ctypes.c_size_t)]
        L.vsr_bvh_build_boxes.argtypes = [P, ctypes.c_uint32, P, ctypes.POINTER(ctypes.c_void_p),
                                          ctypes.POINTER(ctypes.c_size_t)]
        L.vsr_bvh_free.argtypes = [P]
        L.vsr_bvh_free.restype = None
        L.vsr_bvh_validate.argtypes = [P, ctypes.c_size_t]
        L.vsr_bvh_last_error.restype = ctypes.c_char_p
        L.vsr_inputs_poisson_disc.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                              ctypes.c_uint32, ctypes.c_uint64, P,
                                              ctypes.POINTER(ctypes.c_uint32)]
        _lib = L
    return _lib


def bvh_build(verts: np.ndarray, idx: np.ndarray | None, leaf_max: int = 4,
              bins: int = 32, traversal_cost: float = 1.0) -> np.ndarray:
    """Binned-SAH BVH over indexed triangles; returns the blob as uint8 array."""
    L = lib()
    verts = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
    if idx is not None:
        idx = np.ascontiguousarray(idx, np.uint32).reshape(-1, 3)
        ntri = idx.shape[0]
        ip = idx.ctypes.data
    else:
        ntri = verts.shape[0] // 3
        ip = None
    p = BuildParams(leaf_max, bins, traversal_cost)
    out = ctypes.c_void_p()
    nbytes = ctypes.c_size_t()
    rc = L.vsr_bvh_build(verts.ctypes.data, verts.shape[0], ip, ntri, ctypes.byref(p),
                         ctypes.byref(out), ctypes.byref(nbytes))
    if rc != 0:
        raise ValueError(L.vsr_bvh_last_error().decode())
    try:
        blob = np.frombuffer(ctypes.string_at(out.value, nbytes.value), np.uint8).copy()
    finally:
        L.vsr_bvh_free(out)
    return blob


def bvh_build_boxes(boxes: np.ndarray, leaf_max: int = 4, bins: int = 32,
                    traversal_cost: float = 1.0) -> np.ndarray:
    """Binned-SAH BVH over boxes float32 [n, 6] (lo.xyz, hi.xyz); primitive i
    of the returned blob is box i."""
    L = lib()
    boxes = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    p = BuildParams(leaf_max, bins, traversal_cost)
    out = ctypes.c_void_p()
    nbytes = ctypes.c_size_t()
    rc = L.vsr_bvh_build_boxes(boxes.ctypes.data if boxes.size else None, boxes.shape[0],
                               ctypes.byref(p), ctypes.byref(out), ctypes.byref(nbytes))
    if rc != 0:
        raise ValueError(L.vsr_bvh_last_error().decode())
    try:
        blob = np.frombuffer(ctypes.string_at(out.value, nbytes.value), np.uint8).copy()
    finally:
        L.vsr_bvh_free(out)
    return blob


def bvh_validate(blob: np.ndarray) -> str:
    """'' when the blob is structurally valid, else the reason."""
    L = lib()
    b = np.ascontiguousarray(blob, np.uint8)
    rc = L.vsr_bvh_validate(b.ctypes.data if b.size else None, b.size)
    return "" if rc == 0 else L.vsr_bvh_last_error().decode()


def poisson_disc(w: float, h: float, r: float, max_points: int, seed: int) -> np.ndarray:
    L = lib()
    out = np.zeros((max_points, 2), np.float32)
    n = ctypes.c_uint32()
    rc = L.vsr_inputs_poisson_disc(w, h, r, max_points, seed, out.ctypes.data,
                                   ctypes.byref(n))
    if rc != 0:
        raise ValueError(L.vsr_bvh_last_error().decode())
    return out[: n.value]
