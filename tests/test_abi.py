"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; host-side argument checks reject bad calls before
any CUDA work (no GPU needed)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_1912_12786_gb300 import _build
from paper_1912_12786_gb300.inputs import scenes, bvh_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^(?:vsr_status|const char\s*\*|int32_t|int|void)\s+\*?\s*(vsr_\w+)\s*\(", re.M)


@pytest.fixture(scope="module")
def lib():
    path = _build.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        with open(h) as f:
            names.update(DECL.findall(f.read()))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("vsr_scene_create", "vsr_scene_create_indexed", "vsr_bvh_load", "vsr_trace",
                     "vsr_bvh_build", "vsr_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_boundary():
    from paper_1912_12786_gb300 import vsr
    for n in ("vsr_scene_create", "vsr_scene_create_indexed", "vsr_scene_destroy", "vsr_bvh_load",
              "vsr_trace", "vsr_trace_stats", "vsr_make_shadow_rays", "vsr_get_device_error",
              "vsr_last_error", "vsr_version"):
        assert callable(getattr(vsr, n)), n


def test_host_only_calls(lib):
    lib.vsr_version.restype = ctypes.c_int32
    assert lib.vsr_version() == 100
    lib.vsr_last_error.restype = ctypes.c_char_p
    P = ctypes.c_void_p
    lib.vsr_scene_create.argtypes = [P, P, P, ctypes.c_uint32, P, ctypes.c_uint32, P]
    assert lib.vsr_scene_create(None, None, None, 0, None, 0, None) == 1  # VSR_ERR_ARG
    assert b"out is null" in lib.vsr_last_error()
    lib.vsr_trace.argtypes = [P, P, ctypes.c_uint64, P, ctypes.c_int32, P, P, P, P]
    assert lib.vsr_trace(None, None, 0, None, 0, None, None, None, None) == 1
    assert b"scene is null" in lib.vsr_last_error()
    lib.vsr_bvh_load.argtypes = [P, P, ctypes.c_size_t]
    assert lib.vsr_bvh_load(None, None, 0) == 1


def test_library_builder_matches_input_builder(lib):
    """libvsr exports the same host builder the input generators use."""
    sc, _ = scenes.small_quads(n_quads=64)
    ref = bvh_build(sc.verts, sc.idx)
    P = ctypes.c_void_p
    lib.vsr_bvh_build.argtypes = [P, ctypes.c_uint64, P, ctypes.c_uint32, P,
                                  ctypes.POINTER(P), ctypes.POINTER(ctypes.c_size_t)]
    lib.vsr_bvh_free.argtypes = [P]
    out, nbytes = P(), ctypes.c_size_t()
    v = np.ascontiguousarray(sc.verts)
    i = np.ascontiguousarray(sc.idx)
    assert lib.vsr_bvh_build(v.ctypes.data, v.shape[0], i.ctypes.data, i.shape[0], None,
                             ctypes.byref(out), ctypes.byref(nbytes)) == 0
    got = np.frombuffer(ctypes.string_at(out.value, nbytes.value), np.uint8)
    lib.vsr_bvh_free(out)
    assert np.array_equal(got, ref)


def test_headers_are_plain_c_and_match_the_binding(tmp_path):
    """The boundary headers compile as pedantic C99 (no C++ in the ABI), and
    every struct the binding passes has the size ctypes gives it."""
    import shutil
    import subprocess
    from paper_1912_12786_gb300 import vsr as V
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = ["vsr_ray", "vsr_hit", "vsr_intersector", "vsr_trace_params", "vsr_shade_params",
               "vsr_path_params", "vsr_texture_desc", "vsr_build_params", "vsr_bvh_node"]
    src = tmp_path / "abi.c"
    src.write_text('#include <stdio.h>\n#include "vsr.h"\n#include "vsr_bvh.h"\nint main(void) {\n' +
                   "".join(f'    printf("%zu\\n", sizeof({s}));\n' for s in structs) +
                   "    return 0;\n}\n")
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                    _build.INCLUDE, str(src), "-o", str(exe)], check=True)
    sizes = dict(zip(structs, map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                                      text=True).stdout.split())))
    assert sizes["vsr_ray"] == 32 and sizes["vsr_hit"] == 16 and sizes["vsr_bvh_node"] == 32
    for name in ("vsr_intersector", "vsr_trace_params", "vsr_shade_params", "vsr_path_params",
                 "vsr_texture_desc"):
        assert sizes[name] == ctypes.sizeof(getattr(V, name)), name
    from paper_1912_12786_gb300.inputs import _lib
    assert sizes["vsr_build_params"] == ctypes.sizeof(_lib.BuildParams)
