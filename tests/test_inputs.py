"""The seeded input producers (no GPU): the BVH builder's output does not
depend on its thread count, is structurally valid, and a traversal over it
finds exactly the brute-force closest hits on a scene large enough to use
the parallel subtree builds."""
import numpy as np

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import _lib, bvh_validate, scenes


def test_builder_is_deterministic_across_thread_counts(monkeypatch):
    rng = np.random.default_rng(9)
    corners = scenes.random_quads(rng, 20_000, 0.0, 1.0, 0.01, 0.05)
    verts, idx, _ = scenes._quads_to_tris(corners)
    monkeypatch.setenv("VSR_BUILD_THREADS", "1")
    one = _lib.bvh_build(verts, idx)
    monkeypatch.setenv("VSR_BUILD_THREADS", "7")
    seven = _lib.bvh_build(verts, idx)
    assert bvh_validate(one) == "" and np.array_equal(one, seven)


def test_parallel_build_traversal_equals_brute_force():
    rng = np.random.default_rng(10)
    corners = scenes.random_quads(rng, 12_000, 0.0, 1.0, 0.01, 0.05)
    verts, idx, uvs = scenes._quads_to_tris(corners)
    sc = scenes.Scene("q", verts, idx, uvs, np.zeros(len(idx), np.uint32),
                      [scenes.disc_alpha_u8(64, 0.4)])
    rays = scenes.camera_rays_random(np.random.default_rng(2), 3000)
    blob = sc.bvh()
    for kind in ("default", "alpha_tex"):
        hb, _ = O.trace_bvh(sc, blob, rays, kind, "closest")
        hl, _ = O.trace_list(sc, rays, kind, "closest")
        assert np.array_equal(hb["prim"], hl["prim"]) and np.array_equal(hb["t"], hl["t"])
