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


def test_path_dirs_are_cosine_distributed():
    """Local bounce directions: unit vectors in the upper hemisphere whose
    cos(theta) = z has density 2 z on [0, 1] (cosine-weighted), so
    E[z] = 2/3, E[z^2] = 1/2, and the azimuth is uniform (E[x] = E[y] = 0)."""
    d = scenes.path_dirs(50000, 2, seed=3).astype(np.float64)
    assert d.shape == (100000, 3)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    assert np.all(d[:, 2] >= 0)
    se = 4.0 / np.sqrt(len(d))
    assert abs(d[:, 2].mean() - 2 / 3) < se
    assert abs((d[:, 2] ** 2).mean() - 0.5) < se
    assert abs(d[:, 0].mean()) < se and abs(d[:, 1].mean()) < se
    assert np.array_equal(scenes.path_dirs(10, 3, seed=5), scenes.path_dirs(10, 3, seed=5))


def test_instance_world_boxes_enclose_placed_geometry():
    """Every instance's world box holds its mesh's vertices under the float64
    placement, and the float32 world-to-object map inverts the placement to
    float32 accuracy."""
    for iset, _ in (scenes.instanced_small(), scenes.instanced_small(n_inst=20, seed=4)):
        for i, (mid, a) in enumerate(zip(iset.inst_mesh, iset.o2w)):
            m = iset.meshes[mid]
            v = m.verts[np.asarray(m.idx).reshape(-1)].astype(np.float64)
            w = v @ a[:, :3].T + a[:, 3]
            assert np.all(w >= iset.boxes[i, :3]) and np.all(w <= iset.boxes[i, 3:])
            inv = iset.w2o[i].reshape(3, 4).astype(np.float64)
            back = w @ inv[:, :3].T + inv[:, 3]
            assert np.allclose(back, v, atol=1e-5 * (1 + np.abs(v).max()))
