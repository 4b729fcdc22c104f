"""Instanced traces on the GPU vs the oracle, through the C ABI (needs a GB300).

Bar: hits (t, u, v, prim), instance ids and bvh_costs counters bit-identical
to the oracle's two-level traversal (top-level BVH over the instances, each
mesh's own BVH below, the intersector passed on); near-tie rays excluded as
for single meshes.  Closest-hit ties between coincident instances go to the
lower instance id.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = ["none", "default", "alpha_tex", "proc_alpha", "count"]


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    return vsr


def _upload(V, I):
    ms = [V.scene_from_inputs(m, b) for m, b in zip(I.meshes, I.blobs)]
    return V.vsr_instances_create(ms, I.inst_mesh, I.w2o, I.top)


@pytest.fixture(scope="module")
def small(V):
    I, rays = scenes.instanced_small()
    X = _upload(V, I)
    yield I, rays, X
    X.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _gpu(V, X, rays, kind, query, params=None, dispatch="static"):
    n = rays.shape[0]
    hits = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
    ids = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    cnt = torch.full((n, 2), -1, dtype=torch.int32, device="cuda") if kind == "count" else None
    V.vsr_trace_instances(X, rays, V.intersector(kind, dispatch), query, hits, ids, cnt, params)
    torch.cuda.synchronize()
    return (hits.cpu().numpy(), ids.cpu().numpy().view(np.uint32),
            None if cnt is None else cnt.cpu().numpy().view(np.uint32))


def _oracle(I, rays, kind, query):
    return O.trace_instances(list(zip(I.meshes, I.blobs)), I.inst_mesh, I.w2o, rays, kind, query,
                             I.top)


def _compare(got, ids, ref, rids, st, label):
    r = O.hits_raw(ref)
    ok = st[:, 3] == 0
    bad = (np.any(got.view(np.uint32) != r.view(np.uint32), axis=1) | (ids != rids)) & ok
    assert not bad.any(), f"{label}: {int(bad.sum())} rays differ"
    return ok


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", KINDS)
def test_small_all_intersectors(V, small, kind, query):
    I, rays, X = small
    ref, rids, st = _oracle(I, rays, kind, query)
    got, ids, cnt = _gpu(V, X, _dev(rays), kind, query)
    ok = _compare(got, ids, ref, rids, st, f"{kind}/{query}")
    if cnt is not None:
        assert np.array_equal(cnt[ok], st[ok, :2])
    assert len(np.unique(ids[ids != O.NONE])) >= 4
    assert V.vsr_instances_device_error(X) == 0
    for m in X.meshes:
        assert V.vsr_get_device_error(m) == 0


@pytest.mark.parametrize("n,width", [(1, 0), (33, 0), (4097, 37), (65536, 256)])
def test_ragged_and_pixel_tiles(V, small, n, width):
    I, rays, X = small
    sel = np.resize(rays[::-1], (n, 8))
    ref, rids, st = _oracle(I, sel, "alpha_tex", "closest")
    got, ids, _ = _gpu(V, X, _dev(sel), "alpha_tex", "closest", V.trace_params(image_width=width))
    _compare(got, ids, ref, rids, st, f"n={n} width={width}")


def test_coincident_instances_tie_to_the_lower_id(V):
    from test_oracle_pins import two_tri_scene
    sc, _ = two_tri_scene()
    ident = np.hstack([np.eye(3), np.zeros((3, 1))])
    moved = np.hstack([np.eye(3), np.array([[10.0], [0.0], [0.0]])])
    I = scenes.make_instance_set("two", [sc], [0, 0, 0], [moved, ident, ident])
    X = _upload(V, I)
    try:
        rays = np.array([[0, 0, 0, 0, 0, 0, 1, np.inf], [10, 0, 0, 0, 0, 0, 1, np.inf],
                         [0, 0, 4, 0, 0, 0, -1, np.inf]], np.float32)
        got, ids, _ = _gpu(V, X, _dev(rays), "default", "closest")
        assert list(ids) == [1, 0, 1]
        assert list(got[:, 3].view(np.uint32)) == [0, 0, 1] and list(got[:, 0]) == [1.0, 1.0, 1.0]
    finally:
        X.close()


def test_argument_checks(V, small):
    I, rays, X = small
    d = _dev(rays[:64])
    hits = torch.empty((64, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="lockstep 0"):
        V.vsr_trace_instances(X, d, V.intersector("default"), "closest", hits, None, None,
                              V.trace_params(persistent=1, lockstep=1))
    with pytest.raises(V.VsrError, match="refill_threshold"):
        V.vsr_trace_instances(X, d, V.intersector("default"), "closest", hits, None, None,
                              V.trace_params(persistent=1, refill_threshold=0))
    ms = X.meshes
    with pytest.raises(V.VsrError, match="missing mesh"):
        V.vsr_instances_create(ms, np.full(len(I.inst_mesh), 5, np.uint32), I.w2o, I.top)
    with pytest.raises(V.VsrError, match="different number of instances"):
        V.vsr_instances_create(ms, I.inst_mesh[:-1], I.w2o[:-1], I.top)
    bad = I.w2o.copy()
    bad[2, 5] = np.nan
    with pytest.raises(V.VsrError, match="non-finite"):
        V.vsr_instances_create(ms, I.inst_mesh, bad, I.top)
    bare = V.vsr_scene_create_indexed(I.meshes[0].verts, I.meshes[0].idx, I.meshes[0].uvs,
                                      I.meshes[0].geom_id, I.meshes[0].textures)
    with pytest.raises(V.VsrError, match="no BVH"):
        V.vsr_instances_create([bare, ms[1]], I.inst_mesh, I.w2o, I.top)
    bare.close()


def test_instanced_forest_sample(V):
    """The forest built from 64 turned copies of one tile plus the ground:
    the full 1920x1080 frame, primary closest hits and shadow any hits with
    the alpha intersector in the bench's launch configuration, a seeded
    sample against the oracle."""
    import bench
    I, rays = scenes.instanced_forest()
    X = _upload(V, I)
    try:
        p = bench.default_params(V)
        got, ids, _ = _gpu(V, X, _dev(rays), "alpha_tex", "closest", p)
        rng = np.random.default_rng(17)
        sel = np.sort(rng.choice(len(rays), 4000, replace=False))
        ref, rids, st = _oracle(I, rays[sel], "alpha_tex", "closest")
        ok = _compare(got[sel], ids[sel], ref, rids, st, "forest primary")
        assert ok.mean() > 0.99
        # the ground and the first row of tiles hide the rest of the forest
        seen = np.unique(ids[ids != O.NONE])
        assert 0 in seen and len(seen) >= 3
        light, eps = scenes.light_dir_f32(), np.float32(1e-4 * 100.0 * np.sqrt(3))
        sref = O.shadow_rays(rays[sel], O.hits_raw(ref), light, float(eps))
        sh_ref, sh_ids, sh_st = _oracle(I, sref, "alpha_tex", "any")
        sh, shi, _ = _gpu(V, X, _dev(sref), "alpha_tex", "any", p)
        _compare(sh, shi, sh_ref, sh_ids, sh_st, "forest shadow")
        assert V.vsr_instances_device_error(X) == 0
    finally:
        X.close()


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", KINDS)
def test_dynamic_dispatch_equals_static(V, small, kind, query):
    """Callback dispatch through the instance set (the callbacks see each
    instance's mesh) gives the same hits, instance ids and counters as the
    compiled-in intersector, bit for bit, and so the oracle's."""
    I, rays, X = small
    d = _dev(rays)
    a = _gpu(V, X, d, kind, query)
    b = _gpu(V, X, d, kind, query, dispatch="dynamic")
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert np.array_equal(a[1], b[1])
    if kind == "count":
        assert np.array_equal(a[2], b[2])
    c = _gpu(V, X, d, kind, query, V.trace_params(image_width=128), dispatch="dynamic")
    assert np.array_equal(a[0].view(np.uint32), c[0].view(np.uint32))
    assert V.vsr_instances_device_error(X) == 0


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dispatch", ["static", "dynamic"])
def test_persistent_matches_oracle(V, small, kind, query, dispatch):
    """Persistent warps, each lane's two-level traversal resumable step by
    step (a mesh step, or the top level's advance to the next instance whose
    mesh root the ray hits): hits, instance ids and counters are the
    oracle's."""
    I, rays, X = small
    ref, rids, st = _oracle(I, rays, kind, query)
    d = _dev(rays)
    for c in (dict(refill_threshold=16), dict(refill_threshold=1, block_size=64),
              dict(refill_threshold=32, image_width=128, block_size=256)):
        p = V.trace_params(persistent=1, watchdog_ms=10_000, **c)
        got, ids, cnt = _gpu(V, X, d, kind, query, p, dispatch=dispatch)
        ok = _compare(got, ids, ref, rids, st, f"{dispatch} {kind}/{query} {c}")
        if cnt is not None:
            assert np.array_equal(cnt[ok], st[ok, :2])
    assert V.vsr_instances_device_error(X) == 0
    for m in X.meshes:
        assert V.vsr_get_device_error(m) == 0


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_persistent_ragged(V, small, n):
    I, rays, X = small
    sel = np.resize(rays[::-1], (n, 8))
    for q in ("closest", "any"):
        ref, rids, st = _oracle(I, sel, "alpha_tex", q)
        got, ids, _ = _gpu(V, X, _dev(sel), "alpha_tex", q,
                           V.trace_params(persistent=1, refill_threshold=8, watchdog_ms=10_000))
        _compare(got, ids, ref, rids, st, f"n={n} {q}")


def test_persistent_watchdog(V, small):
    """A watchdog of 3 outer iterations per warp runs out: the instance set's
    error word gets the timeout bit, every record is the full result, a miss
    written for a ray in flight or the fill value of a ray never claimed; a
    run with the default budget afterwards is complete and clean."""
    I, rays, X = small
    d = _dev(rays)
    full, fids, _ = _gpu(V, X, d, "default", "closest")
    cut = V.trace_params(persistent=1, refill_threshold=16, watchdog_iterations=3)
    n = rays.shape[0]
    hits = torch.full((n, 4), -5.0, dtype=torch.float32, device="cuda")
    V.vsr_trace_instances(X, d, V.intersector("default"), "closest", hits, None, None, cut)
    torch.cuda.synchronize()
    word = V.vsr_instances_device_error(X)
    assert word & V.DEVERR_TIMEOUT, word
    h = hits.cpu().numpy()
    same = np.all(h.view(np.uint32) == full.view(np.uint32), axis=1)
    miss = h[:, 3].view(np.uint32) == O.NONE
    fill = np.all(h == -5.0, axis=1)
    assert (same | miss | fill).all() and not same.all()
    got, ids, _ = _gpu(V, X, d, "default", "closest",
                       V.trace_params(persistent=1, refill_threshold=16, watchdog_ms=10_000))
    assert np.array_equal(got.view(np.uint32), full.view(np.uint32))
    assert np.array_equal(ids, fids)
    assert V.vsr_instances_device_error(X) == 0
