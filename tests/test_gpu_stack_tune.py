"""The register short stack and the launch tuner of vsr_trace (needs a GB300).

- Every register-stack depth (0, 1, 2, 4, 8 entries in registers, the rest in
  shared memory) visits nodes in the same LIFO order, so records and counts
  are bit-identical to the oracle's for every intersector and query.
- vsr_trace_tune picks a configuration; vsr_trace with params NULL then gives
  the same bits as the explicit configuration it returned (and as the
  oracle), also when the first NULL call tunes by itself.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    return vsr


@pytest.fixture(scope="module")
def small(V):
    sc, rays = scenes.small_quads()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    yield sc, rays, blob, s, torch.from_numpy(rays).cuda()
    s.close()


def _same_as_oracle(hits, ref, st, label):
    got = hits.cpu().numpy().view(np.uint32)
    want = O.hits_raw(ref).view(np.uint32)
    bad = np.any(got != want, axis=1) & (st[:, 3] == 0)
    assert not bad.any(), f"{label}: {int(bad.sum())} rays differ"


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", ["none", "default", "alpha_tex", "proc_alpha", "count"])
def test_stack_depths_match_oracle(V, small, kind, query):
    sc, rays, blob, s, d_rays = small
    ref, st = O.trace_bvh(sc, blob, rays, kind, query)
    for regs in (0, 1, 2, 4, 8):
        for width in (0, 256):
            p = V.trace_params(block_size=128, stack_regs=regs, image_width=width)
            hits, cnt = V.trace(s, d_rays, kind, query, counters=(kind == "count"), params=p)
            _same_as_oracle(hits, ref, st, f"{kind}/{query}/K={regs}/w={width}")
            if kind == "count":
                assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", ["none", "default", "alpha_tex", "proc_alpha", "count", "clip"])
def test_lockstep_matches_oracle(V, small, kind, query):
    """The warp in lock step (speculative descent for the any-hit query with
    intersectors that keep no counters) gives every ray the oracle's record
    and counts: one ray per thread and persistent, pixel tiles and buffer
    order, stack in shared memory and in registers."""
    sc, rays, blob, s, d_rays = small
    clip = dict(clip_lo=(0.2, 0.1, 0.0), clip_hi=(0.8, 0.7, 0.9)) if kind == "clip" else {}
    ref, st = O.trace_bvh(sc, blob, rays, kind, query, **clip)
    configs = [dict(block_size=128), dict(block_size=64, stack_regs=4, image_width=256),
               dict(block_size=256, persistent=1, refill_threshold=24, watchdog_ms=10_000),
               dict(block_size=96, persistent=1, refill_threshold=8, stack_regs=2,
                    watchdog_ms=10_000)]
    for c in configs:
        p = V.trace_params(lockstep=1, **c)
        hits, cnt = V.trace(s, d_rays, kind, query, counters=(kind == "count"), params=p, **clip)
        _same_as_oracle(hits, ref, st, f"lockstep {kind}/{query}/{c}")
        if kind == "count":
            assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("kind", ["default", "alpha_tex", "proc_alpha", "count"])
def test_dynamic_persistent_and_lockstep_match_oracle(V, small, kind, query):
    """Dynamic dispatch (callbacks bound per ray through the function-pointer
    tables) in the persistent and lock-step launch shapes: per-lane loops and
    lock step, persistent and one ray per thread, pixel tiles and buffer
    order.  Speculative descent runs for the kinds without a box callback;
    count (box and triangle callbacks) keeps every lane's box tests, and its
    counters match the oracle's."""
    sc, rays, blob, s, d_rays = small
    ref, st = O.trace_bvh(sc, blob, rays, kind, query)
    configs = [dict(block_size=128, lockstep=1),
               dict(block_size=64, lockstep=1, image_width=256),
               dict(block_size=256, persistent=1, refill_threshold=24, watchdog_ms=10_000),
               dict(block_size=96, persistent=1, refill_threshold=8, lockstep=1,
                    watchdog_ms=10_000),
               dict(block_size=128, persistent=1, refill_threshold=32, lockstep=1,
                    image_width=256, watchdog_ms=10_000)]
    for c in configs:
        p = V.trace_params(**c)
        hits, cnt = V.trace(s, d_rays, kind, query, dispatch="dynamic",
                            counters=(kind == "count"), params=p)
        _same_as_oracle(hits, ref, st, f"dynamic {kind}/{query}/{c}")
        if kind == "count":
            assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])
    assert V.vsr_get_device_error(s) == 0


def test_dynamic_persistent_ragged(V):
    """Dynamic dispatch, persistent and lock step, on ray counts that leave
    partly filled warps, and at every register budget."""
    sc, rays = scenes.small_quads(seed=scenes.SEED_BASE + 45)
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    for n in (1, 33, 4097):
        sub = np.ascontiguousarray(rays[:n])
        for q in ("closest", "any"):
            ref, st = O.trace_bvh(sc, blob, sub, "proc_alpha", q)
            for pers, ls in ((1, 0), (1, 1), (0, 1)):
                hits, _ = V.trace(s, torch.from_numpy(sub).cuda(), "proc_alpha", q,
                                  dispatch="dynamic",
                                  params=V.trace_params(lockstep=ls, persistent=pers,
                                                        watchdog_ms=10_000))
                _same_as_oracle(hits, ref, st, f"dynamic n={n} {q} pers={pers} ls={ls}")
    # every register budget of the dynamic persistent and lock-step kernels
    d_rays = torch.from_numpy(rays).cuda()
    for q in ("closest", "any"):
        ref, st = O.trace_bvh(sc, blob, rays, "alpha_tex", q)
        for cap in (1, 3, 4):
            for pers, ls in ((1, 0), (1, 1), (0, 1)):
                hits, _ = V.trace(s, d_rays, "alpha_tex", q, dispatch="dynamic",
                                  params=V.trace_params(lockstep=ls, persistent=pers,
                                                        reg_cap_blocks=cap, watchdog_ms=10_000))
                _same_as_oracle(hits, ref, st, f"dynamic {q} cap={cap} pers={pers} ls={ls}")
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="reg_cap_blocks 5 and 6"):
        V.vsr_trace(s, d_rays, V.intersector("default", "dynamic"), "any", hits, None,
                    V.trace_params(persistent=1, reg_cap_blocks=5))
    assert V.vsr_get_device_error(s) == 0
    s.close()


def test_lockstep_ragged_and_single_leaf(V):
    """Ray counts that leave partly filled warps (1, 33, 4,097 rays) and a
    scene whose BVH is one leaf (the root itself), in lock step."""
    sc, rays = scenes.small_quads(seed=scenes.SEED_BASE + 43)
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    for n in (1, 33, 4097):
        sub = np.ascontiguousarray(rays[:n])
        for q in ("closest", "any"):
            ref, st = O.trace_bvh(sc, blob, sub, "alpha_tex", q)
            for pers in (0, 1):
                hits, _ = V.trace(s, torch.from_numpy(sub).cuda(), "alpha_tex", q,
                                  params=V.trace_params(lockstep=1, persistent=pers,
                                                        watchdog_ms=10_000))
                _same_as_oracle(hits, ref, st, f"lockstep n={n} {q} persistent={pers}")
    s.close()
    tiny, trays = scenes.small_quads(seed=scenes.SEED_BASE + 44, n_quads=1)
    tblob = tiny.bvh()
    ts = V.scene_from_inputs(tiny, tblob)
    for q in ("closest", "any"):
        ref, st = O.trace_bvh(tiny, tblob, trays, "default", q)
        hits, _ = V.trace(ts, torch.from_numpy(trays).cuda(), "default", q,
                          params=V.trace_params(lockstep=1))
        _same_as_oracle(hits, ref, st, f"lockstep one leaf {q}")
    assert V.vsr_get_device_error(ts) == 0
    ts.close()


def test_lockstep_rejected_where_unsupported(V, small):
    sc, rays, blob, s, d_rays = small
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="lockstep"):
        V.vsr_trace(s, d_rays, V.intersector("default"), "closest", hits, None,
                    V.trace_params(lockstep=2))
    with pytest.raises(V.VsrError, match="lockstep"):
        V.vsr_trace(s, d_rays, V.intersector("default"), "closest", hits, None,
                    V.trace_params(lockstep=1, reg_cap_blocks=4))


def test_stack_depths_clip_box(V, small):
    sc, rays, blob, s, d_rays = small
    lo, hi = (0.2, 0.1, 0.0), (0.8, 0.7, 0.9)
    ref, st = O.trace_bvh(sc, blob, rays, "clip", "closest", clip_lo=lo, clip_hi=hi)
    for regs in (0, 2, 8):
        p = V.trace_params(stack_regs=regs)
        hits, _ = V.trace(s, d_rays, "clip", "closest", params=p, clip_lo=lo, clip_hi=hi)
        _same_as_oracle(hits, ref, st, f"clip K={regs}")


@pytest.mark.parametrize("kind,query,dispatch", [("none", "closest", "static"),
                                                 ("alpha_tex", "closest", "static"),
                                                 ("alpha_tex", "any", "static"),
                                                 ("proc_alpha", "any", "static"),
                                                 ("count", "closest", "static"),
                                                 ("alpha_tex", "closest", "dynamic"),
                                                 ("proc_alpha", "any", "dynamic")])
def test_trace_coherence_order_matches_oracle(V, small, kind, query, dispatch):
    """vsr_trace with ray_order 1 sorts the rays by origin and direction and
    traces them in that order: every ray's record (and its counts) is the
    oracle's, one ray per thread and persistent, at several stack depths."""
    sc, rays, blob, s, d_rays = small
    ref, st = O.trace_bvh(sc, blob, rays, kind, query)
    configs = [dict(block_size=128), dict(block_size=64, stack_regs=2)]
    if dispatch == "static":
        configs += [dict(block_size=128, persistent=1, refill_threshold=16, stack_regs=4,
                         watchdog_ms=10_000)]
    else:
        configs = configs[:1] + [dict(block_size=128, persistent=1, refill_threshold=16,
                                      lockstep=1, watchdog_ms=10_000)]
    for c in configs:
        p = V.trace_params(ray_order=1, **c)
        hits, cnt = V.trace(s, d_rays, kind, query, dispatch=dispatch,
                            counters=(kind == "count"), params=p)
        _same_as_oracle(hits, ref, st, f"ordered {kind}/{query}/{dispatch}/{c}")
        if kind == "count":
            assert np.array_equal(cnt.cpu().numpy().view(np.uint32), st[:, :2])
    assert V.vsr_get_device_error(s) == 0


def test_trace_coherence_order_ragged_and_empty(V):
    """Ray counts that leave ragged radix tiles (1, 33, 4,097 rays) and an
    empty trace, in coherence order."""
    sc, rays = scenes.small_quads(seed=scenes.SEED_BASE + 42)
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    for n in (1, 33, 4097):
        sub = np.ascontiguousarray(rays[:n])
        ref, st = O.trace_bvh(sc, blob, sub, "alpha_tex", "closest")
        hits, _ = V.trace(s, torch.from_numpy(sub).cuda(), "alpha_tex", "closest",
                          params=V.trace_params(ray_order=1))
        _same_as_oracle(hits, ref, st, f"ordered n={n}")
    empty = torch.empty((0, 8), dtype=torch.float32, device="cuda")
    out = torch.empty((0, 4), dtype=torch.float32, device="cuda")
    V.vsr_trace(s, empty, V.intersector("alpha_tex"), "closest", out, None,
                V.trace_params(ray_order=1))
    torch.cuda.synchronize()
    assert V.vsr_get_device_error(s) == 0
    s.close()


def test_trace_coherence_order_rejected_where_unsupported(V, small):
    sc, rays, blob, s, d_rays = small
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    isect = V.intersector("default")
    with pytest.raises(V.VsrError, match="image_width 0"):
        V.vsr_trace(s, d_rays, isect, "closest", hits, None,
                    V.trace_params(ray_order=1, image_width=256))
    with pytest.raises(V.VsrError, match="ray_order"):
        V.vsr_trace(s, d_rays, isect, "closest", hits, None, V.trace_params(ray_order=2))
    with pytest.raises(V.VsrError, match="ray_order"):
        V.vsr_trace_persistent_noalloc(s, d_rays, isect, "closest", hits, None,
                                       V.trace_params(persistent=1, ray_order=1))


def test_stack_depth_rejected_when_unsupported(V, small):
    sc, rays, blob, s, d_rays = small
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="stack_regs"):
        V.vsr_trace(s, d_rays, V.intersector("default"), "closest", hits, None,
                    V.trace_params(stack_regs=3))


@pytest.mark.parametrize("kind,query,dispatch", [("alpha_tex", "closest", "static"),
                                                 ("alpha_tex", "any", "static"),
                                                 ("proc_alpha", "any", "static"),
                                                 ("count", "closest", "static"),
                                                 ("alpha_tex", "closest", "dynamic"),
                                                 ("count", "any", "dynamic")])
def test_null_params_use_the_tuned_configuration(V, kind, query, dispatch):
    sc, rays = scenes.small_quads(seed=scenes.SEED_BASE + 40)
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    d_rays = torch.from_numpy(rays).cuda()
    isect = V.intersector(kind, dispatch)
    scratch = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    tuned = V.vsr_trace_tune(s, d_rays, isect, query, scratch, image_width=256)
    p = V.params_dict(tuned)
    assert p["block_size"] in (64, 128, 256)
    # the tiled map, or the coherence order (which replaces it)
    assert (p["image_width"], p["ray_order"]) in ((256, 0), (0, 1))
    assert p["stack_regs"] in ((0, 1, 2, 4, 8) if dispatch == "static" else (0,))
    assert p["reg_cap_blocks"] == 0 and p["lockstep"] in (0, 1) and p["persistent"] in (0, 1)
    a = torch.full((len(rays), 4), -3.0, dtype=torch.float32, device="cuda")
    b = torch.full_like(a, -4.0)
    V.vsr_trace(s, d_rays, isect, query, a, None, None)          # tuned (cached)
    V.vsr_trace(s, d_rays, isect, query, b, None, tuned)         # explicit
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    ref, st = O.trace_bvh(sc, blob, rays, kind, query)
    _same_as_oracle(a, ref, st, f"tuned {kind}/{query}/{dispatch}")
    assert V.vsr_get_device_error(s) == 0
    s.close()


def test_first_null_call_tunes_itself(V):
    sc, rays = scenes.small_quads(seed=scenes.SEED_BASE + 41)
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    d_rays = torch.from_numpy(rays).cuda()
    hits, _ = V.trace(s, d_rays, "alpha_tex", "closest")     # tunes, then traces
    again, _ = V.trace(s, d_rays, "alpha_tex", "closest")    # cached configuration
    torch.cuda.synchronize()
    assert torch.equal(hits.view(torch.int32), again.view(torch.int32))
    ref, st = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest")
    _same_as_oracle(hits, ref, st, "self-tuned")
    s.close()


def test_tune_rejects_bad_arguments(V, small):
    sc, rays, blob, s, d_rays = small
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    empty = torch.empty((0, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="at least one ray"):
        V.vsr_trace_tune(s, empty, V.intersector("default"), "closest", hits)
