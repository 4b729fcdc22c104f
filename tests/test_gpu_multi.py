"""Multi-hit query on the GPU vs the oracle, through the C ABI (needs a GB300).

Bar: the first N accepted hits of each ray (t, u, v, prim, in ascending
(t, prim) order, then miss records) are bit-identical to the oracle's
multi-hit traversal, and bvh_costs counters too; rays the oracle flags as near
ties may differ and are excluded, as for closest-hit.  N = 1 must reproduce
vsr_trace's closest hit bit for bit.
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


@pytest.fixture(scope="module")
def small(V):
    sc, rays = scenes.small_quads()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    yield sc, rays, blob, s
    s.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _multi(V, s, rays, kind, nh, params=None, counters=False, dispatch="static"):
    n = rays.shape[0]
    hits = torch.full((n, nh, 4), float("nan"), dtype=torch.float32, device="cuda")
    cnt = torch.full((n, 2), -1, dtype=torch.int32, device="cuda") if counters else None
    V.vsr_trace_multi(s, rays, V.intersector(kind, dispatch), nh, hits, cnt, params)
    torch.cuda.synchronize()
    return hits.cpu().numpy(), (cnt.cpu().numpy().view(np.uint32) if counters else None)


def _compare(got, ref, st, label):
    """got [n, nh, 4] float32; ref dict of [n, nh]; st oracle stats."""
    r = np.stack([ref["t"], ref["u"], ref["v"], ref["prim"].view(np.float32)], -1)
    bad = np.any(got.view(np.uint32) != r.view(np.uint32), axis=(1, 2))
    ties = st[:, 3] != 0
    assert not (bad & ~ties).any(), f"{label}: {int((bad & ~ties).sum())} rays differ"
    return int(ties.sum())


@pytest.mark.parametrize("nh", [1, 3, 4, 5, 8, 9, 16])
@pytest.mark.parametrize("kind", KINDS)
def test_small_all_intersectors(V, small, kind, nh):
    sc, rays, blob, s = small
    ref, st = O.trace_multi(sc, rays, nh, kind, blob)
    got, cnt = _multi(V, s, _dev(rays), kind, nh, counters=(kind == "count"))
    _compare(got, ref, st, f"{kind} nh={nh}")
    if kind == "count":
        ok = st[:, 3] == 0
        assert np.array_equal(cnt[ok], st[ok, :2])
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("kind", KINDS)
def test_one_hit_is_vsr_trace(V, small, kind):
    sc, rays, blob, s = small
    d = _dev(rays)
    got, _ = _multi(V, s, d, kind, 1)
    h, _ = V.trace(s, d, kind, "closest")
    torch.cuda.synchronize()
    assert np.array_equal(got[:, 0].view(np.uint32), h.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("n,width", [(1, 0), (33, 0), (4097, 0), (4097, 37), (65536, 256)])
def test_ragged_and_pixel_tiles(V, small, n, width):
    sc, rays, blob, s = small
    sel = np.resize(rays[::-1], (n, 8))
    ref, st = O.trace_multi(sc, sel, 6, "alpha_tex", blob)
    got, _ = _multi(V, s, _dev(sel), "alpha_tex", 6, V.trace_params(image_width=width))
    _compare(got, ref, st, f"n={n} width={width}")


def test_argument_checks(V, small):
    sc, rays, blob, s = small
    d = _dev(rays[:64])
    hits = torch.empty((64, 16, 4), dtype=torch.float32, device="cuda")
    for nh in (0, 17):
        with pytest.raises(V.VsrError):
            V.vsr_trace_multi(s, d, V.intersector("default"), nh, hits)
    with pytest.raises(V.VsrError, match="persistent 1"):
        V.vsr_trace_multi(s, d, V.intersector("default"), 4, hits, None,
                          V.trace_params(lockstep=1))
    small_hits = torch.empty((64, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="hits"):
        V.vsr_trace_multi(s, _dev(np.resize(rays, (1 << 16, 8))), V.intersector("default"), 16,
                          small_hits)


def test_forest_full_frame_sample(V):
    """1920x1080 primary rays through the alpha-masked forest, 8 hits per
    ray in the bench's launch configuration: a seeded sample against the
    oracle, and the first column against vsr_trace over the whole frame."""
    import bench
    sc, rays = scenes.billboard_forest()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    try:
        d = _dev(rays)
        p = bench.default_params(V)
        got, _ = _multi(V, s, d, "alpha_tex", 8, p)
        h, _ = V.trace(s, d, "alpha_tex", "closest", params=p)
        torch.cuda.synchronize()
        assert np.array_equal(got[:, 0].view(np.uint32), h.cpu().numpy().view(np.uint32))
        rng = np.random.default_rng(11)
        sel = np.sort(rng.choice(len(rays), 4000, replace=False))
        ref, st = O.trace_multi(sc, rays[sel], 8, "alpha_tex", blob)
        assert _compare(got[sel], ref, st, "forest") <= 0.01 * len(sel)
        depth = (got[:, :, 3].view(np.uint32) != O.NONE).sum(1)
        assert depth.mean() > 2.0  # looking through several layers of foliage
        assert V.vsr_get_device_error(s) == 0
    finally:
        s.close()


@pytest.mark.parametrize("nh", [1, 5, 16])
@pytest.mark.parametrize("kind", KINDS)
def test_dynamic_dispatch_equals_static(V, small, kind, nh):
    """The intersector reached through the callback tables gives the same
    records and counters as the compiled-in one, bit for bit (and so the
    oracle's), including pixel tiles."""
    sc, rays, blob, s = small
    d = _dev(rays)
    cnt = kind == "count"
    for p in (None, V.trace_params(image_width=256)):
        a, ca = _multi(V, s, d, kind, nh, p, counters=cnt)
        b, cb = _multi(V, s, d, kind, nh, p, counters=cnt, dispatch="dynamic")
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), kind
        if cnt:
            assert np.array_equal(ca, cb)
    ref, st = O.trace_multi(sc, rays, nh, kind, blob)
    _compare(b, ref, st, f"dynamic {kind} N={nh}")
    assert V.vsr_get_device_error(s) == 0


PERSISTENT = [dict(persistent=1, refill_threshold=16, watchdog_ms=10_000),
              dict(persistent=1, refill_threshold=24, lockstep=1, watchdog_ms=10_000),
              dict(persistent=1, refill_threshold=1, lockstep=1, image_width=256, block_size=64,
                   watchdog_ms=10_000)]


@pytest.mark.parametrize("nh", [1, 4, 16])
@pytest.mark.parametrize("kind", KINDS + ["clip"])
@pytest.mark.parametrize("dispatch", ["static", "dynamic"])
def test_persistent_matches_oracle(V, small, kind, nh, dispatch):
    """Persistent warps (per-lane loops and lock step, whose closest-hit
    speculation bounds boxes by the buffer's last entry) give the oracle's
    records and counters, with either dispatch."""
    if dispatch == "dynamic" and kind == "clip":
        pytest.skip("the clip box is compiled in only (static dispatch)")
    sc, rays, blob, s = small
    clip = dict(clip_lo=(0.2, 0.1, 0.0), clip_hi=(0.8, 0.7, 0.9)) if kind == "clip" else {}
    ref, st = O.trace_multi(sc, rays, nh, kind, blob, **clip)
    d = _dev(rays)
    cnt = kind == "count"
    for c in PERSISTENT:
        n = rays.shape[0]
        hits = torch.full((n, nh, 4), float("nan"), dtype=torch.float32, device="cuda")
        cn = torch.full((n, 2), -1, dtype=torch.int32, device="cuda") if cnt else None
        V.vsr_trace_multi(s, d, V.intersector(kind, dispatch, **clip), nh, hits, cn,
                          V.trace_params(**c))
        torch.cuda.synchronize()
        _compare(hits.cpu().numpy(), ref, st, f"{dispatch} {kind} nh={nh} {c}")
        if cnt:
            ok = st[:, 3] == 0
            assert np.array_equal(cn.cpu().numpy().view(np.uint32)[ok], st[ok, :2])
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("n", [1, 33, 4097])
def test_persistent_ragged(V, small, n):
    sc, rays, blob, s = small
    sel = np.resize(rays[::-1], (n, 8))
    ref, st = O.trace_multi(sc, sel, 6, "proc_alpha", blob)
    for c in PERSISTENT:
        got, _ = _multi(V, s, _dev(sel), "proc_alpha", 6, V.trace_params(**c))
        _compare(got, ref, st, f"n={n} {c}")
