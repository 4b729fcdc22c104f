"""Persistent-warp and batched launches: the watchdog, the procedural-alpha
any-hit query in both loops, and the register short stack (needs a GB300).

- The watchdog bounds both persistent loops: with a budget of a few
  iterations on a workload that needs many, the launch must return, leave
  the timeout bit in the device error word and leave the GPU usable (the
  next launch gives the full result).
- The procedural-alpha any-hit query through the persistent kernel and the
  batched kernel must equal the oracle's same-order traversal bit for bit
  (near ties excepted), at several block/refill settings and stack depths.
- Every register-stack depth gives the same records as the shared-memory
  stack, in the persistent launch and in batches.

Every persistent launch here carries a 10 s watchdog, so a loop that does not
end returns with the timeout bit instead of holding the GPU.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

WD_MS = 10_000


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


def _compare(V, hits, ref, st, label):
    got = hits.cpu().numpy().view(np.uint32)
    want = O.hits_raw(ref).view(np.uint32)
    ties = st[:, 3] != 0
    bad = np.any(got != want, axis=1) & ~ties
    assert not bad.any(), f"{label}: {int(bad.sum())} rays differ (first {np.flatnonzero(bad)[:3]})"


@pytest.mark.parametrize("block,refill,regs", [(128, 16, 0), (32, 1, 0), (256, 32, 4),
                                               (64, 24, 2), (96, 8, 8), (128, 1, 1)])
def test_persistent_proc_alpha_any_matches_oracle(V, small, block, refill, regs):
    sc, rays, blob, s, d_rays = small
    ref, st = O.trace_bvh(sc, blob, rays, "proc_alpha", "any")
    p = V.trace_params(block_size=block, persistent=1, refill_threshold=refill,
                       stack_regs=regs, watchdog_ms=WD_MS)
    hits = torch.full((len(rays), 4), -9.0, dtype=torch.float32, device="cuda")
    V.vsr_trace(s, d_rays, V.intersector("proc_alpha"), "any", hits, None, p)
    torch.cuda.synchronize()
    assert V.vsr_get_device_error(s) == 0
    _compare(V, hits, ref, st, f"persistent proc any {block}/{refill}/{regs}")


def test_persistent_launches_on_two_streams(V, small):
    """Persistent launches of one scene on two streams may overlap: each takes
    its own ray counter, so both give the full result."""
    sc, rays, blob, s, d_rays = small
    isect = V.intersector("alpha_tex")
    ref = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    V.vsr_trace(s, d_rays, isect, "closest", ref, None, V.trace_params())
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [torch.full_like(ref, -3.0) for _ in range(6)]
    torch.cuda.synchronize()  # the fills are on the current stream
    for k, o in enumerate(outs):
        p = V.trace_params(block_size=128, persistent=1, refill_threshold=16, lockstep=k % 2,
                           watchdog_ms=WD_MS)
        V.vsr_trace(s, d_rays, isect, "closest", o, None, p, streams[k % 2])
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o.view(torch.int32), ref.view(torch.int32))
    assert V.vsr_get_device_error(s) == 0


def test_noalloc_proc_alpha_any_matches_persistent(V, small):
    sc, rays, blob, s, d_rays = small
    p = V.trace_params(block_size=128, persistent=1, refill_threshold=16, watchdog_ms=WD_MS)
    ref = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    V.vsr_trace(s, d_rays, V.intersector("proc_alpha"), "any", ref, None, p)
    for _ in range(2):
        got = torch.full_like(ref, -7.0)
        V.vsr_trace_persistent_noalloc(s, d_rays, V.intersector("proc_alpha"), "any", got, None, p)
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("regs", [0, 1, 2, 4, 8])
@pytest.mark.parametrize("kind,query", [("alpha_tex", "closest"), ("count", "any"),
                                        ("default", "closest"), ("proc_alpha", "closest")])
def test_persistent_stack_depths_agree(V, small, kind, query, regs):
    sc, rays, blob, s, d_rays = small
    n = len(rays)
    want = kind == "count"
    base = V.trace_params(block_size=128, persistent=0, stack_regs=0)
    ref, ref_c = V.trace(s, d_rays, kind, query, counters=want, params=base)
    p = V.trace_params(block_size=96, persistent=1, refill_threshold=20, stack_regs=regs,
                       watchdog_ms=WD_MS)
    got, got_c = V.trace(s, d_rays, kind, query, counters=want, params=p)
    torch.cuda.synchronize()
    assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
    if want:
        assert torch.equal(got_c, ref_c)
    assert V.vsr_get_device_error(s) == 0


@pytest.mark.parametrize("lockstep", [0, 1])
def test_watchdog_stops_persistent_loop(V, small, lockstep):
    """Default any-hit (a case that never stalled) with a budget of 3 outer
    iterations per warp: the launch returns with the timeout bit, and the next
    launch with no budget gives the full, correct result."""
    sc, rays, blob, s, d_rays = small
    isect = V.intersector("default")
    full = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    V.vsr_trace(s, d_rays, isect, "any", full, None,
                V.trace_params(persistent=0, watchdog_ms=WD_MS))
    torch.cuda.synchronize()
    assert V.vsr_get_device_error(s) == 0
    cut = V.trace_params(block_size=128, persistent=1, refill_threshold=16,
                         watchdog_iterations=3, lockstep=lockstep)
    hits = torch.full_like(full, -5.0)
    V.vsr_trace(s, d_rays, isect, "any", hits, None, cut)
    torch.cuda.synchronize()
    word = V.vsr_get_device_error(s)
    assert word & V.DEVERR_TIMEOUT, word
    # the launch stopped early: every record is the full result, a miss record
    # written for a ray in flight, or the fill value of a ray never claimed,
    # and not all of them are the full result
    hb, fb = hits.view(torch.int32), full.view(torch.int32)
    same = (hb == fb).all(dim=1)
    miss = hits[:, 3].view(torch.int32) == -1
    fill = (hits == -5.0).all(dim=1)
    assert bool((same | miss | fill).all())
    assert not bool(same.all())
    again = torch.full_like(full, -5.0)
    V.vsr_trace(s, d_rays, isect, "any", again, None,
                V.trace_params(block_size=128, persistent=1, refill_threshold=16,
                               watchdog_ms=WD_MS, lockstep=lockstep))
    torch.cuda.synchronize()
    assert V.vsr_get_device_error(s) == 0
    assert torch.equal(again.view(torch.int32), full.view(torch.int32))


def test_watchdog_time_budget_is_accepted(V, small):
    """A time budget that does not run out changes nothing; 0xFFFFFFFF
    switches the time budget off."""
    sc, rays, blob, s, d_rays = small
    isect = V.intersector("alpha_tex")
    outs = []
    for ms in (0, 1, 0xFFFFFFFF):
        h = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
        V.vsr_trace(s, d_rays, isect, "closest", h, None,
                    V.trace_params(persistent=1, watchdog_ms=ms if ms != 1 else 5_000))
        outs.append(h)
    torch.cuda.synchronize()
    assert V.vsr_get_device_error(s) == 0
    for h in outs[1:]:
        assert torch.equal(h.view(torch.int32), outs[0].view(torch.int32))


@pytest.fixture(scope="module")
def batch(V):
    items = scenes.batch_scenes(seed=77, n_scenes=12, tri_range=(200, 20_000),
                                ray_range=(50, 30_000))
    blobs = scenes.build_bvhs([s for s, _ in items])
    handles = [V.scene_from_inputs(s, b) for (s, _), b in zip(items, blobs)]
    dev_rays = [torch.from_numpy(np.ascontiguousarray(r)).cuda() for _, r in items]
    yield items, blobs, handles, dev_rays
    for h in handles:
        h.close()


def _hits(dev_rays, fill=-5.0):
    return [torch.full((r.shape[0], 4), fill, dtype=torch.float32, device="cuda")
            for r in dev_rays]


@pytest.mark.parametrize("regs", [0, 2, 4])
def test_batch_proc_alpha_any_matches_oracle(V, batch, regs):
    items, blobs, handles, dev_rays = batch
    isect = V.intersector("proc_alpha")
    hits = _hits(dev_rays)
    p = V.trace_params(block_size=128, persistent=1, refill_threshold=16, stack_regs=regs,
                       watchdog_ms=WD_MS)
    b = V.vsr_batch_create(handles, dev_rays, hits, isect, "any", p)
    V.vsr_batch_launch(b)
    torch.cuda.synchronize()
    for h in handles:
        assert V.vsr_get_device_error(h) == 0
    rng = np.random.default_rng(11)
    for k, ((sc, rays), blob) in enumerate(zip(items, blobs)):
        sel = np.sort(rng.choice(len(rays), min(400, len(rays)), replace=False))
        ref, st = O.trace_bvh(sc, blob, rays[sel], "proc_alpha", "any")
        got = hits[k].cpu().numpy()[sel].view(np.uint32)
        want = O.hits_raw(ref).view(np.uint32)
        ties = st[:, 3] != 0
        assert np.array_equal(got[~ties], want[~ties]), k
    b.close()


@pytest.mark.parametrize("kind,query", [("alpha_tex", "any"), ("proc_alpha", "closest"),
                                        ("count", "closest")])
def test_batch_stack_depths_agree(V, batch, kind, query):
    items, blobs, handles, dev_rays = batch
    isect = V.intersector(kind)
    outs = []
    for regs in (0, 2, 4):
        hits = _hits(dev_rays)
        p = V.trace_params(block_size=64, persistent=1, refill_threshold=24, stack_regs=regs,
                           watchdog_ms=WD_MS)
        b = V.vsr_batch_create(handles, dev_rays, hits, isect, query, p)
        V.vsr_batch_launch(b)
        torch.cuda.synchronize()
        b.close()
        outs.append(hits)
    for other in outs[1:]:
        for x, y in zip(outs[0], other):
            assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    for h in handles:
        assert V.vsr_get_device_error(h) == 0


@pytest.mark.parametrize("lockstep", [0, 1])
def test_batch_watchdog(V, batch, lockstep):
    """A batch with a budget of 3 iterations reports the timeout to scene 0;
    the GPU stays usable and a batch with no budget gives per-scene results."""
    items, blobs, handles, dev_rays = batch
    isect = V.intersector("default")
    hits = _hits(dev_rays)
    b = V.vsr_batch_create(handles, dev_rays, hits, isect, "any",
                           V.trace_params(block_size=128, persistent=1, refill_threshold=16,
                                          watchdog_iterations=3, lockstep=lockstep))
    V.vsr_batch_launch(b)
    torch.cuda.synchronize()
    b.close()
    words = [V.vsr_get_device_error(h) for h in handles]
    assert words[0] & V.DEVERR_TIMEOUT
    assert all((w & ~V.DEVERR_TIMEOUT) == 0 for w in words)
    hits = _hits(dev_rays)
    b = V.vsr_batch_create(handles, dev_rays, hits, isect, "any",
                           V.trace_params(block_size=128, persistent=1, refill_threshold=16,
                                          watchdog_ms=WD_MS, lockstep=lockstep))
    V.vsr_batch_launch(b)
    torch.cuda.synchronize()
    b.close()
    for h, r, got in zip(handles, dev_rays, hits):
        ref = torch.empty_like(got)
        V.vsr_trace(h, r, isect, "any", ref, None, V.trace_params())
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
    for h in handles:
        assert V.vsr_get_device_error(h) == 0
