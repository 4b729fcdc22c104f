"""Batched persistent launch over many scenes vs per-scene traces and the
oracle (needs a GB300).

The batched kernel runs the same traversal as vsr_trace, so every ray's
record -- closest or any hit -- must be bit-identical to the per-scene
launch, and (on a sample) to the oracle.  The batch mixes scenes of very
different sizes, one scene with no rays and one with no triangles.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    items = scenes.batch_scenes(seed=77, n_scenes=24, tri_range=(200, 20_000),
                                ray_range=(50, 30_000))
    empty = scenes.Scene("empty", np.zeros((0, 3), np.float32), np.zeros((0, 3), np.uint32),
                         np.zeros((0, 3, 2), np.float32), np.zeros(0, np.uint32),
                         [scenes.disc_alpha_u8(4)])
    items.insert(5, (items[4][0], np.zeros((0, 8), np.float32)))     # no rays
    items.insert(9, (empty, scenes.camera_rays_random(np.random.default_rng(1), 300)))
    blobs = scenes.build_bvhs([s for s, _ in items])
    handles, dev_rays = [], []
    for (s, r), b in zip(items, blobs):
        handles.append(vsr.scene_from_inputs(s, b))
        dev_rays.append(torch.from_numpy(np.ascontiguousarray(r)).cuda())
    yield vsr, items, blobs, handles, dev_rays
    for h in handles:
        h.close()


def _hits_like(dev_rays):
    return [torch.full((max(r.shape[0], 0), 4), -5.0, dtype=torch.float32, device="cuda")
            for r in dev_rays]


@pytest.mark.parametrize("kind,query", [("alpha_tex", "closest"), ("alpha_tex", "any"),
                                        ("default", "closest"), ("default", "any")])
def test_batch_equals_per_scene(batch, kind, query):
    V, items, blobs, handles, dev_rays = batch
    isect = V.intersector(kind)
    hits = _hits_like(dev_rays)
    b = V.vsr_batch_create(handles, dev_rays, hits, isect, query)
    V.vsr_batch_launch(b)
    torch.cuda.synchronize()
    p = V.vsr_batch_params(b)
    assert p.block_size % 32 == 0 and 1 <= p.refill_threshold <= 32
    for k, (h, r) in enumerate(zip(handles, dev_rays)):
        if r.shape[0] == 0:
            continue
        ref = torch.empty_like(hits[k])
        V.vsr_trace(h, r, isect, query, ref)
        torch.cuda.synchronize()
        assert torch.equal(hits[k].view(torch.int32), ref.view(torch.int32)), k
    # replaying the captured graph gives the same records
    again = [x.clone() for x in hits]
    for x in hits:
        x.fill_(-3.0)
    V.vsr_batch_launch(b)
    torch.cuda.synchronize()
    for x, y in zip(hits, again):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    b.close()
    for h in handles:
        assert V.vsr_get_device_error(h) == 0


def test_batch_matches_oracle_sample(batch):
    V, items, blobs, handles, dev_rays = batch
    hits = _hits_like(dev_rays)
    V.vsr_trace_batch(handles, dev_rays, hits, V.intersector("alpha_tex"), "closest")
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for k, ((sc, rays), blob) in enumerate(zip(items, blobs)):
        if len(rays) == 0:
            continue
        sel = np.sort(rng.choice(len(rays), min(300, len(rays)), replace=False))
        ref, st = O.trace_bvh(sc, blob, rays[sel], "alpha_tex", "closest")
        got = hits[k].cpu().numpy()[sel].view(np.uint32)
        want = O.hits_raw(ref).view(np.uint32)
        ties = st[:, 3] != 0
        assert np.array_equal(got[~ties], want[~ties]), k


def test_batch_explicit_params_and_one_call_cache(batch):
    V, items, blobs, handles, dev_rays = batch
    isect = V.intersector("alpha_tex")
    a = _hits_like(dev_rays)
    bb = _hits_like(dev_rays)
    p = V.trace_params(block_size=64, persistent=1, refill_threshold=24, blocks_per_sm=4)
    V.vsr_trace_batch(handles, dev_rays, a, isect, "any", params=p)
    V.vsr_trace_batch(handles, dev_rays, a, isect, "any", params=p)  # cached replay
    V.vsr_trace_batch(handles, dev_rays, bb, isect, "any")
    torch.cuda.synchronize()
    for x, y in zip(a, bb):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))


def test_batch_rejects_bad_arguments(batch):
    V, items, blobs, handles, dev_rays = batch
    hits = _hits_like(dev_rays)
    with pytest.raises(V.VsrError, match="static dispatch"):
        V.vsr_batch_create(handles, dev_rays, hits, V.intersector("default", "dynamic"), "any")
    with pytest.raises(V.VsrError, match="stack_regs"):
        V.vsr_batch_create(handles, dev_rays, hits, V.intersector("default"), "any",
                           V.trace_params(persistent=1, stack_regs=1))
    sc = items[0][0]
    nobvh = V.vsr_scene_create_indexed(sc.verts, sc.idx, sc.uvs, sc.geom_id, sc.textures)
    with pytest.raises(V.VsrError, match="VSR_ERR_STATE"):
        V.vsr_batch_create([nobvh], dev_rays[:1], hits[:1], V.intersector("default"), "any")
    nobvh.close()
    small = [torch.empty((1, 4), dtype=torch.float32, device="cuda")]
    import ctypes
    host = np.zeros((dev_rays[0].shape[0], 8), np.float32)

    class HostTensor:
        shape = host.shape

        def data_ptr(self):
            return host.ctypes.data

    with pytest.raises(V.VsrError, match="device memory"):
        V.vsr_batch_create(handles[:1], [HostTensor()], hits[:1], V.intersector("default"), "any")
    del ctypes, small


@pytest.mark.parametrize("kind,query", [("alpha_tex", "closest"), ("alpha_tex", "any"),
                                        ("proc_alpha", "any"), ("count", "closest")])
def test_coherence_order_equals_buffer_order(batch, kind, query):
    """Tracing in coherence order (the rays sorted by scene, origin and
    direction inside the launch) gives every ray the record of the buffer
    order, bit for bit: each ray is traced exactly once.  The batch holds an
    empty scene and a scene without rays."""
    V, items, blobs, handles, dev_rays = batch
    isect = V.intersector(kind)
    outs = []
    for order, regs in ((0, 0), (1, 0), (1, 4)):
        hits = _hits_like(dev_rays)
        p = V.trace_params(block_size=128, persistent=1, refill_threshold=16, stack_regs=regs,
                           ray_order=order, watchdog_ms=10_000)
        b = V.vsr_batch_create(handles, dev_rays, hits, isect, query, p)
        V.vsr_batch_launch(b)
        V.vsr_batch_launch(b)  # the graph replay sorts again
        torch.cuda.synchronize()
        b.close()
        outs.append(hits)
    for other in outs[1:]:
        for k, (x, y) in enumerate(zip(outs[0], other)):
            assert torch.equal(x.view(torch.int32), y.view(torch.int32)), k
    for h in handles:
        assert V.vsr_get_device_error(h) == 0


@pytest.mark.parametrize("kind,query", [("alpha_tex", "closest"), ("alpha_tex", "any"),
                                        ("proc_alpha", "any"), ("count", "closest"),
                                        ("count", "any"), ("default", "any")])
def test_lockstep_equals_per_lane_loops(batch, kind, query):
    """The batched kernel with the warp in lock step (speculative any-hit
    descent where it applies) gives the records of per-lane loops bit for
    bit, in buffer and coherence order and with registers holding the stack
    top."""
    V, items, blobs, handles, dev_rays = batch
    isect = V.intersector(kind)
    outs = []
    for ls, order, regs in ((0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 0, 4)):
        hits = _hits_like(dev_rays)
        p = V.trace_params(block_size=128, persistent=1, refill_threshold=16, stack_regs=regs,
                           ray_order=order, lockstep=ls, watchdog_ms=10_000)
        b = V.vsr_batch_create(handles, dev_rays, hits, isect, query, p)
        V.vsr_batch_launch(b)
        V.vsr_batch_launch(b)
        torch.cuda.synchronize()
        b.close()
        outs.append(hits)
    for other in outs[1:]:
        for k, (x, y) in enumerate(zip(outs[0], other)):
            assert torch.equal(x.view(torch.int32), y.view(torch.int32)), k
    for h in handles:
        assert V.vsr_get_device_error(h) == 0


def test_coherence_order_rejected_outside_traces_and_batches(batch):
    V, items, blobs, handles, dev_rays = batch
    hits = torch.empty((dev_rays[0].shape[0], 4), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="ray_order"):
        V.vsr_trace_multi(handles[0], dev_rays[0], V.intersector("default"), 2,
                          torch.empty((dev_rays[0].shape[0], 2, 4), dtype=torch.float32,
                                      device="cuda"),
                          None, V.trace_params(ray_order=1))
