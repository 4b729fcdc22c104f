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


def test_stack_depths_clip_box(V, small):
    sc, rays, blob, s, d_rays = small
    lo, hi = (0.2, 0.1, 0.0), (0.8, 0.7, 0.9)
    ref, st = O.trace_bvh(sc, blob, rays, "clip", "closest", clip_lo=lo, clip_hi=hi)
    for regs in (0, 2, 8):
        p = V.trace_params(stack_regs=regs)
        hits, _ = V.trace(s, d_rays, "clip", "closest", params=p, clip_lo=lo, clip_hi=hi)
        _same_as_oracle(hits, ref, st, f"clip K={regs}")


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
                                                 ("alpha_tex", "closest", "dynamic")])
def test_null_params_use_the_tuned_configuration(V, kind, query, dispatch):
    sc, rays = scenes.small_quads(seed=scenes.SEED_BASE + 40)
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    d_rays = torch.from_numpy(rays).cuda()
    isect = V.intersector(kind, dispatch)
    scratch = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    tuned = V.vsr_trace_tune(s, d_rays, isect, query, scratch, image_width=256)
    p = V.params_dict(tuned)
    assert p["block_size"] in (64, 128, 256) and p["image_width"] == 256
    assert p["stack_regs"] in ((0, 1, 2, 4, 8) if dispatch == "static" else (0,))
    if dispatch == "dynamic":
        assert p["persistent"] == 0
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
