"""vsr_trace_persistent_noalloc: the persistent trace whose ray counter lives
in the library's static device array, for callers that must not allocate
device memory while tracing (an application whose device memory is all handed
to its own pool, or a frame loop that cannot take the synchronisation a fresh
cudaMalloc can bring).

Checked through the C ABI against the existing entry point (vsr_trace with a
persistent launch), on two calls in a row: the second call starts from the
counter value the first one left behind, so it also shows that the entry
point clears its scratch.  Results must be bit-identical, the bar of the other
parity tests.  This file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    sc, rays = scenes.small_quads()
    s = vsr.scene_from_inputs(sc, sc.bvh())
    yield vsr, s, torch.from_numpy(rays).cuda()
    s.close()


@pytest.mark.parametrize("kind,query", [("alpha_tex", "closest"), ("count", "any"),
                                        ("default", "any")])
def test_noalloc_matches_persistent_trace_twice(setup, kind, query):
    V, s, rays = setup
    n = rays.shape[0]
    params = V.trace_params(block_size=128, persistent=1, refill_threshold=16)
    isect = V.intersector(kind)
    want = kind == "count"
    ref = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ref_cnt = torch.empty((n, 2), dtype=torch.int32, device="cuda") if want else None
    V.vsr_trace(s, rays, isect, query, ref, ref_cnt, params)
    for _ in range(2):
        got = torch.full((n, 4), -7.0, dtype=torch.float32, device="cuda")
        cnt = torch.full((n, 2), -7, dtype=torch.int32, device="cuda") if want else None
        V.vsr_trace_persistent_noalloc(s, rays, isect, query, got, cnt, params)
        torch.cuda.synchronize()
        assert torch.equal(got.view(torch.int32), ref.view(torch.int32))
        if want:
            assert torch.equal(cnt, ref_cnt)
    assert V.vsr_get_device_error(s) == 0


def test_noalloc_rejects_more_rays_than_supported(setup):
    V, s, rays = setup
    hits = torch.empty((4, 4), dtype=torch.float32, device="cuda")
    limit = ((1 << 31) - 2) * 32  # one launch's limit
    with pytest.raises(V.VsrError, match="maximum of"):
        V.vsr_trace_persistent_noalloc(s, rays, V.intersector("default"), "closest", hits,
                                       n=limit + 1)
    with pytest.raises(V.VsrError, match="static dispatch"):
        V.vsr_trace_persistent_noalloc(s, rays, V.intersector("default", "dynamic"), "closest",
                                       hits)
