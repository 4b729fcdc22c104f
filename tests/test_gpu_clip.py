"""Clip-box intersector on the GPU vs the oracle, through the C ABI (needs a
GB300).  The intersector culls node boxes that miss the clip box and accepts
candidates whose hit point lies in it; hits, box and triangle test counts are
bit-identical to the oracle's culling traversal (near ties excluded).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BOXES = [((0.2, 0.1, 0.0), (0.7, 0.6, 1.0)), ((-1.0, 0.4, 0.35), (2.0, 2.0, 0.6))]


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


def _cmp(got, ref, st):
    r = O.hits_raw(ref).view(np.uint32)
    ok = st[:, 3] == 0
    bad = np.any(got.view(np.uint32) != r, axis=1) & ok
    assert not bad.any(), int(bad.sum())
    return ok


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("query", ["closest", "any"])
@pytest.mark.parametrize("box", BOXES)
def test_clip_vs_oracle(V, small, box, query, persistent):
    sc, rays, blob, s = small
    lo, hi = box
    ref, st = O.trace_bvh(sc, blob, rays, "clip", query, clip_lo=lo, clip_hi=hi)
    isect = V.intersector("clip", clip_lo=lo, clip_hi=hi)
    d = _dev(rays)
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    V.vsr_trace(s, d, isect, query, hits, None, V.trace_params(persistent=persistent))
    torch.cuda.synchronize()
    ok = _cmp(hits.cpu().numpy(), ref, st)
    stats = torch.empty((len(rays), 4), dtype=torch.int32, device="cuda")
    V.vsr_trace_stats(s, d, isect, query, hits, stats)
    torch.cuda.synchronize()
    g = stats.cpu().numpy().view(np.uint32)
    assert np.array_equal(g[ok, :3], st[ok, :3])
    assert (ref["prim"] != O.NONE).sum() > 1000
    assert V.vsr_get_device_error(s) == 0


def test_clip_multi_hit(V, small):
    sc, rays, blob, s = small
    lo, hi = BOXES[0]
    ref, st = O.trace_multi(sc, rays, 5, "clip", blob, clip_lo=lo, clip_hi=hi)
    hits = torch.empty((len(rays), 5, 4), dtype=torch.float32, device="cuda")
    V.vsr_trace_multi(s, _dev(rays), V.intersector("clip", clip_lo=lo, clip_hi=hi), 5, hits)
    torch.cuda.synchronize()
    got = hits.cpu().numpy()
    r = np.stack([ref["t"], ref["u"], ref["v"], ref["prim"].view(np.float32)], -1)
    bad = np.any(got.view(np.uint32) != r.view(np.uint32), axis=(1, 2)) & (st[:, 3] == 0)
    assert not bad.any()


def test_box_around_everything_is_default(V, small):
    sc, rays, blob, s = small
    d = _dev(rays)
    a, _ = V.trace(s, d, "clip", "closest", clip_lo=(-9, -9, -9), clip_hi=(9, 9, 9))
    b, _ = V.trace(s, d, "default", "closest")
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))


def test_refusals(V, small):
    sc, rays, blob, s = small
    d = _dev(rays[:64])
    hits = torch.empty((64, 4), dtype=torch.float32, device="cuda")
    lo, hi = BOXES[0]
    with pytest.raises(V.VsrError, match="static dispatch"):
        V.vsr_trace(s, d, V.intersector("clip", "dynamic", clip_lo=lo, clip_hi=hi), "closest", hits)
    with pytest.raises(V.VsrError, match="clip_lo <= clip_hi"):
        V.vsr_trace(s, d, V.intersector("clip", clip_lo=hi, clip_hi=lo), "closest", hits)
    with pytest.raises(V.VsrError, match="finite"):
        V.vsr_trace(s, d, V.intersector("clip", clip_lo=(0, float("nan"), 0), clip_hi=hi),
                    "closest", hits)
    img = torch.empty((64, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(V.VsrError, match="clip-box"):
        V.vsr_render(s, d, V.intersector("clip", clip_lo=lo, clip_hi=hi), V.shade_params((0, 0, 1)),
                     img)
