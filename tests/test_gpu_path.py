"""Diffuse path tracing on the GPU vs the oracle, through the C ABI (needs a
GB300).  Every segment is a closest-hit query with the intersector and every
bounce is built in FP32 with a fixed operation order, so radiance is
bit-identical to the oracle's for every path whose segments have no near-tie
flag; pixel tiles and dynamic dispatch give the same radiance.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
SKY = (0.7, 0.8, 1.0)
UNTEX = (0.8, 0.75, 0.6)


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


def _gpu(V, s, rays, kind, bounces, dirs, params=None, dispatch="static", eps=1e-4):
    n = rays.shape[0]
    rad = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    seg = torch.zeros(n, dtype=torch.int32, device="cuda")
    V.vsr_path_trace(s, _dev(rays), V.intersector(kind, dispatch),
                     V.path_params(bounces, eps, SKY, UNTEX), _dev(dirs), rad, seg, params)
    torch.cuda.synchronize()
    return rad.cpu().numpy(), seg.cpu().numpy()


@pytest.mark.parametrize("bounces", [0, 1, 3])
@pytest.mark.parametrize("kind", ["default", "alpha_tex", "proc_alpha"])
def test_small_vs_oracle(V, small, kind, bounces):
    sc, rays, blob, s = small
    dirs = scenes.path_dirs(len(rays), bounces)
    ref, flags = O.path_trace(sc, blob, rays, bounces, dirs, 1e-4, SKY, UNTEX, kind)
    got, seg = _gpu(V, s, rays, kind, bounces, dirs)
    ok = flags == 0
    assert np.array_equal(got[ok].view(np.uint32), ref[ok].view(np.uint32)), \
        int((np.any(got[ok] != ref[ok], axis=1)).sum())
    assert ok.mean() > 0.99
    assert np.all((seg >= 1) & (seg <= bounces + 1))
    if bounces:
        assert (ref.sum(1) > 0).mean() > 0.2 and (seg > 1).mean() > 0.2
    assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()


def test_tiles_and_dynamic_dispatch_agree(V, small):
    sc, rays, blob, s = small
    dirs = scenes.path_dirs(len(rays), 3)
    a, sa = _gpu(V, s, rays, "alpha_tex", 3, dirs)
    b, sb = _gpu(V, s, rays, "alpha_tex", 3, dirs, V.trace_params(image_width=256))
    c, sc_ = _gpu(V, s, rays, "alpha_tex", 3, dirs, dispatch="dynamic")
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32)) and np.array_equal(sa, sb)
    assert np.array_equal(a.view(np.uint32), c.view(np.uint32)) and np.array_equal(sa, sc_)
    # every segment in lock step (closest hit with speculative descent), one
    # ray per thread and persistent
    for p in (V.trace_params(lockstep=1),
              V.trace_params(lockstep=1, persistent=1, refill_threshold=16, watchdog_ms=10_000),
              V.trace_params(persistent=1, refill_threshold=8, image_width=256,
                             watchdog_ms=10_000)):
        d, sd = _gpu(V, s, rays, "alpha_tex", 3, dirs, p)
        assert np.array_equal(a.view(np.uint32), d.view(np.uint32)) and np.array_equal(sa, sd)
        # the same shapes with the callbacks reached through the tables
        d, sd = _gpu(V, s, rays, "alpha_tex", 3, dirs, p, dispatch="dynamic")
        assert np.array_equal(a.view(np.uint32), d.view(np.uint32)) and np.array_equal(sa, sd)


def test_ragged_sizes(V, small):
    sc, rays, blob, s = small
    for n in (1, 33, 4097):
        sel = np.resize(rays[::-1], (n, 8))
        dirs = scenes.path_dirs(n, 2, seed=n)
        ref, flags = O.path_trace(sc, blob, sel, 2, dirs, 1e-4, SKY, UNTEX, "alpha_tex")
        got, _ = _gpu(V, s, sel, "alpha_tex", 2, dirs)
        ok = flags == 0
        assert np.array_equal(got[ok].view(np.uint32), ref[ok].view(np.uint32))


def test_compaction_across_scan_chunks(V, small):
    """Live-path compaction between bounces: 300,001 paths make 1,172 blocks
    of 256, more than one 1,024-entry chunk of the block-count scan and a
    partial last block.  Radiance equals the oracle's, and the paths with a
    later segment are exactly those whose earlier segment hit."""
    sc, rays, blob, s = small
    n = 300_001
    sel = np.resize(rays, (n, 8))
    dirs = scenes.path_dirs(n, 2, seed=77)
    ref, flags = O.path_trace(sc, blob, sel, 2, dirs, 1e-4, SKY, UNTEX, "alpha_tex")
    got, seg = _gpu(V, s, sel, "alpha_tex", 2, dirs)
    ok = flags == 0
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok].view(np.uint32), ref[ok].view(np.uint32))
    assert (seg == 1).any() and (seg == 2).any() and (seg == 3).any()
    got_t, seg_t = _gpu(V, s, sel, "alpha_tex", 2, dirs, V.trace_params(octant=1))
    assert np.array_equal(got.view(np.uint32), got_t.view(np.uint32))
    assert np.array_equal(seg, seg_t)
    assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()


def test_argument_checks(V, small):
    sc, rays, blob, s = small
    d = _dev(rays[:64])
    rad = torch.empty((64, 3), dtype=torch.float32, device="cuda")
    dirs = _dev(scenes.path_dirs(64, 3))
    isect = V.intersector("default")
    with pytest.raises(V.VsrError, match="bounces"):
        V.vsr_path_trace(s, d, isect, V.path_params(65), dirs, rad)
    with pytest.raises(V.VsrError, match="ray_order"):
        V.vsr_path_trace(s, d, isect, V.path_params(3), dirs, rad, None,
                         V.trace_params(ray_order=1))
    with pytest.raises(V.VsrError, match="non-finite"):
        V.vsr_path_trace(s, d, isect, V.path_params(3, sky=(1.0, float("inf"), 1.0)), dirs, rad)
    with pytest.raises(V.VsrError, match="dirs"):
        V.vsr_path_trace(s, _dev(np.resize(rays, (1 << 16, 8))), isect, V.path_params(3), dirs,
                         torch.empty((1 << 16, 3), dtype=torch.float32, device="cuda"))


def test_forest_sample(V):
    """1920x1080 paths through the alpha-masked forest, 3 bounces, in the
    bench's launch configuration; a seeded sample against the oracle."""
    import bench
    sc, rays = scenes.billboard_forest()
    blob = sc.bvh()
    s = V.scene_from_inputs(sc, blob)
    try:
        dirs = scenes.path_dirs(len(rays), 3)
        got, seg = _gpu(V, s, rays, "alpha_tex", 3, dirs, bench.default_params(V),
                        eps=scenes.shadow_eps(sc))
        rng = np.random.default_rng(19)
        sel = np.sort(rng.choice(len(rays), 3000, replace=False))
        sdirs = dirs.reshape(len(rays), 3, 3)[sel].reshape(-1, 3)
        ref, flags = O.path_trace(sc, blob, rays[sel], 3, sdirs, scenes.shadow_eps(sc), SKY, UNTEX,
                                  "alpha_tex")
        ok = flags == 0
        assert ok.mean() > 0.98
        assert np.array_equal(got[sel][ok].view(np.uint32), ref[ok].view(np.uint32))
        assert (seg > 1).mean() > 0.5
        assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()
    finally:
        s.close()
