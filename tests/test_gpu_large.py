"""Large incoherent workload on the GPU (needs a GB300): 16 M triangles (7 M
procedurally alpha-masked quads plus a 2 M-triangle heightfield), 1920x1080
primary rays and 4 ambient-occlusion rays per pixel (tmax 0.5).

Checks: primary closest hits on a seeded sample against the oracle; the GPU
ambient-occlusion ray construction against the oracle's (origins bit-exact,
directions within 2e-6); any-hit parity on oracle-made AO rays for the
procedural-alpha and counting intersectors in static and dynamic dispatch;
whole-launch invariants over all 8.3 M AO rays.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
SPP, TMAX = 4, 0.5


@pytest.fixture(scope="module")
def large():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    sc, rays = scenes.large_incoherent()
    blob = sc.bvh()
    s = vsr.scene_from_inputs(sc, blob)
    xi = scenes.ao_random(len(rays), SPP)
    eps = scenes.shadow_eps(sc)
    yield vsr, sc, rays, blob, s, xi, eps
    s.close()


def _cmp(got, ref, st, label):
    g = got.view(np.uint32)
    r = O.hits_raw(ref).view(np.uint32)
    ties = st[:, 3] != 0
    bad = np.any(g != r, axis=1) & ~ties
    assert not bad.any(), f"{label}: {int(bad.sum())} rays differ"


def test_primary_and_ao_parity_on_a_sample(large):
    V, sc, rays, blob, s, xi, eps = large
    proc = V.intersector("proc_alpha")
    d_rays = torch.from_numpy(rays).cuda()
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    V.vsr_trace(s, d_rays, proc, "closest", hits)
    torch.cuda.synchronize()
    rng = np.random.default_rng(21)
    sel = np.sort(rng.choice(len(rays), 6000, replace=False))
    ref, st = O.trace_bvh(sc, blob, rays[sel], "proc_alpha", "closest")
    _cmp(hits.cpu().numpy()[sel], ref, st, "primary")
    # AO rays made by the oracle from its own primary hits, traced by both
    xs = xi.reshape(len(rays), SPP, 2)[sel].reshape(-1, 2)
    ao = O.ao_rays(sc, rays[sel], O.hits_raw(ref), SPP, xs, TMAX, eps)
    d_ao = torch.from_numpy(ao).cuda()
    for kind in ("proc_alpha", "count"):
        r_h, r_st = O.trace_bvh(sc, blob, ao, kind, "any")
        for disp in ("static", "dynamic"):
            h, cnt = V.trace(s, d_ao, kind, "any", disp, counters=(kind == "count"))
            torch.cuda.synchronize()
            _cmp(h.cpu().numpy(), r_h, r_st, f"ao {kind}/{disp}")
            if kind == "count":
                assert np.array_equal(cnt.cpu().numpy().view(np.uint32), r_st[:, :2])
    # the GPU's own AO construction from the same (oracle) primary hits
    d_prim = torch.from_numpy(np.ascontiguousarray(rays[sel])).cuda()
    d_hits = torch.from_numpy(O.hits_raw(ref)).cuda()
    out = torch.empty((len(sel) * SPP, 8), dtype=torch.float32, device="cuda")
    V.vsr_make_ao_rays(s, d_prim, d_hits, SPP, torch.from_numpy(xs).cuda(), TMAX, eps, out)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    assert np.array_equal(g[:, [0, 1, 2, 3, 7]].view(np.uint32), ao[:, [0, 1, 2, 3, 7]].view(np.uint32))
    assert np.abs(g[:, 4:7] - ao[:, 4:7]).max() < 2e-6
    assert V.vsr_get_device_error(s) == 0


def test_full_ao_pass_invariants(large):
    """All 8.3 M AO rays: static == dynamic dispatch and bvh_costs hits ==
    default hits, bit for bit; about half the pixels hit geometry."""
    V, sc, rays, blob, s, xi, eps = large
    d_rays = torch.from_numpy(rays).cuda()
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    V.vsr_trace(s, d_rays, V.intersector("proc_alpha"), "closest", hits)
    ao = torch.empty((len(rays) * SPP, 8), dtype=torch.float32, device="cuda")
    V.vsr_make_ao_rays(s, d_rays, hits, SPP, torch.from_numpy(xi).cuda(), TMAX, eps, ao)
    a, _ = V.trace(s, ao, "proc_alpha", "any")
    b, _ = V.trace(s, ao, "proc_alpha", "any", "dynamic")
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    c, cnt = V.trace(s, ao, "count", "any", counters=True)
    cd, cntd = V.trace(s, ao, "count", "any", "dynamic", counters=True)
    d, _ = V.trace(s, ao, "default", "any")
    assert torch.equal(c.view(torch.int32), d.view(torch.int32))
    assert torch.equal(cd.view(torch.int32), d.view(torch.int32)) and torch.equal(cnt, cntd)
    active = (ao[:, 7] > 0).float().mean().item()
    assert 0.3 < active < 0.99
    assert V.vsr_get_device_error(s) == 0
