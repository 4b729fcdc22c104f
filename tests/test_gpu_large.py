"""Large incoherent workload on the GPU (needs a GB300): 16 M triangles (7 M
procedurally alpha-masked quads plus a 2 M-triangle heightfield), 1920x1080
primary rays and 4 ambient-occlusion rays per pixel (tmax 0.5).

Checks: primary closest hits on a seeded sample against the oracle; the GPU
ambient-occlusion ray construction against the oracle's (origins bit-exact,
directions within 2e-6); any-hit parity on oracle-made AO rays for the
procedural-alpha and counting intersectors in static and dynamic dispatch;
whole-launch invariants over all 8.3 M AO rays; the ambient-occlusion render
and its texel adjoint against the FP64 reference.
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


def test_octant_primary_full_frame(large):
    """The 16 M-triangle frame's primary closest hits with the box test
    specialised to each warp's direction octant (pixel tiles, as the
    benchmark runs them) equal the generic kernel's bit for bit, and a
    seeded sample equals the oracle's."""
    V, sc, rays, blob, s, xi, eps = large
    proc = V.intersector("proc_alpha")
    d_rays = torch.from_numpy(rays).cuda()
    h0 = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    h1 = torch.empty_like(h0)
    V.vsr_trace(s, d_rays, proc, "closest", h0, None, V.trace_params(image_width=1920))
    V.vsr_trace(s, d_rays, proc, "closest", h1, None,
                V.trace_params(image_width=1920, octant=1))
    torch.cuda.synchronize()
    assert torch.equal(h0.view(torch.int32), h1.view(torch.int32))
    sel = np.sort(np.random.default_rng(23).choice(len(rays), 3000, replace=False))
    ref, st = O.trace_bvh(sc, blob, rays[sel], "proc_alpha", "closest")
    _cmp(h1.cpu().numpy()[sel], ref, st, "octant primary")
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


def test_ao_render_and_texel_gradients(large):
    """c = albedo(uv) * (1 - occluded fraction of 4 AO rays) and its gradient
    with respect to the colour texels at fixed visibility, against the FP64
    reference, whose occlusion comes from the oracle's own AO rays and
    traversal and whose uv is interpolated at the oracle's FP32 barycentrics.  Pixels whose primary primitive or occluded count differs
    (primary near-ties; AO directions agree only to 2e-6) are counted and
    bounded, and left out of the comparison by zeroing their adjoint on both
    sides."""
    from oracle import adjoint as A
    V, sc, rays, blob, s, xi, eps = large
    ref, st = O.trace_bvh(sc, blob, rays, "proc_alpha", "closest")
    ao = O.ao_rays(sc, rays, O.hits_raw(ref), SPP, xi, TMAX, eps)
    aoh, _ = O.trace_bvh(sc, blob, ao, "proc_alpha", "any")
    occ = (aoh["prim"] != O.NONE).reshape(-1, SPP).mean(1)
    bary = np.stack([ref["u"], ref["v"]], 1)
    fa = A.FrozenAO(sc, rays, ref["prim"], 1.0 - occ, bary=bary)
    tex = sc.textures[0].texels
    proc = V.intersector("proc_alpha")
    shade = V.shade_params((0.0, 0.0, 1.0), grad_tex=0)
    d_rays = torch.from_numpy(rays).cuda()
    d_xi = torch.from_numpy(xi).cuda()
    hits = torch.empty((len(rays), 4), dtype=torch.float32, device="cuda")
    img = torch.empty((len(rays), 3), dtype=torch.float32, device="cuda")
    gocc = torch.empty(len(rays), dtype=torch.float32, device="cuda")
    V.vsr_render_ao(s, d_rays, proc, SPP, d_xi, TMAX, eps, shade, img, hits, gocc)
    torch.cuda.synchronize()
    _cmp(hits.cpu().numpy(), ref, st, "ao render primary")
    gprim = hits.cpu().numpy()[:, 3].view(np.uint32)
    same = (gprim == ref["prim"]) & (np.abs(gocc.cpu().numpy() - occ) < 1e-6)
    assert (~same).sum() <= 1e-3 * len(rays), int((~same).sum())
    assert np.all(same[(gprim == O.NONE) & (ref["prim"] == O.NONE)])
    ref_img = fa.image(A._t(sc.verts), A._t(tex)).numpy()
    # FP32 uv interpolation (<= 4 ulp(1)) and texel coordinate (<= ulp(1024)/2)
    # move the bilinear weights; times the texture's largest neighbour step
    step = max(np.abs(np.diff(tex[..., :3], axis=a)).max() for a in (0, 1))
    tol = 2 * step * (4 * 2.0 ** -23 * tex.shape[1] + 2.0 ** -14) + 1e-6
    err = np.abs(img.cpu().numpy()[same] - ref_img[same]).max(1)
    assert err.max() < tol, (err.max(), tol)
    rng = np.random.default_rng(31)
    tt = tex.copy()
    tt[..., :3] += (0.01 * rng.standard_normal(tex[..., :3].shape)).astype(np.float32)
    target = fa.image(A._t(sc.verts), A._t(tt)).numpy()
    _, _, _, g = fa.loss_grad(sc.verts, tex, target)
    g[~same] = 0.0
    _, gt_ref = fa.vjp(sc.verts, tex, g)
    gt = torch.zeros(tex.shape, dtype=torch.float32, device="cuda")
    V.vsr_render_ao_backward(s, hits, gocc, shade, torch.from_numpy(g.astype(np.float32)).cuda(),
                             gt)
    torch.cuda.synchronize()
    gt = gt.cpu().numpy()
    rel = np.linalg.norm(gt - gt_ref) / np.linalg.norm(gt_ref)
    assert rel < 1e-3, rel
    assert np.all(gt[..., 3] == 0)
    # central differences of the loss over the agreeing pixels: exact up to
    # rounding, since the loss is quadratic in the texels at fixed visibility
    fa_same = A.FrozenAO(sc, rays, np.where(same, ref["prim"], O.NONE), 1.0 - occ, bary=bary)
    tj = rng.integers(0, tex.shape[0], 256)
    ti = rng.integers(0, tex.shape[1], 256)
    tc = rng.integers(0, 3, 256)
    fd = np.array([fa_same.fd_texel(sc.verts, tex, target, j, i, c)
                   for j, i, c in zip(tj, ti, tc)])
    assert np.count_nonzero(fd) > 128
    assert np.linalg.norm(gt[tj, ti, tc] - fd) <= 1e-3 * np.linalg.norm(fd)
    assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()
