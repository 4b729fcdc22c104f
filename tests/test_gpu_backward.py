"""Differentiable render and its adjoint on the GPU vs the FP64 reference.

Workload: the displaced icosphere (64,980 triangles, 32,492 vertices, RGBA32F
512x512 albedo with alpha cutout at 0.3), 512x512 primary rays, closest hit
with the alpha-texture intersector, diffuse shading under one directional
light, L2 loss to an image rendered from perturbed vertices and texels.

Bars: hits bit-exact with the oracle; image within 2e-5 of the FP64 shading;
gradients within 1e-3 (norm-wise relative) of the FP64 autograd reference and
of central differences (h = 1e-3, Richardson-extrapolated with h = 5e-4; plain
central differences at h = 1e-3 carry about 1.4e-3 truncation error on this
mesh and are held to 2e-3).  The upstream gradient given to the GPU is
computed from the oracle's image, so no reference input comes from the GPU.
"""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import oracle as O
from paper_1912_12786_gb300.inputs import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sphere():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_12786_gb300 import _build, vsr
    _build.build()
    sc, rays, tv, tt = scenes.displaced_icosphere()
    blob = sc.bvh()
    ref_hits, st = O.trace_bvh(sc, blob, rays, "alpha_tex", "closest", cutoff_f=0.3)
    light = scenes.light_dir_f32()
    fs = A.FrozenShading(sc, rays, ref_hits["prim"], light.astype(np.float64))
    target = fs.image(A._t(tv), A._t(tt)).numpy()
    loss, gv_ref, gt_ref, g = fs.loss_grad(sc.verts, sc.textures[0].texels, target)
    s = vsr.scene_from_inputs(sc, blob)
    yield dict(V=vsr, sc=sc, rays=rays, blob=blob, ref_hits=ref_hits, st=st, fs=fs,
               target=target, gv_ref=gv_ref, gt_ref=gt_ref, g=g, s=s, light=light)
    s.close()


def _gpu_grads(d, g, misaligned=False):
    """Vertex and texel gradients of the render; with `misaligned` the texel
    gradient array starts 4 bytes past a 16-byte boundary (scalar atomics)."""
    V, s = d["V"], d["s"]
    rays = torch.from_numpy(d["rays"]).cuda()
    gv = torch.zeros((d["sc"].verts.shape[0], 3), dtype=torch.float32, device="cuda")
    shape = d["sc"].textures[0].texels.shape
    if misaligned:
        gt = torch.zeros(int(np.prod(shape)) + 1, dtype=torch.float32, device="cuda")[1:].view(shape)
        assert gt.data_ptr() % 16 == 4
    else:
        gt = torch.zeros(shape, dtype=torch.float32, device="cuda")
    V.vsr_trace_backward(s, rays, V.intersector("alpha_tex", cutoff_f=0.3),
                         V.shade_params(d["light"]), torch.from_numpy(g.astype(np.float32)).cuda(),
                         gv, gt)
    torch.cuda.synchronize()
    return gv.cpu().numpy(), gt.cpu().numpy()


def test_render_forward(sphere):
    d = sphere
    V = d["V"]
    rays = torch.from_numpy(d["rays"]).cuda()
    img = torch.empty((len(d["rays"]), 3), dtype=torch.float32, device="cuda")
    hits = torch.empty((len(d["rays"]), 4), dtype=torch.float32, device="cuda")
    V.vsr_render(d["s"], rays, V.intersector("alpha_tex", cutoff_f=0.3),
                 V.shade_params(d["light"]), img, hits)
    torch.cuda.synchronize()
    gh = hits.cpu().numpy().view(np.uint32)
    rh = O.hits_raw(d["ref_hits"]).view(np.uint32)
    ties = d["st"][:, 3] != 0
    assert np.array_equal(gh[~ties], rh[~ties])
    ref_img = d["fs"].image(A._t(d["sc"].verts), A._t(d["sc"].textures[0].texels)).numpy()
    assert np.abs(img.cpu().numpy() - ref_img).max() < 2e-5
    hit_frac = float((rh[:, 3] != O.NONE).mean())
    assert 0.3 < hit_frac < 0.6
    assert V.vsr_get_device_error(d["s"]) == 0, V.vsr_last_error()


def test_backward_matches_fp64_reference(sphere):
    d = sphere
    gv, gt = _gpu_grads(d, d["g"])
    assert _rel(gv, d["gv_ref"]) < 1e-3
    assert _rel(gt, d["gt_ref"]) < 1e-3
    big = np.abs(d["gv_ref"]) > 1e-3 * np.abs(d["gv_ref"]).max()
    err = np.abs(gv - d["gv_ref"])[big] / np.abs(d["gv_ref"])[big]
    assert np.quantile(err, 0.99) < 1e-2
    assert np.all(gt[..., 3] == 0)
    # scalar texel atomics (misaligned array) give the same sums
    gv2, gt2 = _gpu_grads(d, d["g"], misaligned=True)
    assert np.allclose(gt2, gt, rtol=1e-4, atol=1e-6 * np.abs(gt).max())
    assert np.allclose(gv2, gv, rtol=1e-4, atol=1e-6 * np.abs(gv).max())
    assert d["V"].vsr_get_device_error(d["s"]) == 0, d["V"].vsr_last_error()


def test_backward_matches_central_differences(sphere):
    d = sphere
    fs, sc, target = d["fs"], d["sc"], d["target"]
    verts, tex = sc.verts, sc.textures[0].texels
    gv, gt = _gpu_grads(d, d["g"])
    rng = np.random.default_rng(11)
    ks = rng.choice(np.unique(fs.idx), 171, replace=False)
    fd1, fdr, got = [], [], []
    for k in ks:
        for ax in range(3):
            a, kink_a = fs.fd_vertex(verts, tex, target, int(k), ax, h=1e-3)
            b, kink_b = fs.fd_vertex(verts, tex, target, int(k), ax, h=5e-4)
            if kink_a or kink_b:
                continue  # stencil crosses a bilinear cell or shading kink
            fd1.append(a)
            fdr.append((4 * b - a) / 3)
            got.append(gv[k, ax])
    assert len(got) > 150
    got, fd1, fdr = map(np.array, (got, fd1, fdr))
    assert _rel(got, fdr) < 1e-3
    assert _rel(got, fd1) < 2e-3
    tj = rng.integers(0, tex.shape[0], 512)
    ti = rng.integers(0, tex.shape[1], 512)
    tc = rng.integers(0, 3, 512)
    fdt = np.array([fs.fd_texel(verts, tex, target, j, i, c) for j, i, c in zip(tj, ti, tc)])
    assert _rel(gt[tj, ti, tc], fdt) < 1e-3


def test_render_in_every_launch_shape(sphere):
    """The render is the trace kernels plus a shading pass, so every launch
    configuration of vsr_trace gives the same image and hit records; the
    re-tracing adjoint likewise."""
    d = sphere
    V, s = d["V"], d["s"]
    rays = torch.from_numpy(d["rays"]).cuda()
    n = len(d["rays"])
    isect = V.intersector("alpha_tex", cutoff_f=0.3)
    shade = V.shade_params(d["light"])
    ref_img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    ref_hits = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    V.vsr_render(s, rays, isect, shade, ref_img, ref_hits)
    for p in (V.trace_params(image_width=512, block_size=64),
              V.trace_params(persistent=1, refill_threshold=16, watchdog_ms=10_000),
              V.trace_params(persistent=1, lockstep=1, refill_threshold=24, watchdog_ms=10_000),
              V.trace_params(lockstep=1, stack_regs=4)):
        img = torch.full_like(ref_img, -1.0)
        hits = torch.full_like(ref_hits, -1.0)
        V.vsr_render(s, rays, isect, shade, img, hits, p)
        img2 = torch.full_like(ref_img, -1.0)
        V.vsr_render(s, rays, isect, shade, img2, None, p)
        torch.cuda.synchronize()
        assert torch.equal(img.view(torch.int32), ref_img.view(torch.int32))
        assert torch.equal(img2.view(torch.int32), ref_img.view(torch.int32))
        assert torch.equal(hits.view(torch.int32), ref_hits.view(torch.int32))
        gv = torch.zeros((d["sc"].verts.shape[0], 3), dtype=torch.float32, device="cuda")
        g = torch.from_numpy(d["g"].astype(np.float32)).cuda()
        V.vsr_trace_backward(s, rays, isect, shade, g, gv, None, p)
        torch.cuda.synchronize()
        assert _rel(gv.cpu().numpy(), d["gv_ref"]) < 1e-3
    assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()


def test_backward_from_saved_hits(sphere):
    """The adjoint from the forward's hit records (no re-trace) equals the
    re-tracing adjoint up to the order of the atomics, and the FP64
    reference; misses and out-of-range records are skipped, the latter
    flagged (error bit 3)."""
    d = sphere
    V, s = d["V"], d["s"]
    rays = torch.from_numpy(d["rays"]).cuda()
    n = len(d["rays"])
    isect = V.intersector("alpha_tex", cutoff_f=0.3)
    shade = V.shade_params(d["light"])
    img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    hits = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    V.vsr_render(s, rays, isect, shade, img, hits)
    g = torch.from_numpy(d["g"].astype(np.float32)).cuda()
    gv = torch.zeros((d["sc"].verts.shape[0], 3), dtype=torch.float32, device="cuda")
    gt = torch.zeros(d["sc"].textures[0].texels.shape, dtype=torch.float32, device="cuda")
    V.vsr_render_backward_hits(s, rays, hits, shade, g, gv, gt)
    torch.cuda.synchronize()
    gv, gt = gv.cpu().numpy(), gt.cpu().numpy()
    rv, rt = _gpu_grads(d, d["g"])
    assert np.allclose(gv, rv, rtol=1e-4, atol=1e-6 * np.abs(rv).max())
    assert np.allclose(gt, rt, rtol=1e-4, atol=1e-6 * np.abs(rt).max())
    assert _rel(gv, d["gv_ref"]) < 1e-3 and _rel(gt, d["gt_ref"]) < 1e-3
    assert np.all(gt[..., 3] == 0)
    assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()
    # vertex gradients only (no texel array)
    gv2 = torch.zeros((d["sc"].verts.shape[0], 3), dtype=torch.float32, device="cuda")
    V.vsr_render_backward_hits(s, rays, hits, shade, g, gv2, None)
    torch.cuda.synchronize()
    assert np.allclose(gv2.cpu().numpy(), rv, rtol=1e-4, atol=1e-6 * np.abs(rv).max())
    # a record out of range is skipped and flagged, never dereferenced
    prim = hits[:, 3].contiguous().view(torch.int32)
    k = int(torch.nonzero(prim != -1)[0].item())
    bad = hits.clone()
    bad[k, 3] = torch.tensor([d["sc"].ntri + 7], dtype=torch.int32).view(torch.float32)[0]
    gk = torch.zeros_like(g)
    gk[k] = 1.0
    gv3 = torch.zeros_like(gv2)
    V.vsr_render_backward_hits(s, rays, bad, shade, gk, gv3, None)
    torch.cuda.synchronize()
    assert torch.count_nonzero(gv3) == 0
    assert V.vsr_get_device_error(s) & 8
    assert V.vsr_get_device_error(s) == 0
    host = np.zeros((n, 4), np.float32)

    class HostTensor:  # host memory where device memory is required
        shape = host.shape

        def data_ptr(self):
            return host.ctypes.data

    with pytest.raises(V.VsrError, match="device memory"):
        V.vsr_render_backward_hits(s, rays, HostTensor(), shade, g, gv2, None)


def test_autograd_function_and_scene_update(sphere):
    """RenderFunction gives the same image and gradients as the direct calls;
    a vertex update refits the BVH so traces stay exact."""
    from paper_1912_12786_gb300.autograd import render
    d = sphere
    V, sc = d["V"], d["sc"]
    rays = torch.from_numpy(d["rays"]).cuda()
    isect = V.intersector("alpha_tex", cutoff_f=0.3)
    shade = V.shade_params(d["light"])
    verts = torch.from_numpy(sc.verts.copy()).cuda().requires_grad_(True)
    tex = torch.from_numpy(sc.textures[0].texels.copy()).cuda().requires_grad_(True)
    img = render(d["s"], rays, verts, tex, isect, shade)
    tgt = torch.from_numpy(d["target"].astype(np.float32)).cuda()
    loss = ((img - tgt) ** 2).sum()
    loss.backward()
    g = 2.0 * (img.detach() - tgt)
    gv, gt = _gpu_grads(d, g.cpu().numpy())
    assert np.allclose(verts.grad.cpu().numpy(), gv, rtol=1e-4, atol=1e-6 * np.abs(gv).max())
    assert np.allclose(tex.grad.cpu().numpy(), gt, rtol=1e-4, atol=1e-6 * np.abs(gt).max())
    # the re-tracing backward (no hit records kept) gives the same gradients
    verts.grad = None
    tex.grad = None
    img2 = render(d["s"], rays, verts, tex, isect, shade, save_hits=False)
    assert torch.equal(img2, img)
    ((img2 - tgt) ** 2).sum().backward()
    assert np.allclose(verts.grad.cpu().numpy(), gv, rtol=1e-4, atol=1e-6 * np.abs(gv).max())
    assert np.allclose(tex.grad.cpu().numpy(), gt, rtol=1e-4, atol=1e-6 * np.abs(gt).max())
    # move the vertices: the refit BVH must give the same closest hits as a
    # BVH built from scratch over the moved mesh (default intersector)
    moved = (sc.verts * np.float32(1.03) + np.float32(0.01)).astype(np.float32)
    V.vsr_scene_update(d["s"], torch.from_numpy(moved).cuda())
    msc = scenes.Scene("moved", moved, sc.idx, sc.uvs, sc.geom_id, sc.textures)
    ref, st = O.trace_bvh(msc, msc.bvh(), d["rays"], "default", "closest")
    hits, _ = V.trace(d["s"], rays, "default", "closest")
    gh = hits.cpu().numpy().view(np.uint32)
    ties = st[:, 3] != 0
    assert np.array_equal(gh[~ties, 3], O.hits_raw(ref).view(np.uint32)[~ties, 3])
    V.vsr_scene_update(d["s"], torch.from_numpy(sc.verts).cuda())
    assert V.vsr_get_device_error(d["s"]) == 0


def test_ao_render_after_tuning_the_any_hit_query(sphere):
    """The AO render traces its occlusion rays at the configuration tuned for
    the scene and the any-hit query; the counts, and so the image, are the
    same whichever configuration runs."""
    d = sphere
    V, sc, s = d["V"], d["sc"], d["s"]
    spp, tmax, eps = 4, 0.5, scenes.shadow_eps(sc)
    n = len(d["rays"])
    rays = torch.from_numpy(d["rays"]).cuda()
    xi = torch.from_numpy(scenes.ao_random(n, spp)).cuda()
    isect = V.intersector("alpha_tex", cutoff_f=0.3)
    shade = V.shade_params((0.0, 0.0, 1.0), grad_tex=0)
    out = []
    for tune in (False, True):
        if tune:
            ao = torch.empty((n * spp, 8), dtype=torch.float32, device="cuda")
            V.vsr_make_ao_rays(s, rays, out[0][1], spp, xi, tmax, eps, ao)
            scratch = torch.empty((n * spp, 4), dtype=torch.float32, device="cuda")
            V.vsr_trace_tune(s, ao, isect, "any", scratch)
        img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        hits = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        occ = torch.empty(n, dtype=torch.float32, device="cuda")
        V.vsr_render_ao(s, rays, isect, spp, xi, tmax, eps, shade, img, hits, occ)
        torch.cuda.synchronize()
        out.append((img, hits, occ))
    for x, y in zip(out[0], out[1]):
        assert torch.equal(x.view(torch.int32), y.view(torch.int32))
    assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()


def test_ao_render_autograd_and_bad_hit_records(sphere):
    """Ambient-occlusion render on the icosphere (4 occlusion rays per pixel,
    tmax 0.5): hits bit-exact with the oracle, occlusion equal to the oracle's
    on all but a few pixels, texel gradients of AORenderFunction equal to the
    direct backward call and within 1e-3 of the FP64 reference on the pixels
    whose occlusion agrees.  A hit record naming a primitive out of range is
    skipped by the backward and by vsr_make_ao_rays, and sets error bit 3."""
    from paper_1912_12786_gb300.autograd import render_ao
    d = sphere
    V, sc, s = d["V"], d["sc"], d["s"]
    spp, tmax, eps = 4, 0.5, scenes.shadow_eps(sc)
    n = len(d["rays"])
    xi_h = scenes.ao_random(n, spp)
    rays, xi = torch.from_numpy(d["rays"]).cuda(), torch.from_numpy(xi_h).cuda()
    isect = V.intersector("alpha_tex", cutoff_f=0.3)
    shade = V.shade_params((0.0, 0.0, 1.0), grad_tex=0)
    tex0 = sc.textures[0].texels
    img = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    hits = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    occ = torch.empty(n, dtype=torch.float32, device="cuda")
    V.vsr_render_ao(s, rays, isect, spp, xi, tmax, eps, shade, img, hits, occ)
    torch.cuda.synchronize()
    ref, st = d["ref_hits"], d["st"]
    gh = hits.cpu().numpy().view(np.uint32)
    ties = st[:, 3] != 0
    assert np.array_equal(gh[~ties], O.hits_raw(ref).view(np.uint32)[~ties])
    ao = O.ao_rays(sc, d["rays"], O.hits_raw(ref), spp, xi_h, tmax, eps)
    aoh, _ = O.trace_bvh(sc, d["blob"], ao, "alpha_tex", "any", cutoff_f=0.3)
    occ_ref = (aoh["prim"] != O.NONE).reshape(-1, spp).mean(1)
    same = (gh[:, 3] == ref["prim"]) & (np.abs(occ.cpu().numpy() - occ_ref) < 1e-6)
    assert (~same).sum() <= 1e-3 * n and 0.05 < occ_ref[ref["prim"] != O.NONE].mean() < 0.95
    fa = A.FrozenAO(sc, d["rays"], ref["prim"], 1.0 - occ_ref,
                    bary=np.stack([ref["u"], ref["v"]], 1))
    ref_img = fa.image(A._t(sc.verts), A._t(tex0)).numpy()
    assert np.abs(img.cpu().numpy()[same] - ref_img[same]).max() < 2e-5
    # upstream gradient from the oracle's image, zero where occlusion differs
    g_ref = np.where(same[:, None], 2.0 * (ref_img - 0.5), 0.0)
    g = torch.from_numpy(g_ref.astype(np.float32)).cuda()
    # autograd against the direct calls (same hits and occlusion, same kernels)
    tex = torch.from_numpy(tex0.copy()).cuda().requires_grad_(True)
    img2 = render_ao(s, rays, tex, isect, spp, xi, tmax, eps, shade)
    assert torch.equal(img2, img)
    img2.backward(g)
    gt = torch.zeros_like(tex)
    V.vsr_render_ao_backward(s, hits, occ, shade, g, gt)
    torch.cuda.synchronize()
    gt = gt.cpu().numpy()
    assert np.allclose(tex.grad.cpu().numpy(), gt, rtol=1e-4, atol=1e-6 * np.abs(gt).max())
    # FP64 reference at the oracle's barycentrics and occlusion
    _, gt_ref = fa.vjp(sc.verts, tex0, g_ref)
    assert _rel(gt, gt_ref) < 1e-3
    assert np.all(gt[..., 3] == 0)
    # a gradient array that is 4- but not 16-byte aligned takes scalar
    # atomics instead of one vector atomic per texel: the same sums
    buf = torch.zeros(tex.numel() + 1, dtype=torch.float32, device="cuda")
    gmis = buf[1:].view(tex.shape)
    assert gmis.data_ptr() % 16 == 4
    V.vsr_render_ao_backward(s, hits, occ, shade, g, gmis)
    torch.cuda.synchronize()
    assert np.allclose(gmis.cpu().numpy(), gt, rtol=1e-4, atol=1e-6 * np.abs(gt).max())
    assert buf[0].item() == 0.0
    assert V.vsr_get_device_error(s) == 0, V.vsr_last_error()
    # hit records out of range: skipped and flagged, never dereferenced
    k = int(np.flatnonzero(gh[:, 3] != O.NONE)[0])
    bad = hits.clone()
    bad[k, 3] = torch.tensor([sc.ntri + 5], dtype=torch.int32).view(torch.float32)[0]
    gt2 = torch.zeros_like(tex)
    gk = torch.zeros_like(g)
    gk[k] = 1.0
    V.vsr_render_ao_backward(s, bad, occ, shade, gk, gt2)
    torch.cuda.synchronize()
    assert torch.count_nonzero(gt2) == 0
    assert V.vsr_get_device_error(s) & 8
    out = torch.empty((n * spp, 8), dtype=torch.float32, device="cuda")
    V.vsr_make_ao_rays(s, rays, bad, spp, xi, tmax, eps, out)
    torch.cuda.synchronize()
    assert torch.all(out[k * spp:(k + 1) * spp, 7] < 0)
    assert V.vsr_get_device_error(s) & 8
    assert V.vsr_get_device_error(s) == 0
