"""FP64 reference for differentiable shading at fixed visibility.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU legs may import this module.  It shares no code with the GPU
library.

The paper defines visibility queries only; gradients are an extension built
on its closest-hit query with a custom intersector.  The shaded image is

    c = albedo_rgb(uv) * max(0, n_f . L)        (hit)
    c = background                              (miss)

where, for the frozen primitive p of each pixel (taken from the oracle's FP32
closest-hit traversal), (t, u, v) solve  o + t d = v0 + u (v1 - v0) + v (v2 - v0)
in FP64 (evaluated even when the point leaves the triangle: visibility is
fixed), uv = (1 - u - v) tc0 + u tc1 + v tc2, albedo is the bilinear lookup
with texel centres at ((i + 0.5)/W, (j + 0.5)/H) and clamp-to-edge texel
indices, n = normalize((v1 - v0) x (v2 - v0)) flipped to face the ray, and L
is the unit vector toward a directional light.  The loss is the squared L2
distance to a target image.

The forward pass is written plainly with float64 torch CPU ops; the reference
gradient is torch autograd of that forward (no hand-derived adjoint), so it is
independent of the GPU kernel's hand-written one.  It is pinned by central
finite differences of the same forward and by closed forms in the tests.
"""
from __future__ import annotations

import numpy as np
import torch

NONE = 0xFFFFFFFF


def _t(x):
    return torch.as_tensor(np.asarray(x), dtype=torch.float64)


class FrozenShading:
    """Shading of the pixels whose primitive is fixed.

    scene   inputs.scenes.Scene with one RGBA32F texture (index `tex`) for
            textured triangles; untextured triangles have albedo 1
    rays    float32 [n, 8]; prims uint32 [n] (0xFFFFFFFF = miss)
    """

    def __init__(self, scene, rays, prims, light, background=(0.0, 0.0, 0.0), tex=0):
        prims = np.asarray(prims, np.uint32)
        self.n = len(prims)
        self.hit = np.flatnonzero(prims != NONE)
        p = prims[self.hit].astype(np.int64)
        self.prim = p
        self.idx = np.asarray(scene.idx, np.int64)[p]                    # [m, 3]
        self.o = _t(rays[self.hit, 0:3])
        self.d = _t(rays[self.hit, 4:7])
        self.tc = _t(scene.uvs[p])                                         # [m, 3, 2]
        geom = np.asarray(scene.geom_id, np.uint32)[p]
        if np.any((geom != NONE) & (geom != tex)):
            raise NotImplementedError("one differentiable texture per scene")
        self.textured = torch.as_tensor(geom == tex)
        self.light = _t(light)
        self.background = _t(background)
        t = scene.textures[tex]
        assert t.fmt == "rgba32f"
        self.W, self.H = t.w, t.h

    # -- forward ---------------------------------------------------------

    def _surface(self, verts, sel):
        """FP64 (uv, e1, e2, d, textured) of the frozen triangles."""
        idx = self.idx if sel is None else self.idx[sel]
        o = self.o if sel is None else self.o[sel]
        d = self.d if sel is None else self.d[sel]
        tc = self.tc if sel is None else self.tc[sel]
        textured = self.textured if sel is None else self.textured[sel]
        a = verts[idx[:, 0]]
        b = verts[idx[:, 1]]
        c = verts[idx[:, 2]]
        e1 = b - a
        e2 = c - a
        # solve [-d, e1, e2] (t, u, v)^T = o - a
        M = torch.stack([-d, e1, e2], dim=2)
        tuv = torch.linalg.solve(M, (o - a).unsqueeze(-1)).squeeze(-1)
        u, v = tuv[:, 1], tuv[:, 2]
        uv = (1 - u - v)[:, None] * tc[:, 0] + u[:, None] * tc[:, 1] + v[:, None] * tc[:, 2]
        return uv, e1, e2, d, textured

    def colours(self, verts, texels, sel=None):
        """FP64 colours of the hit pixels (or of the subset `sel` of them)."""
        uv, e1, e2, d, textured = self._surface(verts, sel)
        alb = self.bilinear(texels, uv)
        alb = torch.where(textured[:, None], alb, torch.ones_like(alb))
        m = torch.linalg.cross(e1, e2)
        n = m / torch.linalg.norm(m, dim=1, keepdim=True)
        facing = (n * d).sum(1) < 0
        nf = torch.where(facing[:, None], n, -n)
        s = torch.clamp((nf * self.light).sum(1), min=0.0)
        return alb * s[:, None]

    def bilinear(self, texels, uv):
        x = uv[:, 0] * self.W - 0.5
        y = uv[:, 1] * self.H - 0.5
        x0 = torch.floor(x.detach())
        y0 = torch.floor(y.detach())
        fx = (x - x0)[:, None]
        fy = (y - y0)[:, None]
        i0 = x0.long().clamp(0, self.W - 1)
        i1 = (x0.long() + 1).clamp(0, self.W - 1)
        j0 = y0.long().clamp(0, self.H - 1)
        j1 = (y0.long() + 1).clamp(0, self.H - 1)
        rgb = texels[..., :3]
        return ((1 - fx) * (1 - fy) * rgb[j0, i0] + fx * (1 - fy) * rgb[j0, i1]
                + (1 - fx) * fy * rgb[j1, i0] + fx * fy * rgb[j1, i1])

    def image(self, verts, texels):
        img = self.background.expand(self.n, 3).clone()
        img[self.hit] = self.colours(verts, texels)
        return img

    # -- reference gradient ---------------------------------------------

    def vjp(self, verts, texels, g):
        """Gradients of sum(image * g) with respect to vertices and texels."""
        v = _t(verts).requires_grad_(True)
        tx = _t(texels).requires_grad_(True)
        col = self.colours(v, tx)
        (col * _t(g)[self.hit]).sum().backward()
        gv = torch.zeros_like(v) if v.grad is None else v.grad
        return gv.numpy(), tx.grad.numpy()

    def loss_grad(self, verts, texels, target):
        """L = sum |image - target|^2 and its gradients (FP64)."""
        with torch.no_grad():
            img = self.image(_t(verts), _t(texels))
        g = 2.0 * (img - _t(target))
        gv, gt = self.vjp(verts, texels, g.numpy())
        return float(((img - _t(target)) ** 2).sum()), gv, gt, g.numpy()

    # -- finite differences ---------------------------------------------

    def pixels_of_vertex(self, k):
        return np.flatnonzero(np.any(self.idx == k, axis=1))

    def fd_vertex(self, verts, texels, target, k, axis, h=1e-3):
        """Central difference of the loss in vertex k's coordinate `axis`,
        evaluated on the pixels that vertex touches; also reports whether the
        stencil crosses a kink (bilinear cell, light cutoff or facing flip)."""
        sel = self.pixels_of_vertex(k)
        if len(sel) == 0:
            return 0.0, False
        tgt = _t(target)[self.hit][sel]
        tx = _t(texels)
        vals, keys = [], []
        for sgn in (1.0, -1.0, 0.0):
            v = _t(verts).clone()
            v[k, axis] += sgn * h
            with torch.no_grad():
                col = self.colours(v, tx, sel)
                vals.append(float(((col - tgt) ** 2).sum()))
                keys.append(self._kink_key(v, sel))
        kink = not (np.array_equal(keys[0], keys[2]) and np.array_equal(keys[1], keys[2]))
        return (vals[0] - vals[1]) / (2 * h), kink

    def _kink_key(self, verts, sel):
        idx, o, d, tc = self.idx[sel], self.o[sel], self.d[sel], self.tc[sel]
        a, b, c = verts[idx[:, 0]], verts[idx[:, 1]], verts[idx[:, 2]]
        e1, e2 = b - a, c - a
        M = torch.stack([-d, e1, e2], dim=2)
        tuv = torch.linalg.solve(M, (o - a).unsqueeze(-1)).squeeze(-1)
        u, v = tuv[:, 1], tuv[:, 2]
        uv = (1 - u - v)[:, None] * tc[:, 0] + u[:, None] * tc[:, 1] + v[:, None] * tc[:, 2]
        cx = torch.floor(uv[:, 0] * self.W - 0.5)
        cy = torch.floor(uv[:, 1] * self.H - 0.5)
        m = torch.linalg.cross(e1, e2)
        facing = (m * d).sum(1) < 0
        nf = torch.where(facing[:, None], m, -m)
        lit = (nf * self.light).sum(1) > 0
        return np.stack([cx.numpy(), cy.numpy(), facing.numpy(), lit.numpy()], 1)

    def fd_texel(self, verts, texels, target, j, i, ch, h=1e-3):
        """Central difference of the loss in texel (j, i) channel ch (exact up
        to rounding: the loss is quadratic in the texels at fixed visibility)."""
        sel = self.pixels_of_texel(verts, j, i)
        if len(sel) == 0:
            return 0.0
        tx = _t(texels)
        tgt = _t(target)[self.hit][sel]
        vals = []
        for sgn in (1.0, -1.0):
            t2 = tx.clone()
            t2[j, i, ch] += sgn * h
            with torch.no_grad():
                col = self.colours(_t(verts), t2, sel)
            vals.append(float(((col - tgt) ** 2).sum()))
        return (vals[0] - vals[1]) / (2 * h)

    def pixels_of_texel(self, verts, j, i):
        """Hit pixels whose bilinear footprint contains texel (j, i)."""
        if getattr(self, "_corners", None) is None:
            with torch.no_grad():
                idx, o, d, tc = self.idx, self.o, self.d, self.tc
                vt = _t(verts)
                a, b, c = vt[idx[:, 0]], vt[idx[:, 1]], vt[idx[:, 2]]
                M = torch.stack([-d, b - a, c - a], dim=2)
                tuv = torch.linalg.solve(M, (o - a).unsqueeze(-1)).squeeze(-1)
                u, v = tuv[:, 1], tuv[:, 2]
                uv = (1 - u - v)[:, None] * tc[:, 0] + u[:, None] * tc[:, 1] \
                    + v[:, None] * tc[:, 2]
                self._corners = self._footprint(uv)
        ii, jj, tex = self._corners
        return np.flatnonzero((ii == i).any(1) & (jj == j).any(1) & tex)

    def _footprint(self, uv):
        """Clamped column and row indices of the 2x2 texels each uv reads."""
        with torch.no_grad():
            x0 = torch.floor(uv[:, 0] * self.W - 0.5).long()
            y0 = torch.floor(uv[:, 1] * self.H - 0.5).long()
            ii = torch.stack([x0.clamp(0, self.W - 1), (x0 + 1).clamp(0, self.W - 1)], 1)
            jj = torch.stack([y0.clamp(0, self.H - 1), (y0 + 1).clamp(0, self.H - 1)], 1)
        return ii.numpy(), jj.numpy(), self.textured.numpy()


class FrozenAO(FrozenShading):
    """Ambient-occlusion shading at fixed visibility:
    c = albedo_rgb(uv) * visibility, visibility = 1 - occluded fraction of the
    pixel's occlusion rays (given, from the oracle's own traversal).

    bary  optional float32 [n, 2]: the (u, v) the closest-hit traversal
          returned for each pixel.  When given, uv is interpolated in FP64 at
          those barycentrics instead of at the FP64 ray-plane solution, so the
          image is the one defined by the traversal's own hit record (on small
          triangles with a texture stretched over each, the FP32 hit point
          moves uv by a sizable part of a texel).  uv is then constant in the
          vertices: only texel gradients are defined.
    """

    def __init__(self, scene, rays, prims, visibility, background=(0.0, 0.0, 0.0), tex=0,
                 bary=None):
        super().__init__(scene, rays, prims, light=(0.0, 0.0, 1.0), background=background,
                         tex=tex)
        self.vis = _t(np.asarray(visibility, np.float64)[self.hit])
        self.bary = None if bary is None else _t(np.asarray(bary, np.float32)[self.hit])

    def _uv_at_bary(self, sel):
        b = self.bary if sel is None else self.bary[sel]
        tc = self.tc if sel is None else self.tc[sel]
        u, v = b[:, 0], b[:, 1]
        return (1 - u - v)[:, None] * tc[:, 0] + u[:, None] * tc[:, 1] + v[:, None] * tc[:, 2]

    def colours(self, verts, texels, sel=None):
        if self.bary is None:
            uv, _, _, _, textured = self._surface(verts, sel)
        else:
            uv = self._uv_at_bary(sel)
            textured = self.textured if sel is None else self.textured[sel]
        alb = self.bilinear(texels, uv)
        alb = torch.where(textured[:, None], alb, torch.ones_like(alb))
        vis = self.vis if sel is None else self.vis[sel]
        return alb * vis[:, None]

    def pixels_of_texel(self, verts, j, i):
        if self.bary is not None and getattr(self, "_corners", None) is None:
            uv = self._uv_at_bary(None)
            self._corners = self._footprint(uv)
        return super().pixels_of_texel(verts, j, i)
