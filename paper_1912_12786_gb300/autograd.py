"""torch.autograd.Functions over the differentiable renders.

RenderFunction (vsr_render / vsr_render_backward_hits or vsr_trace_backward):
forward pushes the vertex and texel tensors into the scene (with a BVH refit
when the vertices change), renders the closest-hit image with the given
intersector and shading, keeps its hit records (16 bytes per ray) and returns
the image.  Backward returns gradients for the vertices and the texels at
fixed visibility from the kept hit records, or, with save_hits=False, by
tracing the same rays again.

AORenderFunction (vsr_render_ao / vsr_render_ao_backward): forward pushes the
texels and renders albedo * (1 - occluded fraction); backward returns the
texel gradient at fixed visibility from the saved hits and occlusion.

The scene must not be updated between a forward and its backward.
"""
from __future__ import annotations

import torch

from . import vsr as V


class RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, verts, texels, scene, rays, isect, shade, save_hits):
        verts = verts.detach().contiguous()
        texels = texels.detach().contiguous()
        V.vsr_scene_update(scene, verts, shade.grad_tex, texels)
        n = rays.shape[0]
        image = torch.empty((n, 3), dtype=torch.float32, device=rays.device)
        hits = (torch.empty((n, 4), dtype=torch.float32, device=rays.device) if save_hits
                else None)
        V.vsr_render(scene, rays, isect, shade, image, hits)
        ctx.scene, ctx.isect, ctx.shade = scene, isect, shade
        if save_hits:
            ctx.save_for_backward(rays, verts, texels, hits)
        else:
            ctx.save_for_backward(rays, verts, texels)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        rays, verts, texels, *hits = ctx.saved_tensors
        gv = torch.zeros_like(verts)
        gt = torch.zeros_like(texels)
        g = grad_image.contiguous().float()
        if hits:
            V.vsr_render_backward_hits(ctx.scene, rays, hits[0], ctx.shade, g, gv, gt)
        else:
            V.vsr_trace_backward(ctx.scene, rays, ctx.isect, ctx.shade, g, gv, gt)
        return gv, gt, None, None, None, None, None


def render(scene, rays, verts, texels, isect, shade, save_hits=True):
    """Differentiable closest-hit render; returns float32 [n, 3].  The
    backward uses the forward's hit records, or traces again when
    save_hits is False (no per-ray state kept)."""
    return RenderFunction.apply(verts, texels, scene, rays, isect, shade, save_hits)


class AORenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, texels, scene, rays, isect, spp, xi, ao_tmax, eps, shade):
        texels = texels.detach().contiguous()
        V.vsr_scene_update(scene, None, shade.grad_tex, texels)
        n = rays.shape[0]
        image = torch.empty((n, 3), dtype=torch.float32, device=rays.device)
        hits = torch.empty((n, 4), dtype=torch.float32, device=rays.device)
        occ = torch.empty(n, dtype=torch.float32, device=rays.device)
        V.vsr_render_ao(scene, rays, isect, spp, xi, ao_tmax, eps, shade, image, hits, occ)
        ctx.scene, ctx.shade = scene, shade
        ctx.save_for_backward(hits, occ, texels)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        hits, occ, texels = ctx.saved_tensors
        gt = torch.zeros_like(texels)
        V.vsr_render_ao_backward(ctx.scene, hits, occ, ctx.shade,
                                 grad_image.contiguous().float(), gt)
        return gt, None, None, None, None, None, None, None, None


def render_ao(scene, rays, texels, isect, spp, xi, ao_tmax, eps, shade):
    """Differentiable ambient-occlusion render (texels only); float32 [n, 3]."""
    return AORenderFunction.apply(texels, scene, rays, isect, spp, xi, ao_tmax, eps, shade)
