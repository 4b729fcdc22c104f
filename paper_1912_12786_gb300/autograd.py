"""torch.autograd.Functions over the differentiable renders.

RenderFunction (vsr_render / vsr_trace_backward): forward pushes the vertex
and texel tensors into the scene (with a BVH refit when the vertices change),
renders the closest-hit image with the given intersector and shading, and
returns it.  Backward traces the same rays again and returns gradients for
the vertices and the texels at fixed visibility.

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
    def forward(ctx, verts, texels, scene, rays, isect, shade):
        verts = verts.detach().contiguous()
        texels = texels.detach().contiguous()
        V.vsr_scene_update(scene, verts, shade.grad_tex, texels)
        image = torch.empty((rays.shape[0], 3), dtype=torch.float32, device=rays.device)
        V.vsr_render(scene, rays, isect, shade, image)
        ctx.scene, ctx.isect, ctx.shade = scene, isect, shade
        ctx.save_for_backward(rays, verts, texels)
        return image

    @staticmethod
    def backward(ctx, grad_image):
        rays, verts, texels = ctx.saved_tensors
        gv = torch.zeros_like(verts)
        gt = torch.zeros_like(texels)
        V.vsr_trace_backward(ctx.scene, rays, ctx.isect, ctx.shade,
                             grad_image.contiguous().float(), gv, gt)
        return gv, gt, None, None, None, None


def render(scene, rays, verts, texels, isect, shade):
    """Differentiable closest-hit render; returns float32 [n, 3]."""
    return RenderFunction.apply(verts, texels, scene, rays, isect, shade)


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
