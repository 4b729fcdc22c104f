"""torch.autograd.Function over vsr_render / vsr_trace_backward.

Forward pushes the vertex and texel tensors into the scene (with a BVH refit
when the vertices change), renders the closest-hit image with the given
intersector and shading, and returns it.  Backward traces the same rays
again and returns gradients for the vertices and the texels at fixed
visibility.  The scene must not be updated between the two.
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
