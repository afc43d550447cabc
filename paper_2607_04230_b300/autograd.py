"""torch.autograd.Function over the deferred resolve (argument marshalling
only; forward and backward run in libhm's kernels).

forward(layer_verts, albedo) renders one groom (visibility + resolve) and
returns straight-alpha RGBA [H][W][4].  backward calls hm_shade_backward with
the forward's visibility buffers held fixed: gradients reach the hair-mesh
layer vertices [L][V][3] and the per-strand albedo [S][3]; the alpha channel is
constant (its strip counts are discrete) and gets no gradient.

The groom keeps the state of its last render (layer vertices, LOD result,
segment records).  When another forward on the same groom ran in between,
backward first restores this forward's inputs and re-renders its visibility
(deterministic: the same keys) so the adjoint sees the state it
differentiates.
"""
from __future__ import annotations

import itertools

import torch

from . import hm

_forward_ids = itertools.count(1)


class HairRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, layer_verts, albedo, groom, scene, frame, shadows=None):
        lv = layer_verts.detach().float().contiguous()
        alb = albedo.detach().float().contiguous()
        groom.update_layer_verts(lv)
        groom.update_albedo(alb)
        hm.render([groom], scene, frame, shadows=shadows)
        ctx.groom, ctx.scene, ctx.shadows = groom, scene, shadows
        ctx.cam = frame.camera(scene.camera)      # with the frame's key layout
        ctx.vis = (frame.vis_center.clone(), frame.vis_cons.clone())
        ctx.inputs = (lv.clone(), alb.clone())
        ctx.lv_shape, ctx.alb_shape = layer_verts.shape, albedo.shape
        ctx.fid = next(_forward_ids)
        groom.last_forward = ctx.fid
        return frame.rgba.clone()

    @staticmethod
    def backward(ctx, grad_rgba):
        sc = ctx.scene
        dev = grad_rgba.device
        if getattr(ctx.groom, "last_forward", None) != ctx.fid:
            # another forward rendered this groom since: restore this one's state
            ctx.groom.update_layer_verts(ctx.inputs[0])
            ctx.groom.update_albedo(ctx.inputs[1])
            vc, va = torch.empty_like(ctx.vis[0]), torch.empty_like(ctx.vis[1])
            hm.render_visibility([ctx.groom], ctx.cam, vc, va)
            ctx.groom.last_forward = ctx.fid
        glv = torch.zeros(ctx.lv_shape, dtype=torch.float32, device=dev)
        galb = torch.zeros(ctx.alb_shape, dtype=torch.float32, device=dev)
        nbytes = hm.backward_scratch_bytes(sc.camera.width, sc.camera.height)
        scratch = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
        g = grad_rgba.float().contiguous()
        if g.data_ptr() % 16:
            # the adjoint reads float4 rows: a view at an unaligned offset is copied
            g = g.clone(memory_format=torch.contiguous_format)
        hm.shade_backward([ctx.groom], ctx.cam, sc.lights, sc.filt, ctx.vis[0], ctx.vis[1],
                          g, [glv], [galb], scratch, shadows=ctx.shadows)
        return glv, galb, None, None, None, None


def render(groom, scene, frame, layer_verts, albedo, shadows=None):
    """Differentiable RGBA of one groom w.r.t. its layer vertices and albedo
    (shadow maps, when given, are held fixed: gradients flow through the
    receiver's depth, not through the map)."""
    return HairRender.apply(layer_verts, albedo, groom, scene, frame, shadows)
