"""torch.autograd binding of the sphere-splat renderer (forward: wrs_build_lbvh + wrs_trace,
backward: wrs_trace_backward).

The differentiable quantities are the per-splat colour (premultiplied RGBA), opacity and radius
scale, all in compacted splat order.  The single-view Function stores no hit lists: its backward
kernel re-traverses every ray (spec S7).  The radius scale changes the spheres, so every forward call
rebuilds the LBVH with the current scales; :func:`render_views` renders several views from one
build, all views in one launch (wrs_trace_views), and their gradients in one launch into one
set of buffers (wrs_trace_backward_views).  When the per-ray hit lists fit in memory the forward
pass records them (wrs_trace_views_record) and the adjoint runs from them without traversal
(wrs_trace_backward_views_recorded); otherwise the adjoint re-traverses.  Given a RefitTree (splat
centres fixed, only the radius scales change, as in a radius fit) the forward refits that tree
(wrs_refit_lbvh) instead of building a new one.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import (HitLists, RefitTree, SplatBuffers, TraceParams, build_lbvh, trace, trace_backward,
               trace_backward_views, trace_backward_views_recorded, trace_views,
               trace_views_record, tree_layout)

# Hit lists are recorded by the multi-view forward pass (and the adjoint then needs no traversal)
# when they fit in this many bytes; beyond it the adjoint re-traverses every ray.
RECORD_BUDGET_BYTES = 1 << 30
RECORD_CAPACITY = 16


class TraceFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rgba: torch.Tensor, opacity: Optional[torch.Tensor],
                radius_scale: Optional[torch.Tensor], splats: SplatBuffers, cam,
                params: TraceParams, leaf_size: int):
        n = rgba.shape[0]
        if n > splats.capacity:
            raise ValueError("more colours than splats")
        splats.rgba[:n].copy_(rgba.detach())
        op = None if opacity is None else opacity.detach().contiguous()
        sc = None if radius_scale is None else radius_scale.detach().contiguous()
        bvh, sorted_ = build_lbvh(splats, leaf_size, radius_scale=sc, layout=tree_layout(params))
        img = trace(bvh, sorted_, cam, params, opacity=op)
        ctx.state = (bvh, sorted_, cam, params, op, sc, n)
        return img

    @staticmethod
    def backward(ctx, g_img: torch.Tensor):
        bvh, sorted_, cam, params, op, sc, n = ctx.state
        need_rgba, need_op, need_sc = ctx.needs_input_grad[:3]
        g_rgba, g_op, g_sc = trace_backward(bvh, sorted_, cam, g_img.contiguous(), params,
                                            opacity=op, radius_scale=sc,
                                            want_opacity=need_op, want_scale=need_sc)
        return (g_rgba[:n] if need_rgba else None,
                g_op[:n] if need_op else None,
                g_sc[:n] if need_sc else None,
                None, None, None, None)


def render(splats: SplatBuffers, cam, rgba: torch.Tensor, opacity: Optional[torch.Tensor] = None,
           radius_scale: Optional[torch.Tensor] = None, params: TraceParams = TraceParams(),
           leaf_size: int = 1) -> torch.Tensor:
    """Differentiable client image [H,W,4] of the splats (geometry from ``splats``; colour,
    opacity and radius scale from the given per-splat tensors, compacted order)."""
    return TraceFunction.apply(rgba, opacity, radius_scale, splats, cam, params, leaf_size)


class MultiViewTraceFunction(torch.autograd.Function):
    """Several client views of one splat set: one LBVH build and one launch for all views; the
    backward pass, also one launch, accumulates every view's gradient into one buffer (no
    per-view buffers, no sums)."""

    @staticmethod
    def forward(ctx, rgba: torch.Tensor, opacity: Optional[torch.Tensor],
                radius_scale: Optional[torch.Tensor], splats: SplatBuffers, cams,
                params: TraceParams, leaf_size: int, record_hits: int,
                tree: Optional[RefitTree]):
        n = rgba.shape[0]
        if n > splats.capacity:
            raise ValueError("more colours than splats")
        splats.rgba[:n].copy_(rgba.detach())
        op = None if opacity is None else opacity.detach().contiguous()
        sc = None if radius_scale is None else radius_scale.detach().contiguous()
        if tree is not None:
            if tree.splats is not splats or tree.leaf_size != leaf_size:
                raise ValueError("the tree belongs to other splats or another leaf size")
            bvh, sorted_ = tree.update(sc)
        else:
            bvh, sorted_ = build_lbvh(splats, leaf_size, radius_scale=sc,
                                      layout=tree_layout(params))
        c0 = cams[0]
        if any((c.width, c.height) != (c0.width, c0.height) for c in cams):
            raise ValueError("all views must have the same size")
        lists = None
        if record_hits:
            out, lists = trace_views_record(bvh, sorted_, cams, params, record_hits, opacity=op)
        else:
            out = trace_views(bvh, sorted_, cams, params, opacity=op)
        ctx.state = (bvh, sorted_, list(cams), params, op, sc, n, lists)
        return out

    @staticmethod
    def backward(ctx, g_img: torch.Tensor):
        bvh, sorted_, cams, params, op, sc, n, lists = ctx.state
        need_rgba, need_op, need_sc = ctx.needs_input_grad[:3]
        if lists is not None:
            g_rgba, g_op, g_sc = trace_backward_views_recorded(
                bvh, sorted_, cams, lists, g_img.contiguous(), params, opacity=op,
                radius_scale=sc, want_opacity=need_op, want_scale=need_sc)
        else:
            g_rgba, g_op, g_sc = trace_backward_views(bvh, sorted_, cams, g_img.contiguous(),
                                                      params, opacity=op, radius_scale=sc,
                                                      want_opacity=need_op, want_scale=need_sc)
        return (g_rgba[:n] if need_rgba else None,
                g_op[:n] if need_op else None,
                g_sc[:n] if need_sc else None,
                None, None, None, None, None, None)


def render_views(splats: SplatBuffers, cams: Sequence, rgba: torch.Tensor,
                 opacity: Optional[torch.Tensor] = None,
                 radius_scale: Optional[torch.Tensor] = None, params: TraceParams = TraceParams(),
                 leaf_size: int = 1, record_hits: Optional[int] = None,
                 tree: Optional[RefitTree] = None) -> torch.Tensor:
    """Differentiable images [V,H,W,4] of several same-size client views of the splats.

    ``record_hits``: capacity of the per-ray hit lists the forward pass records so that the
    adjoint needs no traversal (rays with more hits are traced again); 0 = always re-traverse;
    None = RECORD_CAPACITY when the lists fit in RECORD_BUDGET_BYTES, else 0.
    ``tree``: a RefitTree over ``splats`` (same leaf size) to refit with the radius scales instead
    of building a new LBVH; the splat centres must not change while it is used."""
    cams = list(cams)
    if record_hits is None:
        rays = len(cams) * cams[0].width * cams[0].height
        record_hits = (RECORD_CAPACITY if HitLists.nbytes(rays, RECORD_CAPACITY)
                       <= RECORD_BUDGET_BYTES else 0)
    return MultiViewTraceFunction.apply(rgba, opacity, radius_scale, splats, cams, params,
                                        leaf_size, int(record_hits), tree)
