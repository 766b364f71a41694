"""Differentiable persistence diagrams (torch.autograd.Function).

Forward: the CUDA library computes the pairs and, for each finite birth and
death, the critical edge (u, v) whose length it is, and leaves both on the
GPU (the device-resident entry points).  Backward: the library's
backward kernel scatters dL/d(birth, death) through those edges onto the
point coordinates (d|x_u - x_v| / dx_u = (x_u - x_v) / |x_u - x_v|).  The
pairing is piecewise constant in the coordinates, so this is the gradient
wherever the pairing does not change.  torch only holds the tensors.

recompute=True keeps no critical edges between forward and backward (the
pairs are recomputed in backward), for when memory matters more than time.
"""
from __future__ import annotations

import numpy as np
import torch

from . import vr


def _edges_of(bc, p, device):
    """Critical edges of dimension p (a device tensor of the device-resident
    result: no host round trip)."""
    e = bc.edges[p]
    return e.to(device) if e is not None else torch.zeros((0, 4), dtype=torch.int32, device=device)


class VRDiagram(torch.autograd.Function):
    """VRDiagram.apply(points (n, D) float32 CUDA, dmax, threshold=inf, recompute=False)
    -> tuple of (k_p, 2) tensors of (birth, death), p = 0..dmax; death = inf for
    essential classes.  Backward launches the library's kernel once per dimension
    whose values received a gradient."""

    @staticmethod
    def forward(ctx, points, dmax, threshold=float("inf"), recompute=False):
        ctx.set_materialize_grads(False)
        x = points.detach().contiguous()
        stream = torch.cuda.current_stream(x.device)
        bc = vr.barcodes_device(points=x, dmax=dmax, threshold=threshold, flags=vr.VR_CRITICAL_EDGES, stream=stream)
        outs = [bc.values[p] for p in range(dmax + 1)]
        ctx.dmax, ctx.threshold, ctx.recompute = dmax, threshold, recompute
        if recompute:
            ctx.save_for_backward(points)
        else:
            ctx.save_for_backward(points, *[_edges_of(bc, p, x.device) for p in range(dmax + 1)])
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grads):
        if ctx.recompute:
            (points,) = ctx.saved_tensors
            x = points.detach().contiguous()
            bc = vr.barcodes_device(points=x, dmax=ctx.dmax, threshold=ctx.threshold, flags=vr.VR_CRITICAL_EDGES,
                                    stream=torch.cuda.current_stream(x.device))
            edges = [_edges_of(bc, p, x.device) for p in range(ctx.dmax + 1)]
        else:
            points, *edges = ctx.saved_tensors
            x = points.detach().contiguous()
        grad = torch.zeros_like(x)
        stream = torch.cuda.current_stream(x.device)
        for p in range(ctx.dmax + 1):
            g = grads[p]
            if g is None or edges[p].shape[0] == 0:
                continue
            g = g.float()
            vr.backward(x, edges[p].contiguous(), g[:, 0].contiguous(), g[:, 1].contiguous(), grad, stream=stream)
        return grad, None, None, None


class VRDiagramBatched(torch.autograd.Function):
    """VRDiagramBatched.apply(points (sum n, D) float32 CUDA, offsets int64 host array,
    dmax, threshold=inf) -> for p = 0..dmax a (K_p, 2) tensor of all clouds' pairs,
    then for p = 0..dmax the int64 (num+1,) offsets of each cloud's pairs (no gradient).
    One persistent launch forward; backward, one launch per dimension whose values
    received a gradient (dimensions without one cost nothing)."""

    @staticmethod
    def forward(ctx, points, offsets, dmax, threshold=float("inf")):
        ctx.set_materialize_grads(False)
        x = points.detach().contiguous()
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        stream = torch.cuda.current_stream(x.device)
        bb = vr.barcodes_batched_device(x, offs, dmax=dmax, threshold=threshold, flags=vr.VR_CRITICAL_EDGES,
                                        stream=stream)
        outs = [bb.values[p] for p in range(dmax + 1)]
        offs_out = [torch.from_numpy(bb.offsets[p].astype(np.int64)) for p in range(dmax + 1)]
        ctx.dmax = dmax
        ctx.save_for_backward(points, *[bb.edges[p] for p in range(dmax + 1)])
        for o in offs_out:
            ctx.mark_non_differentiable(o)
        return tuple(outs) + tuple(offs_out)

    @staticmethod
    def backward(ctx, *grads):
        points, *edges = ctx.saved_tensors
        x = points.detach().contiguous()
        grad = torch.zeros_like(x)
        stream = torch.cuda.current_stream(x.device)
        for p in range(ctx.dmax + 1):
            g = grads[p]
            if g is None or edges[p].shape[0] == 0:
                continue
            g = g.float()
            vr.backward(x, edges[p].contiguous(), g[:, 0].contiguous(), g[:, 1].contiguous(), grad, stream=stream)
        return grad, None, None, None
