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


def _edges_tensor(bc, dmax, device):
    """Critical edges of every dimension, concatenated (device tensors from the
    device-resident result: no host round trip)."""
    parts = [bc.edges[p] for p in range(dmax + 1)]
    return torch.cat(parts).to(device) if parts else torch.zeros((0, 4), dtype=torch.int32, device=device)


class VRDiagram(torch.autograd.Function):
    """VRDiagram.apply(points (n, D) float32 CUDA, dmax, threshold=inf, recompute=False)
    -> tuple of (k_p, 2) tensors of (birth, death), p = 0..dmax; death = inf for
    essential classes."""

    @staticmethod
    def forward(ctx, points, dmax, threshold=float("inf"), recompute=False):
        x = points.detach().contiguous()
        stream = torch.cuda.current_stream(x.device)
        bc = vr.barcodes_device(points=x, dmax=dmax, threshold=threshold, flags=vr.VR_CRITICAL_EDGES, stream=stream)
        outs = [bc.values[p] for p in range(dmax + 1)]
        ctx.dmax, ctx.threshold, ctx.recompute = dmax, threshold, recompute
        ctx.counts = list(bc.counts)
        if recompute:
            ctx.save_for_backward(points)
        else:
            ctx.save_for_backward(points, _edges_tensor(bc, dmax, x.device))
        return tuple(outs)

    @staticmethod
    def backward(ctx, *grads):
        if ctx.recompute:
            (points,) = ctx.saved_tensors
            x = points.detach().contiguous()
            bc = vr.barcodes_device(points=x, dmax=ctx.dmax, threshold=ctx.threshold, flags=vr.VR_CRITICAL_EDGES,
                                    stream=torch.cuda.current_stream(x.device))
            edges = _edges_tensor(bc, ctx.dmax, x.device)
        else:
            points, edges = ctx.saved_tensors
            x = points.detach().contiguous()
        gb, gd = [], []
        for p, k in enumerate(ctx.counts):
            g = grads[p]
            if g is None:
                g = torch.zeros((k, 2), dtype=torch.float32, device=x.device)
            g = g.contiguous().float()
            gb.append(g[:, 0])
            gd.append(g[:, 1])
        gb = torch.cat(gb).contiguous()
        gd = torch.cat(gd).contiguous()
        grad = torch.zeros_like(x)
        if edges.shape[0]:
            vr.backward(x, edges.contiguous(), gb, gd, grad, stream=torch.cuda.current_stream(x.device))
        return grad, None, None, None


class VRDiagramBatched(torch.autograd.Function):
    """VRDiagramBatched.apply(points (sum n, D) float32 CUDA, offsets int64 host array,
    dmax, threshold=inf) -> for p = 0..dmax a (K_p, 2) tensor of all clouds' pairs,
    then for p = 0..dmax the int64 (num+1,) offsets of each cloud's pairs (no gradient).
    One persistent launch forward, one backward launch for the whole batch."""

    @staticmethod
    def forward(ctx, points, offsets, dmax, threshold=float("inf")):
        x = points.detach().contiguous()
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        stream = torch.cuda.current_stream(x.device)
        bb = vr.barcodes_batched_device(x, offs, dmax=dmax, threshold=threshold, flags=vr.VR_CRITICAL_EDGES,
                                        stream=stream)
        outs = [bb.values[p] for p in range(dmax + 1)]
        offs_out = [torch.from_numpy(bb.offsets[p].astype(np.int64)) for p in range(dmax + 1)]
        ctx.counts = [int(bb.offsets[p][-1]) for p in range(dmax + 1)]
        ctx.save_for_backward(points, torch.cat([bb.edges[p] for p in range(dmax + 1)]))
        for o in offs_out:
            ctx.mark_non_differentiable(o)
        return tuple(outs) + tuple(offs_out)

    @staticmethod
    def backward(ctx, *grads):
        points, edges = ctx.saved_tensors
        x = points.detach().contiguous()
        gb, gd = [], []
        for p, k in enumerate(ctx.counts):
            g = grads[p]
            if g is None:
                g = torch.zeros((k, 2), dtype=torch.float32, device=x.device)
            g = g.contiguous().float()
            gb.append(g[:, 0])
            gd.append(g[:, 1])
        grad = torch.zeros_like(x)
        if edges.shape[0]:
            vr.backward(x, edges.contiguous(), torch.cat(gb).contiguous(), torch.cat(gd).contiguous(), grad,
                        stream=torch.cuda.current_stream(x.device))
        return grad, None, None, None
