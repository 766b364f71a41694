"""The oracle over many independent clouds, one cloud per process.

TEST INFRASTRUCTURE ONLY (see the package docstring): used by the tests and
by the CPU-baseline leg of the benchmark.  Each worker runs the plain C
oracle (``cohom`` with clearing, Algorithm 12) on whole clouds; nothing is
shared between clouds, so the work splits across host cores with no change to
what each cloud computes.  Workers are started with ``spawn``, so the pool is
safe to open after CUDA has been initialised in the parent.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _one(args):
    import oracle
    pts, dmax, threshold = args
    n = pts.shape[0]
    D = oracle.distances_f32(pts).astype(np.float64)
    t = oracle.enclosing_radius(D, n) if not np.isfinite(threshold) else float(np.float32(threshold))
    pairs, _ = oracle.cohom(D, n, dmax, t, clearing=True)
    return oracle.diagram(pairs, dmax)


def _one_grad(args):
    """Forward pairing plus the FP64 gradient of sum over H1 of (death - birth)^2."""
    from oracle import grad
    pts, dmax = args
    pairs, edges = grad.fp32_pairing(pts, dmax)
    return grad.loss_grad_h1(pts.astype(np.float64), pairs, edges)


def open_pool(processes: int | None = None):
    """A spawn-started pool of `processes` workers (all host cores by default)."""
    import oracle
    oracle.build()  # compile once in the parent, not racing in the workers
    return mp.get_context("spawn").Pool(processes or os.cpu_count() or 1)


def diagrams(clouds, dmax: int, threshold: float = np.inf, processes: int | None = None, pool=None):
    """oracle.diagram(...) of every cloud (float32 (n_i, D) arrays), in order."""
    if not clouds:
        return []
    work = [(np.ascontiguousarray(c, dtype=np.float32), dmax, threshold) for c in clouds]
    if pool is not None:
        return pool.map(_one, work, chunksize=1)
    procs = max(1, min(processes or os.cpu_count() or 1, len(clouds)))
    if procs == 1:
        return [_one(w) for w in work]
    with open_pool(procs) as pl:
        return pl.map(_one, work, chunksize=max(1, len(work) // (4 * procs)))


def loss_grads(clouds, dmax: int, pool):
    """(loss, FP64 gradient) of every cloud, in order, on an open pool."""
    work = [(np.ascontiguousarray(c, dtype=np.float32), dmax) for c in clouds]
    return pool.map(_one_grad, work, chunksize=1)
