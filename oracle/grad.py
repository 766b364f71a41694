"""FP64 reference gradients of diagram losses (TEST INFRASTRUCTURE ONLY).

Every finite birth or death of a Vietoris-Rips pair is the length of one
edge of its simplex (diam = max pairwise distance, eq. 5.3): the critical
edge (u, v), ties broken by the largest edge index (the reading used
throughout).  For a fixed pairing the loss is a function of those lengths, so
  d loss / d x_u = sum over uses of  dL/dlength * (x_u - x_v) / |x_u - x_v|.
`pairs_with_edges` takes the pairing from the oracle (cohomology, Algorithm
12) and the critical edges from the oracle's own routine; `loss_grad_h1`
evaluates the loss sum over H1 pairs of (death - birth)^2 and its gradient in
float64; `central_differences` checks it numerically, skipping coordinates
whose perturbation changes the pairing.
"""
from __future__ import annotations

import numpy as np

from . import cohom, critical_edge, distances_f32, distances_f64, enclosing_radius


def pairs_with_edges(D, n, dmax, threshold=None):
    """Oracle pairs of every length with (u_b, v_b, u_d, v_d) critical edges."""
    D = np.asarray(D, dtype=np.float64)
    t = enclosing_radius(D, n) if threshold is None else threshold
    pairs, _ = cohom(D, n, dmax, t, clearing=True)
    edges = []
    for r in pairs:
        p = int(r["dim"])
        eb = critical_edge(D, n, int(r["birth_cidx"]), p) if p > 0 else (-1, -1)
        ed = critical_edge(D, n, int(r["death_cidx"]), p + 1) if r["death_cidx"] >= 0 else (-1, -1)
        edges.append(eb + ed)
    return pairs, np.asarray(edges, dtype=np.int64).reshape(-1, 4)


def loss_grad_h1(pts64, pairs, edges):
    """loss = sum over finite H1 pairs of (death - birth)^2, in float64, and its gradient."""
    x = np.asarray(pts64, dtype=np.float64)
    grad = np.zeros_like(x)
    loss = 0.0
    for r, e in zip(pairs, edges):
        if int(r["dim"]) != 1 or r["death_cidx"] < 0:
            continue
        ub, vb, ud, vd = (int(q) for q in e)
        b = np.linalg.norm(x[ub] - x[vb])
        d = np.linalg.norm(x[ud] - x[vd])
        loss += (d - b) ** 2
        gd, gb = 2 * (d - b), -2 * (d - b)
        grad[ud] += gd * (x[ud] - x[vd]) / d
        grad[vd] -= gd * (x[ud] - x[vd]) / d
        grad[ub] += gb * (x[ub] - x[vb]) / b
        grad[vb] -= gb * (x[ub] - x[vb]) / b
    return loss, grad


def _loss64(x, n, dmax):
    D = distances_f64(x)
    pairs, edges = pairs_with_edges(D, n, dmax)
    loss, _ = loss_grad_h1(x, pairs, edges)
    key = sorted((int(r["dim"]), int(r["birth_cidx"]), int(r["death_cidx"])) for r in pairs
                 if r["death"] > r["birth"])
    return loss, key


def central_differences(pts64, coords, h):
    """{(i, k): (L(x + h e) - L(x - h e)) / 2h} for the coordinates whose pairing
    (of nonzero persistence) is the same at x - h, x and x + h; and the count skipped."""
    x = np.array(pts64, dtype=np.float64)
    n = x.shape[0]
    _, base = _loss64(x, n, 1)
    out, skipped = {}, 0
    for (i, k) in coords:
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        lp, kp = _loss64(xp, n, 1)
        lm, km = _loss64(xm, n, 1)
        if kp != base or km != base:
            skipped += 1
            continue
        out[(i, k)] = (lp - lm) / (2 * h)
    return out, skipped


def fp32_pairing(pts32, dmax):
    """Pairs and critical edges of the single-precision distance matrix (the
    pairing the CUDA path computes, bit for bit)."""
    pts32 = np.ascontiguousarray(pts32, dtype=np.float32)
    n = pts32.shape[0]
    return pairs_with_edges(distances_f32(pts32).astype(np.float64), n, dmax)
