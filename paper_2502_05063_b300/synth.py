"""Seeded synthetic point clouds for the Vietoris-Rips workloads.

This module holds no persistence arithmetic: it only draws inputs, so both
the CUDA path and the CPU oracle can be fed byte-identical clouds.  All draws
use numpy's PCG64 generator seeded explicitly; every cloud is rounded to
float32 once, at the end.

The dissertation measures on point-cloud datasets (celegans, dragon, HIV,
o3, sphere_3_192, Vicsek; Sec. 5.6) that are not available here; these
generators stand in for them with the same kind of structure (manifold
samples plus noise, uniform clouds) at the sizes of the workloads below.

Workloads (name -> generator, homology dims, threshold):
  uniform64    n=64 uniform in [0,1]^3, seed 0, H0-H1, no threshold
  torus500     n=500 on the torus R=2, r=1 in R^3 (uniform angles) + N(0, 0.05^2), seed 1, H0-H2
  sphere200    n=200 uniform on S^3 in R^4 + N(0, 0.02^2), seed 2, H0-H3, threshold 1.2
  batch4096    4096 clouds, n ~ U{32..256}, each a noisy circle (radius ~U[0.5,2], sigma 0.05,
               z=0 plane, 3-D noise), noisy sphere S^2 (same radius law and noise) or uniform
               in [0,1]^3 with probability 1/3 each, seed 3, cloud i from stream (3, i), H0-H1
  circles256   256 clouds of n=128 on the unit circle in R^2 + N(0, 0.1^2), seed 4, H0-H1
  o3like4096   n=4096 Haar-random O(3) matrices in R^9, seed 6, H0-H2, threshold 1.4 (sparse mode)
  randperm     distance matrices whose lower triangle is a random permutation of
               1 .. n(n-1)/2 (stored as ordered distinct floats), n = 50 .. 9000,
               seed 5, sample s from stream (5, n, s), H0-H1 of the full 2-skeleton
"""
from __future__ import annotations

import numpy as np


def _rng(*key) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def uniform_cube(n: int, dim: int = 3, seed: int = 0) -> np.ndarray:
    return _rng(seed).random((n, dim)).astype(np.float32)


def torus(n: int = 500, R: float = 2.0, r: float = 1.0, sigma: float = 0.05, seed: int = 1) -> np.ndarray:
    g = _rng(seed)
    th = g.random(n) * (2 * np.pi)
    ph = g.random(n) * (2 * np.pi)
    x = np.stack([(R + r * np.cos(ph)) * np.cos(th), (R + r * np.cos(ph)) * np.sin(th), r * np.sin(ph)], 1)
    x = x + sigma * g.standard_normal((n, 3))
    return x.astype(np.float32)


def sphere(n: int, ambient: int, radius: float = 1.0, sigma: float = 0.0, seed: int = 2,
           g: np.random.Generator | None = None) -> np.ndarray:
    """Uniform on the (ambient-1)-sphere of the given radius, plus isotropic noise."""
    g = g if g is not None else _rng(seed)
    v = g.standard_normal((n, ambient))
    v = v / np.linalg.norm(v, axis=1, keepdims=True) * radius
    if sigma:
        v = v + sigma * g.standard_normal((n, ambient))
    return v.astype(np.float32)


def circle(n: int, radius: float = 1.0, sigma: float = 0.1, ambient: int = 2,
           seed: int = 4, g: np.random.Generator | None = None) -> np.ndarray:
    """Uniform angle on a circle in the first two coordinates, noise in all."""
    g = g if g is not None else _rng(seed)
    th = g.random(n) * (2 * np.pi)
    x = np.zeros((n, ambient))
    x[:, 0] = radius * np.cos(th)
    x[:, 1] = radius * np.sin(th)
    x = x + sigma * g.standard_normal((n, ambient))
    return x.astype(np.float32)


def evenly_spaced_circle(n: int, radius: float = 1.0) -> np.ndarray:
    th = np.arange(n) * (2 * np.pi / n)
    return np.stack([radius * np.cos(th), radius * np.sin(th)], 1).astype(np.float32)


def batch_clouds(num: int = 4096, nmin: int = 32, nmax: int = 256, seed: int = 3):
    """List of float32 (n_i, 3) clouds and their kinds ('circle'|'sphere'|'cube')."""
    clouds, kinds = [], []
    for i in range(num):
        g = _rng(seed, i)
        n = int(g.integers(nmin, nmax + 1))
        kind = int(g.integers(0, 3))
        if kind == 0:
            x = circle(n, radius=float(g.uniform(0.5, 2.0)), sigma=0.05, ambient=3, g=g)
            kinds.append("circle")
        elif kind == 1:
            x = sphere(n, 3, radius=float(g.uniform(0.5, 2.0)), sigma=0.05, g=g)
            kinds.append("sphere")
        else:
            x = g.random((n, 3)).astype(np.float32)
            kinds.append("cube")
        clouds.append(x)
    return clouds, kinds


def circles(num: int = 256, n: int = 128, sigma: float = 0.1, seed: int = 4):
    return [circle(n, 1.0, sigma, 2, g=_rng(seed, i)) for i in range(num)]


def orthogonal_group(n: int, seed: int = 6) -> np.ndarray:
    """n Haar-random 3x3 orthogonal matrices (QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q), flattened to points of R^9: a
    synthetic stand-in for a sample of O(3) (the paper's o3 workload)."""
    g = _rng(seed)
    A = g.standard_normal((n, 3, 3))
    Q, Rr = np.linalg.qr(A)
    d = np.sign(np.diagonal(Rr, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return (Q * d[:, None, :]).reshape(n, 9).astype(np.float32)


def lower_star_grid(m: int, seed: int = 7):
    """Boundary matrix of the lower-star filtration of an m x m grid with
    random vertex values (a workload for the explicit-matrix path): the
    Freudenthal triangulation (edges right, down and down-right; two triangles
    per square), each simplex valued by its largest vertex value, ordered by
    (value, dimension, position in the listing), faces always before cofaces.
    Returns (colptr int64[N+1], rows int32[nnz], dims int8[N]), rows ascending."""
    g = _rng(seed)
    val = g.random(m * m)
    vid = np.arange(m * m).reshape(m, m)
    e_r = np.stack([vid[:, :-1].ravel(), vid[:, 1:].ravel()], 1)
    e_d = np.stack([vid[:-1, :].ravel(), vid[1:, :].ravel()], 1)
    e_x = np.stack([vid[:-1, :-1].ravel(), vid[1:, 1:].ravel()], 1)
    edges = np.concatenate([e_r, e_d, e_x])
    a, b, c, d = vid[:-1, :-1].ravel(), vid[:-1, 1:].ravel(), vid[1:, :-1].ravel(), vid[1:, 1:].ravel()
    tris = np.concatenate([np.stack([a, b, d], 1), np.stack([a, c, d], 1)])
    nv, ne, nt = m * m, len(edges), len(tris)
    # edge numbers: right edges (i, j) at i(m-1)+j, down edges (i, j) after them at
    # i*m+j, diagonals (i, j) last at i(m-1)+j
    nr, nd = m * (m - 1), (m - 1) * m
    ii, jj = np.meshgrid(np.arange(m - 1), np.arange(m - 1), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    right = lambda i, j: i * (m - 1) + j
    down = lambda i, j: nr + i * m + j
    diag = lambda i, j: nr + nd + i * (m - 1) + j
    t_up = np.stack([right(ii, jj), diag(ii, jj), down(ii, jj + 1)], 1)      # (i,j),(i,j+1),(i+1,j+1)
    t_lo = np.stack([down(ii, jj), diag(ii, jj), right(ii + 1, jj)], 1)      # (i,j),(i+1,j),(i+1,j+1)
    tri_edges = np.concatenate([t_up, t_lo]).astype(np.int64)
    value = np.concatenate([val, val[edges].max(1), val[tris].max(1)])
    dims = np.concatenate([np.zeros(nv, np.int8), np.ones(ne, np.int8), np.full(nt, 2, np.int8)])
    order = np.lexsort((np.arange(nv + ne + nt), dims, value))
    pos = np.empty_like(order)
    pos[order] = np.arange(len(order))
    cols = []
    for s_ in order:
        if s_ < nv:
            cols.append(np.zeros(0, np.int64))
        elif s_ < nv + ne:
            cols.append(np.sort(pos[edges[s_ - nv]]))
        else:
            cols.append(np.sort(pos[nv + tri_edges[s_ - nv - ne]]))
    colptr = np.zeros(len(cols) + 1, np.int64)
    colptr[1:] = np.cumsum([len(c_) for c_ in cols])
    rows = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return colptr, rows, dims[order]


def random_permutation_dists(n: int, seed: int = 5, sample: int = 0) -> np.ndarray:
    """Condensed lower triangle whose entries are a uniformly random permutation
    of 1 .. n(n-1)/2 (the random distance matrices of the apparent-fraction
    experiment, Sec. 5.6.6), stored as float32.  Only the order of the
    entries matters (Obs 5.6.8) and integers past 2^24 are not all float32
    values, so rank k is stored as the k-th float32 above 1.0 (bit pattern of
    1.0 plus k): distinct, finite and in the same order."""
    m = n * (n - 1) // 2
    perm = _rng(seed, n, sample).permutation(m).astype(np.uint32) + np.uint32(1)
    return (perm + np.uint32(0x3F800000)).view(np.float32)


def pack(clouds):
    """Concatenate clouds into float32 (sum n, dim) plus int64 offsets (num+1)."""
    offs = np.zeros(len(clouds) + 1, dtype=np.int64)
    offs[1:] = np.cumsum([c.shape[0] for c in clouds])
    pts = np.concatenate(clouds, 0) if clouds else np.zeros((0, 3), np.float32)
    return np.ascontiguousarray(pts, dtype=np.float32), offs


WORKLOADS = {
    "uniform64": dict(make=lambda: uniform_cube(64, 3, seed=0), dmax=1, threshold=np.inf,
                      desc="n=64 uniform in [0,1]^3, seed 0, H0-H1, no threshold"),
    "torus500": dict(make=lambda: torus(500, seed=1), dmax=2, threshold=np.inf,
                     desc="n=500 on the torus R=2, r=1 in R^3 + N(0, 0.05^2), seed 1, H0-H2, no threshold"),
    "sphere200": dict(make=lambda: sphere(200, 4, 1.0, 0.02, seed=2), dmax=3, threshold=1.2,
                      desc="n=200 uniform on S^3 in R^4 + N(0, 0.02^2), seed 2, H0-H3, threshold 1.2"),
    "o3like4096": dict(make=lambda: orthogonal_group(4096, seed=6), dmax=2, threshold=1.4,
                       desc="n=4096 Haar-random O(3) matrices in R^9, seed 6, H0-H2, threshold 1.4"),
}
