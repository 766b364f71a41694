"""Paths of the public call that the workloads do not reach, each compared
with the oracle (or, for H0 at sizes the oracle is slow on, with Kruskal's
algorithm and the elder rule written out here), bit for bit:

* the spanning-tree kernel for n > 8192 (Prim, shared- and global-memory
  variants) and the elder rule with its union-find in global memory;
* the fused filtration/apparent kernel and the reduction for p = 4, 5, 6;
* VR_ERR_INDEX_OVERFLOW from the packed-key check after ranking;
* VR_DEBUG_CHECKS on results that satisfy every identity;
* vr_backward with an edge endpoint outside the cloud.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_2502_05063_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2502_05063_b300 import vr as _vr
    return _vr


def rows_gpu(bc, p):
    return [(float(r["birth"]), float(r["death"]), int(r["birth_simplex"]), int(r["death_simplex"]))
            for r in bc.pairs[p]]


def rows_oracle(dg_p):
    return [(float(np.float32(r["birth"])), float(np.float32(r["death"])) if np.isfinite(r["death"]) else math.inf,
             int(r["birth_cidx"]), int(r["death_cidx"])) for r in dg_p]


def h0_by_kruskal(D, n, thr):
    """H0 under the strict order (diameter ascending, edge index descending):
    Kruskal's algorithm over the edges within the threshold, elder rule for
    the birth vertex (a component is as old as its largest vertex; the
    younger one dies), essential classes at each remaining component's
    largest vertex.  Rows as the library emits them (zero-length omitted)."""
    idx = np.nonzero(D <= thr)[0]
    # condensed index e = i(i-1)/2 + j  ->  (i, j), i > j
    i = np.floor((1 + np.sqrt(1 + 8 * idx.astype(np.float64))) / 2).astype(np.int64)
    i -= (i * (i - 1) // 2 > idx)
    i += ((i + 1) * i // 2 <= idx)
    j = idx - i * (i - 1) // 2
    order = np.lexsort((-idx, D[idx]))
    parent = np.arange(n)
    oldest = np.arange(n)

    def find(x):
        r = x
        while parent[r] != r:
            r = parent[r]
        while parent[x] != r:
            parent[x], x = r, parent[x]
        return r

    rows = []
    for k in order:
        a, b = find(int(i[k])), find(int(j[k]))
        if a == b:
            continue
        young, old = (a, b) if oldest[a] < oldest[b] else (b, a)
        if D[idx[k]] > 0:
            rows.append((0.0, float(D[idx[k]]), int(oldest[young]), int(idx[k])))
        parent[young] = old
    for v in range(n):
        if find(v) == v:
            rows.append((0.0, math.inf, int(oldest[v]), -1))
    rows.sort(key=lambda r: (r[0], r[1], r[2]))
    return rows


# --------------------------------------------------------------------------
# spanning tree for n > 8192
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,q,dmax", [(8300, 0.0005, 1), (8300, 0.002, 0), (9001, 0.0002, 0)])
def test_prim_path_matches_oracle(vr, n, q, dmax):
    """n just above 8192 (Prim, keys in shared memory): H0 (and H1 when asked)
    equal the oracle; the small thresholds leave the graph disconnected or
    barely connected."""
    rng = np.random.default_rng(n + int(q * 1e5))
    pts = rng.random((n, 3)).astype(np.float32)
    D = oracle.distances_f32(pts)
    thr = float(np.quantile(D[:400000], q))
    bc = vr.barcodes(points=pts, dmax=dmax, threshold=thr)
    pairs, _ = oracle.cohom(D.astype(np.float64), n, dmax, float(np.float32(thr)), clearing=True)
    dg = oracle.diagram(pairs, dmax)
    for p in range(dmax + 1):
        assert rows_gpu(bc, p) == rows_oracle(dg[p]), p
    assert rows_gpu(bc, 0) == h0_by_kruskal(D, n, np.float32(thr))


def test_prim_global_memory_path(vr):
    """n = 20000: Prim keeps its keys and the elder rule its union-find in global
    memory.  H0 against Kruskal and the elder rule, at a threshold that leaves
    several components and at one that connects the cloud."""
    n = 20000
    rng = np.random.default_rng(20000)
    pts = rng.random((n, 3)).astype(np.float32)
    D = oracle.distances_f32(pts)
    for q in (0.00005, 0.0003):
        thr = np.float32(np.quantile(D[:1000000], q))
        bc = vr.barcodes(points=pts, dmax=0, threshold=float(thr))
        assert rows_gpu(bc, 0) == h0_by_kruskal(D, n, thr), q


# --------------------------------------------------------------------------
# dimensions 4 to 6
# --------------------------------------------------------------------------

def _high_dim_cases():
    out = []
    for dmax in (4, 5, 6):
        for kind in ("random", "ties"):
            for n in (dmax + 3, dmax + 5, 12):
                out.append((dmax, kind, n))
    return out


@pytest.mark.parametrize("dmax,kind,n", _high_dim_cases())
def test_high_dimensions_exact(vr, dmax, kind, n):
    """p = 4..6 (the fused kernel's and the reduction's largest instances):
    every pair, zero-length ones included, and the critical edges."""
    rng = np.random.default_rng(100 * dmax + n + (kind == "ties"))
    if kind == "random":
        D = oracle.distances_f32(rng.random((n, 3)).astype(np.float32))
    else:
        D = rng.integers(1, 4, size=n * (n - 1) // 2).astype(np.float32)
    flags = vr.VR_KEEP_ZERO_LENGTH | vr.VR_CRITICAL_EDGES | vr.VR_DEBUG_CHECKS
    bc = vr.barcodes(dists=D, n=n, dmax=dmax, flags=flags)
    D64 = D.astype(np.float64)
    R = oracle.enclosing_radius(D64, n)
    pairs, _ = oracle.cohom(D64, n, dmax, R, clearing=True)
    dg = oracle.diagram(pairs, dmax, keep_zero=True)
    if n <= 10:  # the definition itself (Algorithm 2) agrees
        assert sorted(map(tuple, oracle.diagram(oracle.plain(D64, n, dmax, R), dmax, keep_zero=True)[dmax][
            ["birth", "death", "birth_cidx", "death_cidx"]].tolist())) == sorted(
            map(tuple, dg[dmax][["birth", "death", "birth_cidx", "death_cidx"]].tolist()))
    for p in range(dmax + 1):
        assert rows_gpu(bc, p) == rows_oracle(dg[p]), p
        for row, e in zip(bc.pairs[p], bc.critical_edges[p]):
            if p > 0:
                assert tuple(e[:2]) == oracle.critical_edge(D64, n, int(row["birth_simplex"]), p)
            if row["death_simplex"] >= 0:
                assert tuple(e[2:]) == oracle.critical_edge(D64, n, int(row["death_simplex"]), p + 1)


# --------------------------------------------------------------------------
# error paths and checks
# --------------------------------------------------------------------------

def test_index_overflow_after_ranking(vr):
    """3000 random points have about 4.5M distinct distances (23 rank bits); a
    tetrahedron index needs 42 bits, so the dimension-2 row keys would need 65:
    VR_ERR_INDEX_OVERFLOW, reported before any dimension is computed."""
    rng = np.random.default_rng(3000)
    pts = rng.random((3000, 3)).astype(np.float32)
    with pytest.raises(vr.VRError) as e:
        vr.barcodes(points=pts, dmax=3)
    assert e.value.name == "VR_ERR_INDEX_OVERFLOW"
    # with few distinct distances the same sizes fit: integer coordinates 0..3
    small = rng.integers(0, 4, size=(300, 3)).astype(np.float32)
    bc = vr.barcodes(points=small, dmax=1, threshold=1.0, flags=vr.VR_DEBUG_CHECKS)
    assert len(bc.pairs[0]) >= 1


def test_debug_checks_on_workloads(vr):
    """VR_DEBUG_CHECKS accepts correct results (the 200-point sphere workload and
    random clouds) and changes nothing in them."""
    w = synth.WORKLOADS["sphere200"]
    pts = w["make"]()
    a = vr.barcodes(points=pts, dmax=w["dmax"], threshold=w["threshold"])
    b = vr.barcodes(points=pts, dmax=w["dmax"], threshold=w["threshold"], flags=vr.VR_DEBUG_CHECKS)
    for p in range(w["dmax"] + 1):
        assert rows_gpu(a, p) == rows_gpu(b, p)
    clouds = [synth.uniform_cube(int(n), 3, seed=int(n)) for n in (5, 40, 120)]
    pts, offs = synth.pack(clouds)
    vr.barcodes_batched(pts, offs, dmax=1, flags=vr.VR_DEBUG_CHECKS)


def test_backward_rejects_out_of_range_edge(vr):
    """An edge endpoint >= n is skipped and reported as VR_ERR_INVALID_ARG; the
    valid edges still contribute."""
    import torch
    pts = torch.tensor([[0.0, 0.0], [3.0, 4.0], [6.0, 8.0]], device="cuda")
    edges = torch.tensor([[1, 0, -1, -1], [7, 0, 2, 1]], dtype=torch.int32, device="cuda")
    gb = torch.tensor([1.0, 1.0], device="cuda")
    gd = torch.tensor([0.0, 2.0], device="cuda")
    grad = torch.zeros_like(pts)
    with pytest.raises(vr.VRError) as e:
        vr.backward(pts, edges, gb, gd, grad)
    assert e.value.name == "VR_ERR_INVALID_ARG"
    # edge (1,0) with g=1 and edge (2,1) with g=2: unit vector (0.6, 0.8)
    want = np.array([[-0.6, -0.8], [0.6 - 1.2, 0.8 - 1.6], [1.2, 1.6]], np.float32)
    assert np.allclose(grad.cpu().numpy(), want, rtol=0, atol=1e-6)
    grad.zero_()
    ok = edges.clone()
    ok[1, 0] = 2
    vr.backward(pts, ok, gb, gd, grad)
