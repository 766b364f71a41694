"""The sparse (low-threshold) mode, VR_SPARSE (Sec. 5.3.12-5.3.13, Algorithm
15; Sec. 5.5.3; Sec. 5.7.2): the complex listed from neighbour lists gives
the pairs of the oracle, bit for bit, and those of the dense path."""
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


def rows(bc, p):
    return [(float(r["birth"]), float(r["death"]), int(r["birth_simplex"]), int(r["death_simplex"]))
            for r in bc.pairs[p]]


def oracle_rows(dg_p):
    return [(float(np.float32(r["birth"])), float(np.float32(r["death"])) if np.isfinite(r["death"]) else math.inf,
             int(r["birth_cidx"]), int(r["death_cidx"])) for r in dg_p]


@pytest.mark.parametrize("name", ["torus500", "sphere200"])
@pytest.mark.parametrize("q", [0.1, 0.3])
def test_sparse_workloads_at_low_thresholds(vr, name, q):
    """The 500-point torus (H0-H2) and 200-point sphere (H0-H3) at thresholds at
    the 10th and 30th percentile of their distances."""
    w = synth.WORKLOADS[name]
    pts = w["make"]()
    n, dmax = pts.shape[0], w["dmax"]
    D = oracle.distances_f32(pts)
    thr = float(np.quantile(D, q))
    sp = vr.barcodes(points=pts, dmax=dmax, threshold=thr, flags=vr.VR_SPARSE | vr.VR_DEBUG_CHECKS)
    de = vr.barcodes(points=pts, dmax=dmax, threshold=thr)
    pairs, st = oracle.cohom(D.astype(np.float64), n, dmax, float(np.float32(thr)), clearing=True)
    dg = oracle.diagram(pairs, dmax)
    for p in range(dmax + 1):
        assert rows(sp, p) == oracle_rows(dg[p]), p
        assert rows(sp, p) == rows(de, p), p
        if p >= 1:
            for k in ("columns", "apparent", "reduced", "pairs", "essential", "cleared"):
                assert sp.stats[p][k] == de.stats[p][k], (p, k)
            # the listed simplices are exactly the p-simplices within the threshold
            assert sp.stats[p]["candidates"] == de.stats[p]["candidates"] - de.stats[p]["above_threshold"]


@pytest.mark.parametrize("it", range(10))
def test_sparse_random_clouds(vr, it):
    rng = np.random.default_rng(7000 + it)
    n = int(rng.integers(2, 80))
    amb = int(rng.integers(1, 5))
    pts = rng.random((n, amb)).astype(np.float32)
    if it % 3 == 0:
        pts = np.round(pts * 4).astype(np.float32)  # ties and duplicates
    dmax = int(rng.integers(1, 4 if n <= 40 else 3))
    D = oracle.distances_f32(pts)
    thr = float(np.quantile(D, rng.uniform(0.05, 0.6))) if len(D) else 1.0
    flags = vr.VR_SPARSE | (vr.VR_KEEP_ZERO_LENGTH | vr.VR_CRITICAL_EDGES if it % 2 else 0)
    sp = vr.barcodes(points=pts, dmax=dmax, threshold=thr, flags=flags)
    de = vr.barcodes(points=pts, dmax=dmax, threshold=thr, flags=flags & ~vr.VR_SPARSE)
    pairs, _ = oracle.cohom(D.astype(np.float64), n, dmax, float(np.float32(thr)), clearing=True)
    dg = oracle.diagram(pairs, dmax, keep_zero=bool(flags & vr.VR_KEEP_ZERO_LENGTH))
    for p in range(dmax + 1):
        assert rows(sp, p) == oracle_rows(dg[p]), (it, p)
        if flags & vr.VR_CRITICAL_EDGES:
            assert sp.critical_edges[p].tolist() == de.critical_edges[p].tolist()


def test_sparse_empty_and_edgeless(vr):
    pts = synth.uniform_cube(50, 3, seed=1)
    bc = vr.barcodes(points=pts, dmax=2, threshold=1e-6, flags=vr.VR_SPARSE)  # no edge within it
    assert len(bc.pairs[0]) == 50 and all(math.isinf(float(x)) for x in bc.pairs[0]["death"])
    assert len(bc.pairs[1]) == 0 and len(bc.pairs[2]) == 0
    assert bc.stats[1]["candidates"] == 0 and bc.stats[2]["candidates"] == 0


def test_sparse_o3_sample(vr):
    """The O(3)-sample stand-in at the paper's threshold 1.4, 600 points, H0-H2:
    sparse, dense and the oracle agree."""
    pts = synth.orthogonal_group(600, seed=16)
    D = oracle.distances_f32(pts)
    sp = vr.barcodes(points=pts, dmax=2, threshold=1.4, flags=vr.VR_SPARSE | vr.VR_DEBUG_CHECKS)
    pairs, _ = oracle.cohom(D.astype(np.float64), 600, 2, float(np.float32(1.4)), clearing=True)
    dg = oracle.diagram(pairs, 2)
    for p in range(3):
        assert rows(sp, p) == oracle_rows(dg[p]), p
