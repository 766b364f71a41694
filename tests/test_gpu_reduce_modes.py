"""The three reductions of the non-apparent columns (Sec. 5.2.9): the default
(reduced columns kept explicitly by the block engine), the reduction-matrix
technique (VR_REDUCE_V: every finished column keeps only its generators) and
oblivious reduction (VR_REDUCE_OBLIVIOUS: Algorithm 12 as printed, nothing
kept).  Lemma 5.2.10 makes all three give the same pairs; each is compared
with the oracle or its stored output, bit for bit."""
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


MODES = ["default", "v", "oblivious"]


def mode_flag(vr, mode):
    return {"default": 0, "v": vr.VR_REDUCE_V, "oblivious": vr.VR_REDUCE_OBLIVIOUS}[mode]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("it", range(6))
def test_modes_random_clouds(vr, mode, it):
    rng = np.random.default_rng(900 + it)
    n = [30, 60, 90, 45, 120, 70][it]
    pts = rng.random((n, 3)).astype(np.float32)
    if it == 3:
        pts = np.round(pts * 4).astype(np.float32)
    dmax = 2 if n <= 90 else 1
    bc = vr.barcodes(points=pts, dmax=dmax, flags=mode_flag(vr, mode) | vr.VR_DEBUG_CHECKS)
    D = oracle.distances_f32(pts).astype(np.float64)
    pairs, _ = oracle.cohom(D, n, dmax, oracle.enclosing_radius(D, n), clearing=True)
    dg = oracle.diagram(pairs, dmax)
    for p in range(dmax + 1):
        assert rows(bc, p) == oracle_rows(dg[p]), (mode, p)


@pytest.mark.parametrize("mode", ["v", "oblivious"])
@pytest.mark.parametrize("name", ["uniform64", "sphere200", "torus500"])
def test_modes_workload_golden(vr, mode, name):
    from test_gpu_parity import load_golden
    g, pts, thr, dg = load_golden(name)
    bc = vr.barcodes(points=pts, dmax=g["dmax"], threshold=thr, flags=mode_flag(vr, mode))
    for p in range(g["dmax"] + 1):
        assert rows(bc, p) == dg[p], (mode, p)


@pytest.mark.parametrize("n", [40, 60, 75])
def test_modes_random_permutation(vr, n):
    """Random non-metric matrices (Sec. 5.6.6): the three modes agree with the
    oracle, and at n = 100 with each other (the oracle's oblivious reduction
    no longer finishes in seconds there)."""
    D = synth.random_permutation_dists(n, sample=3)
    thr = float(D.max())
    pairs, _ = oracle.cohom(D.astype(np.float64), n, 1, thr, clearing=True)
    dg = oracle.diagram(pairs, 1)
    for mode in MODES:
        bc = vr.barcodes(dists=D, n=n, dmax=1, threshold=thr, flags=mode_flag(vr, mode) | vr.VR_DEBUG_CHECKS)
        for p in range(2):
            assert rows(bc, p) == oracle_rows(dg[p]), (mode, p)


def test_modes_agree_random_permutation_100(vr):
    D = synth.random_permutation_dists(100, sample=1)
    thr = float(D.max())
    got = [vr.barcodes(dists=D, n=100, dmax=1, threshold=thr, flags=mode_flag(vr, m)) for m in MODES]
    for p in range(2):
        assert rows(got[0], p) == rows(got[1], p) == rows(got[2], p), p
