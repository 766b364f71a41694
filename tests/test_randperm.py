"""The random-permutation workload of the apparent-fraction experiment
(Sec. 5.6.6, Fig 5.14): the lower triangle of the distance matrix is a
uniformly random permutation of 1 .. n(n-1)/2, and the quantity is the
fraction of dimension-1 columns (edges of the full 2-skeleton) that are
apparent.

CPU: the generator is a permutation in the stored order, and the oracle's
apparent pairs depend only on that order (Obs 5.6.8) and respect the upper
bound of Thm 5.4.2, (n-2)/n.  GPU: every pair equals the oracle (n <= 70,
where the oracle's oblivious reduction still finishes in seconds), the
apparent count equals Def 5.3.4 taken literally, and at n up to 9000 the
apparent-only run (VR_APPARENT_ONLY) stays within the bound, agrees with the
full run where that completes, and passes the count identities."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_05063_b300 import synth


def test_generator_is_a_permutation_in_float_order():
    for n in (2, 3, 17, 300):
        D = synth.random_permutation_dists(n, sample=1)
        m = n * (n - 1) // 2
        assert D.dtype == np.float32 and len(D) == m and np.all(np.isfinite(D))
        ranks = D.view(np.uint32).astype(np.int64) - 0x3F800000
        assert sorted(ranks.tolist()) == list(range(1, m + 1))
        assert np.array_equal(np.argsort(D, kind="stable"), np.argsort(ranks, kind="stable"))


@pytest.mark.parametrize("n", [6, 12, 25, 40])
def test_oracle_apparent_depends_only_on_order(n):
    """Obs 5.6.8 and Thm 5.4.2 on the oracle: the integer permutation and its
    float coding give the same apparent pairs, at most C(n-1, 2) of them."""
    D = synth.random_permutation_dists(n).astype(np.float64)
    ints = (D.astype(np.float32).view(np.uint32).astype(np.int64) - 0x3F800000).astype(np.float64)
    a = oracle.apparent(D, n, 1, float(D.max()))
    b = oracle.apparent(ints, n, 1, float(ints.max()))
    assert sorted(map(tuple, a.tolist())) == sorted(map(tuple, b.tolist()))
    assert 1 <= len(a) <= math.comb(n - 1, 2)


@pytest.fixture(scope="module")
def vr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2502_05063_b300 import vr as _vr
    return _vr


def _rows(bc, p):
    return [(float(r["birth"]), float(r["death"]), int(r["birth_simplex"]), int(r["death_simplex"]))
            for r in bc.pairs[p]]


@pytest.mark.gpu
@pytest.mark.parametrize("n", [5, 12, 30, 50, 70])
def test_randperm_exact(vr, n):
    D = synth.random_permutation_dists(n, sample=n)
    thr = float(D.max())  # the full 2-skeleton
    bc = vr.barcodes(dists=D, n=n, dmax=1, threshold=thr, flags=vr.VR_DEBUG_CHECKS)
    D64 = D.astype(np.float64)
    pairs, _ = oracle.cohom(D64, n, 1, thr, clearing=True)
    dg = oracle.diagram(pairs, 1)
    for p in range(2):
        want = [(float(np.float32(r["birth"])), float(np.float32(r["death"])) if np.isfinite(r["death"]) else math.inf,
                 int(r["birth_cidx"]), int(r["death_cidx"])) for r in dg[p]]
        assert _rows(bc, p) == want, p
    assert bc.stats[1]["apparent"] == len(oracle.apparent(D64, n, 1, thr))
    only = vr.barcodes(dists=D, n=n, dmax=1, threshold=thr, flags=vr.VR_APPARENT_ONLY | vr.VR_DEBUG_CHECKS)
    assert only.stats[1]["apparent"] == bc.stats[1]["apparent"]
    assert only.stats[1]["reduced"] == bc.stats[1]["reduced"]
    assert len(only.pairs[1]) == 0 and _rows(only, 0) == _rows(bc, 0)


@pytest.mark.gpu
def test_randperm_apparent_fraction_large(vr):
    """n = 100 .. 9000: within the Thm 5.4.2 bound (n-2)/n; at n = 100 equal to
    the full run; and increasing with n, as the paper's curve does."""
    import torch
    fr = []
    for n in (100, 400, 2000, 9000):
        D = synth.random_permutation_dists(n)
        d = torch.from_numpy(D).cuda()
        thr = float(D.max())
        bc = vr.barcodes(dists=d, n=n, dmax=1, threshold=thr, flags=vr.VR_APPARENT_ONLY | vr.VR_DEBUG_CHECKS)
        st = bc.stats[1]
        m = n * (n - 1) // 2
        assert st["candidates"] == m and st["above_threshold"] == 0 and st["cleared"] == n - 1
        assert st["apparent"] <= math.comb(n - 1, 2)
        fr.append(st["apparent"] / m)
        if n == 100:
            full = vr.barcodes(dists=d, n=n, dmax=1, threshold=thr)
            assert full.stats[1]["apparent"] == st["apparent"]
    assert fr == sorted(fr) and fr[-1] > 0.98, fr
