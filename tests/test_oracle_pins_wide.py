"""Further pins of the CPU oracle, each against something other than itself.

* ``or_distances_f32`` against an independent float32 evaluation of the
  distance formula, one IEEE single rounding per operation, k ascending
  (numpy float32 ufuncs), bit for bit, on inputs where the order of the sum
  and a fused multiply-add change the last bit.
* ``or_cohom`` (Algorithm 12, with and without clearing) against ``or_plain``
  (Algorithm 2 on the explicit boundary matrix), index for index, on 1000
  random inputs of up to 40 points and dimension up to 3, a third of them
  tie-heavy integer matrices, and on the 64-point uniform cloud in full.  The
  equality rests on Prop 4.3.5 (cohomology gives the same pairs), Lemma
  5.2.10 (oblivious reduction) and the clearing lemma of Sec. 5.2.3.  These
  inputs are large enough that the oracle's pivot table outgrows its initial
  size (more than 512 pivots in a dimension), which the stats counters show.
"""
import math

import numpy as np

import oracle
from paper_2502_05063_b300 import synth


def full_rows(pairs):
    return sorted((int(r["dim"]), float(r["birth"]), float(r["death"]), int(r["birth_cidx"]),
                   int(r["death_cidx"])) for r in pairs)


# --------------------------------------------------------------------------
# the single-precision distance formula
# --------------------------------------------------------------------------

def _stepwise_f32(pts, order=None):
    """sqrt(sum_k (x_ik - x_jk)^2) over all pairs i > j, every operation an
    IEEE single-precision operation (numpy float32 arithmetic), k in `order`."""
    pts = np.asarray(pts, dtype=np.float32)
    n, dim = pts.shape
    ii, jj = np.tril_indices(n, -1)          # row-major lower triangle: (1,0), (2,0), (2,1), ...
    acc = np.zeros(len(ii), dtype=np.float32)
    for k in (range(dim) if order is None else order):
        diff = pts[ii, k] - pts[jj, k]      # float32 - float32 -> float32, rounded once
        acc = acc + diff * diff             # product rounded, then the sum rounded
    return np.sqrt(acc)                     # IEEE correctly rounded float32 square root


def _fma_f32(pts):
    """The same sum with each multiply-add fused (one rounding for d*d + acc),
    emulated exactly: d*d is exact in float64, and the rounding of the
    float64 sum to float32 differs from one exact rounding only on ties far
    below what the check below needs."""
    pts = np.asarray(pts, dtype=np.float32)
    n, dim = pts.shape
    ii, jj = np.tril_indices(n, -1)
    acc = np.zeros(len(ii), dtype=np.float32)
    for k in range(dim):
        diff = (pts[ii, k] - pts[jj, k]).astype(np.float64)
        acc = (diff * diff + acc.astype(np.float64)).astype(np.float32)
    return np.sqrt(acc)


def _hard_clouds():
    """Inputs on which summation order and contraction matter."""
    rng = np.random.default_rng(20250207)
    out = []
    for amb in (1, 2, 3, 4, 7, 8, 16):
        n = 48
        scale = 10.0 ** rng.uniform(-3, 3, size=(n, amb))       # mixed magnitudes per coordinate
        x = rng.standard_normal((n, amb)) * scale
        x[1::2] = x[0::2] + rng.standard_normal((n // 2, amb)) * 1e-4 * scale[0::2]  # near-cancelling
        out.append(x.astype(np.float32))
        out.append(rng.random((n, amb)).astype(np.float32) + np.float32(1000.0))   # large offset, small spread
    return out


def test_distances_f32_stepwise_bit_exact():
    """The oracle's distances are the k-ascending single-rounding evaluation,
    bit for bit, on every pair of every input."""
    for pts in _hard_clouds():
        got = oracle.distances_f32(pts)
        want = _stepwise_f32(pts)
        assert got.dtype == np.float32 and want.dtype == np.float32
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), pts.shape


def test_distance_pin_detects_order_and_fma():
    """The inputs above do tell the evaluation orders apart: reversing k, or
    fusing the multiply-add, changes some distances, so the bit-exact pin
    would catch either change in the oracle."""
    rev = fma = 0
    for pts in _hard_clouds():
        ref = _stepwise_f32(pts).view(np.uint32)
        if pts.shape[1] > 1:
            rev += int(np.sum(_stepwise_f32(pts, order=range(pts.shape[1] - 1, -1, -1)).view(np.uint32) != ref))
        fma += int(np.sum(_fma_f32(pts).view(np.uint32) != ref))
    assert rev > 100 and fma > 100, (rev, fma)


def test_distances_are_symmetric_and_sqrt_exact_on_squares():
    """(a-b)^2 = (b-a)^2 exactly, so swapping the two points changes no bit;
    integer coordinates with a perfect-square sum give the exact root."""
    rng = np.random.default_rng(3)
    x = rng.standard_normal((30, 5)).astype(np.float32)
    a = oracle.distances_f32(x)
    b = oracle.distances_f32(x[::-1].copy())
    n = 30
    # pair (i, j) of x is pair (n-1-j, n-1-i) of the reversed cloud
    S = np.zeros((n, n), np.float32)
    S[np.tril_indices(n, -1)] = b
    S = S + S.T
    A = np.zeros((n, n), np.float32)
    A[np.tril_indices(n, -1)] = a
    A = A + A.T
    assert np.array_equal(A.view(np.uint32), S[::-1, ::-1].view(np.uint32))
    pts = np.array([[0, 0, 0], [3, 4, 0], [2, 3, 6], [1, 4, 8]], dtype=np.float32)
    # 5 = |(3,4,0)|, 7 = |(2,3,6)|, 9 = |(1,4,8)|
    d = oracle.distances_f32(pts)
    assert d[0] == 5.0 and d[1] == 7.0 and d[3] == 9.0


# --------------------------------------------------------------------------
# O-cohom against O-plain on inputs of up to 40 points
# --------------------------------------------------------------------------

def _instance(rng, it):
    n = int(rng.integers(2, 41))
    tie_heavy = it % 3 == 0
    if tie_heavy:
        D = rng.integers(1, 5, size=n * (n - 1) // 2).astype(np.float64)
    else:
        amb = int(rng.integers(1, 5))
        D = oracle.distances_f32(rng.random((n, amb)).astype(np.float32)).astype(np.float64)
    # dimension and threshold keep every instance at a fraction of a second
    if n <= 12:
        dmax = int(rng.integers(0, 4))
    elif n <= 24:
        dmax = int(rng.integers(0, 3))
    else:
        dmax = int(rng.integers(0, 2)) if it % 5 else 2
    thr = math.inf
    if len(D) and (it % 4 == 0 or n > 30 or (dmax >= 2 and n > 16)):
        q = 0.35 if (dmax >= 2 and n > 16) else float(rng.uniform(0.3, 0.9))
        thr = float(np.quantile(D, q))
    if n > 30 and dmax == 3:
        dmax = 2
    return n, D, dmax, thr


def test_plain_equals_cohom_up_to_40_points():
    rng = np.random.default_rng(4040)
    grown = 0
    sizes = []
    for it in range(1000):
        n, D, dmax, thr = _instance(rng, it)
        a = full_rows(oracle.plain(D, n, dmax, thr))
        pb, sb = oracle.cohom(D, n, dmax, thr)
        pc, sc = oracle.cohom(D, n, dmax, thr, clearing=True)
        assert a == full_rows(pb) == full_rows(pc), (it, n, dmax, thr)
        grown += int(np.any(sb[:, 2] > 512))
        sizes.append(n)
    assert max(sizes) == 40 and sum(s > 30 for s in sizes) > 150
    assert grown > 20  # pivot tables grew past their initial 1024 slots in these instances


def test_plain_equals_cohom_uniform64_in_full():
    """The 64-point uniform cloud (H0-H1) with and without the enclosing-radius
    truncation: all three reductions agree on every pair, and the dimension-1
    pivot table grows (more than 512 pivots)."""
    pts = synth.uniform_cube(64, 3, seed=0)
    n = 64
    D = oracle.distances_f32(pts).astype(np.float64)
    R = oracle.enclosing_radius(D, n)
    for thr in (math.inf, R):
        a = full_rows(oracle.plain(D, n, 1, thr))
        pb, sb = oracle.cohom(D, n, 1, thr)
        pc, sc = oracle.cohom(D, n, 1, thr, clearing=True)
        assert a == full_rows(pb) == full_rows(pc)
        assert sb[1, 2] > 512
        # the clearing run skips exactly the 63 tree edges (H0 deaths) among the edges
        assert sb[1, 0] - sc[1, 0] == n - 1
