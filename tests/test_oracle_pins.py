"""Pins that hold the CPU oracle to the dissertation (arXiv 2502.05063) and to
mathematics outside it.  None of these compares the oracle with itself: each
expected value comes from a printed example, a closed form, a textbook
routine or an independent computation (rank-based brute force)."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse
import scipy.sparse.csgraph

import oracle
from oracle import brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def condensed(square):
    n = len(square)
    return np.array([square[i][j] for i in range(1, n) for j in range(i)], dtype=np.float64)


def square_of(D, n):
    S = np.zeros((n, n))
    k = 0
    for i in range(1, n):
        for j in range(i):
            S[i, j] = S[j, i] = D[k]
            k += 1
    return S


def as_multiset(pairs, dmax):
    """{(p, birth, death)} with death > birth, as a sorted list."""
    out = []
    for p in range(dmax + 1):
        for r in pairs[pairs["dim"] == p]:
            if r["death"] > r["birth"]:
                out.append((p, float(r["birth"]), float(r["death"])))
    return sorted(out)


def full_rows(pairs):
    return sorted((int(r["dim"]), float(r["birth"]), float(r["death"]), int(r["birth_cidx"]),
                   int(r["death_cidx"])) for r in pairs)


# --------------------------------------------------------------------------
# Worked examples printed in the paper
# --------------------------------------------------------------------------

def test_fig_4_1_standard_reduction():
    """Figs 4.1/4.2: pivots (2,3), (1,4), (5,6); column 5 reduces to zero."""
    cols, lows = {}, None
    for line in open(os.path.join(GOLDEN, "fig_4_1_boundary.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, _, rest = line.partition(":")
        if key == "lows":
            lows = [int(x) for x in rest.split()]
        else:
            cols[int(key)] = [int(x) for x in rest.split()]
    got = oracle.reduce_explicit([cols[j] for j in range(len(cols))])
    assert list(got) == lows
    pivots = sorted((int(l), j) for j, l in enumerate(got) if l >= 0)
    assert pivots == [(1, 4), (2, 3), (5, 6)]


def test_fig_5_1_square():
    """Fig 5.1: four corners of a square; one H1 bar born at 1, dying at sqrt(2)."""
    pts = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)
    D = oracle.distances_f32(pts)
    s2 = float(np.sqrt(np.float32(2.0)))
    for pairs in (oracle.plain(D, 4, 1), oracle.cohom(D, 4, 1)[0], oracle.cohom(D, 4, 1, clearing=True)[0]):
        dg = oracle.diagram(pairs, 1)
        assert [(float(r["birth"]), float(r["death"])) for r in dg[1]] == [(1.0, s2)]
        assert sorted(float(r["death"]) for r in dg[0]) == [1.0, 1.0, 1.0, math.inf]
    assert brute.barcode(square_of(D, 4), 4, 1) == sorted(
        [(0, 0.0, 1.0)] * 3 + [(0, 0.0, math.inf), (1, 1.0, s2)])


def _fig_5_5_5_6():
    rows, pairs = {}, []
    for line in open(os.path.join(GOLDEN, "fig_5_5_5_6_apparent.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        key, _, rest = line.partition(":")
        if key == "pairs":
            e, t = rest.split(";")
            pairs.append((tuple(int(x) for x in e.split()), tuple(int(x) for x in t.split())))
        else:
            rows[key] = [float(x) for x in rest.split()]
    return rows, pairs


@pytest.mark.parametrize("fig", ["fig5.5", "fig5.6"])
def test_fig_5_5_and_5_6_apparent_pairs(fig):
    rows, pairs = _fig_5_5_5_6()
    D = np.array(rows[fig])
    got = oracle.apparent(D, 5, 1)
    want = sorted((oracle.simplex_index(e, 5), oracle.simplex_index(t, 5)) for e, t in pairs)
    assert sorted(map(tuple, got.tolist())) == want


# --------------------------------------------------------------------------
# Closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n0,d", [(4, 1), (5, 1), (7, 1), (6, 2), (7, 3)])
def test_thm_5_4_2_upper_bound_all_equal(n0, d):
    """Thm 5.4.2: with all diameters equal exactly C(n0-1, d+1) apparent pairs."""
    D = np.ones(n0 * (n0 - 1) // 2)
    assert len(oracle.apparent(D, n0, d)) == math.comb(n0 - 1, d + 1)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_thm_5_4_2_single_simplex(d):
    """Tightness of the lower bound: one (d+1)-simplex has exactly one apparent pair."""
    n0 = d + 2
    rng = np.random.default_rng(d)
    D = rng.permutation(n0 * (n0 - 1) // 2).astype(np.float64) + 1
    assert len(oracle.apparent(D, n0, d)) == 1


def test_thm_5_4_2_bounds_random():
    """(n0-d-1)/n0 >= apparent fraction >= ... on random distinct distances (upper bound)."""
    rng = np.random.default_rng(5)
    for n0 in (6, 8, 10):
        for d in (1, 2):
            D = rng.permutation(n0 * (n0 - 1) // 2).astype(np.float64) + 1
            a = len(oracle.apparent(D, n0, d))
            assert a <= math.comb(n0 - 1, d + 1)
            assert a >= 1


def test_combinatorial_number_system():
    """eq. 5.6 is a bijection onto 0..C(n,k)-1 and orders subsets colexicographically."""
    n = 11
    for k in range(1, 5):
        subsets = list(itertools.combinations(range(n), k))
        idx = [oracle.simplex_index(s, n) for s in subsets]
        assert sorted(idx) == list(range(math.comb(n, k)))
        colex = sorted(subsets, key=lambda s: tuple(reversed(s)))
        assert [oracle.simplex_index(s, n) for s in colex] == list(range(math.comb(n, k)))
        for s, c in zip(subsets, idx):
            assert oracle.simplex_vertices(c, k - 1, n) == list(s)


def test_evenly_spaced_circle_one_bar():
    """n evenly spaced points with exact chord ties: H1 is one bar
    [chord(1), chord(ceil(n/3))) (Adamaszek-Adams, outside the paper)."""
    for n in range(5, 25):
        chord = [np.float32(2 * math.sin(math.pi * k / n)) for k in range(n // 2 + 1)]
        S = [[float(chord[min(abs(i - j), n - abs(i - j))]) for j in range(n)] for i in range(n)]
        D = condensed(S)
        for pairs in (oracle.plain(D, n, 1) if n <= 16 else None, oracle.cohom(D, n, 1)[0]):
            if pairs is None:
                continue
            dg = oracle.diagram(pairs, 1)
            bars = [(float(r["birth"]), float(r["death"])) for r in dg[1]]
            assert bars == [(float(chord[1]), float(chord[math.ceil(n / 3)]))], n


def test_circle_points_one_long_bar():
    """Evenly spaced points (float coordinates): exactly one H1 bar much longer than the
    spread of the one-step chords, born at the largest one-step chord."""
    for n in (12, 24, 40):
        th = np.arange(n) * (2 * np.pi / n)
        pts = np.stack([np.cos(th), np.sin(th)], 1).astype(np.float32)
        D = oracle.distances_f32(pts)
        S = square_of(D, n)
        steps = [S[i, (i + 1) % n] for i in range(n)]
        spread = max(steps) - min(steps)
        dg = oracle.diagram(oracle.cohom(D, n, 1)[0], 1)
        long = [r for r in dg[1] if r["death"] - r["birth"] > 10 * spread + 1e-6]
        assert len(long) == 1
        assert float(long[0]["birth"]) == max(steps)


# --------------------------------------------------------------------------
# Textbook routines and invariants
# --------------------------------------------------------------------------

def kruskal(D, n):
    """Kruskal's algorithm under the strict total order (diam asc, edge index desc)."""
    edges = sorted(((D[i * (i - 1) // 2 + j], -(i * (i - 1) // 2 + j), i, j)
                    for i in range(1, n) for j in range(i)))
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    tree = []
    for d, negc, i, j in edges:
        a, b = find(i), find(j)
        if a != b:
            parent[a] = b
            tree.append((d, -negc))
    return tree


@pytest.mark.parametrize("seed", range(6))
def test_h0_is_kruskal(seed):
    """Sec. 5.2.5: H0 deaths are the minimum spanning tree edges."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 40))
    pts = rng.random((n, 3)).astype(np.float32)
    if seed % 2:
        pts = np.round(pts * 4).astype(np.float32)  # many ties, some duplicate points
    D = oracle.distances_f32(pts).astype(np.float64)
    pairs, _ = oracle.cohom(D, n, 0)
    h0 = pairs[(pairs["dim"] == 0) & np.isfinite(pairs["death"])]
    tree = kruskal(D, n)
    assert sorted(int(c) for c in h0["death_cidx"]) == sorted(c for _, c in tree)
    assert sorted(h0["death"].tolist()) == sorted(d for d, _ in tree)
    # scipy's MST (a library routine) gives the same total weight
    S = square_of(D, n)
    mst = scipy.sparse.csgraph.minimum_spanning_tree(scipy.sparse.csr_matrix(S + (S == 0) * 0))
    if np.all(S[np.triu_indices(n, 1)] > 0):
        assert math.isclose(mst.sum(), sum(d for d, _ in tree), rel_tol=1e-12)
    # one essential class, born at the oldest vertex n-1 (Sec. 5.1.4 order)
    ess = pairs[(pairs["dim"] == 0) & ~np.isfinite(pairs["death"])]
    assert len(ess) == 1 and int(ess[0]["birth_cidx"]) == n - 1


def _random_instance(rng, tie_heavy):
    n = int(rng.integers(2, 11))
    if tie_heavy:
        D = rng.integers(1, 4, size=n * (n - 1) // 2).astype(np.float64)
    else:
        D = oracle.distances_f32(rng.random((n, int(rng.integers(1, 4)))).astype(np.float32)).astype(np.float64)
    return n, D


def test_plain_equals_cohom_random():
    """Prop 4.3.5 / Thm 3.2.28 (cohomology gives the same pairs), Lemma 5.2.10
    (oblivious reduction), clearing lemma: all three agree on every pair, index
    by index, on 1000 random inputs, a third of them tie-heavy."""
    rng = np.random.default_rng(1234)
    for it in range(1000):
        n, D = _random_instance(rng, tie_heavy=(it % 3 == 0))
        dmax = int(rng.integers(0, 4 if n <= 8 else 3))
        thr = math.inf if it % 4 else float(np.quantile(D, 0.6)) if len(D) else math.inf
        a = full_rows(oracle.plain(D, n, dmax, thr))
        b = full_rows(oracle.cohom(D, n, dmax, thr)[0])
        c = full_rows(oracle.cohom(D, n, dmax, thr, clearing=True)[0])
        assert a == b == c, (it, n, dmax, thr)


def test_plain_equals_brute_force():
    """Bars from Algorithm 2 equal bars from persistent Betti numbers (ranks)."""
    rng = np.random.default_rng(99)
    for it in range(40):
        n = int(rng.integers(3, 8))
        if it % 2:
            D = rng.integers(1, 5, size=n * (n - 1) // 2).astype(np.float64)
        else:
            D = oracle.distances_f32(rng.random((n, 2)).astype(np.float32)).astype(np.float64)
        dmax = int(rng.integers(0, 3))
        thr = math.inf if it % 3 else float(np.median(D))
        got = as_multiset(oracle.plain(D, n, dmax, thr), dmax)
        want = brute.barcode(square_of(D, n), n, dmax, thr)
        assert got == want, (it, n, dmax)


def _count_simplices(S, n, p, v):
    c = 0
    for s in itertools.combinations(range(n), p + 1):
        if max((S[a, b] for a, b in itertools.combinations(s, 2)), default=0.0) <= v:
            c += 1
    return c


@pytest.mark.parametrize("seed", range(4))
def test_euler_and_count_identities(seed):
    """Obs 3.2.14 (each simplex is a birth or a death) and the Euler-Poincare
    relation with the truncation term, at every filtration value."""
    rng = np.random.default_rng(seed)
    n, dmax = 9, 2
    D = oracle.distances_f32(rng.random((n, 3)).astype(np.float32)).astype(np.float64)
    S = square_of(D, n)
    pairs = oracle.plain(D, n, dmax)
    for p in range(dmax + 1):
        births = np.sum(pairs["dim"] == p)
        deaths_below = np.sum((pairs["dim"] == p - 1) & np.isfinite(pairs["death"])) if p else 0
        assert births + deaths_below == math.comb(n, p + 1)
    for v in sorted(set(D.tolist()) | {0.0}):
        lhs = 0
        for p in range(dmax + 1):
            sel = pairs[pairs["dim"] == p]
            alive = np.sum((sel["birth"] <= v) & (v < sel["death"]))
            lhs += (-1) ** p * int(alive)
        rhs = sum((-1) ** p * _count_simplices(S, n, p, v) for p in range(dmax + 1))
        top = pairs[(pairs["dim"] == dmax) & (pairs["death"] <= v)]
        rhs += (-1) ** (dmax + 1) * len(top)
        assert lhs == rhs, v


def test_enclosing_radius_truncation():
    """Prop 5.2.13: truncating at R changes no pair of nonzero persistence."""
    rng = np.random.default_rng(7)
    for it in range(30):
        n = int(rng.integers(4, 12))
        D = oracle.distances_f32(rng.random((n, 3)).astype(np.float32)).astype(np.float64)
        R = oracle.enclosing_radius(D, n)
        S = square_of(D, n)
        assert R == min(max(S[x, y] for y in range(n) if y != x) for x in range(n))
        dmax = 2 if n <= 9 else 1
        full = oracle.diagram(oracle.plain(D, n, dmax), dmax)
        cut = oracle.diagram(oracle.plain(D, n, dmax, R), dmax)
        for p in range(dmax + 1):
            f = [tuple(r) for r in full[p][["birth", "death", "birth_cidx", "death_cidx"]].tolist()]
            c = [tuple(r) for r in cut[p][["birth", "death", "birth_cidx", "death_cidx"]].tolist()]
            assert f == c


def test_order_preserving_remap():
    """Obs 5.6.8: replacing distances by their ranks keeps every simplex pair."""
    rng = np.random.default_rng(11)
    for it in range(20):
        n = int(rng.integers(4, 11))
        D = oracle.distances_f32(rng.random((n, 3)).astype(np.float32)).astype(np.float64)
        if it % 2:
            D = np.round(D * 3) / 3 + 0.1
        Rk = np.searchsorted(np.unique(D), D).astype(np.float64) + 1
        a = oracle.plain(D, n, 2 if n <= 8 else 1)
        b = oracle.plain(Rk, n, 2 if n <= 8 else 1)
        key = lambda P: sorted((int(r["dim"]), int(r["birth_cidx"]), int(r["death_cidx"])) for r in P)
        assert key(a) == key(b)


def test_apparent_pairs_are_pairs_and_never_cleared():
    """Def 5.3.4 pairs are persistence pairs (zero persistence), and their birth
    simplex is never a death simplex one dimension down (Prop 5.3.9)."""
    rng = np.random.default_rng(3)
    for it in range(30):
        n, D = _random_instance(rng, tie_heavy=(it % 2 == 0))
        if n < 3:
            continue
        pairs = oracle.plain(D, n, 2)
        for p in (1,):
            app = oracle.apparent(D, n, p)
            rows = {(int(r["birth_cidx"]), int(r["death_cidx"])) for r in pairs[pairs["dim"] == p]}
            deaths_below = {int(r["death_cidx"]) for r in pairs[pairs["dim"] == p - 1]}
            for s, t in app.tolist():
                assert (s, t) in rows
                assert s not in deaths_below


def test_critical_edge():
    rng = np.random.default_rng(2)
    n = 9
    D = np.round(rng.random(n * (n - 1) // 2) * 3)
    S = square_of(D, n)
    for q in (1, 2, 3):
        for s in itertools.combinations(range(n), q + 1):
            c = oracle.simplex_index(s, n)
            u, v = oracle.critical_edge(D, n, c, q)
            dm = max(S[a, b] for a, b in itertools.combinations(s, 2))
            ties = [(b, a) for a, b in itertools.combinations(s, 2) if S[a, b] == dm]
            best = max(ties, key=lambda e: e[0] * (e[0] - 1) // 2 + e[1])
            assert (u, v) == best
