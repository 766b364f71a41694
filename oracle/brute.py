"""Brute-force persistence by Z/2 ranks (TEST INFRASTRUCTURE ONLY).

An independent route to the barcode that uses no matrix reduction at all:
persistent Betti numbers beta_p^{a,c} = dim Z_p(K_a) - dim(B_p(K_c) cap Z_p(K_a))
of the filtration K_a = Rips_{v_a} (eq. 5.3) at its distinct values v_a, from
which the number of bars [v_a, v_c) follows by inclusion-exclusion; a bar is
an interval summand of the persistence module (Gabriel's theorem, eq. 3.70;
Thm 3.2.20 ties the pivots of Algorithm 2 to these summands).

dim(B_p(K_c) cap C_p(K_a)) = rank(M) - rank(M restricted to the rows not in
K_a), where M is the boundary matrix of the (p+1)-simplices of K_c; this
intersection already lies in Z_p(K_a) because boundaries are cycles.

Pure Python on bitsets; meant for n <= 10.
"""
from __future__ import annotations

import itertools
import math


def _rank(cols):
    """Z/2 rank of a list of column bitsets (Python ints)."""
    basis = {}  # leading bit -> vector
    r = 0
    for v in cols:
        while v:
            h = v.bit_length() - 1
            if h in basis:
                v ^= basis[h]
            else:
                basis[h] = v
                r += 1
                break
    return r


def barcode(D, n, dmax, threshold=math.inf):
    """Multiset {(p, birth, death)} of bars with death > birth, death=inf for
    essential classes, for p = 0..dmax.  D(i, j) is a callable or a square
    nested list / array."""
    dist = D if callable(D) else (lambda i, j: D[i][j])
    simp = {q: [] for q in range(dmax + 2)}
    for q in range(dmax + 2):
        for s in itertools.combinations(range(n), q + 1):
            d = max((dist(a, b) for a, b in itertools.combinations(s, 2)), default=0.0)
            if d <= threshold:
                simp[q].append((s, d))
    values = sorted({d for q in simp for _, d in simp[q]})
    m = len(values)
    index = {q: {s: i for i, (s, _) in enumerate(simp[q])} for q in simp}

    def boundary_cols(q, vmax):
        """columns (bitsets over index[q-1]) of q-simplices with diam <= vmax."""
        out = []
        for s, d in simp[q]:
            if d <= vmax:
                b = 0
                for k in range(len(s)):
                    b |= 1 << index[q - 1][s[:k] + s[k + 1:]]
                out.append(b)
        return out

    def mask_rows(q, vmax):
        """bitset of the q-simplices with diam <= vmax."""
        b = 0
        for i, (s, d) in enumerate(simp[q]):
            if d <= vmax:
                b |= 1 << i
        return b

    def z(p, a):
        n_p = sum(1 for _, d in simp[p] if d <= values[a])
        if p == 0:
            return n_p
        return n_p - _rank(boundary_cols(p, values[a]))

    beta = {}
    for p in range(dmax + 1):
        for a in range(m):
            zp = z(p, a)
            inside = mask_rows(p, values[a])
            for c in range(a, m):
                M = boundary_cols(p + 1, values[c])
                outside = [col & ~inside for col in M]
                beta[p, a, c] = zp - (_rank(M) - _rank(outside))

    def B(p, a, c):
        if a < 0:
            return 0
        return beta[p, a, c]

    bars = []
    for p in range(dmax + 1):
        for a in range(m):
            for c in range(a + 1, m):
                mu = B(p, a, c - 1) - B(p, a, c) - B(p, a - 1, c - 1) + B(p, a - 1, c)
                bars += [(p, values[a], values[c])] * mu
            mu = B(p, a, m - 1) - B(p, a - 1, m - 1)
            bars += [(p, values[a], math.inf)] * mu
    return sorted(bars)
