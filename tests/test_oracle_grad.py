"""Pins of the FP64 reference gradient: the analytic formula against central
finite differences of the oracle's own loss (no gradient code involved in the
differences), and the closed form on the square of Fig 5.1."""
import numpy as np

import oracle
from oracle import grad as og


def test_square_closed_form():
    """Fig 5.1 square, one H1 bar [1, sqrt 2): loss = (sqrt2 - 1)^2; only the
    endpoints of the two critical edges get a gradient."""
    pts = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float64)
    pairs, edges = og.pairs_with_edges(oracle.distances_f64(pts), 4, 1)
    loss, g = og.loss_grad_h1(pts, pairs, edges)
    assert abs(loss - (np.sqrt(2) - 1) ** 2) < 1e-15
    h1 = [e for r, e in zip(pairs, edges) if r["dim"] == 1 and r["death"] > r["birth"]]
    assert len(h1) == 1
    touched = set(int(q) for q in h1[0])
    for i in range(4):
        if i not in touched:
            assert np.all(g[i] == 0)
    assert np.abs(g).sum() > 0


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    for trial in range(3):
        n = 14
        th = np.sort(rng.random(n)) * 2 * np.pi
        pts = np.stack([np.cos(th), np.sin(th)], 1) + 0.05 * rng.standard_normal((n, 2))
        pairs, edges = og.pairs_with_edges(oracle.distances_f64(pts), n, 1)
        _, g = og.loss_grad_h1(pts, pairs, edges)
        coords = [(i, k) for i in range(n) for k in range(2)]
        fd, skipped = og.central_differences(pts, coords, 1e-6)
        assert len(fd) >= len(coords) - 4
        for (i, k), v in fd.items():
            assert abs(v - g[i, k]) <= 1e-6 * max(1.0, np.abs(g).max()), (trial, i, k, v, g[i, k])
