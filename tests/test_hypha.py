"""HYPHA on explicit boundary matrices (Ch. 4, Algorithm 10: GPU scan,
clearing, compression, then the standard reduction of what remains) against
the oracle's Algorithm 2 on the same matrix: the pivot row of every column,
exactly.  Inputs: the worked example of Fig 4.1, lower-star filtrations of
triangulated grids with random vertex values, and Vietoris-Rips filtrations
listed explicitly."""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2502_05063_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def csc_columns(colptr, rows):
    return [rows[colptr[j]:colptr[j + 1]].tolist() for j in range(len(colptr) - 1)]


def rips_boundary(n, dim_top, seed):
    """Explicit boundary matrix of the Rips filtration of n random points, all
    simplices up to dimension dim_top, ordered by (diameter, dimension, vertex
    tuple); CSC with rows ascending."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    S = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    if seed % 2:
        S = np.round(S * 4) / 4  # ties
    simp = []
    for k in range(dim_top + 1):
        for s in itertools.combinations(range(n), k + 1):
            d = max((S[a, b] for a, b in itertools.combinations(s, 2)), default=0.0)
            simp.append((d, k, s))
    simp.sort()
    pos = {s: i for i, (_, _, s) in enumerate(simp)}
    cols = []
    for _, k, s in simp:
        cols.append(sorted(pos[f] for f in itertools.combinations(s, k)) if k > 0 else [])
    colptr = np.zeros(len(cols) + 1, np.int64)
    colptr[1:] = np.cumsum([len(c) for c in cols])
    rows = np.array([r for c in cols for r in c], dtype=np.int32)
    return colptr, rows, np.array([k for _, k, _ in simp])


def fig41():
    cols = {}
    for line in open(os.path.join(GOLDEN, "fig_4_1_boundary.txt")):
        line = line.split("#")[0].strip()
        if line and not line.startswith("lows"):
            key, _, rest = line.partition(":")
            cols[int(key)] = [int(x) for x in rest.split()]
    cols = [sorted(cols[j]) for j in range(len(cols))]
    colptr = np.zeros(len(cols) + 1, np.int64)
    colptr[1:] = np.cumsum([len(c) for c in cols])
    return colptr, np.array([r for c in cols for r in c], dtype=np.int32)


# --------------------------------------------------------------------------
# CPU: the workloads are boundary matrices, and the oracle's pins on them
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m", [2, 5, 17])
def test_lower_star_grid_is_a_boundary_matrix(m):
    colptr, rows, dims = synth.lower_star_grid(m, seed=m)
    N = len(colptr) - 1
    assert N == m * m + 3 * m * m - 4 * m + 1 + 2 * (m - 1) ** 2
    for j in range(N):
        r = rows[colptr[j]:colptr[j + 1]]
        assert np.all(r < j) and np.all(np.diff(r) > 0) and len(r) == (dims[j] + 1 if dims[j] > 0 else 0)
        if dims[j] == 2:  # the boundary of a boundary vanishes over Z/2
            acc = {}
            for e in r:
                for v in rows[colptr[e]:colptr[e + 1]]:
                    acc[v] = acc.get(v, 0) ^ 1
            assert not any(acc.values())


def test_oracle_on_a_grid_has_the_homology_of_a_disc():
    """The triangulated square is contractible: one essential class, in
    dimension 0 (a closed form for the oracle's Algorithm 2 on this input)."""
    colptr, rows, dims = synth.lower_star_grid(12, seed=3)
    low = oracle.reduce_explicit(csc_columns(colptr, rows))
    lows = set(int(x) for x in low if x >= 0)
    essential = [int(dims[j]) for j in range(len(low)) if low[j] < 0 and j not in lows]
    assert essential == [0]


# --------------------------------------------------------------------------
# GPU
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def vr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2502_05063_b300 import vr as _vr
    return _vr


@pytest.mark.gpu
def test_hypha_fig_4_1(vr):
    colptr, rows = fig41()
    low, st = vr.hypha_pairs(colptr, rows)
    assert low.tolist() == oracle.reduce_explicit(csc_columns(colptr, rows)).tolist()
    assert sorted((int(l), j) for j, l in enumerate(low) if l >= 0) == [(1, 4), (2, 3), (5, 6)]


@pytest.mark.gpu
@pytest.mark.parametrize("m,seed", [(2, 1), (3, 2), (10, 3), (40, 4), (100, 5), (160, 6)])
def test_hypha_lower_star_grids(vr, m, seed):
    import torch
    colptr, rows, _ = synth.lower_star_grid(m, seed=seed)
    want = oracle.reduce_explicit(csc_columns(colptr, rows))
    low, st = vr.hypha_pairs(colptr, rows)
    assert low.tolist() == want.tolist()
    # device-resident input gives the same
    low_d, _ = vr.hypha_pairs(torch.from_numpy(colptr).cuda(), torch.from_numpy(rows).cuda())
    assert low_d.tolist() == want.tolist()
    assert st["columns"] == len(colptr) - 1 and 0 <= st["unstable"] <= st["columns"]


@pytest.mark.gpu
@pytest.mark.parametrize("n,top,seed", [(8, 3, 0), (12, 2, 1), (14, 3, 2), (18, 2, 3), (25, 2, 5)])
def test_hypha_rips_boundary(vr, n, top, seed):
    colptr, rows, _ = rips_boundary(n, top, seed)
    want = oracle.reduce_explicit(csc_columns(colptr, rows))
    low, st = vr.hypha_pairs(colptr, rows)
    assert low.tolist() == want.tolist()


@pytest.mark.gpu
def test_hypha_rejects_malformed(vr):
    colptr = np.array([0, 0, 1], np.int64)
    rows = np.array([1], np.int32)  # column 1 with row 1: not below the column
    with pytest.raises(vr.VRError) as e:
        vr.hypha_pairs(colptr, rows)
    assert e.value.name == "VR_ERR_INVALID_ARG"
    colptr = np.array([0, 0, 0, 2], np.int64)
    rows = np.array([1, 0], np.int32)  # rows not ascending
    with pytest.raises(vr.VRError):
        vr.hypha_pairs(colptr, rows)


@pytest.mark.gpu
@pytest.mark.parametrize("shared_rows", [1, 4, 64])
def test_hypha_global_working_buffers(vr, shared_rows, monkeypatch):
    """The final phase keeps the working column in shared memory while it fits
    (4096 rows) and moves to global buffers past that; lowering the limit
    (read on each call) sends the same reductions through the global path."""
    monkeypatch.setenv("VR_HYPHA_SHARED_ROWS", str(shared_rows))
    for m, seed in [(10, 3), (40, 4)]:
        colptr, rows, _ = synth.lower_star_grid(m, seed=seed)
        low, _ = vr.hypha_pairs(colptr, rows)
        assert low.tolist() == oracle.reduce_explicit(csc_columns(colptr, rows)).tolist()
    for n, top, seed in [(14, 3, 2), (25, 2, 5)]:
        colptr, rows, _ = rips_boundary(n, top, seed)
        low, _ = vr.hypha_pairs(colptr, rows)
        assert low.tolist() == oracle.reduce_explicit(csc_columns(colptr, rows)).tolist()
