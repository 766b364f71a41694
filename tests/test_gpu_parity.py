"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: bit-exact.  Distances use one fixed single-precision formula on both
sides, so every birth and death is a distance-matrix entry and every pair
(birth, death, birth simplex, death simplex) must match exactly.
"""
import json
import math
import os
import struct
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2502_05063_b300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def vr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2502_05063_b300 import vr as _vr
    return _vr


def rows_gpu(bc, p):
    a = bc.pairs[p]
    return [(float(r["birth"]), float(r["death"]), int(r["birth_simplex"]), int(r["death_simplex"])) for r in a]


def rows_oracle(dg_p):
    return [(float(np.float32(r["birth"])), float(np.float32(r["death"])) if np.isfinite(r["death"]) else math.inf,
             int(r["birth_cidx"]), int(r["death_cidx"])) for r in dg_p]


def oracle_diagram(D32, n, dmax, thr, keep_zero=False):
    D = D32.astype(np.float64)
    t = oracle.enclosing_radius(D, n) if not np.isfinite(thr) else float(np.float32(thr))
    pairs, stats = oracle.cohom(D, n, dmax, t, clearing=True)
    return oracle.diagram(pairs, dmax, keep_zero=keep_zero), stats, t


def assert_same(bc, dg, dmax, ctx=""):
    for p in range(dmax + 1):
        g, o = rows_gpu(bc, p), rows_oracle(dg[p])
        assert g == o, "dim %d differs %s: gpu %d rows, oracle %d rows; first diff %s" % (
            p, ctx, len(g), len(o), next(((a, b) for a, b in zip(g, o) if a != b), None))


# --------------------------------------------------------------------------
# distances and sort
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,dim", [(2, 1), (17, 3), (64, 3), (300, 4), (129, 7)])
def test_distances_bit_exact(vr, n, dim):
    import torch
    rng = np.random.default_rng(n * 10 + dim)
    pts = (rng.standard_normal((n, dim)) * rng.uniform(0.1, 100)).astype(np.float32)
    want = oracle.distances_f32(pts)
    x = torch.from_numpy(pts).cuda()
    out = torch.zeros(n * (n - 1) // 2, dtype=torch.float32, device="cuda")
    vr.distances(x, out)
    got = out.cpu().numpy()
    assert got.view(np.uint32).tolist() == want.view(np.uint32).tolist()


@pytest.mark.parametrize("num,bits", [(0, 64), (1, 64), (4095, 20), (4097, 33), (100000, 57), (12345, 64)])
def test_radix_sort_matches_numpy(vr, num, bits):
    import torch
    rng = np.random.default_rng(num + bits)
    keys = rng.integers(0, 2 ** 63, size=num, dtype=np.int64).astype(np.uint64)
    if bits < 64:
        keys &= np.uint64((1 << bits) - 1)
    keys[: num // 3] = keys[num // 3: 2 * (num // 3)] if num >= 3 else keys[: num // 3]  # duplicates
    vals = np.arange(num, dtype=np.uint64)
    kd = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    vd = torch.from_numpy(vals.view(np.int64).copy()).cuda()
    vr.sort_u64(kd, vd, bits)
    order = np.argsort(keys, kind="stable")
    assert kd.cpu().numpy().view(np.uint64).tolist() == keys[order].tolist()
    assert vd.cpu().numpy().view(np.uint64).tolist() == vals[order].tolist()


@pytest.mark.parametrize("num,bits", [(300, 20), (4096, 36), (9000, 40), (4097, 64), (32768, 30), (40000, 28)])
def test_radix_sort_ignores_bits_above(vr, num, bits):
    """Only the low `bits` bits order the keys (stably); the keys keep their high bits."""
    import torch
    rng = np.random.default_rng(7 * num + bits)
    keys = rng.integers(0, 2 ** 63, size=num, dtype=np.int64).astype(np.uint64)
    low = keys & np.uint64((1 << bits) - 1)
    low[: num // 4] = low[num // 4: 2 * (num // 4)]  # equal low parts, different high parts
    keys = (keys & ~np.uint64((1 << bits) - 1)) | low
    vals = np.arange(num, dtype=np.uint64)
    kd = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    vd = torch.from_numpy(vals.view(np.int64).copy()).cuda()
    vr.sort_u64(kd, vd, bits)
    order = np.argsort(low, kind="stable")
    assert kd.cpu().numpy().view(np.uint64).tolist() == keys[order].tolist()
    assert vd.cpu().numpy().view(np.uint64).tolist() == vals[order].tolist()


# --------------------------------------------------------------------------
# barcodes: random small clouds, all dimensions, exact
# --------------------------------------------------------------------------

def _cases():
    rng = np.random.default_rng(2024)
    out = []
    for it in range(40):
        n = int(rng.integers(1, 60))
        amb = int(rng.integers(1, 5))
        dmax = int(rng.integers(0, 4 if n <= 25 else 3))
        kind = it % 4
        out.append((it, n, amb, dmax, kind))
    return out


@pytest.mark.parametrize("it,n,amb,dmax,kind", _cases())
def test_random_clouds_exact(vr, it, n, amb, dmax, kind):
    rng = np.random.default_rng(1000 + it)
    if kind == 0:
        pts = rng.random((n, amb)).astype(np.float32)
    elif kind == 1:  # integer grid: many equal distances, duplicate points
        pts = rng.integers(0, 3, size=(n, amb)).astype(np.float32)
    elif kind == 2:
        pts = synth.circle(n, 1.0, 0.1, max(amb, 2), seed=it)
    else:
        pts = (rng.standard_normal((n, amb)) * 10).astype(np.float32)
    thr = np.inf if it % 3 else float(np.quantile(oracle.distances_f32(pts), 0.7)) if n > 1 else np.inf
    D32 = oracle.distances_f32(pts)
    dg, stats, t = oracle_diagram(D32, n, dmax, thr)
    bc = vr.barcodes(points=pts, dmax=dmax, threshold=thr)
    assert_same(bc, dg, dmax, "case %d" % it)
    for p in range(1, dmax + 1):
        assert bc.stats[p]["columns"] == stats[p][0]
        assert bc.stats[p]["essential"] == stats[p][3]
        assert bc.stats[p]["pairs"] == stats[p][2]
        if n <= 40:
            assert bc.stats[p]["apparent"] == len(oracle.apparent(D32.astype(np.float64), n, p, t))


@pytest.mark.parametrize("it", range(12))
def test_tie_heavy_dists_exact(vr, it):
    """Integer-valued distance matrices (not metrics), heavy ties, keep zero-length pairs."""
    rng = np.random.default_rng(77 + it)
    n = int(rng.integers(3, 30))
    dmax = int(rng.integers(1, 3))
    D32 = rng.integers(1, 4 + it, size=n * (n - 1) // 2).astype(np.float32)
    dg, stats, t = oracle_diagram(D32, n, dmax, np.inf, keep_zero=True)
    bc = vr.barcodes(dists=D32, n=n, dmax=dmax, flags=vr.VR_KEEP_ZERO_LENGTH)
    assert_same(bc, dg, dmax, "ties %d" % it)


@pytest.mark.parametrize("n0,d", [(5, 1), (9, 1), (8, 2), (9, 3)])
def test_thm_5_4_2_all_equal(vr, n0, d):
    """Thm 5.4.2 / Fig 5.5: all diameters equal -> C(n0-1, d+1) apparent pairs."""
    D32 = np.ones(n0 * (n0 - 1) // 2, dtype=np.float32)
    bc = vr.barcodes(dists=D32, n=n0, dmax=d)
    # clearing removes the (d-1)-deaths; the apparent count is unchanged (Prop 5.3.9)
    assert bc.stats[d]["apparent"] == math.comb(n0 - 1, d + 1)


def test_fig_5_6_distinct_diameters(vr):
    # the figure is the full complex: a finite threshold above every distance
    # (no threshold would truncate at the enclosing radius, here 4)
    D32 = np.array([10, 9, 8, 7, 6, 5, 4, 3, 2, 1], dtype=np.float32)
    bc = vr.barcodes(dists=D32, n=5, dmax=1, threshold=100.0)
    assert bc.stats[1]["apparent"] == 6


def test_square_fig_5_1(vr):
    pts = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], dtype=np.float32)
    bc = vr.barcodes(points=pts, dmax=1)
    assert [(float(r["birth"]), float(r["death"])) for r in bc.pairs[1]] == [(1.0, float(np.sqrt(np.float32(2))))]


def test_critical_edges(vr):
    rng = np.random.default_rng(5)
    pts = rng.integers(0, 4, size=(30, 2)).astype(np.float32)
    n = 30
    D = oracle.distances_f32(pts).astype(np.float64)
    bc = vr.barcodes(points=pts, dmax=2, flags=vr.VR_CRITICAL_EDGES | vr.VR_KEEP_ZERO_LENGTH)
    for p in range(3):
        for r, e in zip(bc.pairs[p], bc.critical_edges[p]):
            if p > 0:
                assert tuple(e[:2]) == oracle.critical_edge(D, n, int(r["birth_simplex"]), p)
            else:
                assert tuple(e[:2]) == (-1, -1)
            if r["death_simplex"] >= 0:
                assert tuple(e[2:]) == oracle.critical_edge(D, n, int(r["death_simplex"]), p + 1)
            else:
                assert tuple(e[2:]) == (-1, -1)


def test_edge_cases(vr):
    one = np.zeros((1, 3), np.float32)
    bc = vr.barcodes(points=one, dmax=2)
    assert len(bc.pairs[0]) == 1 and math.isinf(bc.pairs[0][0]["death"])
    two = np.array([[0, 0], [3, 4]], np.float32)
    bc = vr.barcodes(points=two, dmax=1)
    assert [(float(r["birth"]), float(r["death"])) for r in bc.pairs[0]] == [(0.0, 5.0), (0.0, math.inf)]
    assert len(bc.pairs[1]) == 0
    bc = vr.barcodes(points=two, dmax=1, threshold=-1.0)
    assert all(len(a) == 0 for a in bc.pairs)
    dup = np.zeros((6, 2), np.float32)  # all points equal: one essential H0 class, nothing else
    bc = vr.barcodes(points=dup, dmax=2)
    assert len(bc.pairs[0]) == 1 and len(bc.pairs[1]) == 0 and len(bc.pairs[2]) == 0
    with pytest.raises(vr.VRError) as e:
        vr.barcodes(dists=np.array([1.0, np.nan, 2.0], np.float32), n=3, dmax=1)
    assert e.value.name == "VR_ERR_INVALID_ARG"
    with pytest.raises(vr.VRError):
        vr.barcodes(dists=np.array([1.0, -2.0, 2.0], np.float32), n=3, dmax=1)
    with pytest.raises(vr.VRError):
        vr.barcodes(points=two, dmax=7)


def test_device_input_matches_host_input(vr):
    import torch
    pts = synth.uniform_cube(80, 3, seed=9)
    a = vr.barcodes(points=pts, dmax=2)
    b = vr.barcodes(points=torch.from_numpy(pts).cuda(), dmax=2)
    for p in range(3):
        assert rows_gpu(a, p) == rows_gpu(b, p)


def test_repeatable(vr):
    pts = synth.torus(150, seed=3)
    first = vr.barcodes(points=pts, dmax=2)
    for _ in range(3):
        again = vr.barcodes(points=pts, dmax=2)
        for p in range(3):
            assert rows_gpu(first, p) == rows_gpu(again, p)
            counts = lambda st: {k: v for k, v in st.items() if not k.startswith("ms_")}
            assert counts(first.stats[p]) == counts(again.stats[p])


# --------------------------------------------------------------------------
# full-size workloads against stored oracle output
# --------------------------------------------------------------------------

def load_golden(name):
    g = json.load(open(os.path.join(GOLDEN, name + ".json")))
    pts = np.frombuffer(bytes.fromhex(g["points_f32_hex"]), dtype="<f4").reshape(g["n"], g["ambient"]).copy()
    thr = math.inf if g["threshold"] == "inf" else struct.unpack("<f", bytes.fromhex(g["threshold"]))[0]

    def f(h):
        return math.inf if h == "inf" else struct.unpack("<f", bytes.fromhex(h))[0]

    dg = {int(p): [(f(r[0]), f(r[1]), int(r[2]), int(r[3])) for r in rows] for p, rows in g["diagram"].items()}
    return g, pts, thr, dg


@pytest.mark.parametrize("name", ["uniform64", "sphere200", "torus500"])
def test_workload_golden(vr, name):
    g, pts, thr, dg = load_golden(name)
    bc = vr.barcodes(points=pts, dmax=g["dmax"], threshold=thr)
    assert struct.pack("<f", bc.threshold).hex() == g["threshold_used"]
    for p in range(g["dmax"] + 1):
        assert rows_gpu(bc, p) == dg[p], "dim %d" % p
        if p >= 1:
            assert bc.stats[p]["columns"] == g["columns"][p]
            assert bc.stats[p]["apparent"] == g["apparent"][p]
            assert bc.stats[p]["pairs"] == g["pairs"][p]
            assert bc.stats[p]["essential"] == g["essential"][p]


@pytest.mark.parametrize("arena_log2", [16, 21])
def test_back_buffer_regrowth_matches_golden(vr, arena_log2):
    """Columns whose back buffers overflow restart with more room; the pairing is unchanged.

    With a 2^16- or 2^21-row arena for the block engine's back buffers (64K
    rows per column) the long cocycle columns of torus500 (several 100K rows)
    overflow again and again; each overflow of the first unfinished column,
    in any round of a batch, must enlarge the buffers, and columns finished
    before a regrowth keep their reduced forms for the columns they own
    pivots of.  Runs in a child process, which reads the arena size from its
    environment.
    """
    here = os.path.dirname(os.path.abspath(__file__))
    script = (
        "import sys\n"
        "sys.path[:0] = [%r, %r]\n"
        "from test_gpu_parity import load_golden, rows_gpu\n"
        "from paper_2502_05063_b300 import vr\n"
        "g, pts, thr, dg = load_golden('torus500')\n"
        "bc = vr.barcodes(points=pts, dmax=g['dmax'], threshold=thr)\n"
        "bad = [p for p in range(g['dmax'] + 1) if rows_gpu(bc, p) != dg[p]]\n"
        "print('MISMATCH' if bad else 'OK', bad)\n" % (os.path.dirname(here), here))
    env = dict(os.environ, VR_HEAVY_ARENA_LOG2=str(arena_log2))
    out = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    assert out.stdout.strip().startswith("OK"), out.stdout
