"""The batched form (one persistent launch over many clouds) against the
single-cloud path and against the oracle.  Bit-exact, like every parity test."""
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


def rows(a):
    return [(float(r["birth"]), float(r["death"]), int(r["birth_simplex"]), int(r["death_simplex"])) for r in a]


def mixed_clouds(num, seed, nmax=256):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(num):
        n = int(rng.integers(1, nmax + 1)) if i % 5 else int(rng.integers(1, 6))
        kind = i % 4
        if kind == 0:
            x = synth.circle(n, float(rng.uniform(0.5, 2)), 0.05, 3, g=rng)
        elif kind == 1:
            x = synth.sphere(n, 3, float(rng.uniform(0.5, 2)), 0.05, g=rng)
        elif kind == 2:
            x = rng.random((n, 3)).astype(np.float32)
        else:
            x = rng.integers(0, 3, size=(n, 3)).astype(np.float32)  # ties and duplicates
        out.append(x)
    return out


@pytest.mark.parametrize("dmax,thr,flags", [(1, np.inf, 0), (1, 0.8, 2), (0, np.inf, 0)])
def test_batched_equals_single(vr, dmax, thr, flags):
    clouds = mixed_clouds(60, seed=dmax * 10 + int(np.isfinite(thr)))
    pts, offs = synth.pack(clouds)
    bb = vr.barcodes_batched(pts, offs, dmax=dmax, threshold=thr, flags=flags)
    assert bb.recomputed == 0
    for i, c in enumerate(clouds):
        single = vr.barcodes(points=c, dmax=dmax, threshold=thr, flags=flags)
        for p in range(dmax + 1):
            assert rows(bb.cloud(i, p)) == rows(single.pairs[p]), (i, p)
            if flags & vr.VR_CRITICAL_EDGES:
                e = bb.critical_edges[p][bb.offsets[p][i]:bb.offsets[p][i + 1]]
                local = np.where(e >= 0, e - offs[i], -1)  # batched edges index the packed array
                assert local.tolist() == single.critical_edges[p].tolist(), (i, p)
        assert bb.thresholds[i] == np.float32(single.threshold)


def test_batch4096_workload(vr):
    """The full 4096-cloud workload: every cloud equals the single-cloud path,
    and every 8th cloud (512 clouds, all three kinds, sizes 32..256) equals the
    oracle, which runs one cloud per process on the host cores."""
    import torch
    from oracle import pool
    clouds, kinds = synth.batch_clouds()
    pts, offs = synth.pack(clouds)
    bb = vr.barcodes_batched(torch.from_numpy(pts).cuda(), offs, dmax=1)
    assert bb.recomputed == 0  # every cloud came from the persistent launch itself
    sample = list(range(0, len(clouds), 8))
    dgs = pool.diagrams([clouds[i] for i in sample], 1)
    for i, dg in zip(sample, dgs):
        for p in range(2):
            want = [(float(np.float32(r["birth"])), float(np.float32(r["death"])) if np.isfinite(r["death"]) else math.inf,
                     int(r["birth_cidx"]), int(r["death_cidx"])) for r in dg[p]]
            assert rows(bb.cloud(i, p)) == want, (i, p, kinds[i])
    for i in range(len(clouds)):
        single = vr.barcodes(points=clouds[i], dmax=1)
        for p in range(2):
            assert rows(bb.cloud(i, p)) == rows(single.pairs[p]), (i, p)
        assert bb.thresholds[i] == np.float32(single.threshold), i


def test_batched_repeat_and_shapes(vr):
    clouds = mixed_clouds(10, seed=5)
    pts, offs = synth.pack(clouds)
    a = vr.barcodes_batched(pts, offs, dmax=1)
    b = vr.barcodes_batched(pts, offs, dmax=1)  # graph replay
    for p in range(2):
        assert rows(a.pairs[p]) == rows(b.pairs[p])
    c = vr.barcodes_batched(pts[: offs[3]], offs[:4], dmax=1)  # another shape
    for i in range(3):
        for p in range(2):
            assert rows(c.cloud(i, p)) == rows(a.cloud(i, p))
    with pytest.raises(vr.VRError):
        big = np.zeros((300, 3), np.float32)
        vr.barcodes_batched(big, np.array([0, 300]), dmax=1)


@pytest.mark.parametrize("n", [100, 150, 256])
def test_lattice_ties(vr, n):
    """Points of a 3x3x3 grid: few distinct distances, so most diameter
    buckets hold many edges and the edge keys crowd a few distance ranges;
    one size per storage variant of the dimension-1 engine (everything in
    shared memory up to 128 points, the ranks up to 172, neither above)."""
    rng = np.random.default_rng(n)
    clouds = [rng.integers(0, 3, size=(n, 3)).astype(np.float32) for _ in range(3)]
    pts, offs = synth.pack(clouds)
    bb = vr.barcodes_batched(pts, offs, dmax=1)
    assert bb.recomputed == 0
    for i, c in enumerate(clouds):
        single = vr.barcodes(points=c, dmax=1)
        for p in range(2):
            assert rows(bb.cloud(i, p)) == rows(single.pairs[p]), (i, p)


def test_sizes_where_the_kernel_switches_storage(vr):
    """Clouds at each size where the batched kernel changes where it keeps
    data: the dimension-1 engine's bitmap and bucket starts leave shared
    memory above 128 points and its ranks above 172; steps 1-3 keep the
    distances in shared memory up to 197 points.  A noisy circle (one long
    cocycle column) and a uniform cube at each size, one batch; every cloud
    equals the single-cloud path, and the circles at the four outer sizes
    equal the oracle."""
    sizes = [128, 129, 172, 173, 197, 198, 255, 256]
    rng = np.random.default_rng(2025)
    clouds = []
    for n in sizes:
        clouds.append(synth.circle(n, 1.0, 0.1, 3, g=rng).astype(np.float32))
        clouds.append(rng.random((n, 3)).astype(np.float32))
    pts, offs = synth.pack(clouds)
    bb = vr.barcodes_batched(pts, offs, dmax=1)
    assert bb.recomputed == 0
    for i, c in enumerate(clouds):
        single = vr.barcodes(points=c, dmax=1)
        for p in range(2):
            assert rows(bb.cloud(i, p)) == rows(single.pairs[p]), (i, len(c), p)
    from oracle import pool
    sample = [0, 2, 12, 14]
    for i, dg in zip(sample, pool.diagrams([clouds[i] for i in sample], 1)):
        for p in range(2):
            want = [(float(np.float32(r["birth"])), float(np.float32(r["death"])) if np.isfinite(r["death"]) else math.inf,
                     int(r["birth_cidx"]), int(r["death_cidx"])) for r in dg[p]]
            assert rows(bb.cloud(i, p)) == want, (i, p)


def test_recompute_when_generators_overflow(vr, monkeypatch):
    """With the per-cloud store of generators cut to 8 entries (read when a
    plan is built; this shape is used by no other test, so the plan is new),
    the long cocycle column of each circle outgrows it: those clouds are
    handed to the single-cloud path, and every cloud still equals it."""
    monkeypatch.setenv("VR_BATCH_POOL_CAP", "8")
    circ = synth.circles(num=24, n=100, seed=9)
    pts, offs = synth.pack(circ)
    bb = vr.barcodes_batched(pts, offs, dmax=1)
    assert bb.recomputed > 0
    for i, c in enumerate(circ):
        single = vr.barcodes(points=c, dmax=1)
        for p in range(2):
            assert rows(bb.cloud(i, p)) == rows(single.pairs[p]), (i, p)


def test_circles_need_no_recompute(vr):
    """The 256 noisy circles of the differentiable workload: the persistent
    launch computes every cloud itself (none is handed to the single-cloud
    path), and each equals the single-cloud path."""
    circ = synth.circles()
    pts, offs = synth.pack(circ)
    bb = vr.barcodes_batched(pts, offs, dmax=1)
    assert bb.recomputed == 0
    for i in range(0, len(circ), 5):
        single = vr.barcodes(points=circ[i], dmax=1)
        for p in range(2):
            assert rows(bb.cloud(i, p)) == rows(single.pairs[p]), (i, p)


def test_batched_output_larger_than_planned(vr):
    """More H1 pairs than the first call's estimate for the shape (64 per cloud
    plus 1024): the host grows the output buffers and reruns, and no pair lands
    outside them meanwhile.  Every fourth cloud equals the single-cloud path,
    and the pair counts of all clouds match it."""
    rng = np.random.default_rng(77)
    clouds = [rng.random((256, 3)).astype(np.float32) for _ in range(64)]
    clouds[5] = clouds[5][:255]  # a total no other test uses: a fresh plan
    pts, offs = synth.pack(clouds)
    bb = vr.barcodes_batched(pts, offs, dmax=1)
    counts = [len(rows(bb.cloud(i, 1))) for i in range(len(clouds))]
    assert sum(counts) > 64 * len(clouds) + 1024  # the case this test is for
    for i in range(len(clouds)):
        single = vr.barcodes(points=clouds[i], dmax=1)
        assert counts[i] == len(single.pairs[1]), i
        if i % 4 == 0:
            for p in range(2):
                assert rows(bb.cloud(i, p)) == rows(single.pairs[p]), (i, p)


def test_batched_device_on_a_side_stream(vr):
    """The device-resident batched result on a stream other than torch's
    current one: the call returns without waiting for its copies, and the
    binding makes the current stream wait before reading them; the values and
    critical edges equal the host result's."""
    import torch
    circ = synth.circles(num=16, n=64, seed=11)
    pts, offs = synth.pack(circ)
    want = vr.barcodes_batched(pts, offs, dmax=1, flags=vr.VR_CRITICAL_EDGES)
    x = torch.from_numpy(pts).cuda()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    got = vr.barcodes_batched_device(x, offs, dmax=1, flags=vr.VR_CRITICAL_EDGES, stream=side)
    for p in range(2):
        v = got.values[p].cpu().numpy()
        assert np.array_equal(v[:, 0], want.pairs[p]["birth"]), p
        assert np.array_equal(v[:, 1], want.pairs[p]["death"]), p
        assert np.array_equal(got.edges[p].cpu().numpy(), want.critical_edges[p]), p
        assert np.array_equal(got.offsets[p], want.offsets[p]), p
