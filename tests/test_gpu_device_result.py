"""The device-resident entry points (vr_barcodes_points_device,
vr_barcodes_dists_device, vr_barcodes_batched_device) return exactly the
pairs, order and critical edges of the host-result entry points, with the
pairs ordered and filtered on the GPU."""
import math

import numpy as np
import pytest

from paper_2502_05063_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2502_05063_b300 import vr as _vr
    return _vr


def _host_rows(bc, p):
    a = bc.pairs[p]
    return [(float(r["birth"]), float(r["death"]), int(r["birth_simplex"]), int(r["death_simplex"])) for r in a]


def _dev_rows(db, p):
    v = db.values[p].cpu().numpy()
    sm = db.simplices[p].cpu().numpy()
    return [(float(v[k, 0]), float(v[k, 1]), int(np.uint64(sm[k, 0])), int(sm[k, 1])) for k in range(len(v))]


@pytest.mark.parametrize("case", range(8))
def test_device_result_equals_host_result(vr, case):
    import torch
    rng = np.random.default_rng(500 + case)
    n = [1, 2, 17, 60, 120, 200, 45, 90][case]
    amb = 3 if case % 2 else 2
    pts = rng.random((n, amb)).astype(np.float32)
    if case == 6:
        pts = np.round(pts * 3).astype(np.float32)  # ties and duplicate points
    dmax = 2 if n <= 120 else 1
    flags = [0, vr.VR_CRITICAL_EDGES, vr.VR_KEEP_ZERO_LENGTH | vr.VR_CRITICAL_EDGES, vr.VR_APPARENT_ONLY][case % 4]
    thr = [math.inf, 0.4, math.inf, 0.7][case % 4]
    x = torch.from_numpy(pts).cuda()
    h = vr.barcodes(points=x, dmax=dmax, threshold=thr, flags=flags)
    d = vr.barcodes_device(points=x, dmax=dmax, threshold=thr, flags=flags)
    assert d.threshold == h.threshold
    for p in range(dmax + 1):
        assert d.counts[p] == len(h.pairs[p])
        assert _dev_rows(d, p) == _host_rows(h, p), p
        if flags & vr.VR_CRITICAL_EDGES:
            assert d.edges[p].cpu().numpy().tolist() == h.critical_edges[p].tolist()
        else:
            assert d.edges[p] is None
        for k in ("columns", "apparent", "reduced", "additions", "pairs", "essential", "emitted"):
            assert d.stats[p][k] == h.stats[p][k], (p, k)


def test_device_result_dists_and_workload(vr):
    import torch
    w = synth.WORKLOADS["sphere200"]
    pts = w["make"]()
    h = vr.barcodes(points=pts, dmax=w["dmax"], threshold=w["threshold"], flags=vr.VR_CRITICAL_EDGES)
    d = vr.barcodes_device(points=torch.from_numpy(pts).cuda(), dmax=w["dmax"], threshold=w["threshold"],
                           flags=vr.VR_CRITICAL_EDGES)
    for p in range(w["dmax"] + 1):
        assert _dev_rows(d, p) == _host_rows(h, p)
        assert d.edges[p].cpu().numpy().tolist() == h.critical_edges[p].tolist()
    D = synth.random_permutation_dists(40)
    h = vr.barcodes(dists=D, n=40, dmax=1, threshold=float(D.max()))
    d = vr.barcodes_device(dists=torch.from_numpy(D).cuda(), n=40, dmax=1, threshold=float(D.max()))
    for p in range(2):
        assert _dev_rows(d, p) == _host_rows(h, p)


@pytest.mark.parametrize("flags", [0, 2])
def test_batched_device_equals_batched_host(vr, flags):
    import torch
    clouds, _ = synth.batch_clouds(num=300, seed=11)
    pts, offs = synth.pack(clouds)
    x = torch.from_numpy(pts).cuda()
    h = vr.barcodes_batched(x, offs, dmax=1, flags=flags)
    d = vr.barcodes_batched_device(x, offs, dmax=1, flags=flags)
    assert np.array_equal(d.thresholds, h.thresholds)
    for p in range(2):
        assert np.array_equal(d.offsets[p], h.offsets[p])
        v = d.values[p].cpu().numpy()
        assert np.array_equal(v[:, 0], h.pairs[p]["birth"]) and np.array_equal(v[:, 1], h.pairs[p]["death"])
        if flags:
            assert d.edges[p].cpu().numpy().tolist() == h.critical_edges[p].tolist()
