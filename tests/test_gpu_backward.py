"""Gradient of sum over H1 pairs of (death - birth)^2 with respect to the point
coordinates: the CUDA backward (through torch.autograd) against the FP64
oracle gradient on the same pairing and against central finite differences,
relative error <= 1e-4 (max-norm)."""
import numpy as np
import pytest

import oracle
from oracle import grad as og
from paper_2502_05063_b300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def ag():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for the gpu tests")
    from paper_2502_05063_b300 import autograd
    return autograd


def h1_loss(out):
    import torch
    h1 = out[1]
    fin = torch.isfinite(h1[:, 1])
    return ((h1[fin, 1] - h1[fin, 0]) ** 2).sum()


def gpu_grad(ag, pts, recompute=False):
    import torch
    x = torch.from_numpy(pts).cuda().requires_grad_(True)
    loss = h1_loss(ag.VRDiagram.apply(x, 1, float("inf"), recompute))
    loss.backward()
    return float(loss.detach()), x.grad.cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_grad_vs_fp64_oracle_same_pairing(ag, i):
    pts = synth.circles(num=4)[i]                     # n=128 noisy circle in R^2, sigma 0.1
    loss, g = gpu_grad(ag, pts)
    pairs, edges = og.fp32_pairing(pts, 1)
    loss64, g64 = og.loss_grad_h1(pts.astype(np.float64), pairs, edges)
    assert abs(loss - loss64) <= TOL * max(loss64, 1e-12)
    assert rel(g, g64) <= TOL
    _, g_re = gpu_grad(ag, pts, recompute=True)
    assert rel(g_re, g64) <= TOL


def test_grad_vs_central_differences(ag):
    pts = synth.circles(num=1, n=40)[0]
    _, g = gpu_grad(ag, pts)
    rng = np.random.default_rng(0)
    pairs, edges = og.fp32_pairing(pts, 1)
    crit = sorted({int(q) for r, e in zip(pairs, edges) if r["dim"] == 1 for q in e if q >= 0})
    coords = [(v, k) for v in crit[:12] for k in range(2)] + [(int(rng.integers(0, 40)), int(rng.integers(0, 2))) for _ in range(8)]
    fd, skipped = og.central_differences(pts.astype(np.float64), coords, 1e-4)
    assert len(fd) >= len(coords) // 2, skipped
    scale = np.abs(g).max()
    for (v, k), d in fd.items():
        assert abs(g[v, k] - d) <= TOL * scale + 1e-6, (v, k, g[v, k], d)


def test_batched_grad(ag):
    """256 clouds of 128 points: one batched forward and one backward launch."""
    import torch
    clouds = synth.circles()
    pts, offs = synth.pack(clouds)
    x = torch.from_numpy(pts).cuda().requires_grad_(True)
    out = ag.VRDiagramBatched.apply(x, offs, 1)
    h1 = out[1]
    fin = torch.isfinite(h1[:, 1])
    loss = ((h1[fin, 1] - h1[fin, 0]) ** 2).sum()
    loss.backward()
    g = x.grad.cpu().numpy().astype(np.float64)
    for i in range(0, 256, 37):
        c = clouds[i]
        pairs, edges = og.fp32_pairing(c, 1)
        _, g64 = og.loss_grad_h1(c.astype(np.float64), pairs, edges)
        assert rel(g[offs[i]:offs[i + 1]], g64) <= TOL, i
