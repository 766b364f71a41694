#!/usr/bin/env python3
"""Benchmark of the Vietoris-Rips barcode hot path on B300.

One step = one call of the public C ABI (vr_barcodes_points) on the
500-point torus workload (n=500 on the torus R=2, r=1 in R^3 plus N(0,0.05^2)
noise, seed 1, H0-H2, no threshold, i.e. truncation at the enclosing
radius): distances, ranks, H0, and for p = 1, 2 the fused filtration /
clearing / apparent-pair kernel, the radix sort of the non-apparent columns
and their Z/2 reduction, then the result copy.

metric: filtration simplices per second, sum over p = 1..dmax of the
C(n, p+1) candidate p-simplices enumerated per step (20,833,250 for this
workload), divided by the whole step time.  `value` times steps on inputs
already resident on the device; `e2e` times the same call on pinned host
input, host-to-device copy and result copy inside the timed region.

Further keys: `roofline` -- the fused filtration/apparent kernel of the top
dimension, its algorithmic bytes per launch (per-unit figures of the
filtration and apparent steps, see roofline_bytes) over its CUDA-event time,
against the measured HBM copy bandwidth and a project-written L2 read probe;
`cpu_baseline` -- the oracle on a bounded sample of the same workload (the
same cloud, dimensions 0-1), single thread, median of 5; `batched` -- the
4096-cloud forward and the 256-circle forward+backward (median of 20 and the
spread), each against a per-cloud loop of the same library, with the oracle
on all host cores beside them (`cpu_baseline_batched`); `other_workloads` --
stage rates of the 64-point uniform and 200-point sphere workloads.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 (torchrun), single clouds do not shard: every rank runs a replica
and the value is the work of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "torus500"
METRIC = "simplices/sec filtration+apparent-pairs; batched VR fwd+bwd clouds/sec vs plain"
UNIT = "simplices/s"
L2_FLUSH_BYTES = 256 << 20
# The oracle's bounded sample of the benched workload: the same 500-point torus
# cloud (seed 1), dimensions 0-1 (the whole H0-H2 computation takes the oracle
# about two minutes).  Rate = dimension-1 candidates C(500, 2) per second.
CPU_SAMPLE_DMAX = 1
CPU_SAMPLE_REPEATS = 5


def candidates(n: int, dmax: int) -> int:
    return sum(math.comb(n, p + 1) for p in range(1, dmax + 1))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        """Start sampling every 50 ms; returns once the first sample is written
        (at most 5 s), so that the samples span the region timed next."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def count_launches(fn):
    """Kernels of libvrgpu launched by one call (CUPTI through torch.profiler)."""
    import torch
    from torch.profiler import ProfilerActivity, profile
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        fn()
        torch.cuda.synchronize()
    n = 0
    for ev in prof.events():
        if ev.device_type.name == "CUDA" and ("vr::" in ev.name or "k_" in ev.name):
            n += 1
    return n


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_sample_seconds(pts, dmax):
    """One run of the oracle as it stands (single thread, cohomology with
    clearing), distances and enclosing radius included, input generation not."""
    import numpy as np
    import oracle
    n = pts.shape[0]
    t0 = time.perf_counter()
    D = oracle.distances_f32(pts).astype(np.float64)
    R = oracle.enclosing_radius(D, n)
    oracle.cohom(D, n, dmax, R, clearing=True)
    return time.perf_counter() - t0


def cpu_baseline_single(repeats=CPU_SAMPLE_REPEATS):
    """Median of `repeats` oracle runs on the bounded sample, after one warm-up."""
    import oracle
    from paper_2502_05063_b300 import synth
    oracle.build()
    pts = synth.WORKLOADS[WORKLOAD]["make"]()
    n = pts.shape[0]
    oracle_sample_seconds(pts, CPU_SAMPLE_DMAX)
    times = [oracle_sample_seconds(pts, CPU_SAMPLE_DMAX) for _ in range(repeats)]
    med = statistics.median(times)
    return {"value": candidates(n, CPU_SAMPLE_DMAX) / med, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds_median": med, "seconds_all": times, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": "oracle (plain C, cohomology with clearing, single thread) on the benched 500-point torus "
                      "cloud (seed 1, enclosing radius), dimensions 0-1: C(500,2) = 124,750 candidate simplices "
                      "per run; median of %d runs after one warm-up" % repeats}


def cpu_baseline_batched():
    """The oracle on bounded samples of the two batched workloads, one cloud per
    process on all host cores (spawn-started pool, warmed before timing)."""
    from oracle import pool as opool
    from paper_2502_05063_b300 import synth
    procs = os.cpu_count() or 1
    clouds, _ = synth.batch_clouds()
    c4 = clouds[::32]
    circ = synth.circles()
    c5 = circ[::4]
    with opool.open_pool(procs) as pl:
        opool.diagrams(c4[:procs], 1, pool=pl)  # warm the workers (imports, library load)
        t0 = time.perf_counter()
        opool.diagrams(c4, 1, pool=pl)
        t4 = time.perf_counter() - t0
        t0 = time.perf_counter()
        opool.loss_grads(c5, 1, pl)
        t5 = time.perf_counter() - t0
    return {
        "batch4096_forward": {"clouds_per_s": len(c4) / t4, "cores": procs, "kind": "oracle", "seconds": t4,
                              "sample": "every 32nd cloud of the 4096-cloud workload (%d clouds), H0-H1, "
                                        "one cloud per process" % len(c4)},
        "circles256_fwd_bwd": {"clouds_per_s": len(c5) / t5, "cores": procs, "kind": "oracle", "seconds": t5,
                               "sample": "every 4th cloud of the 256-circle workload (%d clouds): pairing "
                                         "(cohomology) plus the FP64 gradient of sum over H1 of (death-birth)^2, "
                                         "one cloud per process" % len(c5)},
        "cpu_model": cpu_model(),
    }


def roofline_bytes(p, st):
    """Algorithmic bytes of one launch of the fused filtration/apparent kernel of
    dimension p, by the per-unit figures of the filtration and apparent steps:
      filtration (Alg 17/18): per candidate C(p+1,2) 4-byte diameter lookups and
        one clearing bit; per kept column an 8-byte key;
      apparent search (Lemma 5.3.6): per kept column an 8-byte key read, up to
        16 bytes of output and (p+2) C(p+1,2) 4-byte lookups for the facet test;
        per cofacet examined (p+1) 4-byte lookups."""
    cand, kept, cof = st["candidates"], st["columns"], st["cofacets_scanned"]
    pairs = (p + 1) * p // 2
    a3 = cand * pairs * 4 + cand / 8.0 + kept * 8
    a5 = kept * (8 + 16 + (p + 2) * pairs * 4) + cof * (p + 1) * 4
    return a3 + a5, {"filtration": a3, "apparent": a5}


def stage_rates_of(stats, dmax, stage):
    dims = range(1, dmax + 1)
    f_ms = sum(stage["dim%d" % p]["ms_filtration"] for p in dims)
    s_ms = sum(stage["dim%d" % p]["ms_sort"] for p in dims)
    return {
        "filtration_simplices_per_s": (sum(stats[p]["candidates"] for p in dims) / ((f_ms + s_ms) / 1e3)
                                       if f_ms + s_ms > 0 else None),
        "apparent_columns_per_s": sum(stats[p]["columns"] for p in dims) / (f_ms / 1e3) if f_ms > 0 else None,
        "cofacets_per_s": sum(stats[p]["cofacets_scanned"] for p in dims) / (f_ms / 1e3) if f_ms > 0 else None,
    }


def other_workload_rates(stream, reps=5):
    """M1/M2 stage rates of the 64-point uniform and 200-point sphere workloads
    (library stage timers, mean over `reps` calls after two warm-up calls)."""
    from paper_2502_05063_b300 import synth, vr
    import torch
    out = {}
    for name in ("uniform64", "sphere200"):
        w = synth.WORKLOADS[name]
        x = torch.from_numpy(w["make"]()).cuda()
        dmax = w["dmax"]
        for _ in range(2):
            vr.barcodes(points=x, dmax=dmax, threshold=w["threshold"], stream=stream)
        rs = [vr.barcodes(points=x, dmax=dmax, threshold=w["threshold"], stream=stream) for _ in range(reps)]
        stage = {"dim%d" % p: {k: statistics.mean(r.stats[p][k] for r in rs)
                               for k in ("ms_filtration", "ms_sort", "ms_reduce")} for p in range(dmax + 1)}
        rates = stage_rates_of(rs[-1].stats, dmax, stage)
        rates["stages_ms"] = {k: {kk: round(vv, 4) for kk, vv in v.items()} for k, v in stage.items()}
        rates["counts"] = {"dim%d" % p: {k: rs[-1].stats[p][k] for k in ("candidates", "columns", "apparent",
                                                                           "reduced", "additions", "cofacets_scanned")}
                           for p in range(1, dmax + 1)}
        rates["workload"] = w["desc"]
        out[name] = rates
    return out


def reduction_ablation(stream, reps=3):
    """Sec. 5.2.9 ablation: the reduction of the non-apparent columns with reduced
    columns kept explicitly (default), with only their generators kept
    (reduction-matrix technique, VR_REDUCE_V) and with nothing kept (oblivious,
    VR_REDUCE_OBLIVIOUS).  Per mode and dimension: column additions and the
    reduction's stage time (median of `reps` calls after one warm-up); the
    pairs are the same in every mode (tested)."""
    import numpy as np
    import torch
    from paper_2502_05063_b300 import synth, vr
    modes = {"explicit_default": 0, "v_matrix": vr.VR_REDUCE_V, "oblivious": vr.VR_REDUCE_OBLIVIOUS}
    cases = {"torus500": (torch.from_numpy(synth.WORKLOADS["torus500"]["make"]()).cuda(), None, 2, np.inf)}
    for n in (100,):
        D = synth.random_permutation_dists(n)
        cases["randperm%d" % n] = (None, torch.from_numpy(D).cuda(), 1, float(D.max()))
    out = {}
    for cname, (pts, dists, dmax, thr) in cases.items():
        res = {}
        for mname, fl in modes.items():
            def call():
                if pts is not None:
                    return vr.barcodes(points=pts, dmax=dmax, threshold=thr, flags=fl, stream=stream)
                return vr.barcodes(dists=dists, n=int(round((1 + (1 + 8 * dists.shape[0]) ** 0.5) / 2)), dmax=dmax,
                                   threshold=thr, flags=fl, stream=stream)
            try:
                call()
                runs = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = call()
                    e1.record(stream)
                    e1.synchronize()
                    runs.append((e0.elapsed_time(e1), r))
                runs.sort(key=lambda t: t[0])
                ms, r = runs[len(runs) // 2]
                res[mname] = {"call_ms": ms, "dims": {"dim%d" % p: {"additions": r.stats[p]["additions"],
                                                                    "reduced_columns": r.stats[p]["reduced"],
                                                                    "ms_reduce": r.stats[p]["ms_reduce"]}
                                                      for p in range(1, dmax + 1)}}
            except Exception as e:  # noqa: BLE001  (a mode that runs out of memory is a result)
                res[mname] = {"error": str(e)}
        out[cname] = res
    return out


def sparse_mode(stream, reps=3):
    """The sparse (low-threshold) mode against the dense enumeration on the same
    call: the O(3)-sample stand-in (n=4096 in R^9, threshold 1.4, 2.8% of the
    pairs, H0-H2) and the 500-point torus at the 10th percentile of its
    distances.  Median call time of `reps` calls (CUDA events, device-resident
    input) after one warm-up, and per dimension the listed simplices and the
    fused kernel's time."""
    import numpy as np
    import torch
    from paper_2502_05063_b300 import synth, vr
    out = {}
    tor = synth.WORKLOADS["torus500"]["make"]()
    dt = np.sort(np.linalg.norm(tor[:, None, :] - tor[None, :, :], axis=2)[np.tril_indices(500, -1)])
    cases = {"o3like4096": (synth.WORKLOADS["o3like4096"]["make"](), 2, 1.4),
             "torus500_q10": (tor, 2, float(dt[len(dt) // 10]))}
    for name, (pts, dmax, thr) in cases.items():
        x = torch.from_numpy(pts).cuda()
        res = {"n": int(pts.shape[0]), "dmax": dmax, "threshold": thr}
        for mode, fl in (("sparse", vr.VR_SPARSE), ("dense", 0)):
            try:
                vr.barcodes(points=x, dmax=dmax, threshold=thr, flags=fl, stream=stream)
                runs = []
                for _ in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    r = vr.barcodes(points=x, dmax=dmax, threshold=thr, flags=fl, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    runs.append((e0.elapsed_time(e1), r))
                runs.sort(key=lambda t: t[0])
                ms, r = runs[len(runs) // 2]
                res[mode] = {"call_ms": ms, "dims": {"dim%d" % p: {k: r.stats[p][k] for k in (
                    "candidates", "columns", "apparent", "reduced", "ms_filtration", "ms_reduce")}
                    for p in range(1, dmax + 1)}, "bars": [len(a) for a in r.pairs]}
            except Exception as e:  # noqa: BLE001
                res[mode] = {"error": str(e)}
        out[name] = res
    return out


def hypha_bench(stream, reps=5):
    """HYPHA (Ch. 4) on the explicit boundary matrix of the lower-star
    filtration of a 512 x 512 triangulated grid with random vertex values
    (1,568,771 columns, 3,135,496 entries), device-resident input: the whole
    call (median of `reps` after one warm-up), its phases (library stage
    timers) and the GPU scan's rate in columns and entries per second."""
    import torch
    from paper_2502_05063_b300 import synth, vr
    colptr, rows, _ = synth.lower_star_grid(512, seed=7)
    cp, rw = torch.from_numpy(colptr).cuda(), torch.from_numpy(rows).cuda()
    vr.hypha_pairs(cp, rw, stream=stream)
    runs = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        low, st = vr.hypha_pairs(cp, rw, stream=stream)
        e1.record(stream)
        e1.synchronize()
        runs.append((e0.elapsed_time(e1), st))
    runs.sort(key=lambda t: t[0])
    ms, st = runs[len(runs) // 2]
    ncol, nnz = len(colptr) - 1, len(rows)
    return {"workload": "lower-star filtration of a 512x512 Freudenthal-triangulated grid, random vertex values, "
                        "seed 7 (boundary matrix %d columns, %d entries)" % (ncol, nnz),
            "call_ms": ms, "stats": st,
            "scan_columns_per_s": ncol / (st["ms_scan"] / 1e3) if st["ms_scan"] > 0 else None,
            "scan_entries_per_s": nnz / (st["ms_scan"] / 1e3) if st["ms_scan"] > 0 else None}


RANDPERM_NS = (50, 100, 200, 400, 1000, 2000, 4000, 9000)


def randperm_curve(stream):
    """The apparent-fraction experiment (Sec. 5.6.6, Fig 5.14): distance matrices
    whose lower triangle is a random permutation of 1..n(n-1)/2, the full
    2-skeleton, dimension 1.  Per n: the apparent fraction (mean, min, max over
    the samples) beside the Thm 5.4.2 bound (n-2)/n, and the rate of the fused
    filtration/apparent kernel (library stage timer) and of the whole
    apparent-only call (CUDA events; device-resident input)."""
    import numpy as np
    import torch
    from paper_2502_05063_b300 import synth, vr
    out = {}
    for n in RANDPERM_NS:
        samples = 10 if n <= 1000 else 3
        m = n * (n - 1) // 2
        fr, kms, cms, cof = [], [], [], []
        for smp in range(samples):
            D = synth.random_permutation_dists(n, sample=smp)
            d = torch.from_numpy(D).cuda()
            thr = float(D.max())
            flags = vr.VR_APPARENT_ONLY
            vr.barcodes(dists=d, n=n, dmax=1, threshold=thr, flags=flags, stream=stream)  # warm
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bc = vr.barcodes(dists=d, n=n, dmax=1, threshold=thr, flags=flags, stream=stream)
            e1.record(stream)
            e1.synchronize()
            st = bc.stats[1]
            fr.append(st["apparent"] / m)
            kms.append(st["ms_filtration"])
            cms.append(e0.elapsed_time(e1))
            cof.append(st["cofacets_scanned"])
        k = statistics.median(kms)
        out[str(n)] = {"samples": samples, "apparent_fraction_mean": statistics.mean(fr),
                       "apparent_fraction_min": min(fr), "apparent_fraction_max": max(fr),
                       "upper_bound": (n - 2) / n, "kernel_ms": k,
                       "kernel_simplices_per_s": m / (k / 1e3) if k > 0 else None,
                       "kernel_cofacets_per_s": statistics.median(cof) / (k / 1e3) if k > 0 else None,
                       "call_ms": statistics.median(cms), "call_simplices_per_s": m / (statistics.median(cms) / 1e3)}
    return {"curve": out, "workload": "random permutation of 1..n(n-1)/2 as the lower triangle (ordered distinct "
                                      "floats), full 2-skeleton, H0 and the dimension-1 apparent search "
                                      "(VR_APPARENT_ONLY), seed 5, sample s from stream (5, n, s)"}


def probe_peaks(stream):
    """Project-written read probes (vr_probe_read_gbs): L2-resident and HBM."""
    from paper_2502_05063_b300 import vr
    l2 = max(vr.probe_read_gbs(mb << 20, 200, stream) for mb in (16, 32, 48))
    hbm = vr.probe_read_gbs(4 << 30, 10, stream)
    return {"l2_read_gbs": l2, "hbm_read_gbs": hbm,
            "how": "vr_probe_read_gbs: 16-byte ld.global.cg loads over 4 blocks of 512 threads per SM; L2: best of "
                   "16/32/48 MB buffers x 200 passes; HBM: 4 GB x 10 passes; CUDA events, one untimed pass first"}


def batched_metrics(stream, steps=20):
    """The batched forms: 4096 clouds (forward, H0-H1) and 256 clouds of 128
    points in R^2 (forward + backward of sum (death - birth)^2 over H1), each in
    clouds/s, against a loop of per-cloud calls of the same library."""
    import torch
    from paper_2502_05063_b300 import autograd, synth, vr

    def timeit(fn, k):
        """Median ms of k timed calls (CUDA events per call) after 3 warm-up calls, and the spread.
        Python's cyclic garbage collector is paused during the timed calls (as the
        standard timeit module does), so an interpreter-wide collection over the
        bench process's objects does not land in one call's time."""
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ms = []
        gc.collect()
        gc.disable()
        try:
            for _ in range(k):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        finally:
            gc.enable()
        ms.sort()
        spread = {"min": ms[0], "p10": ms[len(ms) // 10], "median": statistics.median(ms),
                  "p90": ms[(9 * len(ms)) // 10], "max": ms[-1], "repeats": k, "python_gc": "paused while timed"}
        return statistics.median(ms), spread

    clouds, _ = synth.batch_clouds()
    pts, offs = synth.pack(clouds)
    dev = torch.from_numpy(pts).cuda()
    fwd_ms, fwd_spread = timeit(lambda: vr.barcodes_batched(dev, offs, dmax=1, stream=stream), steps)
    sample = [torch.from_numpy(c).cuda() for c in clouds[::32]]
    loop_ms = timeit(lambda: [vr.barcodes(points=d, dmax=1, stream=stream) for d in sample], 3)[0] / len(sample)

    circ = synth.circles()
    cp, co = synth.pack(circ)
    x = torch.from_numpy(cp).cuda()

    def h1_loss(h1):
        """sum over the finite H1 pairs of (death - birth)^2, with no host sync
        (a boolean-mask index would wait for the device to size its result)"""
        d = h1[:, 1] - h1[:, 0]
        d = torch.where(torch.isfinite(d), d, torch.zeros_like(d))  # masked before squaring: no inf * 0
        return (d * d).sum()

    def fwd_bwd_batched():
        xx = x.detach().requires_grad_(True)
        out = autograd.VRDiagramBatched.apply(xx, co, 1)
        h1_loss(out[1]).backward()

    singles = [torch.from_numpy(c).cuda() for c in circ[::8]]

    def fwd_bwd_loop():
        for d in singles:
            xx = d.detach().requires_grad_(True)
            h1_loss(autograd.VRDiagram.apply(xx, 1)[1]).backward()

    fb_ms, fb_spread = timeit(fwd_bwd_batched, steps)
    fb_loop_ms = timeit(fwd_bwd_loop, 3)[0] / len(singles)
    return {
        "batch4096_forward": {"clouds_per_s": len(clouds) / (fwd_ms / 1000), "ms_per_batch": fwd_ms,
                              "ms_spread": fwd_spread,
                              "per_cloud_loop_clouds_per_s": 1000 / loop_ms, "speedup_vs_loop": loop_ms * len(clouds) / fwd_ms,
                              "workload": "4096 clouds, n~U{32..256}, circle/sphere/cube in R^3, H0-H1, seed 3",
                              "loop_sample": "every 32nd cloud, one vr_barcodes call each"},
        "circles256_fwd_bwd": {"clouds_per_s": len(circ) / (fb_ms / 1000), "ms_per_batch": fb_ms,
                               "ms_spread": fb_spread,
                               "per_cloud_loop_clouds_per_s": 1000 / fb_loop_ms,
                               "speedup_vs_loop": fb_loop_ms * len(circ) / fb_ms,
                               "workload": "256 noisy circles, n=128 in R^2, sigma 0.1, seed 4; loss sum over H1 of "
                                           "(death-birth)^2; forward+backward",
                               "loop_sample": "every 8th cloud, VRDiagram forward+backward each"},
    }


def run_reference(args):
    """The reference arm: the oracle as it stands (the paper ships no code), on the
    host cores, each step one bounded sample of the benched workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2502_05063_b300 import synth
    oracle.build()
    pts = synth.WORKLOADS[WORKLOAD]["make"]()
    n = pts.shape[0]
    for _ in range(args.warmup):
        oracle_sample_seconds(pts, CPU_SAMPLE_DMAX)
    t0 = time.perf_counter()
    total = 0.0
    for _ in range(args.steps):
        total += oracle_sample_seconds(pts, CPU_SAMPLE_DMAX)
    wall = time.perf_counter() - t0
    value = candidates(n, CPU_SAMPLE_DMAX) * args.steps / total
    sample = ("oracle (plain C, cohomology with clearing, single thread) on the benched 500-point torus cloud "
              "(seed 1, enclosing radius), dimensions 0-1 per step: C(500,2) = 124,750 candidate simplices")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "ambient_dim": 3, "dmax": 2, "threshold": "enclosing radius",
                       "reference_sample": "dimensions 0-1 of the same cloud"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2502_05063_b300 import build as _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2502_05063_b300 import synth, vr

    w = synth.WORKLOADS[WORKLOAD]
    pts = w["make"]()
    n, dmax, thr = pts.shape[0], w["dmax"], w["threshold"]
    per_step = candidates(n, dmax)
    stream = torch.cuda.current_stream()
    dev = torch.from_numpy(pts).cuda()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step(x):
        return vr.barcodes(points=x, dmax=dmax, threshold=thr, stream=stream)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        step(dev)

    def timed(x):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        results = []
        barrier()
        for k in range(args.steps):
            flush.zero_()  # L2 flush between steps, outside the timed pair
            ev[k][0].record(stream)
            results.append(step(x))
            ev[k][1].record(stream)
        barrier()
        return sum(a.elapsed_time(b) for a, b in ev), results

    clocks = Clocks(local)
    clocks.start()
    total_ms, results = timed(dev)
    clk = clocks.stop()
    pinned = torch.from_numpy(pts).pin_memory()
    e2e_ms, e2e_results = timed(pinned)
    if dist is not None:
        t = torch.tensor([total_ms, e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms, e2e_ms = float(t[0]), float(t[1])
    launches = count_launches(lambda: step(dev))
    if rank != 0:
        return 0

    last = results[-1]
    value = world * per_step * args.steps / (total_ms / 1000.0)
    e2e_value = world * per_step * args.steps / (e2e_ms / 1000.0)
    h2d = pts.nbytes
    d2h = sum(a.nbytes for a in last.pairs)  # pair records returned to the host
    d2h += 24 * (n + sum(last.stats[p]["reduced"] for p in range(1, dmax + 1)))  # device pair records read back
    d2h += 4 * (n * (n - 1) // 2 + 1)  # diameter value table (upper bound)

    # Roofline of the fused filtration/apparent kernel of the top dimension: its
    # algorithmic bytes (roofline_bytes) over its CUDA-event time per launch
    # (the library's stage timer around that launch, on the call's stream),
    # against the measured HBM copy bandwidth and the probed L2 read bandwidth.
    peaks, peak_src = load_peaks()
    probes = probe_peaks(stream)
    st = last.stats[dmax]
    fa_ms = statistics.mean(r.stats[dmax]["ms_filtration"] for r in results)
    nbytes, parts = roofline_bytes(dmax, st)
    achieved = nbytes / (fa_ms / 1000.0) / 1e9
    hbm_peak = float(peaks["hbm_gbs"])
    stage = {}
    for p in range(dmax + 1):
        stage["dim%d" % p] = {k: round(statistics.mean(r.stats[p][k] for r in results), 4)
                              for k in ("ms_filtration", "ms_sort", "ms_reduce")}
    traffic = None
    issue = None
    prof = os.path.join(ROOT, "profiles", "traffic_filtration_apparent_torus500.json")
    if os.path.exists(prof):
        try:
            import hashlib
            rec = json.load(open(prof))
            # the kernel's source: its file and the shared device helpers it inlines
            src = b"".join(open(os.path.join(ROOT, "paper_2502_05063_b300", "csrc", f), "rb").read()
                           for f in ("apparent.cu", "vr_common.cuh"))
            if rec.get("source_sha256") == hashlib.sha256(src).hexdigest():
                traffic = rec.get("bytes_per_launch")
                if rec.get("warp_instructions"):
                    issue = {"warp_instructions_per_launch": rec["warp_instructions"],
                             "lookups_per_launch": st["lookups"],
                             "thread_instructions_per_lookup": rec["warp_instructions"] * rec.get("active_lanes", 32)
                             / max(st["lookups"], 1),
                             "active_lanes_per_instruction": rec.get("active_lanes"),
                             "issue_active_pct": rec.get("issue_active_pct"),
                             "source": "ncu capture recorded in profiles/ (same kernel source)"}
        except (OSError, ValueError):
            traffic = None

    # The step's dominant kernel is the block engine's reduction (k_reduce_heavy):
    # a chain of dependent column additions, bound by their latency, not by a
    # bandwidth or an issue rate; its share of the step and time per addition.
    red_ms = sum(stage["dim%d" % p]["ms_reduce"] for p in range(1, dmax + 1))
    dominant = {"kernel": "k_reduce_heavy<1..%d> (with the warp-engine round)" % dmax,
                "bound": "latency of dependent additions",
                "share_of_step": red_ms / (total_ms / args.steps),
                "per_dimension": {"dim%d" % p: {"ms_reduce": stage["dim%d" % p]["ms_reduce"],
                                                "additions": last.stats[p]["additions"],
                                                "us_per_addition": 1000 * stage["dim%d" % p]["ms_reduce"]
                                                / max(last.stats[p]["additions"], 1)}
                                  for p in range(1, dmax + 1)},
                "profile": "profiles/reduce_heavy_torus500.md, profiles/launches_torus500.md"}
    stage_rates = stage_rates_of(last.stats, dmax, stage)
    stage_rates["note"] = "dimensions 1-%d; filtration and apparent search run as one fused kernel" % dmax

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "ambient_dim": 3, "dmax": dmax, "threshold": "enclosing radius",
                   "simplices_per_step": per_step, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between steps (256 MiB write)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms / args.steps},
        "gpu_launches": launches * args.steps,
        "roofline": {"kernel": "k_filtration_apparent<%d>" % dmax, "bound": "hbm",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": traffic, "ms_per_launch": fa_ms, "algorithmic_bytes_per_launch": nbytes,
                     "bytes_by_step": parts,
                     "peak_source": "hbm_gbs of MEASURED_PEAKS.json (%s; burst copy)" % peak_src,
                     "l2": {"peak": probes["l2_read_gbs"], "frac": achieved / probes["l2_read_gbs"],
                            "peak_source": "project L2-resident read probe, this run"},
                     "target_frac": 0.5,
                     "dominant": dominant},
        "peaks_probe": probes,
        "issue": issue,
        "stages_ms": stage,
        "stage_rates": stage_rates,
        "clocks": clk,
        "counts": {"dim%d" % p: {k: last.stats[p][k] for k in ("candidates", "columns", "apparent", "reduced",
                                                                 "additions", "cofacets_scanned", "lookups")}
                   for p in range(1, dmax + 1)},
    }
    if not args.no_batched:
        line["batched"] = batched_metrics(stream)
        line["other_workloads"] = other_workload_rates(stream)
        line["randperm"] = randperm_curve(stream)
        line["reduction_ablation"] = reduction_ablation(stream)
        line["sparse_mode"] = sparse_mode(stream)
        line["hypha"] = hypha_bench(stream)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_single()
        if not args.no_batched:
            line["cpu_baseline_batched"] = cpu_baseline_batched()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_single():
    import torch
    from paper_2502_05063_b300 import build as _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_2502_05063_b300 import synth, vr
    w = synth.WORKLOADS[WORKLOAD]
    dev = torch.from_numpy(w["make"]()).cuda()
    r = vr.barcodes(points=dev, dmax=w["dmax"], threshold=w["threshold"])
    torch.cuda.synchronize()
    print(json.dumps({"workload": WORKLOAD, "bars": [len(a) for a in r.pairs], "stats": r.stats}))
    return 0


def run_single_batched(num, circles=False):
    """One batched call on the first `num` clouds of the 4096-cloud workload, or
    on the 256 circles of the differentiable workload (for profiler captures of
    the persistent kernel)."""
    import torch
    from paper_2502_05063_b300 import synth, vr
    clouds = synth.circles() if circles else synth.batch_clouds()[0][:num]
    pts, offs = synth.pack(clouds)
    bb = vr.barcodes_batched(torch.from_numpy(pts).cuda(), offs, dmax=1)
    torch.cuda.synchronize()
    print(json.dumps({"clouds": len(clouds), "pairs": [int(o[-1]) for o in bb.offsets]}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form measurements")
    ap.add_argument("--single", action="store_true",
                    help="one untimed call of the workload (for profiler captures), prints its stage counts")
    ap.add_argument("--single-batched", type=int, default=0, metavar="N",
                    help="one batched call on the first N clouds of the 4096-cloud workload (profiler captures)")
    ap.add_argument("--single-circles", action="store_true",
                    help="one batched call on the 256 circles of the differentiable workload (profiler captures)")
    args = ap.parse_args()
    if args.single:
        return run_single()
    if args.single_batched:
        return run_single_batched(args.single_batched)
    if args.single_circles:
        return run_single_batched(0, circles=True)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
