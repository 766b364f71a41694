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

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 (torchrun), single clouds do not shard: every rank runs a replica
and the value is the work of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
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
# oracle sample for the CPU baseline: the same torus generator at fewer points
CPU_SAMPLE_N = 320
REF_STEP_N = 140


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
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

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


def cpu_oracle_throughput(n: int):
    """The oracle as it stands (single thread) on the same generator at n points."""
    import numpy as np
    import oracle
    from paper_2502_05063_b300 import synth
    pts = synth.torus(n, seed=1)
    t0 = time.perf_counter()
    D = oracle.distances_f32(pts).astype(np.float64)
    R = oracle.enclosing_radius(D, n)
    oracle.cohom(D, n, 2, R, clearing=True)
    dt = time.perf_counter() - t0
    return candidates(n, 2) / dt, dt


def batched_metrics(stream, steps=3):
    """The batched forms: 4096 clouds (forward, H0-H1) and 256 clouds of 128
    points in R^2 (forward + backward of sum (death - birth)^2 over H1), each in
    clouds/s, against a loop of per-cloud calls of the same library."""
    import torch
    from paper_2502_05063_b300 import autograd, synth, vr

    def timeit(fn, k):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / k

    clouds, _ = synth.batch_clouds()
    pts, offs = synth.pack(clouds)
    dev = torch.from_numpy(pts).cuda()
    fwd_ms = timeit(lambda: vr.barcodes_batched(dev, offs, dmax=1, stream=stream), steps)
    sample = [torch.from_numpy(c).cuda() for c in clouds[::32]]
    loop_ms = timeit(lambda: [vr.barcodes(points=d, dmax=1, stream=stream) for d in sample], 1) / len(sample)

    circ = synth.circles()
    cp, co = synth.pack(circ)
    x = torch.from_numpy(cp).cuda()

    def fwd_bwd_batched():
        xx = x.detach().requires_grad_(True)
        out = autograd.VRDiagramBatched.apply(xx, co, 1)
        h1 = out[1]
        fin = torch.isfinite(h1[:, 1])
        ((h1[fin, 1] - h1[fin, 0]) ** 2).sum().backward()

    singles = [torch.from_numpy(c).cuda() for c in circ[::8]]

    def fwd_bwd_loop():
        for d in singles:
            xx = d.detach().requires_grad_(True)
            h1 = autograd.VRDiagram.apply(xx, 1)[1]
            fin = torch.isfinite(h1[:, 1])
            ((h1[fin, 1] - h1[fin, 0]) ** 2).sum().backward()

    fb_ms = timeit(fwd_bwd_batched, steps)
    fb_loop_ms = timeit(fwd_bwd_loop, 1) / len(singles)
    return {
        "batch4096_forward": {"clouds_per_s": len(clouds) / (fwd_ms / 1000), "ms_per_batch": fwd_ms,
                              "per_cloud_loop_clouds_per_s": 1000 / loop_ms, "speedup_vs_loop": loop_ms * len(clouds) / fwd_ms,
                              "workload": "4096 clouds, n~U{32..256}, circle/sphere/cube in R^3, H0-H1, seed 3",
                              "loop_sample": "every 32nd cloud, one vr_barcodes call each"},
        "circles256_fwd_bwd": {"clouds_per_s": len(circ) / (fb_ms / 1000), "ms_per_batch": fb_ms,
                               "per_cloud_loop_clouds_per_s": 1000 / fb_loop_ms,
                               "speedup_vs_loop": fb_loop_ms * len(circ) / fb_ms,
                               "workload": "256 noisy circles, n=128 in R^2, sigma 0.1, seed 4; loss sum over H1 of "
                                           "(death-birth)^2; forward+backward",
                               "loop_sample": "every 8th cloud, VRDiagram forward+backward each"},
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        cpu_oracle_throughput(REF_STEP_N)
    t0 = time.perf_counter()
    total = 0.0
    for _ in range(args.steps):
        _, dt = cpu_oracle_throughput(REF_STEP_N)
        total += dt
    wall = time.perf_counter() - t0
    value = candidates(REF_STEP_N, 2) * args.steps / total
    sample = ("oracle (plain C, cohomology with clearing, single thread) on the torus generator at n=%d "
              "(seed 1, H0-H2, enclosing radius) per step" % REF_STEP_N)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "reference_sample_n": REF_STEP_N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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

    # roofline of the fused filtration/apparent kernel of the top dimension: integer-issue bound
    # (ncu: issue ~73%, ALU pipe ~66%, L1 ~21%, DRAM a few MB); one algorithmic op = one
    # diameter-rank lookup and comparison, counted by the kernel (candidate diameters, p+1 per
    # examined cofacet, all pairs of t per facet test)
    peaks, peak_src = load_peaks()
    st = last.stats[dmax]
    fa_ms = statistics.mean(r.stats[dmax]["ms_filtration"] for r in results)
    ops = st["lookups"]
    achieved = ops / (fa_ms / 1000.0) / 1e9
    sm_max = peaks.get("sm_max_mhz", 2032.0)
    alu_peak = 148 * 128 * sm_max * 1e6 / 1e9  # INT32 lane operations per second, in G
    stage = {}
    for p in range(dmax + 1):
        stage["dim%d" % p] = {k: round(statistics.mean(r.stats[p][k] for r in results), 4)
                              for k in ("ms_filtration", "ms_sort", "ms_reduce")}
    traffic = None
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
        except (OSError, ValueError):
            traffic = None

    # the stage rates of the method's data-parallel steps (library stage timers of the last
    # timed calls): filtration simplices over filtration + sort time, apparent-search columns
    # and cofacets over the fused filtration/apparent kernel's time
    dims = range(1, dmax + 1)
    f_ms = sum(stage["dim%d" % p]["ms_filtration"] for p in dims)
    s_ms = sum(stage["dim%d" % p]["ms_sort"] for p in dims)
    stage_rates = {
        "filtration_simplices_per_s": (sum(last.stats[p]["candidates"] for p in dims) / ((f_ms + s_ms) / 1e3)
                                       if f_ms + s_ms > 0 else None),
        "apparent_columns_per_s": (sum(last.stats[p]["columns"] for p in dims) / (f_ms / 1e3)
                                   if f_ms > 0 else None),
        "cofacets_per_s": sum(last.stats[p]["cofacets_scanned"] for p in dims) / (f_ms / 1e3) if f_ms > 0 else None,
        "note": "dimensions 1-%d; filtration and apparent search run as one fused kernel" % dmax,
    }

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
        "roofline": {"kernel": "k_filtration_apparent<%d>" % dmax, "bound": "alu",
                     "achieved": achieved, "peak": alu_peak, "unit": "Gop/s", "frac": achieved / alu_peak,
                     "traffic": traffic, "ms_per_launch": fa_ms, "ops_per_launch": ops,
                     "peak_source": "derived: 148 SMs x 128 INT32 lanes x %.0f MHz (%s sm_max)" % (sm_max, peak_src),
                     "op": "one diameter-rank lookup and comparison"},
        "stages_ms": stage,
        "stage_rates": stage_rates,
        "clocks": clk,
        "counts": {"dim%d" % p: {k: last.stats[p][k] for k in ("candidates", "columns", "apparent", "reduced",
                                                                 "additions", "cofacets_scanned")}
                   for p in range(1, dmax + 1)},
    }
    if not args.no_batched:
        line["batched"] = batched_metrics(stream)
    if world == 1 and not args.no_cpu_baseline:
        v, dt = cpu_oracle_throughput(CPU_SAMPLE_N)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt,
                                "sample": "oracle (plain C, cohomology with clearing, single thread) on the same "
                                          "torus generator at n=%d, H0-H2, enclosing radius" % CPU_SAMPLE_N}
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
    args = ap.parse_args()
    if args.single:
        return run_single()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
