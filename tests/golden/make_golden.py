"""Write the stored expected barcodes of the single-cloud workloads.

Calls only the CPU oracle (``oracle/``) and the seeded input generators; it
never touches the CUDA library.  Each JSON file holds the exact float32 input
(hex of the little-endian bytes, so the test does not depend on the host's
libm), the threshold actually used, the nonzero-persistence diagram of every
dimension with the birth/death simplex indices, and per-dimension counts:

  columns   p-simplices left after threshold and clearing (Sec. 5.5.2)
  pairs     persistence pairs of dimension p, zero-length ones included
  essential classes that never die
  apparent  apparent pairs (s, t) with s of dimension p (Def 5.3.4)

Usage:  python tests/golden/make_golden.py [uniform64 torus500 sphere200]
(torus500 takes a few minutes of single-threaded CPU time).
"""
import json
import os
import struct
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2502_05063_b300 import synth  # noqa: E402


def fhex(x):
    if np.isinf(x):
        return "inf"
    return struct.pack("<f", np.float32(x)).hex()


def make(name):
    w = synth.WORKLOADS[name]
    pts = w["make"]()
    n, amb = pts.shape
    dmax = w["dmax"]
    D32 = oracle.distances_f32(pts)
    D = D32.astype(np.float64)
    thr = w["threshold"]
    thr_used = oracle.enclosing_radius(D, n) if not np.isfinite(thr) else float(np.float32(thr))
    t0 = time.time()
    pairs, stats = oracle.cohom(D, n, dmax, thr_used, clearing=True)
    t1 = time.time()
    dg = oracle.diagram(pairs, dmax)
    apparent = [len(oracle.apparent(D, n, p, thr_used)) for p in range(dmax + 1)]
    t2 = time.time()
    out = {
        "workload": name,
        "doc": w["desc"],
        "n": int(n), "ambient": int(amb), "dmax": int(dmax),
        "threshold": "inf" if not np.isfinite(thr) else fhex(thr),
        "threshold_used": fhex(thr_used),
        "points_f32_hex": np.ascontiguousarray(pts, dtype="<f4").tobytes().hex(),
        "diagram": {str(p): [[fhex(r["birth"]), fhex(r["death"]), int(r["birth_cidx"]), int(r["death_cidx"])]
                             for r in dg[p]] for p in range(dmax + 1)},
        "columns": [int(x) for x in stats[:, 0]],
        "pairs": [int(x) for x in stats[:, 2]],
        "essential": [int(x) for x in stats[:, 3]],
        "apparent": apparent,
        "oracle_seconds": {"cohom": round(t1 - t0, 2), "apparent": round(t2 - t1, 2)},
    }
    with open(os.path.join(HERE, name + ".json"), "w") as f:
        json.dump(out, f, indent=0)
    print(name, "columns", out["columns"], "apparent", apparent, "bars",
          [len(out["diagram"][str(p)]) for p in range(dmax + 1)], out["oracle_seconds"])


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["uniform64", "sphere200", "torus500"]):
        make(name)
