"""Host-side logic of bench.py, without a GPU: the roofline's algorithmic
byte count, the clock-sample parser, and the reference arm's JSON line."""
import json
import math
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_bytes_by_the_per_unit_figures():
    """Dimension 2 of torus500 (counts of a measured step), counted term by term:
    a candidate triangle reads its 3 pair ranks (4 B each) and one clearing bit,
    a kept column writes an 8-byte key; the search reads that key, writes up to
    16 B and reads 4 x 3 ranks for the facet test, and each cofacet examined
    reads the 3 ranks of its new pairs."""
    st = {"candidates": 20_708_500, "columns": 10_600_504, "cofacets_scanned": 65_125_249}
    filtration = 20_708_500 * 3 * 4 + 20_708_500 / 8 + 10_600_504 * 8
    apparent = 10_600_504 * (8 + 16 + 4 * 3 * 4) + 65_125_249 * 3 * 4
    total, parts = bench.roofline_bytes(2, st)
    assert parts["filtration"] == filtration
    assert parts["apparent"] == apparent
    assert total == filtration + apparent == 1_880_633_870.5


def test_roofline_bytes_dimension_one():
    """Edges: one pair rank per candidate, (p+2) C(p+1,2) = 3 ranks for the
    facet test of a kept column, and two ranks per cofacet examined."""
    st = {"candidates": 1000, "columns": 10, "cofacets_scanned": 50}
    total, _ = bench.roofline_bytes(1, st)
    assert total == 1000 * 4 + 1000 / 8 + 10 * 8 + 10 * (8 + 16 + 3 * 4) + 50 * 2 * 4


class _Done:
    def terminate(self):
        pass

    def wait(self):
        return 0


def test_clock_samples_are_parsed(tmp_path):
    """Median SM clock, the maximum, the sample count, and every throttle reason
    seen active in any sample; malformed lines are skipped."""
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("0, 2032, 2032, 700.1, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1965, 2032, 1090.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2032, 2032, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage\n")
    c.proc = _Done()
    got = c.stop()
    assert got == {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "samples": 3, "reasons": ["sw_power_cap"]}
    assert not os.path.exists(c.path)


def test_clocks_without_nvidia_smi():
    c = bench.Clocks(0)
    c.proc = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def _run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r


def test_reference_arm_line():
    """One step of the reference arm (the oracle on its bounded sample): one JSON
    line with the same metric, unit and workload as the library's arm, marked
    as the reference, with its CPU baseline and an e2e that moves no bytes."""
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["higher_is_better"] is True and d["steps"] == 1
    assert d["value"] > 0 and math.isfinite(d["value"])
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    """Under torchrun only rank 0 runs the reference arm; the others exit 0 silently."""
    r = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0
    assert r.stdout.strip() == ""
