"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/vr.h, and rejects bad arguments before touching CUDA.
Host-only arithmetic (the simplex index map of eq. 5.6) is compared with the
oracle."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vr():
    from paper_2502_05063_b300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2502_05063_b300 import vr as _vr
    return _vr


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:vr_status|void|const char\s*\*)\s+(vr_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(vr):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(vr.lib, name), name


def test_status_strings(vr):
    for code, name in vr.STATUS.items():
        s = vr.lib.vr_status_string(code).decode()
        assert s and s != "unknown status", name


def test_simplex_vertices_matches_oracle(vr):
    rng = np.random.default_rng(0)
    for q in range(0, 5):
        n = int(rng.integers(q + 1, 60))
        total = math.comb(n, q + 1)
        for c in set(rng.integers(0, total, size=20).tolist()) | {0, total - 1}:
            assert vr.simplex_vertices(c, q, n) == oracle.simplex_vertices(c, q, n)
    with pytest.raises(vr.VRError):
        vr.simplex_vertices(math.comb(10, 3), 2, 10)  # out of range


def test_argument_checks_before_cuda(vr):
    out = ctypes.POINTER(vr.Result)()
    pts = np.zeros((4, 3), np.float32)
    p = pts.ctypes.data
    assert vr.lib.vr_barcodes_points(p, 0, 3, 1, float("inf"), 0, None, ctypes.byref(out)) == 1
    assert vr.lib.vr_barcodes_points(p, 4, 3, 7, float("inf"), 0, None, ctypes.byref(out)) == 1
    assert vr.lib.vr_barcodes_points(p, 4, 0, 1, float("inf"), 0, None, ctypes.byref(out)) == 1
    assert vr.lib.vr_barcodes_points(p, 4, 3, 1, float("nan"), 0, None, ctypes.byref(out)) == 1
    assert vr.lib.vr_barcodes_points(p, 4, 3, 1, 1.0, 0x80, None, ctypes.byref(out)) == 1
    assert not out
    assert vr.lib.vr_sort_u64_noalloc(None, None, vr.VR_SORT_NOALLOC_MAX_KEYS + 1, 64, None) == 1
    assert vr.lib.vr_sort_u64(None, None, -1, 64, None) == 1
    assert vr.lib.vr_backward(None, 0, 3, None, 0, None, None, None, None) == 1
    # VR_DEBUG_CHECKS is a known flag: the call gets past the flag check (and then
    # fails on the size, before any CUDA call)
    assert vr.lib.vr_barcodes_points(p, 0, 3, 1, 1.0, vr.VR_DEBUG_CHECKS, None, ctypes.byref(out)) == 1


@pytest.mark.parametrize("n,dmax", [(65536, 6), (40000, 5), (65536, 4)])
def test_index_overflow_before_cuda(vr, n, dmax):
    """C(n, dmax+2) >= 2^63: the simplex indices of dimension dmax+1 do not fit,
    reported as VR_ERR_INDEX_OVERFLOW before any device work (no GPU needed)."""
    assert math.comb(n, dmax + 2) >= 2 ** 63
    out = ctypes.POINTER(vr.Result)()
    dummy = np.zeros(3, np.float32)  # never read: the check comes first
    assert vr.lib.vr_barcodes_points(dummy.ctypes.data, n, 3, dmax, float("inf"), 0, None,
                                     ctypes.byref(out)) == 3
    assert vr.lib.vr_barcodes_dists(dummy.ctypes.data, n, dmax, 1.0, 0, None, ctypes.byref(out)) == 3
    assert not out


def test_product_path_has_no_oracle_dependency():
    """The library and its binding never load the oracle."""
    src = open(os.path.join(ROOT, "paper_2502_05063_b300", "vr.py")).read()
    assert "oracle" not in src.split('"""', 2)[2]
    for f in os.listdir(os.path.join(ROOT, "paper_2502_05063_b300", "csrc")):
        text = open(os.path.join(ROOT, "paper_2502_05063_b300", "csrc", f)).read()
        assert "vr_oracle" not in text and "or_cohom" not in text


def test_binding_structs_match_the_header(vr, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets of
    its C struct in include/vr.h (a C program built here prints them), so a
    field added to the header without the binding, or in another order, fails."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"vr_pair": vr.Pair, "vr_stats": vr.Stats, "vr_result": vr.Result,
               "vr_batch_result": vr.BatchResult, "vr_device_result": vr.DeviceResult,
               "vr_batch_device_result": vr.BatchDeviceResult, "vr_hypha_stats": vr.HyphaStats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "vr.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
