"""Python binding of libvrgpu (argument marshalling only).

Every computation runs in the CUDA library behind the C ABI declared in
``include/vr.h``; this module converts arrays and tensors to pointers and the
returned ``vr_result`` into numpy arrays.  Importing it raises if the library
has not been built (``python -m paper_2502_05063_b300.build``): there is no
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvrgpu.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libvrgpu.so is not built; run `python -m paper_2502_05063_b300.build`")

lib = ctypes.CDLL(LIB_PATH)

VR_MAX_DIM = 6
VR_BATCH_MAX_N = 256
VR_KEEP_ZERO_LENGTH = 0x1
VR_CRITICAL_EDGES = 0x2
VR_DEBUG_CHECKS = 0x4
VR_APPARENT_ONLY = 0x8
VR_REDUCE_V = 0x10
VR_REDUCE_OBLIVIOUS = 0x20
VR_SPARSE = 0x40

STATUS = {0: "VR_OK", 1: "VR_ERR_INVALID_ARG", 2: "VR_ERR_OOM", 3: "VR_ERR_INDEX_OVERFLOW",
          4: "VR_ERR_CUDA", 5: "VR_ERR_TIMEOUT", 6: "VR_ERR_INTERNAL"}


class VRError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__("%s failed: %s (%s)" % (where, self.name, lib.vr_status_string(code).decode()))


class Pair(ctypes.Structure):
    _fields_ = [("birth", ctypes.c_float), ("death", ctypes.c_float),
                ("birth_simplex", ctypes.c_uint64), ("death_simplex", ctypes.c_int64)]


STAT_FIELDS = ["candidates", "above_threshold", "cleared", "columns", "apparent", "reduced",
               "additions", "pairs", "essential", "emitted", "cofacets_scanned", "lookups"]


TIME_FIELDS = ["ms_filtration", "ms_sort", "ms_reduce"]


class Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in STAT_FIELDS] + [(f, ctypes.c_float) for f in TIME_FIELDS]


class Result(ctypes.Structure):
    _fields_ = [("dmax", ctypes.c_int32), ("n", ctypes.c_int64), ("threshold", ctypes.c_float),
                ("count", ctypes.c_int64 * (VR_MAX_DIM + 1)),
                ("pairs", ctypes.POINTER(Pair) * (VR_MAX_DIM + 1)),
                ("critical_edges", ctypes.POINTER(ctypes.c_int32) * (VR_MAX_DIM + 1)),
                ("stats", Stats * (VR_MAX_DIM + 1))]


class BatchResult(ctypes.Structure):
    _fields_ = [("num_clouds", ctypes.c_int32), ("dmax", ctypes.c_int32),
                ("pair_offsets", ctypes.POINTER(ctypes.c_int64) * 2),
                ("pairs", ctypes.POINTER(Pair) * 2),
                ("critical_edges", ctypes.POINTER(ctypes.c_int32) * 2),
                ("thresholds", ctypes.POINTER(ctypes.c_float)), ("recomputed", ctypes.c_int32)]


class DeviceResult(ctypes.Structure):
    _fields_ = [("dmax", ctypes.c_int32), ("n", ctypes.c_int64), ("threshold", ctypes.c_float),
                ("count", ctypes.c_int64 * (VR_MAX_DIM + 1)),
                ("pairs", ctypes.c_void_p * (VR_MAX_DIM + 1)),
                ("critical_edges", ctypes.c_void_p * (VR_MAX_DIM + 1)),
                ("stats", Stats * (VR_MAX_DIM + 1)), ("stream", ctypes.c_void_p)]


class BatchDeviceResult(ctypes.Structure):
    _fields_ = [("num_clouds", ctypes.c_int32), ("dmax", ctypes.c_int32),
                ("pair_offsets", ctypes.POINTER(ctypes.c_int64) * 2),
                ("pairs", ctypes.c_void_p * 2),
                ("critical_edges", ctypes.c_void_p * 2),
                ("thresholds", ctypes.POINTER(ctypes.c_float)), ("stream", ctypes.c_void_p),
                ("recomputed", ctypes.c_int32)]


PAIR_DTYPE = np.dtype([("birth", "<f4"), ("death", "<f4"), ("birth_simplex", "<u8"), ("death_simplex", "<i8")])
assert PAIR_DTYPE.itemsize == ctypes.sizeof(Pair)

_vp, _i64, _i32, _u32, _f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_float
lib.vr_status_string.restype = ctypes.c_char_p
lib.vr_status_string.argtypes = [ctypes.c_int]
lib.vr_barcodes_points.argtypes = [_vp, _i64, _i32, _i32, _f32, _u32, _vp, ctypes.POINTER(ctypes.POINTER(Result))]
lib.vr_barcodes_dists.argtypes = [_vp, _i64, _i32, _f32, _u32, _vp, ctypes.POINTER(ctypes.POINTER(Result))]
lib.vr_result_free.argtypes = [ctypes.POINTER(Result)]
lib.vr_result_free.restype = None
lib.vr_simplex_vertices.argtypes = [ctypes.c_uint64, _i32, _i64, _vp]
lib.vr_distances.argtypes = [_vp, _i64, _i32, _vp, _vp]
lib.vr_sort_u64.argtypes = [_vp, _vp, _i64, _i32, _vp]
lib.vr_sort_u64_noalloc.argtypes = [_vp, _vp, _i64, _i32, _vp]
VR_SORT_NOALLOC_MAX_KEYS = 1 << 18
lib.vr_backward.argtypes = [_vp, _i64, _i32, _vp, _i64, _vp, _vp, _vp, _vp]
lib.vr_barcodes_points_device.argtypes = [_vp, _i64, _i32, _i32, _f32, _u32, _vp,
                                          ctypes.POINTER(ctypes.POINTER(DeviceResult))]
lib.vr_barcodes_dists_device.argtypes = [_vp, _i64, _i32, _f32, _u32, _vp, ctypes.POINTER(ctypes.POINTER(DeviceResult))]
lib.vr_device_result_free.argtypes = [ctypes.POINTER(DeviceResult)]
lib.vr_device_result_free.restype = None
lib.vr_barcodes_batched_device.argtypes = [_vp, _vp, _i32, _i32, _i32, _f32, _u32, _vp,
                                           ctypes.POINTER(ctypes.POINTER(BatchDeviceResult))]
lib.vr_batch_device_result_free.argtypes = [ctypes.POINTER(BatchDeviceResult)]
lib.vr_batch_device_result_free.restype = None
lib.vr_hypha_pairs.argtypes = [_vp, _vp, _i64, _i64, _u32, _vp, _vp, _vp]
lib.vr_probe_read_gbs.argtypes = [_i64, _i32, _vp, ctypes.POINTER(ctypes.c_double)]
if hasattr(lib, "vr_barcodes_batched"):
    lib.vr_barcodes_batched.argtypes = [_vp, _vp, _i32, _i32, _i32, _f32, _u32, _vp,
                                        ctypes.POINTER(ctypes.POINTER(BatchResult))]
    lib.vr_batch_result_free.argtypes = [ctypes.POINTER(BatchResult)]
    lib.vr_batch_result_free.restype = None


def _check(code, where):
    if code != 0:
        raise VRError(code, where)


def _ptr_of(x):
    """(pointer, keepalive) for a numpy array (host) or a torch tensor (host or CUDA)."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), x
    raise TypeError("expected a numpy array or a torch tensor")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Barcodes:
    """Per-dimension pairs of one cloud.

    pairs[p]          structured array (birth, death, birth_simplex, death_simplex)
    critical_edges[p] int32 (m, 4) (u_b, v_b, u_d, v_d) if requested, else None
    stats[p]          dict of the vr_stats counters
    threshold         the threshold actually used
    """

    def __init__(self, res: Result):
        self.dmax = res.dmax
        self.n = res.n
        self.threshold = res.threshold
        self.pairs, self.critical_edges, self.stats = [], [], []
        for p in range(res.dmax + 1):
            m = res.count[p]
            if m:
                buf = ctypes.cast(res.pairs[p], ctypes.POINTER(ctypes.c_char * (m * PAIR_DTYPE.itemsize))).contents
                self.pairs.append(np.frombuffer(buf, dtype=PAIR_DTYPE).copy())
            else:
                self.pairs.append(np.zeros(0, dtype=PAIR_DTYPE))
            if res.critical_edges[p]:
                e = np.ctypeslib.as_array(res.critical_edges[p], shape=(max(m, 1) * 4,))[: 4 * m]
                self.critical_edges.append(e.reshape(m, 4).copy())
            else:
                self.critical_edges.append(None)
            self.stats.append({f: getattr(res.stats[p], f) for f in STAT_FIELDS + TIME_FIELDS})


def barcodes(points=None, dists=None, n=None, dmax=1, threshold=np.inf, flags=0, stream=None) -> Barcodes:
    """Vietoris-Rips barcodes of a point cloud (float32 (n, D)) or of a
    condensed lower-triangular distance vector (float32 n(n-1)/2), given as a
    numpy array or a torch tensor on the host or the GPU."""
    out = ctypes.POINTER(Result)()
    if points is not None:
        ptr, keep = _ptr_of(points)
        nn, amb = int(points.shape[0]), int(points.shape[1])
        code = lib.vr_barcodes_points(ptr, nn, amb, int(dmax), float(threshold), int(flags),
                                      _stream_ptr(stream), ctypes.byref(out))
    else:
        ptr, keep = _ptr_of(dists)
        if n is None:
            m = int(dists.shape[0])
            n = int(round((1 + (1 + 8 * m) ** 0.5) / 2))
        code = lib.vr_barcodes_dists(ptr, int(n), int(dmax), float(threshold), int(flags),
                                     _stream_ptr(stream), ctypes.byref(out))
    _check(code, "vr_barcodes")
    try:
        return Barcodes(out.contents)
    finally:
        lib.vr_result_free(out)


class _ResultHolder:
    """Frees a library result once the last array viewing its memory is gone."""

    def __init__(self, ptr, free):
        self.ptr, self.free = ptr, free

    def __del__(self):
        try:
            self.free(self.ptr)
        except Exception:  # interpreter shutdown: the library may already be unloaded
            pass


def _view(ptr, nbytes, dtype, holder):
    """numpy view of nbytes of library-owned host memory, keeping `holder` (and so
    the memory) alive as long as the view or any array derived from it."""
    buf = ctypes.cast(ptr, ctypes.POINTER(ctypes.c_char * nbytes)).contents
    buf.holder = holder
    return np.frombuffer(buf, dtype=dtype)


class BatchBarcodes:
    """Pairs of many clouds: pairs[p] (structured array of all clouds, cloud i at
    offsets[p][i]:offsets[p][i+1]), critical_edges[p] or None, thresholds[i].
    The pair and edge arrays view the library's result in place (no copy); it
    is released when the last of them is gone."""

    def __init__(self, res: BatchResult, holder=None):
        self.num_clouds, self.dmax = res.num_clouds, res.dmax
        self.recomputed = res.recomputed  # clouds computed by the single-cloud path instead
        self.pairs, self.offsets, self.critical_edges = [], [], []
        nc = res.num_clouds
        self.thresholds = np.ctypeslib.as_array(res.thresholds, shape=(max(nc, 1),))[:nc].copy()
        for p in range(res.dmax + 1):
            off = np.ctypeslib.as_array(res.pair_offsets[p], shape=(nc + 1,)).copy()
            m = int(off[-1])
            if m and holder is not None:
                arr = _view(res.pairs[p], m * PAIR_DTYPE.itemsize, PAIR_DTYPE, holder)
            elif m:
                buf = ctypes.cast(res.pairs[p], ctypes.POINTER(ctypes.c_char * (m * PAIR_DTYPE.itemsize))).contents
                arr = np.frombuffer(buf, dtype=PAIR_DTYPE).copy()
            else:
                arr = np.zeros(0, dtype=PAIR_DTYPE)
            edges = None
            if res.critical_edges[p]:
                if m and holder is not None:
                    edges = _view(res.critical_edges[p], m * 16, np.int32, holder).reshape(m, 4)
                else:
                    edges = np.ctypeslib.as_array(res.critical_edges[p], shape=(max(m, 1) * 4,))[: 4 * m].reshape(m, 4).copy()
            self.pairs.append(arr)
            self.offsets.append(off)
            self.critical_edges.append(edges)

    def cloud(self, i, p):
        return self.pairs[p][self.offsets[p][i]:self.offsets[p][i + 1]]


def barcodes_batched(points, offsets, dmax=1, threshold=np.inf, flags=0, stream=None) -> BatchBarcodes:
    """Barcodes of clouds stored back to back in `points` (float32 (sum n, D),
    numpy or torch, host or GPU); offsets: int64 (num+1,) host array."""
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    ptr, keep = _ptr_of(points)
    out = ctypes.POINTER(BatchResult)()
    code = lib.vr_barcodes_batched(ptr, offs.ctypes.data, len(offs) - 1, int(points.shape[1]), int(dmax),
                                   float(threshold), int(flags), _stream_ptr(stream), ctypes.byref(out))
    _check(code, "vr_barcodes_batched")
    holder = _ResultHolder(out, lib.vr_batch_result_free)  # frees `out` when its last view goes
    return BatchBarcodes(out.contents, holder)


def simplex_vertices(cidx: int, q: int, n: int):
    v = np.zeros(q + 1, dtype=np.int32)
    _check(lib.vr_simplex_vertices(int(cidx), int(q), int(n), v.ctypes.data), "vr_simplex_vertices")
    return [int(x) for x in v]


def distances(pts_dev, out_dev, stream=None):
    """Condensed distances of a CUDA float32 (n, D) tensor into a CUDA float32 tensor."""
    _check(lib.vr_distances(pts_dev.data_ptr(), int(pts_dev.shape[0]), int(pts_dev.shape[1]),
                            out_dev.data_ptr(), _stream_ptr(stream)), "vr_distances")


def sort_u64(keys_dev, values_dev=None, bits=64, stream=None):
    """In-place stable ascending radix sort of CUDA int64/uint64 tensors by the low `bits` bits."""
    _check(lib.vr_sort_u64(keys_dev.data_ptr(), values_dev.data_ptr() if values_dev is not None else None,
                           int(keys_dev.numel()), int(bits), _stream_ptr(stream)), "vr_sort_u64")


def sort_u64_noalloc(keys_dev, values_dev=None, bits=64, stream=None):
    """Like sort_u64, but the library allocates nothing: its scratch is a fixed
    static device array (at most VR_SORT_NOALLOC_MAX_KEYS keys).  Calls that
    overlap on the GPU share that array and must not run concurrently."""
    _check(lib.vr_sort_u64_noalloc(keys_dev.data_ptr(), values_dev.data_ptr() if values_dev is not None else None,
                                   int(keys_dev.numel()), int(bits), _stream_ptr(stream)), "vr_sort_u64_noalloc")


def backward(pts_dev, edges_dev, grad_birth_dev, grad_death_dev, grad_pts_dev, stream=None):
    _check(lib.vr_backward(pts_dev.data_ptr(), int(pts_dev.shape[0]), int(pts_dev.shape[1]), edges_dev.data_ptr(),
                           int(edges_dev.shape[0]), grad_birth_dev.data_ptr(), grad_death_dev.data_ptr(),
                           grad_pts_dev.data_ptr(), _stream_ptr(stream)), "vr_backward")


def probe_read_gbs(nbytes: int, iters: int, stream=None) -> float:
    """Read bandwidth (GB/s) of a device buffer of nbytes, streamed iters times."""
    out = ctypes.c_double()
    _check(lib.vr_probe_read_gbs(int(nbytes), int(iters), _stream_ptr(stream), ctypes.byref(out)),
           "vr_probe_read_gbs")
    return out.value


class _DevArray:
    """__cuda_array_interface__ view of library-owned device memory (borrowed)."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _copies_done(stream):
    """The copies out of a device result were queued on torch's current stream
    and the library frees the result in the order of the call's stream: on the
    same stream the free follows the copies; on another, let them finish."""
    import torch
    cur = torch.cuda.current_stream()
    if (_stream_ptr(stream) or 0) != cur.cuda_stream:
        cur.synchronize()


def _library_done(stream):
    """A device result is written in the order of the call's stream; torch's
    current stream, where its arrays are copied out, waits for it when the
    two differ (an event wait on the device, not a host wait)."""
    import torch
    ptr = _stream_ptr(stream) or 0
    cur = torch.cuda.current_stream()
    if ptr != cur.cuda_stream:
        if ptr:
            cur.wait_stream(torch.cuda.ExternalStream(ptr))
        else:
            torch.cuda.synchronize()


def _own(ptr, count, per, torch_dtype, cols):
    """A torch CUDA tensor (count, cols) copied from `count` records of `per`
    bytes at a library device pointer (a device-to-device copy)."""
    import torch
    if count == 0 or not ptr:
        return torch.zeros((0, cols), dtype=torch_dtype, device="cuda")
    raw = torch.as_tensor(_DevArray(ptr, count * per), device="cuda")
    return raw.view(torch_dtype).view(count, -1)[:, :cols].clone()


class DeviceBarcodes:
    """Pairs of one cloud kept on the GPU (vr_barcodes_*_device).

    values[p]   torch float32 (k_p, 2) CUDA tensor of (birth, death), sorted as in Barcodes
    simplices[p] torch int64 (k_p, 2) CUDA tensor of (birth simplex, death simplex)
    edges[p]    torch int32 (k_p, 4) CUDA tensor of critical edges, or None
    stats[p], threshold, counts as in Barcodes.
    """

    def __init__(self, res: DeviceResult):
        import torch
        self.dmax, self.n, self.threshold = res.dmax, res.n, res.threshold
        self.values, self.simplices, self.edges, self.stats, self.counts = [], [], [], [], []
        for p in range(res.dmax + 1):
            k = int(res.count[p])
            self.counts.append(k)
            self.values.append(_own(res.pairs[p], k, PAIR_DTYPE.itemsize, torch.float32, 2))
            sim = _own(res.pairs[p], k, PAIR_DTYPE.itemsize, torch.int64, 3)
            self.simplices.append(sim[:, 1:3].contiguous() if k else torch.zeros((0, 2), dtype=torch.int64,
                                                                                  device="cuda"))
            self.edges.append(_own(res.critical_edges[p], k, 16, torch.int32, 4) if res.critical_edges[p] else None)
            self.stats.append({f: getattr(res.stats[p], f) for f in STAT_FIELDS + TIME_FIELDS})


def barcodes_device(points=None, dists=None, n=None, dmax=1, threshold=np.inf, flags=0, stream=None):
    """Like barcodes(), with the pairs left on the GPU (DeviceBarcodes)."""
    out = ctypes.POINTER(DeviceResult)()
    if points is not None:
        ptr, keep = _ptr_of(points)
        code = lib.vr_barcodes_points_device(ptr, int(points.shape[0]), int(points.shape[1]), int(dmax),
                                             float(threshold), int(flags), _stream_ptr(stream), ctypes.byref(out))
    else:
        ptr, keep = _ptr_of(dists)
        if n is None:
            m = int(dists.shape[0])
            n = int(round((1 + (1 + 8 * m) ** 0.5) / 2))
        code = lib.vr_barcodes_dists_device(ptr, int(n), int(dmax), float(threshold), int(flags),
                                            _stream_ptr(stream), ctypes.byref(out))
    _check(code, "vr_barcodes_device")
    try:
        return DeviceBarcodes(out.contents)
    finally:
        _copies_done(stream)
        lib.vr_device_result_free(out)


class DeviceBatchBarcodes:
    """Pairs of many clouds on the GPU: values[p] (K_p, 2) float32 and edges[p]
    (K_p, 4) int32 (rows of the packed point array) CUDA tensors, offsets[p]
    host int64 (num+1,), thresholds host float32."""

    def __init__(self, res: BatchDeviceResult):
        import torch
        nc = res.num_clouds
        self.num_clouds, self.dmax = nc, res.dmax
        self.recomputed = res.recomputed
        self.thresholds = np.ctypeslib.as_array(res.thresholds, shape=(max(nc, 1),))[:nc].copy()
        self.values, self.edges, self.offsets = [], [], []
        for p in range(res.dmax + 1):
            off = np.ctypeslib.as_array(res.pair_offsets[p], shape=(nc + 1,)).copy()
            k = int(off[-1])
            self.offsets.append(off)
            self.values.append(_own(res.pairs[p], k, PAIR_DTYPE.itemsize, torch.float32, 2))
            self.edges.append(_own(res.critical_edges[p], k, 16, torch.int32, 4) if res.critical_edges[p] else None)


def barcodes_batched_device(points, offsets, dmax=1, threshold=np.inf, flags=0, stream=None):
    """Like barcodes_batched(), with the pairs left on the GPU (DeviceBatchBarcodes)."""
    offs = np.ascontiguousarray(offsets, dtype=np.int64)
    ptr, keep = _ptr_of(points)
    out = ctypes.POINTER(BatchDeviceResult)()
    code = lib.vr_barcodes_batched_device(ptr, offs.ctypes.data, len(offs) - 1, int(points.shape[1]), int(dmax),
                                          float(threshold), int(flags), _stream_ptr(stream), ctypes.byref(out))
    _check(code, "vr_barcodes_batched_device")
    _library_done(stream)
    try:
        return DeviceBatchBarcodes(out.contents)
    finally:
        _copies_done(stream)
        lib.vr_batch_device_result_free(out)


class HyphaStats(ctypes.Structure):
    _fields_ = [("columns", ctypes.c_int64), ("unstable", ctypes.c_int64), ("compression_passes", ctypes.c_int64),
                ("compression_additions", ctypes.c_int64), ("additions", ctypes.c_int64),
                ("ms_scan", ctypes.c_float), ("ms_compression", ctypes.c_float), ("ms_reduce", ctypes.c_float)]


def hypha_pairs(colptr, rows, stream=None):
    """low(R_j) of every column of an explicit boundary matrix (CSC, numpy or
    torch, host or GPU): numpy int32 array, -1 for zero columns; and the stats."""
    cp, keep_cp = _ptr_of(colptr)
    rw, keep_rw = _ptr_of(rows)
    n = int(colptr.shape[0]) - 1
    out = np.zeros(max(n, 1), dtype=np.int32)
    st = HyphaStats()
    _check(lib.vr_hypha_pairs(cp, rw, n, int(rows.shape[0]), 0, _stream_ptr(stream), out.ctypes.data,
                              ctypes.byref(st)), "vr_hypha_pairs")
    return out[:n], {f: getattr(st, f) for f, _ in HyphaStats._fields_}
