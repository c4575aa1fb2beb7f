"""ctypes binding of ``libsfcoct.so`` (the C ABI in ``include/sfcoct.h``).

Argument marshalling only: every step of the path runs in the library's CUDA kernels.
PyTorch provides device memory and the current stream.  If the library has not been
built, or a call fails, a Python exception is raised; there is no CPU fallback.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import threading

import torch

from .build import LIB

__all__ = [
    "SFCError", "Octree", "octree_build", "radius_search", "radius_count", "radius_fill", "radius_search_csr",
    "radius_search_ranges", "knn_locality", "choose_encoding", "use_torch_allocator", "live_allocations",
    "Batch", "batch_search", "BatchPlan", "batch_autotune", "Server",
    "knn", "encode_cells", "launch_count", "profile_enable", "profile_read", "stats_enable", "stats_read",
    "search_stats", "library_path", "ENCODINGS", "KERNELS",
]

ENCODINGS = {"none": 0, "morton": 1, "hilbert": 2}
KERNELS = {"sphere": 0, "circle": 1, "cube": 2, "square": 3}

SFC_OK = 0
STATUS_NAMES = {0: "SFC_OK", 1: "SFC_ERR_INVALID", 2: "SFC_ERR_OOM", 3: "SFC_ERR_CUDA", 4: "SFC_ERR_TIMEOUT",
                5: "SFC_ERR_TOO_LARGE", 6: "SFC_ERR_NOT_DEVICE_PTR", 7: "SFC_ERR_NOT_FINITE",
                8: "SFC_ERR_INTERNAL"}


class SFCError(RuntimeError):
    def __init__(self, status: int, call: str, detail: str = ""):
        self.status = status
        msg = f"{call} failed: {STATUS_NAMES.get(status, status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


class _BuildOpts(C.Structure):
    _fields_ = [("leaf_capacity", C.c_int32), ("prune", C.c_int32)]


class _Csr(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("cols", C.c_void_p)]


class _Info(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_leaves", C.c_int64), ("n_internal", C.c_int64),
                ("n_nodes", C.c_int64), ("encoding", C.c_int32), ("leaf_capacity", C.c_int32),
                ("prune", C.c_int32), ("device", C.c_int32), ("lo", C.c_float * 3), ("scale", C.c_float)]


_lib = None
_lock = threading.Lock()

_SIGNATURES = {
    "sfc_build_opts_default": (C.c_int, [C.c_void_p]),
    "octree_build": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "octree_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "octree_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "radius_search": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_int, C.c_void_p, C.c_void_p]),
    "radius_count": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    "radius_fill": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_int, C.c_void_p, C.c_void_p,
                              C.c_void_p]),
    "sfc_csr_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "radius_count_static": (C.c_int, [C.c_void_p, C.c_float, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "radius_count_static_max_points": (C.c_int64, []),
    "knn": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "octree_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "octree_export_nodes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p]),
    "sfc_encode_cells": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "radius_search_ranges": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_int, C.c_void_p,
                                       C.c_void_p]),
    "sfc_ranges_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "knn_locality": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    "choose_encoding": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sfc_set_allocator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sfc_live_allocations": (C.c_int64, []),
    "batch_search": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "batch_cloud_result": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "batch_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "batch_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int, C.c_void_p, C.c_void_p, C.c_int32,
                                 C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                 C.c_void_p]),
    "sfc_server_opts_default": (C.c_int, [C.c_void_p]),
    "server_create": (C.c_int, [C.c_void_p, C.c_void_p]),
    "server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "server_wait": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "server_result": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    "server_release": (C.c_int, [C.c_void_p, C.c_int64]),
    "server_stats": (C.c_int, [C.c_void_p, C.c_void_p]),
    "server_destroy": (C.c_int, [C.c_void_p]),
    "batch_plan_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "batch_plan_points": (C.c_int, [C.c_void_p, C.c_void_p]),
    "batch_plan_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "batch_plan_finish": (C.c_int, [C.c_void_p, C.c_void_p]),
    "batch_plan_result": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "batch_plan_free": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sfc_status_string": (C.c_char_p, [C.c_int]),
    "sfc_last_error": (C.c_char_p, []),
    "sfc_launch_count": (C.c_uint64, []),
    "sfc_profile_enable": (C.c_int, [C.c_int32]),
    "sfc_profile_read": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "sfc_stats_enable": (C.c_int, [C.c_int32]),
    "sfc_stats_read": (C.c_int, [C.c_void_p]),
}


def library_path() -> str:
    return LIB


def lib():
    """The loaded library; raises if ``libsfcoct.so`` has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"{LIB} is missing: build it with paper_2603_06771_gb300.build.build()")
            L = C.CDLL(LIB)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(status: int, call: str):
    if status != SFC_OK:
        detail = lib().sfc_last_error().decode() if status == 3 else ""
        raise SFCError(status, call, detail)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _enc(encoding) -> int:
    return ENCODINGS[encoding] if isinstance(encoding, str) else int(encoding)


def _kern(kernel) -> int:
    return KERNELS[kernel] if isinstance(kernel, str) else int(kernel)


def _xyz(t: torch.Tensor | None, what: str) -> torch.Tensor | None:
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == 3):
        raise ValueError(f"{what} must be a CUDA float32 tensor of shape (n, 3)")
    return t.contiguous()


def _ptr(t: torch.Tensor | None):
    return None if t is None or t.numel() == 0 else C.c_void_p(t.data_ptr())


class Octree:
    """A built linear octree (handle of the C ABI).  Release with :meth:`free`."""

    def __init__(self, handle: C.c_void_p, stream):
        self._h = handle
        self._stream = stream
        info = _Info()
        _check(lib().octree_info(self._h, C.byref(info)), "octree_info")
        self.n = int(info.n_points)
        self.n_leaves = int(info.n_leaves)
        self.n_internal = int(info.n_internal)
        self.n_nodes = int(info.n_nodes)
        self.encoding = int(info.encoding)
        self.leaf_capacity = int(info.leaf_capacity)
        self.prune = bool(info.prune)
        self.lo = tuple(float(v) for v in info.lo)
        self.scale = float(info.scale)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("octree already freed")
        return self._h

    def free(self, stream=None):
        if self._h is not None:
            _check(lib().octree_free(self._h, C.c_void_p(_stream(stream))), "octree_free")
            self._h = None

    def __del__(self):
        try:
            if self._h is not None and lib() is not None:
                lib().octree_free(self._h, C.c_void_p(_stream(self._stream)))
                self._h = None
        except Exception:
            pass

    def export(self, stream=None) -> dict:
        """Sorted codes, permutation, leaves array and leaf counts as CUDA tensors."""
        dev = torch.device("cuda", torch.cuda.current_device())
        keys = torch.empty(self.n, dtype=torch.int64, device=dev)
        perm = torch.empty(self.n, dtype=torch.int32, device=dev)
        leaves = torch.empty(self.n_leaves + 1, dtype=torch.int64, device=dev)
        counts = torch.empty(self.n_leaves, dtype=torch.int32, device=dev)
        _check(lib().octree_export(self.handle, C.c_void_p(_stream(stream)), _ptr(keys), _ptr(perm), _ptr(leaves),
                                   _ptr(counts)), "octree_export")
        return {"keys": keys, "perm": perm, "leaves": leaves, "counts": counts}

    def export_nodes(self, stream=None) -> dict:
        """Node table: code, level, [start, end), first child (-1 leaf), tight box."""
        dev = torch.device("cuda", torch.cuda.current_device())
        m = self.n_nodes
        out = {"key": torch.empty(m, dtype=torch.int64, device=dev),
               "level": torch.empty(m, dtype=torch.int32, device=dev),
               "start": torch.empty(m, dtype=torch.int32, device=dev),
               "end": torch.empty(m, dtype=torch.int32, device=dev),
               "child": torch.empty(m, dtype=torch.int32, device=dev),
               "box": torch.empty((m, 6), dtype=torch.float32, device=dev)}
        _check(lib().octree_export_nodes(self.handle, C.c_void_p(_stream(stream)), _ptr(out["key"]),
                                         _ptr(out["level"]), _ptr(out["start"]), _ptr(out["end"]),
                                         _ptr(out["child"]), _ptr(out["box"])), "octree_export_nodes")
        return out


def octree_build(points: torch.Tensor, encoding="hilbert", leaf_capacity: int = 32, prune: bool = True,
                 stream=None) -> Octree:
    """``octree_build`` of the C ABI: encode, sort, gather and link the linear octree."""
    pts = _xyz(points, "points")
    opts = _BuildOpts(int(leaf_capacity), 1 if prune else 0)
    h = C.c_void_p()
    s = _stream(stream)
    _check(lib().octree_build(_ptr(pts), pts.shape[0], _enc(encoding), C.byref(opts), C.c_void_p(s), C.byref(h)),
           "octree_build")
    return Octree(h, stream)


def radius_count(tree: Octree, queries: torch.Tensor | None, r: float, kernel="sphere", stream=None):
    """Row pointers (int64 CUDA tensor, rows + 1) and the neighbour total."""
    q = _xyz(queries, "queries")
    rows = tree.n if q is None else q.shape[0]
    row_ptr = torch.empty(rows + 1, dtype=torch.int64, device="cuda")
    nnz = C.c_int64()
    _check(lib().radius_count(tree.handle, _ptr(q), 0 if q is None else rows, C.c_float(r), _kern(kernel),
                              C.c_void_p(_stream(stream)), _ptr(row_ptr), C.byref(nnz)), "radius_count")
    return row_ptr, int(nnz.value)


def radius_fill(tree: Octree, queries: torch.Tensor | None, r: float, kernel, row_ptr: torch.Tensor, nnz: int,
                stream=None) -> torch.Tensor:
    q = _xyz(queries, "queries")
    cols = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
    rows = tree.n if q is None else q.shape[0]
    _check(lib().radius_fill(tree.handle, _ptr(q), 0 if q is None else rows, C.c_float(r), _kern(kernel),
                             C.c_void_p(_stream(stream)), _ptr(row_ptr), _ptr(cols)), "radius_fill")
    return cols[:nnz]


def radius_search(tree: Octree, queries: torch.Tensor | None, r: float, kernel="sphere", stream=None):
    """CSR (row_ptr int64, cols int32) of the fixed-radius search, torch-allocated."""
    row_ptr, nnz = radius_count(tree, queries, r, kernel, stream)
    return row_ptr, radius_fill(tree, queries, r, kernel, row_ptr, nnz, stream)


class _DeviceArray:
    """Exposes library-owned device memory through ``__cuda_array_interface__``."""

    def __init__(self, owner, ptr: int, n: int, typestr: str):
        self._owner = owner
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
                                         "stream": None}


class _CsrOwner:
    def __init__(self, csr: _Csr, stream: int):
        self.csr = csr
        self.stream = stream

    def __del__(self):
        try:
            lib().sfc_csr_free(C.byref(self.csr), C.c_void_p(self.stream))
        except Exception:
            pass


def radius_search_csr(tree: Octree, queries: torch.Tensor | None, r: float, kernel="sphere", stream=None):
    """``radius_search`` of the C ABI (library-allocated CSR) viewed as torch tensors."""
    q = _xyz(queries, "queries")
    rows = tree.n if q is None else q.shape[0]
    csr = _Csr()
    s = _stream(stream)
    _check(lib().radius_search(tree.handle, _ptr(q), 0 if q is None else rows, C.c_float(r), _kern(kernel),
                               C.c_void_p(s), C.byref(csr)), "radius_search")
    owner = _CsrOwner(csr, s)
    row_ptr = torch.as_tensor(_DeviceArray(owner, csr.row_ptr, csr.n_rows + 1, "<i8"), device="cuda")
    cols = torch.as_tensor(_DeviceArray(owner, csr.cols, csr.nnz, "<i4"), device="cuda")
    return row_ptr, cols


class _Ranges(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_runs", C.c_int64), ("run_ptr", C.c_void_p), ("runs", C.c_void_p)]


class _RangesOwner:
    def __init__(self, ranges: _Ranges, stream: int):
        self.ranges = ranges
        self.stream = stream

    def __del__(self):
        try:
            lib().sfc_ranges_free(C.byref(self.ranges), C.c_void_p(self.stream))
        except Exception:
            pass


def radius_search_ranges(tree: Octree, queries: torch.Tensor | None, r: float, kernel="sphere", stream=None):
    """``radius_search_ranges`` of the C ABI: (run_ptr int64 [rows + 1], runs int32 [n_runs, 2])
    of [start, end) sorted positions, library-allocated, viewed as torch tensors."""
    q = _xyz(queries, "queries")
    rows = tree.n if q is None else q.shape[0]
    rg = _Ranges()
    s = _stream(stream)
    _check(lib().radius_search_ranges(tree.handle, _ptr(q), 0 if q is None else rows, C.c_float(r), _kern(kernel),
                                      C.c_void_p(s), C.byref(rg)), "radius_search_ranges")
    owner = _RangesOwner(rg, s)
    run_ptr = torch.as_tensor(_DeviceArray(owner, rg.run_ptr, rg.n_rows + 1, "<i8"), device="cuda")
    if rg.n_runs == 0:
        return run_ptr, torch.empty((0, 2), dtype=torch.int32, device="cuda")
    runs = torch.as_tensor(_DeviceArray(owner, rg.runs, 2 * rg.n_runs, "<i4"), device="cuda").view(-1, 2)
    return run_ptr, runs


def _ids(centre_ids: torch.Tensor) -> torch.Tensor:
    if not (isinstance(centre_ids, torch.Tensor) and centre_ids.is_cuda and centre_ids.dim() == 1):
        raise ValueError("centre_ids must be a 1-D CUDA tensor")
    return centre_ids.to(torch.int32).contiguous()


def knn_locality(tree: Octree, centre_ids: torch.Tensor, k: int, order="hilbert", histogram: bool = True,
                 stream=None):
    """``knn_locality`` of the C ABI: (H_k as an int64 CUDA tensor of n entries or None, G1)."""
    ids = _ids(centre_ids)
    hist = torch.zeros(max(tree.n, 1), dtype=torch.int64, device="cuda") if histogram else None
    g1 = C.c_double()
    _check(lib().knn_locality(tree.handle, _ptr(ids), ids.shape[0], int(k), _enc(order), C.c_void_p(_stream(stream)),
                              _ptr(hist) if hist is not None else None, C.byref(g1)), "knn_locality")
    return (hist[:tree.n] if hist is not None else None), g1.value


def choose_encoding(tree: Octree, centre_ids: torch.Tensor, k: int, stream=None):
    """``choose_encoding`` of the C ABI: (name of the order with the largest G1, {order: G1})."""
    ids = _ids(centre_ids)
    best = C.c_int()
    g = (C.c_double * 3)()
    _check(lib().choose_encoding(tree.handle, _ptr(ids), ids.shape[0], int(k), C.c_void_p(_stream(stream)),
                                 C.byref(best), g), "choose_encoding")
    names = {v: k for k, v in ENCODINGS.items()}
    return names[best.value], {"none": g[0], "morton": g[1], "hilbert": g[2]}


def knn(tree: Octree, queries: torch.Tensor | None, k: int, stream=None):
    """(idx int32 [rows, k], d2 float32 [rows, k]) of the k nearest points."""
    q = _xyz(queries, "queries")
    rows = tree.n if q is None else q.shape[0]
    idx = torch.empty((rows, k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((rows, k), dtype=torch.float32, device="cuda")
    _check(lib().knn(tree.handle, _ptr(q), 0 if q is None else rows, int(k), C.c_void_p(_stream(stream)),
                     _ptr(idx), _ptr(d2)), "knn")
    return idx, d2


def encode_cells(cells: torch.Tensor, encoding="hilbert", stream=None) -> torch.Tensor:
    """63-bit codes (int64 tensor) of integer cells (n, 3) < 2^21."""
    if not (cells.is_cuda and cells.dim() == 2 and cells.shape[1] == 3 and cells.dtype == torch.int32):
        raise ValueError("cells must be a CUDA int32 tensor of shape (n, 3)")
    cells = cells.contiguous()
    keys = torch.empty(cells.shape[0], dtype=torch.int64, device=cells.device)
    _check(lib().sfc_encode_cells(_ptr(cells), cells.shape[0], _enc(encoding), C.c_void_p(_stream(stream)),
                                  _ptr(keys)), "sfc_encode_cells")
    return keys


def launch_count() -> int:
    return int(lib().sfc_launch_count())


def profile_enable(on: bool = True):
    _check(lib().sfc_profile_enable(1 if on else 0), "sfc_profile_enable")


def profile_read() -> dict:
    """{kernel name: (launches, total ms)} of the launches recorded since profile_enable."""
    cap = 256
    names = C.create_string_buffer(64 * cap)
    launches = (C.c_int64 * cap)()
    ms = (C.c_double * cap)()
    n = lib().sfc_profile_read(names, launches, ms, cap)
    out = {}
    for i in range(min(n, cap)):
        name = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[name] = (int(launches[i]), float(ms[i]))
    return out


class _SearchStats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in ("walks", "expansions", "box_tests", "leaves", "point_tests",
                                               "needed_tests", "passed", "whole", "inserts")]


def stats_enable(on: bool = True):
    """Zero the search work counters and count (``on``), or stop counting.  While counting,
    the searches run instrumented kernels: same results, slower; do not time them."""
    _check(lib().sfc_stats_enable(1 if on else 0), "sfc_stats_enable")


def stats_read() -> dict:
    """The work counters summed since ``stats_enable`` (``sfc_search_stats``), as a dict."""
    st = _SearchStats()
    _check(lib().sfc_stats_read(C.byref(st)), "sfc_stats_read")
    return {name: int(getattr(st, name)) for name, _ in _SearchStats._fields_}


@contextlib.contextmanager
def search_stats():
    """``with search_stats() as st: ...`` counts the searches of the block; ``st`` is filled
    with ``stats_read()`` when the block ends."""
    out: dict = {}
    stats_enable(True)
    try:
        yield out
    finally:
        try:
            out.update(stats_read())
        finally:
            stats_enable(False)


# ----------------------------------------------------------------------------- batched path
class _BatchCloud(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("search", C.c_int32), ("kernel", C.c_int32), ("r", C.c_float),
                ("k", C.c_int32), ("leaf_capacity", C.c_int32), ("knn_window", C.c_int32),
                ("queries_per_warp", C.c_int32), ("record_slots", C.c_int32)]


def _cloud_array(clouds: list):
    arr = (_BatchCloud * len(clouds))()
    for i, c in enumerate(clouds):
        radius = c.get("search", "radius") == "radius"
        arr[i] = _BatchCloud(int(c["n"]), 0 if radius else 1, _kern(c.get("kernel", "sphere")) if radius else 0,
                             float(c.get("r", 0.0)), int(c.get("k", 0)), int(c.get("leaf_capacity", 0)),
                             int(c.get("knn_window", 0)), int(c.get("queries_per_warp", 0)),
                             int(c.get("record_slots", 0)))
    return arr


class Batch:
    """Results of ``batch_search`` (library-owned device memory, released by :meth:`free`)."""

    _result = "batch_cloud_result"

    def __init__(self, handle: C.c_void_p, clouds: list, stream):
        self._h = handle
        self._stream = stream
        self.clouds = clouds

    def _views(self, i: int):
        rp, cols, knn_i, knn_d = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        nnz = C.c_int64()
        _check(getattr(lib(), self._result)(self._h, int(i), C.byref(rp), C.byref(cols), C.byref(nnz),
                                            C.byref(knn_i), C.byref(knn_d)), self._result)
        return rp.value, cols.value, int(nnz.value), knn_i.value, knn_d.value

    def radius(self, i: int):
        """(row_ptr, cols) of radius cloud i as the library hands them out: row_ptr starts at
        0 and cols at the cloud's first neighbour (torch views of library memory)."""
        if self._h is None:
            raise RuntimeError("batch already freed")
        rp, cols, nnz, _, _ = self._views(i)
        n = self.clouds[i]["n"]
        row_ptr = torch.as_tensor(_DeviceArray(self, rp, n + 1, "<i8"), device="cuda")
        if nnz == 0:  # (the address may lie just past the output array)
            return row_ptr, torch.empty(0, dtype=torch.int32, device="cuda")
        return row_ptr, torch.as_tensor(_DeviceArray(self, cols, nnz, "<i4"), device="cuda")

    def knn(self, i: int):
        """(idx [n, k], d2 [n, k]) of kNN cloud i (torch tensors)."""
        if self._h is None:
            raise RuntimeError("batch already freed")
        _, _, _, ki, kd = self._views(i)
        n, k = self.clouds[i]["n"], self.clouds[i]["k"]
        if n == 0:
            return (torch.empty((0, k), dtype=torch.int32, device="cuda"),
                    torch.empty((0, k), dtype=torch.float32, device="cuda"))
        idx = torch.as_tensor(_DeviceArray(self, ki, n * k, "<i4"), device="cuda").view(n, k)
        d2 = torch.as_tensor(_DeviceArray(self, kd, n * k, "<f4"), device="cuda").view(n, k)
        return idx, d2

    def free(self, stream=None):
        if self._h is not None:
            _check(lib().batch_free(self._h, C.c_void_p(_stream(stream))), "batch_free")
            self._h = None

    def __del__(self):
        try:
            if self._h is not None:
                lib().batch_free(self._h, C.c_void_p(_stream(self._stream)))
                self._h = None
        except Exception:
            pass


def batch_search(points: torch.Tensor, clouds: list, encoding="hilbert", leaf_capacity: int = 32, prune: bool = True,
                 stream=None) -> Batch:
    """``batch_search`` of the C ABI.  ``clouds``: list of dicts with ``n`` (points, in order
    of the concatenated ``points``), ``search`` ("radius" or "knn"), and ``kernel`` / ``r``
    or ``k``."""
    pts = _xyz(points, "points")
    if sum(int(c["n"]) for c in clouds) != pts.shape[0]:
        raise ValueError("the clouds' sizes must add up to the number of points")
    arr = _cloud_array(clouds)
    opts = _BuildOpts(int(leaf_capacity), 1 if prune else 0)
    h = C.c_void_p()
    _check(lib().batch_search(_ptr(pts), C.byref(arr), len(clouds), _enc(encoding), C.byref(opts),
                              C.c_void_p(_stream(stream)), C.byref(h)), "batch_search")
    return Batch(h, [dict(c) for c in clouds], stream)


class BatchPlan(Batch):
    """``batch_plan_*`` of the C ABI: the batched pass of a fixed list of clouds recorded
    once as a CUDA graph.  Write the points into :attr:`points`, then :meth:`run` (or
    :meth:`launch` + :meth:`finish`); :meth:`radius` / :meth:`knn` view the last run."""

    _result = "batch_plan_result"

    def __init__(self, clouds: list, encoding="hilbert", leaf_capacity: int = 32, prune: bool = True,
                 nnz_capacity: int = 0, stream=None):
        arr = _cloud_array(clouds)
        opts = _BuildOpts(int(leaf_capacity), 1 if prune else 0)
        h = C.c_void_p()
        _check(lib().batch_plan_create(C.byref(arr), len(clouds), _enc(encoding), C.byref(opts), int(nnz_capacity),
                                       C.c_void_p(_stream(stream)), C.byref(h)), "batch_plan_create")
        super().__init__(h, [dict(c) for c in clouds], stream)
        ptr = C.c_void_p()
        _check(lib().batch_plan_points(self._h, C.byref(ptr)), "batch_plan_points")
        n = sum(int(c["n"]) for c in clouds)
        self.points = torch.as_tensor(_DeviceArray(self, ptr.value, 3 * n, "<f4"), device="cuda").view(n, 3)

    def launch(self, stream=None):
        _check(lib().batch_plan_launch(self._h, C.c_void_p(_stream(stream))), "batch_plan_launch")

    def finish(self, stream=None):
        _check(lib().batch_plan_finish(self._h, C.c_void_p(_stream(stream))), "batch_plan_finish")

    def run(self, stream=None):
        self.launch(stream)
        self.finish(stream)
        return self

    def free(self, stream=None):
        if self._h is not None:
            _check(lib().batch_plan_free(self._h, C.c_void_p(_stream(stream))), "batch_plan_free")
            self._h = None

    def __del__(self):
        try:
            if self._h is not None:
                lib().batch_plan_free(self._h, C.c_void_p(_stream(self._stream)))
                self._h = None
        except Exception:
            pass


def batch_autotune(points: torch.Tensor, clouds: list, encoding="hilbert", leaf_capacity: int = 32,
                   prune: bool = True, leaf_candidates=(16, 32, 64, 128, 256), window_candidates=(8, 16, 32, 64),
                   qpw_candidates=(16, 32), slot_candidates=(16, 32, 64), stream=None) -> list:
    """``batch_autotune`` of the C ABI: the clouds with ``leaf_capacity``, (kNN)
    ``knn_window``, ``queries_per_warp`` and (radius) ``record_slots`` filled in from timing
    this batch on the device."""
    pts = _xyz(points, "points")
    if sum(int(c["n"]) for c in clouds) != pts.shape[0]:
        raise ValueError("the clouds' sizes must add up to the number of points")
    arr = _cloud_array(clouds)
    opts = _BuildOpts(int(leaf_capacity), 1 if prune else 0)

    def ints(v):
        return (C.c_int32 * max(len(v), 1))(*v), len(v)

    lc, nl = ints(leaf_candidates)
    wc, nw = ints(window_candidates)
    qc, nq = ints(qpw_candidates)
    sc, ns = ints(slot_candidates)
    out = (_BatchCloud * len(clouds))()
    _check(lib().batch_autotune(_ptr(pts), C.byref(arr), len(clouds), _enc(encoding), C.byref(opts), lc, nl, wc, nw,
                                qc, nq, sc, ns, C.c_void_p(_stream(stream)), out), "batch_autotune")
    return [dict(c, leaf_capacity=int(out[i].leaf_capacity), knn_window=int(out[i].knn_window),
                 queries_per_warp=int(out[i].queries_per_warp), record_slots=int(out[i].record_slots))
            for i, c in enumerate(clouds)]


# ----------------------------------------------------------------------------- serving
class _ServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("batch_points", C.c_int64),
                ("hbm_budget", C.c_int64), ("enc", C.c_int), ("leaf_capacity", C.c_int32)]


class _Request(C.Structure):
    _fields_ = [("points_xyz", C.c_void_p), ("n_points", C.c_int64), ("queries_xyz", C.c_void_p),
                ("n_queries", C.c_int64), ("search", C.c_int32), ("kernel", C.c_int32), ("r", C.c_float),
                ("k", C.c_int32)]


class _RequestResult(C.Structure):
    _fields_ = [("row_ptr", C.c_void_p), ("cols", C.c_void_p), ("nnz", C.c_int64), ("row_base", C.c_int64),
                ("knn_idx", C.c_void_p), ("knn_d2", C.c_void_p), ("n_rows", C.c_int64), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double), ("batched_with", C.c_int32), ("pad", C.c_int32)]


class _ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("running", C.c_int64), ("admitted", C.c_int64),
                ("reserved_bytes", C.c_int64)]


def _host_xyz(a, what: str):
    """A C-contiguous float32 (n, 3) host array (numpy or CPU tensor) the server may read."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise ValueError(f"{what} must be in host memory")
        a = a.contiguous()
        if a.dtype != torch.float32 or a.dim() != 2 or a.shape[1] != 3:
            raise ValueError(f"{what} must be float32 of shape (n, 3)")
        return a, a.data_ptr(), a.shape[0]
    import numpy as np

    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError(f"{what} must be of shape (n, 3)")
    return a, a.ctypes.data, a.shape[0]


class Server:
    """``server_*`` of the C ABI: requests queued at any time, admitted against a device
    memory budget, run on ``slots`` streams, small all-points requests merged."""

    def __init__(self, slots: int = 4, max_batch: int = 64, batch_points: int = 4_000_000,
                 hbm_budget: int = 150 << 30, encoding="hilbert", leaf_capacity: int = 64):
        o = _ServerOpts(int(slots), int(max_batch), int(batch_points), int(hbm_budget), _enc(encoding),
                        int(leaf_capacity))
        h = C.c_void_p()
        _check(lib().server_create(C.byref(o), C.byref(h)), "server_create")
        self._h = h
        self._keep = {}

    def submit(self, points, search: str = "radius", kernel: str = "sphere", r: float = 0.0, k: int = 0,
               queries=None) -> int:
        pts, pptr, n = _host_xyz(points, "points")
        q, qptr, nq = (None, None, 0) if queries is None else _host_xyz(queries, "queries")
        radius = search == "radius"
        req = _Request(pptr if n else None, n, qptr if q is not None else None, nq, 0 if radius else 1,
                       _kern(kernel) if radius else 0, float(r), int(k))
        rid = C.c_int64()
        _check(lib().server_submit(self._h, C.byref(req), C.byref(rid)), "server_submit")
        self._keep[rid.value] = (pts, q, search, int(k))
        return rid.value

    def wait(self, rid: int, timeout_ms: int = -1) -> int:
        st = C.c_int()
        _check(lib().server_wait(self._h, int(rid), int(timeout_ms), C.byref(st)), "server_wait")
        return st.value

    def result(self, rid: int) -> dict:
        """Copies of a finished request's results (torch, on the device) and its timings."""
        res = _RequestResult()
        _check(lib().server_result(self._h, int(rid), C.byref(res)), "server_result")
        _, _, search, k = self._keep[rid]
        out = {"latency_ms": res.latency_ms, "queue_ms": res.queue_ms, "batched_with": res.batched_with,
               "rows": res.n_rows}
        n = res.n_rows
        if search == "radius":
            rp = torch.as_tensor(_DeviceArray(self, res.row_ptr, n + 1, "<i8"), device="cuda").clone()
            out["row_ptr"] = rp
            out["cols"] = (torch.as_tensor(_DeviceArray(self, res.cols, res.nnz, "<i4"), device="cuda").clone()
                           if res.nnz else torch.empty(0, dtype=torch.int32, device="cuda"))
        else:
            if n:
                out["knn_idx"] = torch.as_tensor(_DeviceArray(self, res.knn_idx, n * k, "<i4"),
                                                 device="cuda").view(n, k).clone()
                out["knn_d2"] = torch.as_tensor(_DeviceArray(self, res.knn_d2, n * k, "<f4"),
                                                device="cuda").view(n, k).clone()
            else:
                out["knn_idx"] = torch.empty((0, k), dtype=torch.int32, device="cuda")
                out["knn_d2"] = torch.empty((0, k), dtype=torch.float32, device="cuda")
        return out

    def timings(self, rid: int) -> dict:
        res = _RequestResult()
        _check(lib().server_result(self._h, int(rid), C.byref(res)), "server_result")
        return {"latency_ms": res.latency_ms, "queue_ms": res.queue_ms, "batched_with": res.batched_with,
                "rows": res.n_rows}

    def release(self, rid: int):
        _check(lib().server_release(self._h, int(rid)), "server_release")
        self._keep.pop(rid, None)

    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib().server_stats(self._h, C.byref(st)), "server_stats")
        return {"queued": st.queued, "running": st.running, "admitted": st.admitted,
                "reserved_bytes": st.reserved_bytes}

    def close(self):
        if self._h is not None:
            _check(lib().server_destroy(self._h), "server_destroy")
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- device memory
_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


def _torch_alloc(nbytes, ctx, stream):
    s = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
    return torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(), stream=s)


def _torch_free(ptr, ctx, stream):
    torch.cuda.caching_allocator_delete(ptr)


_HOOKS = (_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free))  # kept alive for the library


def use_torch_allocator(on: bool = True):
    """``sfc_set_allocator`` with torch's caching allocator (``on``) or back to the
    stream-ordered allocator; only while no library allocation is alive."""
    if on:
        _check(lib().sfc_set_allocator(C.cast(_HOOKS[0], C.c_void_p), C.cast(_HOOKS[1], C.c_void_p), None),
               "sfc_set_allocator")
    else:
        _check(lib().sfc_set_allocator(None, None, None), "sfc_set_allocator")


def live_allocations() -> int:
    return int(lib().sfc_live_allocations())
