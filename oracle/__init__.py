"""CPU oracle for the SFC + linear-octree neighbour search (arXiv 2603.06771).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library and its
Python binding never import it; the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, -O2 -ffp-contract=off); this module
compiles it on first use and marshals numpy arrays through ctypes.  Every function
names the passage of the paper it follows:

* section 4  discretisation: :func:`bbox`, :func:`discretise`
* section 4.1 / 4.2 codes:   :func:`encode_cells`, :func:`decode_codes`, :func:`morton`, :func:`hilbert`
* section 4 reordering:      :func:`sort_keys`
* section 5.1 leaves:       :func:`leaves`
* section 3.1 pointer octree: :class:`PointerOctree`
* section 3.2 kernels:      :func:`pred`, :func:`radius_brute`, :meth:`PointerOctree.radius`
* section 3.3 kNN:          :func:`knn_brute`, :meth:`PointerOctree.knn`
* section 5.1 range output: :func:`runs_of_rows`, :meth:`Pipeline.radius_runs`,
  :meth:`Pipeline.neighbours_struct`
* section 5.2 histogram:    :func:`locality_histogram`
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")

SPHERE, CIRCLE, CUBE, SQUARE = 0, 1, 2, 3
KERNELS = {"sphere": SPHERE, "circle": CIRCLE, "cube": CUBE, "square": SQUARE}
ENC_NONE, ENC_MORTON, ENC_HILBERT = 0, 1, 2
ENCODINGS = {"none": ENC_NONE, "morton": ENC_MORTON, "hilbert": ENC_HILBERT}
L = 21

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liborc.so`` (gcc, -O2 -ffp-contract=off)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i64, i32, f32, u64 = C.c_int64, C.c_int, C.c_float, C.c_uint64
        sig = {
            "orc_free": (None, [P]),
            "orc_num_cpus": (i32, []),
            "orc_bbox": (i32, [P, i64, P, P, P]),
            "orc_discretise": (None, [P, i64, P, f32, P]),
            "orc_morton_encode": (u64, [C.c_uint32, C.c_uint32, C.c_uint32, i32]),
            "orc_hilbert_encode": (u64, [C.c_uint32, C.c_uint32, C.c_uint32, i32]),
            "orc_encode_cells": (None, [P, i64, i32, i32, P]),
            "orc_decode_codes": (None, [P, i64, i32, i32, P]),
            "orc_sort": (None, [P, i64, P, P]),
            "orc_leaves": (i64, [P, i64, i64, P, P]),
            "orc_tree_build": (P, [P, P, i64, i64]),
            "orc_tree_free": (None, [P]),
            "orc_tree_num_nodes": (i64, [P]),
            "orc_tree_num_leaves": (i64, [P]),
            "orc_tree_nodes": (None, [P, i32, P, P, P, P, P, P, P, P, P, P]),
            "orc_pred": (i32, [i32, P, P, f32]),
            "orc_radius_brute": (i64, [P, i64, P, i64, f32, i32, i32, P, P]),
            "orc_radius_tree": (i64, [P, P, i64, f32, i32, i32, P, P]),
            "orc_knn_brute": (None, [P, i64, P, i64, i32, i32, P, P]),
            "orc_knn_tree": (None, [P, P, i64, i32, i32, P, P]),
            "orc_boundary_disagreements": (i64, [P, i64, P, i64, f32, i32, i32]),
            "orc_locality_histogram": (None, [P, i64, i32, P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f32x3(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("expected an (n, 3) float32 array")
    return a


def num_cpus() -> int:
    return int(_load().orc_num_cpus())


# ----------------------------------------------------------------------------- section 4
def bbox(xyz) -> tuple[np.ndarray, float, float]:
    """Lower corner, largest extent and scale 2^21 / extent (binary32), section 4."""
    xyz = _f32x3(xyz)
    lo = np.zeros(3, np.float32)
    ext = np.zeros(1, np.float32)
    s = np.zeros(1, np.float32)
    if _load().orc_bbox(_ptr(xyz), len(xyz), _ptr(lo), _ptr(ext), _ptr(s)):
        raise ValueError("non-finite coordinates or extent")
    return lo, float(ext[0]), float(s[0])


def discretise(xyz, lo, scale) -> np.ndarray:
    """Integer cells in [0, 2^21)^3, shape (n, 3) uint32, section 4 steps 1-2."""
    xyz = _f32x3(xyz)
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    cell = np.empty((len(xyz), 3), np.uint32)
    _load().orc_discretise(_ptr(xyz), len(xyz), _ptr(lo), C.c_float(scale), _ptr(cell))
    return cell


# ----------------------------------------------------------------------------- sections 4.1, 4.2
def morton(x: int, y: int, z: int, L: int = L) -> int:
    return int(_load().orc_morton_encode(x, y, z, L))


def hilbert(x: int, y: int, z: int, L: int = L) -> int:
    return int(_load().orc_hilbert_encode(x, y, z, L))


def encode_cells(cell, enc: int, L: int = L) -> np.ndarray:
    """Codes of integer cells; ``enc`` NONE uses Morton codes (section 4.1 / 4.2)."""
    cell = np.ascontiguousarray(cell, dtype=np.uint32).reshape(-1, 3)
    out = np.empty(len(cell), np.uint64)
    _load().orc_encode_cells(_ptr(cell), len(cell), int(enc), int(L), _ptr(out))
    return out


def decode_codes(codes, enc: int, L: int = L) -> np.ndarray:
    codes = np.ascontiguousarray(codes, dtype=np.uint64)
    out = np.empty((len(codes), 3), np.uint32)
    _load().orc_decode_codes(_ptr(codes), len(codes), int(enc), int(L), _ptr(out))
    return out


# ----------------------------------------------------------------------------- section 4 reorder
def sort_keys(keys) -> tuple[np.ndarray, np.ndarray]:
    """(perm, sorted keys): ascending codes, equal codes in input order."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    perm = np.empty(len(keys), np.uint32)
    srt = np.empty(len(keys), np.uint64)
    _load().orc_sort(_ptr(keys), len(keys), _ptr(perm), _ptr(srt))
    return perm, srt


# ----------------------------------------------------------------------------- section 5.1
def leaves(sorted_keys, ncap: int) -> tuple[np.ndarray, np.ndarray]:
    """(leaves[nL + 1], counts[nL]) by repeated splitting of over-full ranges."""
    sk = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
    lp, cp = C.c_void_p(), C.c_void_p()
    lib = _load()
    nl = lib.orc_leaves(_ptr(sk), len(sk), int(ncap), C.byref(lp), C.byref(cp))
    lv = np.ctypeslib.as_array(C.cast(lp, C.POINTER(C.c_uint64)), shape=(nl + 1,)).copy()
    ct = np.ctypeslib.as_array(C.cast(cp, C.POINTER(C.c_uint32)), shape=(max(nl, 1),))[:nl].copy()
    lib.orc_free(lp)
    lib.orc_free(cp)
    return lv, ct


# ----------------------------------------------------------------------------- section 3.2
def pred(kern: int, p, c, r: float) -> bool:
    p = np.ascontiguousarray(p, dtype=np.float32)
    c = np.ascontiguousarray(c, dtype=np.float32)
    return bool(_load().orc_pred(int(kern), _ptr(p), _ptr(c), C.c_float(r)))


def _take_csr(nq: int, row_ptr: np.ndarray, colp) -> tuple[np.ndarray, np.ndarray]:
    total = int(row_ptr[-1])
    cols = np.ctypeslib.as_array(C.cast(colp, C.POINTER(C.c_int32)), shape=(max(total, 1),))[:total].copy()
    _load().orc_free(colp)
    return row_ptr, cols


def radius_brute(xyz, queries, r: float, kern: int, nthreads: int = 0):
    """CSR (row_ptr, cols) of {p : kernel(p, c, r)} for every centre, by testing every point."""
    xyz, q = _f32x3(xyz), _f32x3(queries)
    row_ptr = np.empty(len(q) + 1, np.int64)
    colp = C.c_void_p()
    _load().orc_radius_brute(_ptr(xyz), len(xyz), _ptr(q), len(q), C.c_float(r), int(kern), int(nthreads),
                             _ptr(row_ptr), C.byref(colp))
    return _take_csr(len(q), row_ptr, colp)


def knn_brute(xyz, queries, k: int, nthreads: int = 0):
    """(idx[nq, k], d2[nq, k]) by a full scan: the k smallest (d2, index) pairs."""
    xyz, q = _f32x3(xyz), _f32x3(queries)
    idx = np.empty((len(q), k), np.int32)
    d2 = np.empty((len(q), k), np.float32)
    _load().orc_knn_brute(_ptr(xyz), len(xyz), _ptr(q), len(q), int(k), int(nthreads), _ptr(idx), _ptr(d2))
    return idx, d2


def boundary_disagreements(xyz, queries, r: float, kern: int, nthreads: int = 0) -> int:
    xyz, q = _f32x3(xyz), _f32x3(queries)
    return int(_load().orc_boundary_disagreements(_ptr(xyz), len(xyz), _ptr(q), len(q), C.c_float(r),
                                                  int(kern), int(nthreads)))


# ----------------------------------------------------------------------------- section 3.1 / 3.3
class PointerOctree:
    """Pointer octree over the discretised cloud (section 3.1) with the searches of 3.2 and 3.3."""

    def __init__(self, xyz, ncap: int, cell=None):
        self.xyz = _f32x3(xyz)
        if cell is None:
            lo, _, s = bbox(self.xyz)
            cell = discretise(self.xyz, lo, s)
        self.cell = np.ascontiguousarray(cell, dtype=np.uint32)
        self.ncap = int(ncap)
        self._lib = _load()
        self._t = self._lib.orc_tree_build(_ptr(self.xyz), _ptr(self.cell), len(self.xyz), self.ncap)

    def __del__(self):
        if getattr(self, "_t", None):
            self._lib.orc_tree_free(self._t)
            self._t = None

    @property
    def num_nodes(self) -> int:
        return int(self._lib.orc_tree_num_nodes(self._t))

    @property
    def num_leaves(self) -> int:
        return int(self._lib.orc_tree_num_leaves(self._t))

    def nodes(self, enc: int, perm, sorted_keys) -> dict:
        """Every node with its code range start, level, count and sorted-position range."""
        m = self.num_nodes
        perm = np.asarray(perm, dtype=np.int64)
        rank = np.empty(len(perm), np.uint32)
        rank[perm] = np.arange(len(perm), dtype=np.uint32)
        sk = np.ascontiguousarray(sorted_keys, dtype=np.uint64)
        out = dict(key=np.empty(m, np.uint64), level=np.empty(m, np.int32), count=np.empty(m, np.int64),
                   is_leaf=np.empty(m, np.int32), start=np.empty(m, np.int64), end=np.empty(m, np.int64),
                   contiguous=np.empty(m, np.int32), box=np.empty((m, 6), np.float32))
        self._lib.orc_tree_nodes(self._t, int(enc), _ptr(rank), _ptr(sk), _ptr(out["key"]), _ptr(out["level"]),
                                 _ptr(out["count"]), _ptr(out["is_leaf"]), _ptr(out["start"]), _ptr(out["end"]),
                                 _ptr(out["contiguous"]), _ptr(out["box"]))
        return out

    def radius(self, queries, r: float, kern: int, nthreads: int = 0):
        """CSR of the naive octree search (section 3.2), rows sorted by original index."""
        q = _f32x3(queries)
        row_ptr = np.empty(len(q) + 1, np.int64)
        colp = C.c_void_p()
        self._lib.orc_radius_tree(self._t, _ptr(q), len(q), C.c_float(r), int(kern), int(nthreads),
                                  _ptr(row_ptr), C.byref(colp))
        return _take_csr(len(q), row_ptr, colp)

    def knn(self, queries, k: int, nthreads: int = 0):
        """(idx, d2) by the best-first priority queue of section 3.3."""
        q = _f32x3(queries)
        idx = np.empty((len(q), k), np.int32)
        d2 = np.empty((len(q), k), np.float32)
        self._lib.orc_knn_tree(self._t, _ptr(q), len(q), int(k), int(nthreads), _ptr(idx), _ptr(d2))
        return idx, d2


# ----------------------------------------------------------------------------- section 5.2
def locality_histogram(nbr_pos, row_pos, n: int) -> np.ndarray:
    """H_k(d), d = 0..n-1, from neighbour storage positions (rows) and row positions."""
    nbr = np.ascontiguousarray(nbr_pos, dtype=np.int64)
    rows = np.ascontiguousarray(row_pos, dtype=np.int64)
    hist = np.empty(n, np.int64)
    _load().orc_locality_histogram(_ptr(nbr), nbr.shape[0], nbr.shape[1], _ptr(rows), n, _ptr(hist))
    return hist


def skewness(hist) -> float:
    """Section 5.2: the Fisher-Pearson coefficient G1 = E[((d - mu) / sigma)^3] of the
    distribution with frequencies hist[d], d = 0, 1, ... (float64; 0 when sigma = 0)."""
    h = np.asarray(hist, dtype=np.float64)
    d = np.arange(len(h), dtype=np.float64)
    w = h.sum()
    if w == 0:
        return 0.0
    mu = (h * d).sum() / w
    x = d - mu
    m2 = (h * x * x).sum() / w
    m3 = (h * x * x * x).sum() / w
    return float(m3 / m2 ** 1.5) if m2 > 0 else 0.0


# ----------------------------------------------------------------------------- section 5.1 range output
def runs_of_rows(row_ptr, positions) -> tuple[np.ndarray, np.ndarray]:
    """Every row's neighbours, given as ascending sorted positions, as the maximal runs
    [start, end) of consecutive positions (run_ptr[rows + 1], runs[n_runs, 2])."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    pos = np.asarray(positions, dtype=np.int64)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    new = np.ones(len(pos), bool)
    if len(pos) > 1:
        new[1:] = (rows[1:] != rows[:-1]) | (pos[1:] != pos[:-1] + 1)
    first = np.flatnonzero(new)
    last = np.append(first[1:], len(pos)) - 1
    runs = np.stack([pos[first], pos[last] + 1], axis=1) if len(pos) else np.zeros((0, 2), np.int64)
    run_ptr = np.zeros(len(rp), np.int64)
    np.add.at(run_ptr, rows[first] + 1, 1)
    return np.cumsum(run_ptr), runs


# ----------------------------------------------------------------------------- whole pipeline
class Pipeline:
    """The full reference pipeline for one cloud: bbox, cells, codes, order, leaves, tree."""

    def __init__(self, xyz, enc: int, ncap: int):
        self.xyz = _f32x3(xyz)
        self.enc = int(enc)
        self.ncap = int(ncap)
        self.lo, self.ext, self.scale = bbox(self.xyz)
        self.cell = discretise(self.xyz, self.lo, self.scale)
        tree_enc = ENC_MORTON if self.enc == ENC_NONE else self.enc
        self.keys = encode_cells(self.cell, tree_enc)
        self.perm, self.sorted_keys = sort_keys(self.keys)
        self.rank = np.empty(len(self.perm), np.int64)
        self.rank[self.perm.astype(np.int64)] = np.arange(len(self.perm))
        self.leaves, self.counts = leaves(self.sorted_keys, self.ncap)
        self.tree = PointerOctree(self.xyz, self.ncap, cell=self.cell)

    def nodes(self) -> dict:
        tree_enc = ENC_MORTON if self.enc == ENC_NONE else self.enc
        return self.tree.nodes(tree_enc, self.perm, self.sorted_keys)

    def radius_runs(self, queries, r: float, kern: int, nthreads: int = 0):
        """The range output of the fixed-radius search: every row's neighbours (the naive
        octree search) as maximal runs of consecutive sorted positions."""
        rp, cols = self.tree.radius(queries, r, kern, nthreads)
        pos = self.rank[self.rows_by_rank(rp, cols).astype(np.int64)]
        return runs_of_rows(rp, pos)

    def neighbours_struct(self, centre, r: float, kern: int) -> list:
        """Section 5.1 neighboursStruct for one centre, step by step on the pointer octree:
        a branch wholly inside the kernel contributes its index range (step 1a with the
        range insertion), a disjoint branch is pruned (1b), any other branch is searched
        (1c); a leaf contributes each point inside the kernel (step 2).  Containment and
        disjointness are decided on the node's tight box: the corner farthest from the
        centre inside the kernel, the point of the box nearest to it outside.  Returns the
        (start, end) entries in walk order (sorted positions)."""
        if not hasattr(self, "_node_index"):
            nd = self.nodes()
            self._nodes = nd
            self._node_index = {(int(k), int(l)): i for i, (k, l) in enumerate(zip(nd["key"], nd["level"]))}
        nd, index = self._nodes, self._node_index
        c = np.asarray(centre, dtype=np.float32)
        out = []

        def visit(i):
            if nd["count"][i] == 0:
                return
            start, end = int(nd["start"][i]), int(nd["end"][i])
            if nd["is_leaf"][i]:
                for p in range(start, end):
                    if pred(kern, self.xyz[self.perm[p]], c, r):
                        out.append((p, p + 1))
                return
            lo, hi = nd["box"][i, :3], nd["box"][i, 3:]
            far = np.where(np.abs(hi - c) >= np.abs(lo - c), hi, lo).astype(np.float32)
            near = np.minimum(np.maximum(c, lo), hi).astype(np.float32)
            if pred(kern, far, c, r):
                out.append((start, end))
                return
            if not pred(kern, near, c, r):
                return
            level = int(nd["level"][i])
            shift = 3 * (L - level - 1)
            for digit in range(8):
                j = index.get((int(nd["key"][i]) + (digit << shift), level + 1))
                if j is not None:
                    visit(j)

        visit(index[(0, 0)])
        return out

    def locality(self, centre_ids, k: int, order: int):
        """Section 5.2: H_k of the given centres (original ids) and its skewness G1, with
        the storage positions of `order` (ENC_NONE: original index; a curve: rank in the
        stable order of its codes of this cloud's cells)."""
        ids = np.asarray(centre_ids, dtype=np.int64)
        nbr, _ = self.tree.knn(self.xyz[ids], k)
        if order == ENC_NONE:
            rank = np.arange(len(self.xyz), dtype=np.int64)
        else:
            perm, _ = sort_keys(encode_cells(self.cell, order))
            rank = np.empty(len(perm), np.int64)
            rank[perm.astype(np.int64)] = np.arange(len(perm))
        nb = nbr.astype(np.int64)
        pos = np.where(nb >= 0, rank[np.maximum(nb, 0)], -1)
        hist = locality_histogram(pos, rank[ids], len(self.xyz))
        return hist, skewness(hist)

    def rows_by_rank(self, row_ptr, cols) -> np.ndarray:
        """Reorder every row by the sorted position of its points (the CUDA path's row order)."""
        cols = np.asarray(cols, dtype=np.int64)
        out = np.empty_like(cols)
        rp = np.asarray(row_ptr, dtype=np.int64)
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        order = np.lexsort((self.rank[cols] if len(cols) else cols, rows))
        out[:] = cols[order]
        return out.astype(np.int32)
