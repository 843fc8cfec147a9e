"""Python entry points of the CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this module.  It loads ``liboracle.so`` built from
``vdmc_oracle.c`` in this folder (plain C, no GPU code), and adds the
G(n, p) expectation of Eq. 4.  Nothing here is shared with, or imported by,
the CUDA library or its Python binding.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vdmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        lib.oracle_canonical_index.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_canonical_index.restype = ctypes.c_int
        lib.oracle_classes.argtypes = [ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_uint16),
                                       ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        lib.oracle_classes.restype = ctypes.c_int
        lib.oracle_count_esu.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int,
                                         i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int, u64p]
        lib.oracle_count_esu.restype = ctypes.c_int64
        lib.oracle_count_esu_masked.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int, i32p,
                                                ctypes.POINTER(ctypes.c_uint8), ctypes.c_int, u64p]
        lib.oracle_count_esu_masked.restype = ctypes.c_int64
        lib.oracle_classes_undirected.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint16),
                                                  ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        lib.oracle_classes_undirected.restype = ctypes.c_int
        lib.oracle_count_mode.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, i32p, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int, u64p]
        lib.oracle_count_mode.restype = ctypes.c_int64
        lib.oracle_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p]
        lib.oracle_edges.restype = ctypes.c_int64
        lib.oracle_count_brute.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int, u64p]
        lib.oracle_count_brute.restype = ctypes.c_int64
        lib.oracle_degree_rank.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p]
        lib.oracle_degree_rank.restype = ctypes.c_int
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def canonical_index(k: int, idx: int) -> int:
    """Minimum motif index over all k! vertex orderings (Fig. 1: 53 -> 30)."""
    return int(_load().oracle_canonical_index(k, idx))


def classes(k: int, connected_only: bool = True):
    """(canonical indices ascending, number of labelled isomorphs N_Iso) per class."""
    lib = _load()
    cap = 512
    canon = np.zeros(cap, np.uint16)
    niso = np.zeros(cap, np.uint32)
    nc = lib.oracle_classes(k, 1 if connected_only else 0, _ptr(canon, ctypes.c_uint16),
                            _ptr(niso, ctypes.c_uint32), cap)
    if nc < 0:
        raise ValueError("k must be 2..4")
    return canon[:nc].astype(np.int64), niso[:nc].astype(np.int64)


def num_classes(k: int) -> int:
    return len(classes(k)[0])


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def count(n, src, dst, k, threads: int | None = None):
    """Per-vertex counts uint64[n, C_k] by ESU over every connected k-set.

    Returns (counts, number_of_sets)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    nc = num_classes(k)
    out = np.zeros((n, nc), np.uint64)
    got = lib.oracle_count_esu(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32), k,
                               None, 0, 0, threads or default_threads(), _ptr(out, ctypes.c_uint64))
    if got < 0:
        raise ValueError("oracle_count_esu failed (%d)" % got)
    return out, int(got)


def degree_rank(n, src, dst):
    """rank[v]: position of v in the order (undirected degree desc, id asc)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    rank = np.zeros(n, np.int32)
    rc = lib.oracle_degree_rank(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32),
                                _ptr(rank, ctypes.c_int32))
    if rc:
        raise ValueError("oracle_degree_rank failed (%d)" % rc)
    return rank


def count_roots(n, src, dst, k, rank, lo, hi, threads: int | None = None):
    """Counts over the connected k-sets whose lowest-rank member has rank in [lo, hi)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    rank = _i32(rank)
    nc = num_classes(k)
    out = np.zeros((n, nc), np.uint64)
    got = lib.oracle_count_esu(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32), k,
                               _ptr(rank, ctypes.c_int32), int(lo), int(hi),
                               threads or default_threads(), _ptr(out, ctypes.c_uint64))
    if got < 0:
        raise ValueError("oracle_count_esu failed (%d)" % got)
    return out, int(got)


def count_root_ranges(n, src, dst, k, rank, ranges, threads: int | None = None):
    """Counts over the connected k-sets whose lowest-rank member has rank in any of
    the disjoint ``ranges`` [(lo, hi), ...] (one graph build for all of them)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    rank = _i32(rank)
    mask = np.zeros(n, np.uint8)
    for lo, hi in ranges:
        mask[(rank >= lo) & (rank < hi)] = 1
    nc = num_classes(k)
    out = np.zeros((n, nc), np.uint64)
    got = lib.oracle_count_esu_masked(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32), k,
                                      _ptr(rank, ctypes.c_int32), _ptr(mask, ctypes.c_uint8),
                                      threads or default_threads(), _ptr(out, ctypes.c_uint64))
    if got < 0:
        raise ValueError("oracle_count_esu_masked failed (%d)" % got)
    return out, int(got)


def classes_undirected(k: int):
    """Undirected connected classes: (minimum symmetric indices ascending, labelled graphs per class)."""
    lib = _load()
    cap = 64
    canon = np.zeros(cap, np.uint16)
    niso = np.zeros(cap, np.uint32)
    nc = lib.oracle_classes_undirected(k, _ptr(canon, ctypes.c_uint16), _ptr(niso, ctypes.c_uint32), cap)
    if nc < 0:
        raise ValueError("k must be 2..4")
    return canon[:nc].astype(np.int64), niso[:nc].astype(np.int64)


def edges(n, src, dst):
    """Edges {u, v} of G_U, u < v, in (u, v) order: the rows of per-edge counts. Returns (u, v)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    ne = lib.oracle_edges(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32), None, None)
    if ne < 0:
        raise ValueError("oracle_edges failed (%d)" % ne)
    u = np.zeros(ne, np.int32)
    v = np.zeros(ne, np.int32)
    lib.oracle_edges(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32), _ptr(u, ctypes.c_int32),
                     _ptr(v, ctypes.c_int32))
    return u, v


def count_mode(n, src, dst, k, undirected=False, per_edge=False, rank=None, ranges=None,
               threads: int | None = None):
    """Counts of the undirected and/or per-edge variants.

    Rows: vertices, or the edges of G_U in the order of :func:`edges` when
    per_edge; columns: the directed classes, or :func:`classes_undirected`
    when undirected.  With rank and ranges: only the sets whose lowest-rank
    member has rank in one of the ranges.  Returns (counts, number_of_sets)."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    nc = len(classes_undirected(k)[0]) if undirected else num_classes(k)
    rows = len(edges(n, src, dst)[0]) if per_edge else n
    out = np.zeros((rows, nc), np.uint64)
    key = mask = None
    if ranges is not None:
        key = _i32(rank)
        m8 = np.zeros(n, np.uint8)
        for lo, hi in ranges:
            m8[(key >= lo) & (key < hi)] = 1
        mask = _ptr(m8, ctypes.c_uint8)
    got = lib.oracle_count_mode(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32), k,
                                1 if undirected else 0, 1 if per_edge else 0,
                                _ptr(key, ctypes.c_int32) if key is not None else None, mask,
                                threads or default_threads(), _ptr(out, ctypes.c_uint64))
    if got < 0:
        raise ValueError("oracle_count_mode failed (%d)" % got)
    return out, int(got)


def count_brute(n, src, dst, k):
    """Per-vertex counts by brute force over all C(n, k) vertex subsets."""
    lib = _load()
    src, dst = _i32(src), _i32(dst)
    nc = num_classes(k)
    out = np.zeros((n, nc), np.uint64)
    got = lib.oracle_count_brute(n, src.size, _ptr(src, ctypes.c_int32), _ptr(dst, ctypes.c_int32), k,
                                 _ptr(out, ctypes.c_uint64))
    if got < 0:
        raise ValueError("oracle_count_brute failed (%d)" % got)
    return out, int(got)


def motif_edges(k: int, idx: int) -> int:
    """n_e(m): number of arcs of a motif = number of set bits of its index."""
    return bin(int(idx)).count("1")


def gnp_expected_local(n: int, p: float, k: int, undirected: bool = False):
    """Eq. 4: E[X_{k,m}(i)] = C(n-1, k-1) * N_Iso(m) * p^{n_e} * (1-p)^{n_max - n_e}.

    n_max(k) = k(k-1) for directed graphs and C(k, 2) for undirected ones
    (the text after Eq. 4's definitions); for an undirected motif n_e is its
    number of edges, half the set bits of its symmetric index.  Returns a
    float64 array over the connected classes."""
    canon, niso = classes_undirected(k) if undirected else classes(k)
    nmax = k * (k - 1) // 2 if undirected else k * (k - 1)
    ne = np.array([motif_edges(k, c) for c in canon], dtype=np.float64) / (2.0 if undirected else 1.0)
    return math.comb(n - 1, k - 1) * niso * (p ** ne) * ((1 - p) ** (nmax - ne))
