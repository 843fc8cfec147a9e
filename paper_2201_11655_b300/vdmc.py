"""Thin Python binding of the C ABI in ``include/vdmc.h`` (argument marshalling only).

Every step of the counting runs in ``libvdmc.so``; this module converts torch
tensors / numpy arrays into pointers, sizes and a ``cudaStream_t`` and
checks status codes.  There is no CPU fallback: if the library or a CUDA
device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvdmc.so")

VDMC_OK = 0
STATUS_NAMES = {
    0: "VDMC_OK", 1: "VDMC_ERR_INVALID_ARG", 2: "VDMC_ERR_OUT_OF_RANGE_VERTEX", 3: "VDMC_ERR_OOM",
    4: "VDMC_ERR_CUDA", 5: "VDMC_ERR_DEVICE_LIMIT", 6: "VDMC_ERR_BUSY",
}


class VdmcError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        msg = _lib().vdmc_status_string(int(status)).decode() if _LIB is not None else str(status)
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(int(status), status), msg))


class GraphInfo(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32), ("max_degree", ctypes.c_int32), ("arcs_in", ctypes.c_int64),
        ("self_loops", ctypes.c_int64), ("duplicate_arcs", ctypes.c_int64), ("arcs_kept", ctypes.c_int64),
        ("edges_u", ctypes.c_int64), ("reciprocal_pairs", ctypes.c_int64), ("num_tasks", ctypes.c_int64),
        ("num_hub_roots", ctypes.c_int64), ("num_graphs", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Schedule(ctypes.Structure):
    _fields_ = [("a_chunk", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("hub_min_l", ctypes.c_int32),
                ("hub_blocks_per_sm", ctypes.c_int32), ("hub_split", ctypes.c_int32),
                ("hub_split_roots", ctypes.c_int32), ("hub_warps", ctypes.c_int32), ("d3_bits", ctypes.c_int32)]


class WorkModel(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "bytes", "bytes_per_use", "entries_root", "entries_depth1", "entries_depth2", "entries_depth2_per_use",
        "output_bytes")]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class CountStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "sets_plain", "sets_hub", "sets_hub_enumerated", "sets_by_signature", "sets_enumerated")]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


SCHEDULE_KEYS = ("a_chunk", "warps_per_block", "blocks_per_sm", "hub_min_l", "hub_blocks_per_sm", "hub_split",
                 "hub_split_roots", "hub_warps", "d3_bits")


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libvdmc.so not built (%s); run paper_2201_11655_b300.build" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "vdmc_graph_create": ([i32, i64, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)], ctypes.c_int),
            "vdmc_graph_create_ex": ([i32, i64, vp, vp, ctypes.c_int, ctypes.c_uint32, vp, ctypes.POINTER(vp)],
                                     ctypes.c_int),
            "vdmc_num_classes_undirected": ([ctypes.c_int], ctypes.c_int),
            "vdmc_undirected_class_masks": ([ctypes.c_int, vp], ctypes.c_int),
            "vdmc_graph_num_classes": ([vp, ctypes.c_int], ctypes.c_int),
            "vdmc_count_edges": ([vp, ctypes.c_int, vp, vp], ctypes.c_int),
            "vdmc_graph_edges": ([vp, vp, vp, vp], ctypes.c_int),
            "vdmc_graph_destroy": ([vp], ctypes.c_int),
            "vdmc_graph_create_batch": ([ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)],
                                        ctypes.c_int),
            "vdmc_count_csr_noalloc": ([i32, i64, vp, vp, vp, vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
            "vdmc_graph_info": ([vp, ctypes.POINTER(GraphInfo)], ctypes.c_int),
            "vdmc_graph_export_csr": ([vp, vp, vp, vp], ctypes.c_int),
            "vdmc_num_classes": ([ctypes.c_int], ctypes.c_int),
            "vdmc_class_masks": ([ctypes.c_int, vp], ctypes.c_int),
            "vdmc_class_lut": ([ctypes.c_int, vp], ctypes.c_int),
            "vdmc_count": ([vp, ctypes.c_int, vp, vp], ctypes.c_int),
            "vdmc_count_roots": ([vp, ctypes.c_int, i32, i32, vp, vp], ctypes.c_int),
            "vdmc_count_batch": ([vp, ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
            "vdmc_get_device_status": ([vp], ctypes.c_int),
            "vdmc_work_bytes": ([vp, ctypes.c_int, vp], ctypes.c_int),
            "vdmc_work_model": ([vp, ctypes.c_int, ctypes.POINTER(WorkModel)], ctypes.c_int),
            "vdmc_count_stats": ([vp, ctypes.POINTER(CountStats)], ctypes.c_int),
            "vdmc_root_costs": ([vp, ctypes.c_int, vp, vp], ctypes.c_int),
            "vdmc_set_schedule": ([ctypes.POINTER(Schedule)], ctypes.c_int),
            "vdmc_get_schedule": ([ctypes.POINTER(Schedule)], ctypes.c_int),
            "vdmc_status_string": ([ctypes.c_int], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = lib
    return _LIB


def load():
    """Load libvdmc.so (raises if it is missing) and return the ctypes handle."""
    return _lib()


def _check(st, where):
    if st != VDMC_OK:
        raise VdmcError(st, where)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def num_classes(k: int) -> int:
    return _lib().vdmc_num_classes(k)


def class_masks(k: int) -> np.ndarray:
    nc = num_classes(k)
    if nc < 0:
        raise ValueError("k must be 3 or 4")
    out = np.zeros(nc, np.uint16)
    _check(_lib().vdmc_class_masks(k, out.ctypes.data), "vdmc_class_masks")
    return out


def num_classes_undirected(k: int) -> int:
    return _lib().vdmc_num_classes_undirected(k)


def undirected_class_masks(k: int) -> np.ndarray:
    nc = num_classes_undirected(k)
    if nc < 0:
        raise ValueError("k must be 3 or 4")
    out = np.zeros(nc, np.uint16)
    _check(_lib().vdmc_undirected_class_masks(k, out.ctypes.data), "vdmc_undirected_class_masks")
    return out


def class_lut(k: int) -> np.ndarray:
    """Output column of every motif index (255 = not weakly connected)."""
    if k not in (3, 4):
        raise ValueError("k must be 3 or 4")
    out = np.zeros(1 << (k * (k - 1)), np.uint8)
    _check(_lib().vdmc_class_lut(k, out.ctypes.data), "vdmc_class_lut")
    return out


class Graph:
    """A device graph built by ``vdmc_graph_create``; freed by ``close()``."""

    def __init__(self, handle, n, undirected=False):
        self._h = handle
        self.n = n
        self.undirected = undirected

    def num_classes(self, k: int) -> int:
        """Columns of this graph's counts (directed or undirected classes)."""
        nc = _lib().vdmc_graph_num_classes(self.handle, int(k))
        if nc < 0:
            raise ValueError("k must be 3 or 4")
        return nc

    def edges(self):
        """(u, v, flags) of the rows of per-edge counts: u < v original ids, ascending."""
        ne = self.info()["edges_u"]
        u = np.zeros(ne, np.int32)
        v = np.zeros(ne, np.int32)
        f = np.zeros(ne, np.uint8)
        _check(_lib().vdmc_graph_edges(self.handle, u.ctypes.data, v.ctypes.data, f.ctypes.data), "vdmc_graph_edges")
        return u, v, f

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("graph is closed")
        return self._h

    def info(self) -> dict:
        inf = GraphInfo()
        _check(_lib().vdmc_graph_info(self.handle, ctypes.byref(inf)), "vdmc_graph_info")
        return inf.as_dict()

    def export_csr(self):
        info = self.info()
        rowptr = np.zeros(self.n + 1, np.int64)
        col = np.zeros(2 * info["edges_u"], np.uint32)
        new2old = np.zeros(self.n, np.int32)
        _check(_lib().vdmc_graph_export_csr(self.handle, rowptr.ctypes.data, col.ctypes.data,
                                            new2old.ctypes.data), "vdmc_graph_export_csr")
        return rowptr, col, new2old

    def work_bytes(self, k: int) -> int:
        """Algorithmic bytes of one count (the roofline numerator)."""
        b = np.zeros(1, np.uint64)
        _check(_lib().vdmc_work_bytes(self.handle, int(k), b.ctypes.data), "vdmc_work_bytes")
        return int(b[0])

    def work_model(self, k: int) -> dict:
        """The algorithmic byte model of one count (vdmc_work_model_t as a dict)."""
        m = WorkModel()
        _check(_lib().vdmc_work_model(self.handle, int(k), ctypes.byref(m)), "vdmc_work_model")
        return m.as_dict()

    def count_stats(self) -> dict:
        """Sets found one by one vs by signature in the last count (vdmc_count_stats_t)."""
        st = CountStats()
        _check(_lib().vdmc_count_stats(self.handle, ctypes.byref(st)), "vdmc_count_stats")
        return st.as_dict()

    def device_status(self) -> int:
        return _lib().vdmc_get_device_status(self.handle)

    def close(self):
        if self._h is not None:
            _check(_lib().vdmc_graph_destroy(self._h), "vdmc_graph_destroy")
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def graph_create(n: int, src, dst, stream=None, undirected: bool = False) -> Graph:
    """Build a graph from arcs src[e] -> dst[e] (int32; numpy/CPU tensors or CUDA tensors).

    undirected=True: count the undirected motifs of G_U (arc directions ignored)."""
    import torch
    lib = _lib()
    on_device = 0
    keep = []
    if isinstance(src, torch.Tensor) and src.is_cuda:
        s = src.to(torch.int32).contiguous()
        d = dst.to(device=s.device, dtype=torch.int32).contiguous()
        on_device = 1
        keep += [s, d]
        ps, pd, m = s.data_ptr(), d.data_ptr(), s.numel()
    else:
        s = np.ascontiguousarray(np.asarray(src.cpu() if isinstance(src, torch.Tensor) else src, dtype=np.int32))
        d = np.ascontiguousarray(np.asarray(dst.cpu() if isinstance(dst, torch.Tensor) else dst, dtype=np.int32))
        keep += [s, d]
        ps, pd, m = s.ctypes.data, d.ctypes.data, s.size
    if (d.numel() if on_device else d.size) != m:
        raise ValueError("src and dst differ in length")
    h = ctypes.c_void_p()
    _check(lib.vdmc_graph_create_ex(int(n), int(m), ctypes.c_void_p(ps), ctypes.c_void_p(pd), on_device,
                                    1 if undirected else 0, _stream_ptr(stream), ctypes.byref(h)),
           "vdmc_graph_create_ex")
    return Graph(h, int(n), undirected)


def graph_create_batch(graphs, stream=None) -> Graph:
    """Build the disjoint union of many graphs [(n, src, dst), ...] (local ids) as one device graph.

    Graph i's counts are rows offsets[i] .. offsets[i+1]-1 of a count on the
    returned graph; ``Graph.offsets`` holds those offsets."""
    lib = _lib()
    num = len(graphs)
    ns = np.array([int(g[0]) for g in graphs], dtype=np.int32)
    ms = np.array([len(g[1]) for g in graphs], dtype=np.int64)
    src = np.ascontiguousarray(np.concatenate([np.asarray(g[1], np.int32) for g in graphs]) if num else
                               np.zeros(0, np.int32))
    dst = np.ascontiguousarray(np.concatenate([np.asarray(g[2], np.int32) for g in graphs]) if num else
                               np.zeros(0, np.int32))
    h = ctypes.c_void_p()
    _check(lib.vdmc_graph_create_batch(num, ns.ctypes.data, ms.ctypes.data, src.ctypes.data, dst.ctypes.data, 0,
                                       _stream_ptr(stream), ctypes.byref(h)), "vdmc_graph_create_batch")
    g = Graph(h, int(ns.sum()))
    g.offsets = np.concatenate([[0], np.cumsum(ns.astype(np.int64))])
    return g


def _out_tensor(g: Graph, k: int, out, rows=None):
    import torch
    if k not in (3, 4):
        raise ValueError("k must be 3 or 4")
    nc = g.num_classes(k)
    rows = g.n if rows is None else rows
    if out is None:
        out = torch.empty((rows, nc), dtype=torch.uint64, device="cuda")
    if out.dtype != torch.uint64 or not out.is_cuda or out.numel() != rows * nc or not out.is_contiguous():
        raise ValueError("out must be a contiguous CUDA uint64 tensor of %d x %d elements" % (rows, nc))
    return out


def count(g: Graph, k: int, out=None, stream=None):
    """Per-vertex counts, uint64[n, C_k] CUDA tensor (overwritten)."""
    out = _out_tensor(g, k, out)
    _check(_lib().vdmc_count(g.handle, int(k), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)), "vdmc_count")
    return out


def count_edges(g: Graph, k: int, out=None, stream=None):
    """Per-edge counts, uint64[edges_u, columns] CUDA tensor (rows: Graph.edges() order)."""
    out = _out_tensor(g, k, out, rows=g.info()["edges_u"])
    _check(_lib().vdmc_count_edges(g.handle, int(k), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
           "vdmc_count_edges")
    return out


def count_roots(g: Graph, k: int, rank_lo: int, rank_hi: int, out=None, stream=None):
    """Counts of the sets whose lowest-rank member has rank in [rank_lo, rank_hi)."""
    out = _out_tensor(g, k, out)
    _check(_lib().vdmc_count_roots(g.handle, int(k), int(rank_lo), int(rank_hi), ctypes.c_void_p(out.data_ptr()),
                                   _stream_ptr(stream)), "vdmc_count_roots")
    return out


def count_batch(graphs, k: int, outs=None, stream=None):
    """Count many graphs in one launch; returns the list of output tensors."""
    outs = [_out_tensor(g, k, None if outs is None else outs[i]) for i, g in enumerate(graphs)]
    num = len(graphs)
    harr = (ctypes.c_void_p * max(num, 1))(*[g.handle.value for g in graphs])
    oarr = (ctypes.c_void_p * max(num, 1))(*[o.data_ptr() for o in outs])
    _check(_lib().vdmc_count_batch(harr, num, int(k), oarr, _stream_ptr(stream)), "vdmc_count_batch")
    return outs


def set_schedule(**kw):
    """Set any of the launch-schedule knobs (see vdmc_schedule_t); the rest keep their values."""
    bad = set(kw) - set(SCHEDULE_KEYS)
    if bad:
        raise TypeError("unknown schedule keys %s" % sorted(bad))
    cur = get_schedule()
    cur.update({k: v for k, v in kw.items() if v is not None})
    s = Schedule(*[int(cur[k]) for k in SCHEDULE_KEYS])
    _check(_lib().vdmc_set_schedule(ctypes.byref(s)), "vdmc_set_schedule")


def get_schedule() -> dict:
    s = Schedule()
    _check(_lib().vdmc_get_schedule(ctypes.byref(s)), "vdmc_get_schedule")
    return {k: getattr(s, k) for k in SCHEDULE_KEYS}
