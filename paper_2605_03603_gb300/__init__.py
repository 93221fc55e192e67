"""Balanced (p,q)-biclique counting in signed bipartite graphs on GB300.

Thin ctypes binding over libsbc.so (include/sbc.h): the same entry points,
argument marshalling only. Every step of the count runs in the library's CUDA
kernels; there is no CPU fallback, and importing this package fails loudly if
the library has not been built (`paper_2605_03603_gb300.build.build()`).

PyTorch is used only to hand over device memory and streams: device inputs
may be torch CUDA tensors, and `stream` may be a torch.cuda.Stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "SbcError", "Graph", "sbc_graph_create", "sbc_graph_destroy", "sbc_graph_info",
    "sbc_count", "sbc_count_ex", "sbc_count_csr", "sbc_last_error", "sbc_version",
    "sbc_launch_count", "sbc_count_csr_noalloc", "sbc_count_batch", "Batch", "Server",
    "lib", "LIB_PATH",
]

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libsbc.so is not built ({LIB_PATH}); run paper_2605_03603_gb300.build.build() "
        "(nvcc for sm_103a) first. There is no CPU fallback."
    )

lib = ctypes.CDLL(LIB_PATH)

SBC_OFFS_I64 = 1
SBC_SIGN_BITS = 2
SBC_DEVICE_PTRS = 4
SBC_SIDE_AUTO, SBC_SIDE_U, SBC_SIDE_V = -1, 0, 1
SBC_COUNT_PAPER_TUPLES = 1
SBC_COUNT_CANDIDATE_SIDE = 2
SBC_COUNT_POSITION_SIDE = 4
SBC_COUNT_CHECK = 8

STATUS = {0: "SBC_OK", 1: "SBC_E_INVAL", 2: "SBC_E_GRAPH", 3: "SBC_E_NOMEM", 4: "SBC_E_CUDA",
          5: "SBC_E_TIMEOUT", 6: "SBC_E_BUSY", 7: "SBC_E_UNSUPPORTED", 8: "SBC_E_OVERFLOW"}


class U128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]

    def value(self) -> int:
        return int(self.lo) | (int(self.hi) << 64)


class GraphInfo(ctypes.Structure):
    _fields_ = [("n_u", ctypes.c_int64), ("n_v", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("max_deg_u", ctypes.c_int64), ("max_deg_v", ctypes.c_int64),
                ("wedges_anchor_u", ctypes.c_uint64), ("wedges_anchor_v", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64)]


class Tune(ctypes.Structure):
    """sbc_tune_t: launch parameters of the counting kernels (0 = default)."""
    _fields_ = [("small_wedges", ctypes.c_int32), ("pos_node_cost", ctypes.c_int32),
                ("split_per_warp", ctypes.c_int32), ("tc_min_words", ctypes.c_int32),
                ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {"small_wedges": int(self.small_wedges), "pos_node_cost": int(self.pos_node_cost),
                "split_per_warp": int(self.split_per_warp), "tc_min_words": int(self.tc_min_words),
                "ms": float(self.ms)}


def _tune(t) -> "Tune | None":
    if t is None:
        return None
    if isinstance(t, Tune):
        return t
    return Tune(int(t.get("small_wedges", 0)), int(t.get("pos_node_cost", 0)),
                int(t.get("split_per_warp", 0)), int(t.get("tc_min_words", 0)), 0.0)


class CountOpts(ctypes.Structure):
    _fields_ = [("anchor_side", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("per_anchor", ctypes.c_void_p), ("shard", ctypes.c_int32),
                ("shard_count", ctypes.c_int32), ("tune", ctypes.POINTER(Tune))]


class CountStats(ctypes.Structure):
    _fields_ = [("count", U128), ("anchor_tuples", U128), ("candidates", ctypes.c_uint64),
                ("wedges", ctypes.c_uint64), ("work_items", ctypes.c_uint64),
                ("tuples_tested", ctypes.c_uint64), ("tuples_typed", ctypes.c_uint64),
                ("popc_words", ctypes.c_uint64),
                ("anchor_side", ctypes.c_int32), ("kernels", ctypes.c_int32),
                ("ms_prepare", ctypes.c_float), ("ms_twohop", ctypes.c_float),
                ("ms_tuples", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ms_tc", ctypes.c_float), ("tc_anchors", ctypes.c_uint64),
                ("tc_tiles", ctypes.c_uint64), ("tc_kblocks", ctypes.c_uint64),
                ("twohop_reads", ctypes.c_uint64), ("twohop_anchors", ctypes.c_uint64 * 4),
                ("twohop_share", ctypes.c_float * 4), ("twohop_tail_ms", ctypes.c_float),
                ("pool_bytes", ctypes.c_uint64), ("twohop_split_classes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {"count": self.count.value(), "anchor_tuples": self.anchor_tuples.value(),
                "candidates": int(self.candidates), "wedges": int(self.wedges),
                "work_items": int(self.work_items), "tuples_tested": int(self.tuples_tested),
                "tuples_typed": int(self.tuples_typed), "popc_words": int(self.popc_words),
                "anchor_side": int(self.anchor_side),
                "kernels": int(self.kernels), "ms_prepare": float(self.ms_prepare),
                "ms_twohop": float(self.ms_twohop), "ms_tuples": float(self.ms_tuples),
                "ms_total": float(self.ms_total), "ms_tc": float(self.ms_tc),
                "tc_anchors": int(self.tc_anchors), "tc_tiles": int(self.tc_tiles),
                "tc_kblocks": int(self.tc_kblocks), "twohop_reads": int(self.twohop_reads),
                "twohop_anchors": [int(x) for x in self.twohop_anchors],
                "twohop_share": [round(float(x), 4) for x in self.twohop_share],
                "twohop_tail_ms": float(self.twohop_tail_ms), "pool_bytes": int(self.pool_bytes),
                "twohop_split_classes": int(self.twohop_split_classes)}


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def _declare(name, restype, argtypes):
    fn = getattr(lib, name)
    fn.restype = restype
    fn.argtypes = argtypes
    return fn


_declare("sbc_graph_create", ctypes.c_int,
         [ctypes.POINTER(_vp), _i64, _i64, _i64, _vp, _vp, _vp, ctypes.c_uint32, _vp])
_declare("sbc_graph_destroy", ctypes.c_int, [_vp])
_declare("sbc_graph_info", ctypes.c_int, [_vp, ctypes.POINTER(GraphInfo)])
_declare("sbc_count", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(U128), _vp])
_declare("sbc_count_ex", ctypes.c_int,
         [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(CountOpts), ctypes.POINTER(CountStats), _vp])
_declare("sbc_count_csr", ctypes.c_int,
         [_i64, _i64, _i64, _vp, _vp, _vp, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
          ctypes.POINTER(U128), _vp])
_declare("sbc_last_error", ctypes.c_char_p, [])
_declare("sbc_version", ctypes.c_char_p, [])
_declare("sbc_launch_count", ctypes.c_uint64, [])
_declare("sbc_count_batch", ctypes.c_int,
         [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(U128), _vp])
_declare("sbc_batch_create", ctypes.c_int,
         [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp), _vp])
_declare("sbc_batch_create_ex", ctypes.c_int,
         [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Tune),
          ctypes.POINTER(_vp), _vp])
_declare("sbc_autotune", ctypes.c_int,
         [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int32,
          ctypes.POINTER(Tune), _vp])
_declare("sbc_autotune_cached", ctypes.c_int,
         [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int32,
          ctypes.c_char_p, ctypes.POINTER(Tune), ctypes.POINTER(ctypes.c_int32), _vp])
_declare("sbc_batch_run", ctypes.c_int, [_vp, ctypes.POINTER(U128), _vp])
_declare("sbc_batch_destroy", ctypes.c_int, [_vp])


class ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("lanes", ctypes.c_int32),
                ("max_batch", ctypes.c_int32), ("small_edges", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("jobs", ctypes.c_uint64),
                ("fused_requests", ctypes.c_uint64), ("peak_admitted_bytes", ctypes.c_uint64),
                ("mem_budget_bytes", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("throughput_rps", ctypes.c_double)]


_declare("sbc_server_create", ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)])
_declare("sbc_server_add_graph", ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_uint32)])
_declare("sbc_server_submit", ctypes.c_int,
         [_vp, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)])
_declare("sbc_server_wait", ctypes.c_int,
         [_vp, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(U128), ctypes.POINTER(ctypes.c_double)])
_declare("sbc_server_stats", ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)])
_declare("sbc_server_reset_stats", ctypes.c_int, [_vp])
_declare("sbc_server_destroy", ctypes.c_int, [_vp])
_declare("sbc_measure_alu_rates", ctypes.c_int,
         [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _vp])


def sbc_measure_alu_rates(stream=None) -> dict:
    """Measured POPC and LOP3 rates of the current device (operations/s)."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib.sbc_measure_alu_rates(ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)))
    return {"popc_per_s": a.value, "lop3_per_s": b.value}


_declare("sbc_count_csr_noalloc", ctypes.c_int,
         [_i64, _i64, _i64, _vp, _vp, _vp, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
          ctypes.POINTER(U128), _vp])

# sbc_count_csr_noalloc limits (include/sbc.h)
SBC_NOALLOC_SCRATCH_BYTES = 32 << 20
SBC_NOALLOC_MAX_VERTICES = 65536
SBC_NOALLOC_MAX_EDGES = 65536


def sbc_launch_count() -> int:
    """Kernel launches issued by the library so far in this process."""
    return int(lib.sbc_launch_count())


class SbcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def sbc_last_error() -> str:
    return lib.sbc_last_error().decode()


def sbc_version() -> str:
    return lib.sbc_version().decode()


def _check(rc: int):
    if rc != 0:
        raise SbcError(rc, sbc_last_error())


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return getattr(stream, "cuda_stream", None)


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor."""
    if a is None:
        return None, False
    if isinstance(a, np.ndarray):
        return a.ctypes.data, False
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), bool(getattr(a, "is_cuda", False))
    raise TypeError(f"unsupported buffer type {type(a)}")


class Graph:
    """Owning handle of a device-resident graph (sbc_graph*)."""

    def __init__(self, handle: int, n_u: int, n_v: int, nnz: int):
        self.handle = handle
        self.n_u, self.n_v, self.nnz = n_u, n_v, nnz

    def close(self):
        if self.handle:
            _check(lib.sbc_graph_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sbc_graph_create(n_u: int, n_v: int, row_offsets, cols, signs, sign_bits: bool = False,
                     stream=None) -> Graph:
    """sbc_graph_create: signed CSR over U -> device graph.

    row_offsets int32/int64, cols int32, signs int8 (+1/-1) or packed uint8
    bits (sign_bits=True). numpy arrays are host memory; torch CUDA tensors are
    device memory (all three must be on the same side)."""
    off_p, off_dev = _ptr(row_offsets)
    col_p, col_dev = _ptr(cols)
    sg_p, sg_dev = _ptr(signs)
    nnz = int(cols.shape[0])
    flags = 0
    dt = str(getattr(row_offsets, "dtype", ""))
    if dt.endswith("int64"):
        flags |= SBC_OFFS_I64
    elif not dt.endswith("int32"):
        raise TypeError("row_offsets must be int32 or int64")
    if not str(getattr(cols, "dtype", "")).endswith("int32"):
        raise TypeError("cols must be int32")
    if sign_bits:
        flags |= SBC_SIGN_BITS
    if off_dev or col_dev or sg_dev:
        if not (off_dev and (col_dev or nnz == 0) and (sg_dev or nnz == 0)):
            raise ValueError("row_offsets, cols and signs must all be host or all be device")
        flags |= SBC_DEVICE_PTRS
    out = _vp()
    _check(lib.sbc_graph_create(ctypes.byref(out), n_u, n_v, nnz, off_p, col_p, sg_p, flags,
                                _stream_ptr(stream)))
    return Graph(out.value, n_u, n_v, nnz)


def sbc_graph_destroy(g: Graph):
    g.close()


def sbc_graph_info(g: Graph) -> dict:
    info = GraphInfo()
    _check(lib.sbc_graph_info(g.handle, ctypes.byref(info)))
    return {f: int(getattr(info, f)) for f, _ in GraphInfo._fields_}


def sbc_count(g: Graph, p: int, q: int, stream=None) -> int:
    """Exact number of balanced (p,q)-bicliques (p from U, q from V)."""
    out = U128()
    _check(lib.sbc_count(g.handle, p, q, ctypes.byref(out), _stream_ptr(stream)))
    return out.value()


def sbc_count_ex(g: Graph, p: int, q: int, anchor_side: int = SBC_SIDE_AUTO,
                 per_anchor: bool = False, paper_tuples: bool = False, shard: int = 0,
                 shard_count: int = 0, method: str = "auto", tune=None, stream=None,
                 check: bool = False):
    """sbc_count_ex: returns (count, stats dict, per-anchor list or None).
    method: "auto" (cheaper side per anchor), "candidate" or "position".
    tune: launch parameters (a dict with sbc_tune_t's fields, e.g. from
    sbc_autotune, or None for the defaults). check: device self-checks
    (SBC_COUNT_CHECK)."""
    opts = CountOpts()
    t = _tune(tune)
    if t is not None:
        opts.tune = ctypes.pointer(t)
    opts.anchor_side = anchor_side
    opts.flags = (SBC_COUNT_PAPER_TUPLES if paper_tuples else 0) | {
        "auto": 0, "candidate": SBC_COUNT_CANDIDATE_SIDE, "position": SBC_COUNT_POSITION_SIDE}[method]
    if check:
        opts.flags |= SBC_COUNT_CHECK
    opts.shard = shard
    opts.shard_count = shard_count
    per = None
    if per_anchor:
        # room for either side when the library picks it
        n_alloc = (max(g.n_u, g.n_v) if anchor_side == SBC_SIDE_AUTO
                   else (g.n_u if anchor_side == 0 else g.n_v))
        per = np.zeros(2 * max(n_alloc, 1), dtype=np.uint64)
        opts.per_anchor = per.ctypes.data
    st = CountStats()
    _check(lib.sbc_count_ex(g.handle, p, q, ctypes.byref(opts), ctypes.byref(st),
                            _stream_ptr(stream)))
    d = st.as_dict()
    pa = None
    if per is not None:
        n_side = g.n_u if d["anchor_side"] == 0 else g.n_v
        pa = [int(per[2 * i]) | (int(per[2 * i + 1]) << 64) for i in range(n_side)]
    return d["count"], d, pa


def sbc_count_csr(n_u: int, n_v: int, row_offsets, cols, signs, p: int, q: int,
                  sign_bits: bool = False, stream=None) -> int:
    """One call: host CSR in, exact count out (uploads, counts, frees)."""
    off_p, off_dev = _ptr(row_offsets)
    col_p, _ = _ptr(cols)
    sg_p, _ = _ptr(signs)
    flags = SBC_OFFS_I64 if str(row_offsets.dtype).endswith("int64") else 0
    if sign_bits:
        flags |= SBC_SIGN_BITS
    if off_dev:
        flags |= SBC_DEVICE_PTRS
    out = U128()
    _check(lib.sbc_count_csr(n_u, n_v, int(cols.shape[0]), off_p, col_p, sg_p, flags, p, q,
                             ctypes.byref(out), _stream_ptr(stream)))
    return out.value()


def sbc_count_csr_noalloc(n_u: int, n_v: int, row_offsets, cols, signs, p: int, q: int,
                          sign_bits: bool = False, stream=None) -> int:
    """sbc_count_csr for callers that cannot allocate device memory: the
    library takes all scratch from a fixed device array (see include/sbc.h)."""
    off_p, off_dev = _ptr(row_offsets)
    col_p, _ = _ptr(cols)
    sg_p, _ = _ptr(signs)
    flags = SBC_OFFS_I64 if str(row_offsets.dtype).endswith("int64") else 0
    if sign_bits:
        flags |= SBC_SIGN_BITS
    if off_dev:
        flags |= SBC_DEVICE_PTRS
    out = U128()
    _check(lib.sbc_count_csr_noalloc(n_u, n_v, int(cols.shape[0]), off_p, col_p, sg_p, flags, p,
                                     q, ctypes.byref(out), _stream_ptr(stream)))
    return out.value()


def _handles(graphs):
    arr = (_vp * max(len(graphs), 1))()
    for i, g in enumerate(graphs):
        arr[i] = g.handle
    return arr


def sbc_count_batch(graphs, p: int, q: int, stream=None) -> list:
    """sbc_count_batch: one pass of the counting kernels over a batch of
    resident graphs; returns each graph's exact count."""
    out = (U128 * max(len(graphs), 1))()
    _check(lib.sbc_count_batch(_handles(graphs), len(graphs), p, q, out, _stream_ptr(stream)))
    return [out[i].value() for i in range(len(graphs))]


def sbc_autotune(graphs, p: int, q: int, reps: int = 0, stream=None, cache: str | None = None) -> dict:
    """sbc_autotune: the fastest launch parameters for counting this batch of
    graphs (one graph is a batch of one); returns sbc_tune_t's fields as a
    dict, with "ms" the time of one count under them. With `cache` (a file
    path), sbc_autotune_cached: a tuning stored there for this GPU and kind
    of batch is reused (the dict's "from_cache" says so), else the search
    runs and its result is stored."""
    out = Tune()
    gl = list(graphs)
    if cache is None:
        _check(lib.sbc_autotune(_handles(gl), len(gl), p, q, reps, ctypes.byref(out),
                                _stream_ptr(stream)))
        return out.as_dict()
    hit = ctypes.c_int32(0)
    _check(lib.sbc_autotune_cached(_handles(gl), len(gl), p, q, reps, str(cache).encode(),
                                   ctypes.byref(out), ctypes.byref(hit), _stream_ptr(stream)))
    d = out.as_dict()
    d["from_cache"] = bool(hit.value)
    return d


class Batch:
    """A planned batch (sbc_batch_create); run() replays its counting kernels
    from a captured CUDA graph."""

    def __init__(self, graphs, p: int, q: int, tune=None, stream=None):
        self.graphs = list(graphs)  # keep the graphs alive
        h = _vp()
        t = _tune(tune)
        _check(lib.sbc_batch_create_ex(_handles(self.graphs), len(self.graphs), p, q,
                                       ctypes.byref(t) if t is not None else None,
                                       ctypes.byref(h), _stream_ptr(stream)))
        self.handle = h.value

    def run(self, stream=None) -> list:
        n = len(self.graphs)
        out = (U128 * max(n, 1))()
        _check(lib.sbc_batch_run(self.handle, out, _stream_ptr(stream)))
        return [out[i].value() for i in range(n)]

    def close(self):
        if self.handle:
            _check(lib.sbc_batch_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request server over resident graphs (sbc_server_*): submit() queues a
    count and returns a ticket at once; wait() returns (count, latency_s)."""

    def __init__(self, mem_budget_bytes: int = 0, lanes: int = 0, max_batch: int = 0,
                 small_edges: int = 0):
        o = ServerOpts(mem_budget_bytes, lanes, max_batch, small_edges)
        h = _vp()
        _check(lib.sbc_server_create(ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value
        self.graphs = []

    def add_graph(self, g: Graph) -> int:
        gid = ctypes.c_uint32()
        _check(lib.sbc_server_add_graph(self.handle, g.handle, ctypes.byref(gid)))
        self.graphs.append(g)
        return int(gid.value)

    def submit(self, gid: int, p: int, q: int) -> int:
        t = ctypes.c_uint64()
        _check(lib.sbc_server_submit(self.handle, gid, p, q, ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int, timeout_us: int = -1):
        out = U128()
        lat = ctypes.c_double()
        _check(lib.sbc_server_wait(self.handle, ticket, timeout_us, ctypes.byref(out),
                                   ctypes.byref(lat)))
        return out.value(), float(lat.value)

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib.sbc_server_stats(self.handle, ctypes.byref(st)))
        return {f: (float(getattr(st, f)) if t is ctypes.c_double else int(getattr(st, f)))
                for f, t in ServerStats._fields_}

    def reset_stats(self):
        _check(lib.sbc_server_reset_stats(self.handle))

    def close(self):
        if self.handle:
            _check(lib.sbc_server_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def graph_from_synth(g, device: bool = False, sign_bits: bool = False, stream=None) -> Graph:
    """Convenience: a sbc_synth.SignedBipartite to a device graph (host or
    device-resident inputs)."""
    signs = g.packed_sign_bits() if sign_bits else g.signs
    if device:
        import torch

        off = torch.from_numpy(np.ascontiguousarray(g.offsets)).cuda()
        col = torch.from_numpy(np.ascontiguousarray(g.cols)).cuda()
        sg = torch.from_numpy(np.ascontiguousarray(signs)).cuda()
        return sbc_graph_create(g.n_u, g.n_v, off, col, sg, sign_bits=sign_bits, stream=stream)
    return sbc_graph_create(g.n_u, g.n_v, np.ascontiguousarray(g.offsets),
                            np.ascontiguousarray(g.cols), np.ascontiguousarray(signs),
                            sign_bits=sign_bits, stream=stream)


# ---- dynamic graphs: a count kept exact under edge updates

SBC_DYN_INSERT, SBC_DYN_DELETE, SBC_DYN_SET_SIGN = 0, 1, 2

_declare("sbc_dyn_create", ctypes.c_int,
         [ctypes.POINTER(_vp), _i64, _i64, _i64, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp])
_declare("sbc_dyn_update", ctypes.c_int,
         [_vp, ctypes.c_int, _i64, _i64, ctypes.c_int8, ctypes.POINTER(U128), _vp])
_declare("sbc_dyn_count", ctypes.c_int, [_vp, ctypes.POINTER(U128), ctypes.POINTER(_i64)])
_declare("sbc_dyn_destroy", ctypes.c_int, [_vp])
_declare("sbc_edge_local_graph", ctypes.c_int,
         [_i64, _i64, _i64, _vp, _vp, _vp, _i64, _i64, ctypes.c_int8, ctypes.POINTER(_i64),
          ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp, _vp, _i64])


def _host_csr(n_u, offsets, cols, signs):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    col = np.ascontiguousarray(cols, dtype=np.int32)
    sgn = np.ascontiguousarray(signs, dtype=np.int8)
    if off.shape[0] != n_u + 1 or col.shape[0] != sgn.shape[0]:
        raise ValueError("CSR arrays of inconsistent lengths")
    return off, col, sgn


class Dynamic:
    """A balanced (p,q) count (p, q in [3, 8]) kept exact while edges are
    inserted, deleted or change sign (sbc_dyn_*). Each update counts the
    balanced bicliques through the edge on the GPU. Use as a context manager
    or call close()."""

    def __init__(self, n_u: int, n_v: int, offsets, cols, signs, p: int, q: int, stream=None):
        off, col, sgn = _host_csr(n_u, offsets, cols, signs)
        h = _vp()
        _check(lib.sbc_dyn_create(ctypes.byref(h), n_u, n_v, int(col.shape[0]), off.ctypes.data,
                                  col.ctypes.data, sgn.ctypes.data, p, q, _stream_ptr(stream)))
        self.h = h.value
        self.p, self.q = p, q

    @classmethod
    def from_synth(cls, g, p: int, q: int, stream=None) -> "Dynamic":
        return cls(g.n_u, g.n_v, g.offsets, g.cols, g.signs, p, q, stream)

    def _update(self, op: int, u: int, v: int, sign: int, stream) -> int:
        out = U128()
        _check(lib.sbc_dyn_update(self.h, op, u, v, sign, ctypes.byref(out), _stream_ptr(stream)))
        return out.value()

    def insert(self, u: int, v: int, sign: int, stream=None) -> int:
        """Add edge (u, v) with sign +1 / -1; returns the new count."""
        return self._update(SBC_DYN_INSERT, u, v, sign, stream)

    def delete(self, u: int, v: int, stream=None) -> int:
        """Remove edge (u, v); returns the new count."""
        return self._update(SBC_DYN_DELETE, u, v, 1, stream)

    def set_sign(self, u: int, v: int, sign: int, stream=None) -> int:
        """Give edge (u, v) the sign +1 / -1; returns the new count."""
        return self._update(SBC_DYN_SET_SIGN, u, v, sign, stream)

    def count(self) -> int:
        out, nnz = U128(), _i64()
        _check(lib.sbc_dyn_count(self.h, ctypes.byref(out), ctypes.byref(nnz)))
        return out.value()

    def edges(self) -> int:
        out, nnz = U128(), _i64()
        _check(lib.sbc_dyn_count(self.h, ctypes.byref(out), ctypes.byref(nnz)))
        return nnz.value

    def close(self):
        if self.h:
            lib.sbc_dyn_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def edge_local_graph(n_u: int, n_v: int, offsets, cols, signs, u: int, v: int, sign: int):
    """H(u, v) of sbc_edge_local_graph (host only): (n_l, n_r, offsets, cols)
    of the graph whose complete (p-1, q-1) subgraphs are the balanced
    (p,q)-bicliques through edge (u, v) with sign `sign`."""
    off, col, sgn = _host_csr(n_u, offsets, cols, signs)
    n_l, n_r, nnz = _i64(), _i64(), _i64()
    args = (n_u, n_v, int(col.shape[0]), off.ctypes.data, col.ctypes.data, sgn.ctypes.data, u, v,
            sign, ctypes.byref(n_l), ctypes.byref(n_r), ctypes.byref(nnz))
    _check(lib.sbc_edge_local_graph(*args, None, None, 0))
    h_off = np.zeros(n_l.value + 1, dtype=np.int64)
    h_col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    _check(lib.sbc_edge_local_graph(*args, h_off.ctypes.data, h_col.ctypes.data, h_col.shape[0]))
    return n_l.value, n_r.value, h_off, h_col[:nnz.value]


# ---- checkpoint / resume of long counts

def sbc_count_resumable(g: Graph, p: int, q: int, shards: int, state_path: str,
                        anchor_side: int = SBC_SIDE_AUTO, stream=None, count_fn=None) -> int:
    """The exact count taken in `shards` anchor shards (sbc_count_ex's
    shard / shard_count: anchors of rank r with r % shards == i form shard i),
    each shard's exact partial sum recorded in the JSON file `state_path`
    (replaced atomically) as soon as it is known. A later call with the same
    graph shape, (p, q), shard number and side resumes after the shards
    already recorded; a state file of another count raises ValueError.
    count_fn (tests only) replaces sbc_count_ex."""
    import json
    import os

    count_fn = count_fn or sbc_count_ex
    key = {"n_u": int(g.n_u), "n_v": int(g.n_v), "nnz": int(g.nnz), "p": p, "q": q,
           "shards": int(shards)}
    state = {**key, "side": None if anchor_side == SBC_SIDE_AUTO else int(anchor_side),
             "done": [], "partial": "0"}
    if os.path.exists(state_path):
        with open(state_path) as f:
            old = json.load(f)
        if any(old.get(k) != v for k, v in key.items()) or (
                anchor_side != SBC_SIDE_AUTO and old.get("side") not in (None, anchor_side)):
            raise ValueError(f"{state_path} records another count: {old}")
        state = old
    done, total = set(state["done"]), int(state["partial"])

    def save():
        tmp = f"{state_path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(state, f)
        os.replace(tmp, state_path)

    for i in range(int(shards)):
        if i in done:
            continue
        side = SBC_SIDE_AUTO if state["side"] is None else state["side"]
        c, st, _ = count_fn(g, p, q, anchor_side=side, shard=i, shard_count=int(shards),
                            stream=stream)
        if state["side"] is None:
            state["side"] = int(st["anchor_side"])
        total += int(c)
        done.add(i)
        state["done"] = sorted(done)
        state["partial"] = str(total)
        save()
    return total
