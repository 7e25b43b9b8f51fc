"""Python binding of the C ABI declared in ``include/pgabb.h``.

Argument marshalling only: every step (ingest, ordering, partition, queue,
counting, reduction) runs in the CUDA library ``libpgabb.so``.  Functions
keep the C names.  Arrays may be numpy arrays (host) or torch tensors (host
or CUDA); the memory kind passed to the library follows the array.  Streams
default to torch's current CUDA stream.  When CUDA is available the library
is pointed at torch's caching allocator, so all device memory comes from
torch.

If the shared library is missing and cannot be built, importing it raises:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

PGB_OK = 0
PGB_E_INVAL = -1
PGB_E_NOMEM = -2
PGB_E_OVERFLOW = -3
PGB_E_CUDA = -4
PGB_E_BUDGET = -5
PGB_E_TIMEOUT = -6
PGB_E_CANCELLED = -7
PGB_E_STATE = -8

PGB_MEM_HOST = 0
PGB_MEM_DEVICE = 1

PGB_CUT_NNZ = 0
PGB_CUT_UNIFORM = 1

PGB_MODE_PLAIN = 0
PGB_MODE_PERSISTENT = 1
PGB_MODE_HYBRID = 2

PGB_VAR_AUTO = 0
PGB_VAR_BSEARCH = 1
PGB_VAR_MERGE = 2
PGB_VAR_HASH = 3
PGB_VAR_MIXED = 4
PGB_VAR_HOST = 5

PGB_ORDER_WEIGHT = 0
PGB_ORDER_LOCALITY = 1
PGB_ORDER_HILBERT = 2

PGB_EXPORT_PERM = 0
PGB_EXPORT_ROWPTR = 1
PGB_EXPORT_COL = 2
PGB_EXPORT_CUTS = 3
PGB_EXPORT_BLOCK_EDGES = 4
PGB_EXPORT_TRIPLES = 5
PGB_EXPORT_WEIGHTS = 6
PGB_EXPORT_PART_PROBES = 7
PGB_LAYOUT_ROWMAJOR = 0
PGB_LAYOUT_HILBERT = 1
PGB_FMT_CSR = 0
PGB_FMT_COO = 1
PGB_FMT_CCOO = 2

HEADER = os.path.join(_build.INCLUDE, "pgabb.h")


class PgbError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


class TcOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("variant", ctypes.c_int32), ("per_vertex", ctypes.c_int32),
                ("per_triple", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("order", ctypes.c_int32),
                ("device_budget", ctypes.c_uint64), ("chunk_edges", ctypes.c_uint32),
                ("hash_threads", ctypes.c_uint32), ("cancel", ctypes.c_void_p), ("host_threads", ctypes.c_uint32),
                ("host_share_ppm", ctypes.c_uint32), ("hash_min_lookups", ctypes.c_uint32),
                ("dense_core", ctypes.c_int32)]


class BlocksStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("p", ctypes.c_uint32), ("m", ctypes.c_uint64),
                ("nonempty_blocks", ctypes.c_uint64), ("triples", ctypes.c_uint64),
                ("wedges", ctypes.c_uint64), ("alg_bytes", ctypes.c_uint64),
                ("max_outdeg", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("probes", ctypes.c_uint64)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None
_callbacks = []

_VP = ctypes.c_void_p
_SIGS = {
    "pgb_set_allocator": (ctypes.c_int, [_ALLOC_FN, _FREE_FN, _VP]),
    "pgb_graph_from_edges": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, _VP,
                                            ctypes.POINTER(_VP)]),
    "pgb_graph_from_csr": (ctypes.c_int, [ctypes.c_uint32, _VP, _VP, ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
    "pgb_graph_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_graph_export": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    "pgb_graph_free": (None, [_VP]),
    "pgb_partition": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
    "pgb_blocks_info": (ctypes.c_int, [_VP, ctypes.POINTER(BlocksStats)]),
    "pgb_blocks_export": (ctypes.c_int, [_VP, ctypes.c_int, _VP, ctypes.c_int, _VP]),
    "pgb_blocks_free": (None, [_VP]),
    "pgb_blocks_offload": (ctypes.c_int, [_VP, _VP]),
    "pgb_blocks_resident_bytes": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_tc_opts_default": (None, [ctypes.POINTER(TcOpts)]),
    "pgb_tc_run": (ctypes.c_int, [_VP, ctypes.POINTER(TcOpts), _VP, ctypes.POINTER(_VP)]),
    "pgb_tc_result_get": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64), _VP, ctypes.c_int]),
    "pgb_tc_result_triples": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "pgb_tc_result_kernel_ms": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "pgb_tc_result_dense_core": (ctypes.c_int, [_VP, _VP]),
    "pgb_tc_result_variant": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "pgb_tc_result_part_variants": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint32), _VP]),
    "pgb_tc_result_hybrid": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]),
    "pgb_tc_result_stream": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint32),
                                            ctypes.POINTER(ctypes.c_uint32)]),
    "pgb_blocks_offload_columns": (ctypes.c_int, [_VP, ctypes.c_uint32, _VP]),
    "pgb_blocks_cache_budget": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_tc_result_free": (None, [_VP]),
    "pgb_tc_count_edges": (ctypes.c_int, [_VP, _VP, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_int, ctypes.POINTER(TcOpts), ctypes.c_int, _VP,
                                          ctypes.POINTER(ctypes.c_uint64), _VP]),
    "pgb_last_error": (ctypes.c_char_p, []),
    "pgb_version": (ctypes.c_char_p, []),
    "pgb_kernel_launches": (ctypes.c_uint64, []),
    "pgb_tc_count_oriented_noalloc": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint64, _VP, _VP, _VP, _VP, _VP,
                                                     _VP]),
    "pgb_server_opts_default": (None, [_VP]),
    "pgb_server_job_bytes": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_uint32]),
    "pgb_server_create": (ctypes.c_int, [_VP, ctypes.POINTER(_VP)]),
    "pgb_server_submit": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_server_submit_borrowed": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_server_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]),
    "pgb_server_pause": (ctypes.c_int, [_VP, ctypes.c_int]),
    "pgb_server_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64), _VP,
                                       ctypes.POINTER(ctypes.c_double)]),
    "pgb_server_cancel": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "pgb_server_stats": (ctypes.c_int, [_VP, _VP]),
    "pgb_server_destroy": (None, [_VP]),
    "pgb_block_order": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_int, _VP]),
    "pgb_hilbert_index": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_blocks_block_info": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_uint32, _VP]),
    "pgb_blocks_export_block": (ctypes.c_int, [_VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, _VP, _VP, _VP,
                                               ctypes.c_int, _VP]),
    "pgb_k4_count": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_c4_count": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_cc_run": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "pgb_pagerank_opts_default": (None, [_VP]),
    "pgb_pagerank_run": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_double)]),
    "pgb_cancel_create": (ctypes.c_int, [ctypes.POINTER(_VP)]),
    "pgb_cancel_set": (ctypes.c_int, [_VP]),
    "pgb_cancel_reset": (ctypes.c_int, [_VP]),
    "pgb_cancel_is_set": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "pgb_cancel_free": (None, [_VP]),
}

PGB_NOALLOC_MAX_VERTICES = 1 << 20


def header_functions() -> list[str]:
    """Names of the functions declared in include/pgabb.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(pgb_[a-z0-9_]+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def load(register_torch_allocator: bool = True):
    """Load (building if needed) ``libpgabb.so`` and bind every entry point."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
            if register_torch_allocator:
                _maybe_use_torch_allocator(lib)
    return _lib


def _maybe_use_torch_allocator(lib):
    try:
        import torch
    except ImportError:
        return
    if not torch.cuda.is_available():
        return
    raw_alloc = torch._C._cuda_cudaCachingAllocator_raw_alloc
    raw_delete = torch._C._cuda_cudaCachingAllocator_raw_delete

    def _alloc(size, stream, ctx):
        try:
            return raw_alloc(int(size), int(stream or 0))
        except Exception:
            return None

    def _free(ptr, size, stream, ctx):
        try:
            raw_delete(int(ptr))
        except Exception:
            pass

    fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _callbacks.append((fa, ff))
    _check(lib.pgb_set_allocator(fa, ff, None), "pgb_set_allocator")


def _check(rc: int, where: str):
    if rc != PGB_OK:
        raise PgbError(rc, where, pgb_last_error())


def _stream(stream):
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def _arr(x, dtype):
    """(pointer, mem kind, keep-alive object) for a numpy array or torch tensor."""
    if x is None:
        return None, PGB_MEM_HOST, None
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x, dtype=dtype)
        return x.ctypes.data, PGB_MEM_HOST, x
    import torch
    if isinstance(x, torch.Tensor):
        tdt = {np.uint32: torch.uint32, np.int64: torch.int64, np.uint64: torch.uint64}[dtype]
        if x.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), (PGB_MEM_DEVICE if x.is_cuda else PGB_MEM_HOST), x
    raise TypeError(f"unsupported array type {type(x)}")


class _Handle:
    _free_name = ""

    def __init__(self, ptr, stream):
        self.ptr = ptr
        self.stream = stream

    def free(self):
        if self.ptr:
            getattr(load(), self._free_name)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.ptr:
            raise ValueError("handle already freed")
        return ctypes.c_void_p(self.ptr)


class Graph(_Handle):
    _free_name = "pgb_graph_free"


class Blocks(_Handle):
    _free_name = "pgb_blocks_free"


class Cancel(_Handle):
    _free_name = "pgb_cancel_free"


class Result(_Handle):
    _free_name = "pgb_tc_result_free"

    def __init__(self, ptr, stream, n, ntriples):
        super().__init__(ptr, stream)
        self.n = n
        self.ntriples = ntriples


# ----------------------------------------------------------------- C names

def pgb_last_error() -> str:
    return load().pgb_last_error().decode()


def pgb_version() -> str:
    return load().pgb_version().decode()


def pgb_kernel_launches() -> int:
    return int(load().pgb_kernel_launches())


def pgb_set_allocator(alloc=None, free=None, ctx=None):
    """Install raw ctypes callbacks (``_ALLOC_FN``/``_FREE_FN``) or restore the default."""
    lib = load()
    fa = alloc if alloc is not None else ctypes.cast(None, _ALLOC_FN)
    ff = free if free is not None else ctypes.cast(None, _FREE_FN)
    _check(lib.pgb_set_allocator(fa, ff, ctx), "pgb_set_allocator")


def pgb_graph_from_edges(src, dst, n: int, stream=None) -> Graph:
    lib = load()
    ps, ms, ks = _arr(src, np.uint32)
    pd, md, kd = _arr(dst, np.uint32)
    m = 0 if ks is None else int(ks.numel() if hasattr(ks, "numel") else ks.size)
    if ms != md:
        raise ValueError("src and dst must live in the same memory")
    st = _stream(stream)
    out = ctypes.c_void_p()
    _check(lib.pgb_graph_from_edges(ps, pd, m, n, ms, st, ctypes.byref(out)), "pgb_graph_from_edges")
    return Graph(out.value, st)


def pgb_graph_from_csr(n: int, offs, cols, stream=None) -> Graph:
    lib = load()
    po, mo, _ko = _arr(offs, np.int64)
    pc, mc, _kc = _arr(cols, np.uint32)
    st = _stream(stream)
    out = ctypes.c_void_p()
    _check(lib.pgb_graph_from_csr(n, po, pc, mo, st, ctypes.byref(out)), "pgb_graph_from_csr")
    return Graph(out.value, st)


def pgb_graph_info(g: Graph):
    n, m = ctypes.c_uint32(), ctypes.c_uint64()
    _check(load().pgb_graph_info(g, ctypes.byref(n), ctypes.byref(m)), "pgb_graph_info")
    return int(n.value), int(m.value)


def pgb_graph_export(g: Graph):
    """(a, b, deg) numpy arrays of the cleaned graph (a < b, sorted)."""
    n, m = pgb_graph_info(g)
    a = np.empty(m, np.uint32)
    b = np.empty(m, np.uint32)
    d = np.empty(n, np.uint32)
    _check(load().pgb_graph_export(g, a.ctypes.data if m else None, b.ctypes.data if m else None,
                                   d.ctypes.data if n else None, PGB_MEM_HOST, g.stream), "pgb_graph_export")
    return a, b, d


def pgb_graph_free(g: Graph):
    g.free()


def pgb_partition(g: Graph, p: int, cut_rule: int = PGB_CUT_NNZ, stream=None) -> Blocks:
    st = _stream(stream) if stream is not None else g.stream
    out = ctypes.c_void_p()
    _check(load().pgb_partition(g, p, cut_rule, st, ctypes.byref(out)), "pgb_partition")
    return Blocks(out.value, st)


def pgb_blocks_info(b: Blocks) -> dict:
    s = BlocksStats()
    _check(load().pgb_blocks_info(b, ctypes.byref(s)), "pgb_blocks_info")
    return {k: int(getattr(s, k)) for k, _ in BlocksStats._fields_ if k != "reserved"}


def pgb_blocks_export(b: Blocks, what: int) -> np.ndarray:
    info = pgb_blocks_info(b)
    n, p, m, T = info["n"], info["p"], info["m"], info["triples"]
    spec = {
        PGB_EXPORT_PERM: (np.uint32, n),
        PGB_EXPORT_ROWPTR: (np.int64, n + 1),
        PGB_EXPORT_COL: (np.uint32, m),
        PGB_EXPORT_CUTS: (np.uint32, p + 1),
        PGB_EXPORT_BLOCK_EDGES: (np.uint64, p * p),
        PGB_EXPORT_TRIPLES: (np.uint32, 3 * T),
        PGB_EXPORT_WEIGHTS: (np.uint64, T),
        PGB_EXPORT_PART_PROBES: (np.uint64, p),
    }
    dt, cnt = spec[what]
    out = np.zeros(cnt, dtype=dt)
    _check(load().pgb_blocks_export(b, what, out.ctypes.data if cnt else None, PGB_MEM_HOST, b.stream),
           "pgb_blocks_export")
    if what == PGB_EXPORT_BLOCK_EDGES:
        return out.reshape(p, p)
    if what == PGB_EXPORT_TRIPLES:
        return out.reshape(T, 3)
    return out


def pgb_blocks_free(b: Blocks):
    b.free()


def pgb_blocks_offload(b: Blocks, stream=None):
    """Move the in-edge index of ``b`` to pinned host memory (streamed runs)."""
    st = _stream(stream) if stream is not None else b.stream
    _check(load().pgb_blocks_offload(b, st), "pgb_blocks_offload")


def pgb_tc_opts_default(**kw) -> TcOpts:
    """Default run options with the given fields changed (``cancel`` takes a
    Cancel token, which the caller keeps alive while the run is in use)."""
    o = TcOpts()
    load().pgb_tc_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        if isinstance(v, _Handle):
            v = v.ptr
        setattr(o, k, v)
    return o


class BlockInfo(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint32), ("cols", ctypes.c_uint32), ("nnz", ctypes.c_uint64),
                ("nonempty_rows", ctypes.c_uint32), ("format", ctypes.c_int32), ("bytes_csr", ctypes.c_uint64),
                ("bytes_coo", ctypes.c_uint64), ("bytes_ccoo", ctypes.c_uint64)]


def pgb_block_order(p: int, layout: int = PGB_LAYOUT_ROWMAJOR) -> np.ndarray:
    """The upper blocks (i <= j) as an array of (i, j) rows, in row-major or
    Hilbert-curve order."""
    out = np.zeros(p * (p + 1), dtype=np.uint32)
    _check(load().pgb_block_order(p, layout, out.ctypes.data), "pgb_block_order")
    return out.reshape(-1, 2)


def pgb_hilbert_index(side: int, x: int, y: int) -> int:
    d = ctypes.c_uint64()
    _check(load().pgb_hilbert_index(side, x, y, ctypes.byref(d)), "pgb_hilbert_index")
    return int(d.value)


def pgb_blocks_block_info(b: Blocks, i: int, j: int) -> dict:
    inf = BlockInfo()
    _check(load().pgb_blocks_block_info(b, i, j, ctypes.byref(inf)), "pgb_blocks_block_info")
    return {k: int(getattr(inf, k)) for k, _ in BlockInfo._fields_}


def pgb_blocks_export_block(b: Blocks, i: int, j: int, fmt: int):
    """Block A_ij with block-local IDs: CSR (offsets, columns), COO (rows,
    columns) or CCOO (non-empty rows, their offsets, columns), host arrays."""
    inf = pgb_blocks_block_info(b, i, j)
    nnz, rows, nz = inf["nnz"], inf["rows"], inf["nonempty_rows"]
    na = rows + 1 if fmt == PGB_FMT_CSR else (nnz if fmt == PGB_FMT_COO else nz)
    a = np.zeros(max(na, 1), dtype=np.uint32)
    c = np.zeros(max(nnz, 1), dtype=np.uint32)
    d = np.zeros(nz + 1, dtype=np.uint32)
    _check(load().pgb_blocks_export_block(b, i, j, fmt, a.ctypes.data, c.ctypes.data, d.ctypes.data, PGB_MEM_HOST,
                                          b.stream), "pgb_blocks_export_block")
    if fmt == PGB_FMT_CCOO:
        return a[:nz], d, c[:nnz]
    return a[:na], c[:nnz]


def pgb_k4_count(b: Blocks, stream=None) -> int:
    """Number of 4-cliques."""
    v = ctypes.c_uint64()
    _check(load().pgb_k4_count(b, _stream(stream) if stream is not None else b.stream, ctypes.byref(v)),
           "pgb_k4_count")
    return int(v.value)


def pgb_c4_count(b: Blocks, stream=None) -> int:
    """Number of 4-cycles (the butterflies of a bipartite graph)."""
    v = ctypes.c_uint64()
    _check(load().pgb_c4_count(b, _stream(stream) if stream is not None else b.stream, ctypes.byref(v)),
           "pgb_c4_count")
    return int(v.value)


class PageRankOpts(ctypes.Structure):
    _fields_ = [("damping", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 3)]


def pgb_cc_run(b: Blocks, labels=None, stream=None):
    """Connected components: (labels by original ID, iterations, components).
    ``labels`` may be a uint32 device tensor of n entries to fill; else a
    host numpy array is returned."""
    n = pgb_blocks_info(b)["n"]
    out = labels if labels is not None else np.zeros(n, dtype=np.uint32)
    ptr, mem, keep = _arr(out, np.uint32)
    it, comps = ctypes.c_uint32(), ctypes.c_uint64()
    st = _stream(stream) if stream is not None else b.stream
    _check(load().pgb_cc_run(b, st, ptr, mem, ctypes.byref(it), ctypes.byref(comps)), "pgb_cc_run")
    return (keep if labels is None else labels), int(it.value), int(comps.value)


def pgb_pagerank_opts_default(**kw) -> PageRankOpts:
    o = PageRankOpts()
    load().pgb_pagerank_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def pgb_pagerank_run(b: Blocks, opts: PageRankOpts | None = None, ranks=None, stream=None):
    """PageRank: (ranks float64 by original ID, iterations, last L1 change)."""
    n = pgb_blocks_info(b)["n"]
    out = ranks if ranks is not None else np.zeros(n, dtype=np.float64)
    if isinstance(out, np.ndarray):
        if out.dtype != np.float64 or out.size < n:
            raise ValueError("ranks must be float64 with n entries")
        ptr, mem = out.ctypes.data, PGB_MEM_HOST
    else:
        import torch
        if out.dtype != torch.float64 or out.numel() < n or not out.is_contiguous():
            raise ValueError("ranks must be a contiguous float64 tensor with n entries")
        ptr, mem = out.data_ptr(), (PGB_MEM_DEVICE if out.is_cuda else PGB_MEM_HOST)
    it, err = ctypes.c_uint32(), ctypes.c_double()
    st = _stream(stream) if stream is not None else b.stream
    _check(load().pgb_pagerank_run(b, ctypes.byref(opts) if opts is not None else None, st, ptr, mem,
                                   ctypes.byref(it), ctypes.byref(err)), "pgb_pagerank_run")
    return out, int(it.value), float(err.value)


def pgb_cancel_create() -> Cancel:
    out = ctypes.c_void_p()
    _check(load().pgb_cancel_create(ctypes.byref(out)), "pgb_cancel_create")
    return Cancel(out.value, None)


def pgb_cancel_set(c: Cancel):
    _check(load().pgb_cancel_set(c), "pgb_cancel_set")


def pgb_cancel_reset(c: Cancel):
    _check(load().pgb_cancel_reset(c), "pgb_cancel_reset")


def pgb_cancel_is_set(c: Cancel) -> bool:
    v = ctypes.c_int()
    _check(load().pgb_cancel_is_set(c, ctypes.byref(v)), "pgb_cancel_is_set")
    return bool(v.value)


def pgb_cancel_free(c: Cancel):
    c.free()


def pgb_tc_run(b: Blocks, opts: TcOpts | None = None, stream=None) -> Result:
    st = _stream(stream) if stream is not None else b.stream
    out = ctypes.c_void_p()
    _check(load().pgb_tc_run(b, ctypes.byref(opts) if opts is not None else None, st, ctypes.byref(out)),
           "pgb_tc_run")
    info = pgb_blocks_info(b)
    return Result(out.value, st, info["n"], info["triples"])


def pgb_tc_result_get(r: Result, per_vertex=True):
    """(total, t) with t a numpy uint64[n] in original IDs (or None).

    ``per_vertex`` may also be a CUDA uint64 tensor of length n to receive t
    on the device (then that tensor is returned as t)."""
    tot = ctypes.c_uint64()
    out = None
    ptr, mem = None, PGB_MEM_HOST
    if per_vertex is True:
        out = np.zeros(r.n, np.uint64)
        ptr = out.ctypes.data if r.n else None
    elif per_vertex is not None and per_vertex is not False:
        ptr, mem, out = _arr(per_vertex, np.uint64)
    _check(load().pgb_tc_result_get(r, ctypes.byref(tot), ptr, mem), "pgb_tc_result_get")
    return int(tot.value), out


def pgb_tc_result_triples(r: Result) -> np.ndarray:
    out = np.zeros(r.ntriples, np.uint64)
    _check(load().pgb_tc_result_triples(r, out.ctypes.data if r.ntriples else None, PGB_MEM_HOST),
           "pgb_tc_result_triples")
    return out


def pgb_tc_result_kernel_ms(r: Result) -> float:
    ms = ctypes.c_float()
    _check(load().pgb_tc_result_kernel_ms(r, ctypes.byref(ms)), "pgb_tc_result_kernel_ms")
    return float(ms.value)


class DenseCoreInfo(ctypes.Structure):
    _fields_ = [("ranks", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("triangles", ctypes.c_uint64),
                ("lookups_skipped", ctypes.c_uint64), ("gemm_flop", ctypes.c_double), ("ms", ctypes.c_float),
                ("reserved2", ctypes.c_float)]


def pgb_tc_result_dense_core(r) -> dict:
    """The run's dense top block: ranks (0: none), triangles in it, lookups
    it took off the intersection kernels, GEMM flops, device ms (-1: graph)."""
    i = DenseCoreInfo()
    _check(load().pgb_tc_result_dense_core(r, ctypes.byref(i)), "pgb_tc_result_dense_core")
    return {k: (float(getattr(i, k)) if k in ("gemm_flop", "ms") else int(getattr(i, k)))
            for k in ("ranks", "triangles", "lookups_skipped", "gemm_flop", "ms")}


def pgb_tc_result_variant(r: Result) -> int:
    v = ctypes.c_int()
    _check(load().pgb_tc_result_variant(r, ctypes.byref(v)), "pgb_tc_result_variant")
    return int(v.value)


def pgb_tc_result_part_variants(r: Result) -> np.ndarray:
    """The kernel (PGB_VAR_*) that counted each head part of the run."""
    p = ctypes.c_uint32()
    _check(load().pgb_tc_result_part_variants(r, ctypes.byref(p), None), "pgb_tc_result_part_variants")
    out = np.zeros(p.value, dtype=np.int32)
    _check(load().pgb_tc_result_part_variants(r, ctypes.byref(p), out.ctypes.data if p.value else None),
           "pgb_tc_result_part_variants")
    return out


def pgb_tc_result_hybrid(r: Result) -> dict:
    """HYBRID runs: the host kernel's wall ms, in-edges, parts and threads."""
    ms, ie, parts, th = ctypes.c_float(), ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().pgb_tc_result_hybrid(r, ctypes.byref(ms), ctypes.byref(ie), ctypes.byref(parts), ctypes.byref(th)),
           "pgb_tc_result_hybrid")
    return {"host_ms": float(ms.value), "host_in_edges": int(ie.value), "host_parts": int(parts.value),
            "host_threads": int(th.value)}


def pgb_blocks_offload_columns(b: Blocks, slices: int = 0, stream=None):
    """Move the columns (in ``slices`` row ranges, 0 = p) and a tail-range-major
    in-edge index of ``b`` to pinned host memory (block-cache runs)."""
    st = _stream(stream) if stream is not None else b.stream
    _check(load().pgb_blocks_offload_columns(b, slices, st), "pgb_blocks_offload_columns")


def pgb_blocks_cache_budget(b: Blocks, slices: int, per_vertex: bool = True) -> int:
    """Smallest device_budget whose column cache holds ``slices`` slices."""
    v = ctypes.c_uint64()
    _check(load().pgb_blocks_cache_budget(b, int(per_vertex), slices, ctypes.byref(v)), "pgb_blocks_cache_budget")
    return int(v.value)


def pgb_blocks_resident_bytes(b: Blocks, per_vertex: bool = True) -> int:
    """Device bytes a streamed run holds besides its two slots."""
    v = ctypes.c_uint64()
    _check(load().pgb_blocks_resident_bytes(b, int(per_vertex), ctypes.byref(v)), "pgb_blocks_resident_bytes")
    return int(v.value)


def pgb_tc_result_stream(r: Result, slice_loads: bool = False):
    """(bytes copied host to device, chunks) of a streamed run, plus the column
    slices copied in when ``slice_loads``; zeros for a resident run."""
    nb, nc, nl = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(load().pgb_tc_result_stream(r, ctypes.byref(nb), ctypes.byref(nc), ctypes.byref(nl)),
           "pgb_tc_result_stream")
    if slice_loads:
        return int(nb.value), int(nc.value), int(nl.value)
    return int(nb.value), int(nc.value)


def pgb_tc_result_free(r: Result):
    r.free()


def pgb_tc_count_edges(src, dst, n: int, p: int, cut_rule: int = PGB_CUT_NNZ, opts: TcOpts | None = None,
                       stream=None, per_vertex=True):
    """One call from raw edges to (total, t).  Host arrays in -> host t out."""
    lib = load()
    ps, ms, ks = _arr(src, np.uint32)
    pd, md, kd = _arr(dst, np.uint32)
    if ms != md:
        raise ValueError("src and dst must live in the same memory")
    m = 0 if ks is None else int(ks.numel() if hasattr(ks, "numel") else ks.size)
    st = _stream(stream)
    tot = ctypes.c_uint64()
    t = None
    tptr = None
    if per_vertex is True:
        if ms == PGB_MEM_DEVICE:
            import torch
            t = torch.zeros(n, dtype=torch.uint64, device=ks.device)
            tptr = t.data_ptr()
        else:
            t = np.zeros(n, np.uint64)
            tptr = t.ctypes.data if n else None
    elif per_vertex is not None and per_vertex is not False:
        tptr, _, t = _arr(per_vertex, np.uint64)
    rc = lib.pgb_tc_count_edges(ps, pd, m, n, p, cut_rule, ctypes.byref(opts) if opts is not None else None,
                                ms, st, ctypes.byref(tot), tptr)
    _check(rc, "pgb_tc_count_edges")
    return int(tot.value), t


def pgb_tc_count_oriented_noalloc(n: int, m: int, rowptr, col, perm, total, per_vertex=None, stream=None):
    """Allocation-free count over an oriented graph already in device memory.

    ``rowptr`` (uint32[n+1]), ``col`` (uint32[m]), ``perm`` (uint32[n] or
    None), ``total`` (uint64[1]) and ``per_vertex`` (uint64[n] or None) are
    CUDA tensors; results are written into ``total`` and ``per_vertex``.
    For callers that may not allocate device memory during the call; see
    include/pgabb.h for the limits and the sharing rules.  Tensors shorter
    than ``n`` and ``m`` require raise ValueError before the library is
    called."""
    for name, x, need in (("rowptr", rowptr, n + 1), ("col", col, m), ("perm", perm, n), ("total", total, 1),
                          ("per_vertex", per_vertex, n)):
        if x is None:
            continue
        have = x.size if isinstance(x, np.ndarray) else x.numel()
        if have < need:
            raise ValueError(f"{name} holds {have} entries; n = {n}, m = {m} need at least {need}")
    args = []
    for x, dt in ((rowptr, np.uint32), (col, np.uint32), (perm, np.uint32), (total, np.uint64),
                  (per_vertex, np.uint64)):
        ptr, mem, _ = _arr(x, dt)
        if x is not None and mem != PGB_MEM_DEVICE:
            raise ValueError("pgb_tc_count_oriented_noalloc takes device tensors only")
        args.append(ptr)
    _check(load().pgb_tc_count_oriented_noalloc(n, m, *args, _stream(stream)), "pgb_tc_count_oriented_noalloc")


# ------------------------------------------------------------------ serve

PGB_SERVE_BATCHED = 0
PGB_SERVE_SERIAL = 1
PGB_JOB_QUEUED, PGB_JOB_RUNNING, PGB_JOB_DONE, PGB_JOB_FAILED, PGB_JOB_CANCELLED = range(5)


class ServerOpts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32), ("p", ctypes.c_uint32),
                ("mode", ctypes.c_int32), ("per_vertex", ctypes.c_int32), ("max_batch_jobs", ctypes.c_uint32),
                ("batch_edges", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 8)]


class ServerInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "done", "failed", "cancelled", "queued", "batches",
                                              "jobs_in_batches", "bytes_in_use")]


class Server(_Handle):
    _free_name = "pgb_server_destroy"

    def __init__(self, ptr, per_vertex):
        super().__init__(ptr, None)
        self.per_vertex = per_vertex
        self.n_of = {}
        self.borrowed = {}  # job -> the device tensors it reads, kept alive until wait returns

    def free(self):
        super().free()
        self.borrowed.clear()


def pgb_server_opts_default(**kw) -> ServerOpts:
    o = ServerOpts()
    load().pgb_server_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def pgb_server_job_bytes(m: int, n: int) -> int:
    return int(load().pgb_server_job_bytes(m, n))


def pgb_server_create(opts: ServerOpts | None = None) -> Server:
    opts = opts or pgb_server_opts_default()
    out = ctypes.c_void_p()
    _check(load().pgb_server_create(ctypes.byref(opts), ctypes.byref(out)), "pgb_server_create")
    return Server(out.value, bool(opts.per_vertex))


def pgb_server_submit(srv: Server, src, dst, n: int, borrow: bool = False) -> int:
    """Queue a job.  ``borrow`` (CUDA tensors, or host tensors/arrays, best
    pinned; fully written): the server copies them when the job's batch
    starts instead of at submit; the binding keeps them alive until the job
    is waited for."""
    ps, ms, ks = _arr(src, np.uint32)
    pd, md, kd = _arr(dst, np.uint32)
    if ms != md:
        raise ValueError("src and dst must live in the same memory")
    m = 0 if ks is None else int(ks.numel() if hasattr(ks, "numel") else ks.size)
    jid = ctypes.c_uint64()
    if borrow:
        _check(load().pgb_server_submit_borrowed(srv, ps, pd, m, n, ms, ctypes.byref(jid)),
               "pgb_server_submit_borrowed")
        srv.borrowed[int(jid.value)] = (ks, kd)
    else:
        _check(load().pgb_server_submit(srv, ps, pd, m, n, ms, ctypes.byref(jid)), "pgb_server_submit")
    srv.n_of[int(jid.value)] = n
    return int(jid.value)


def pgb_server_submit_borrowed(srv: Server, src, dst, n: int) -> int:
    """Queue a job on arrays the server borrows (see pgb_server_submit)."""
    return pgb_server_submit(srv, src, dst, n, borrow=True)


def pgb_server_pause(srv: Server, paused: bool = True):
    _check(load().pgb_server_pause(srv, int(paused)), "pgb_server_pause")


def pgb_server_poll(srv: Server, job: int) -> int:
    st = ctypes.c_int()
    _check(load().pgb_server_poll(srv, job, ctypes.byref(st)), "pgb_server_poll")
    return int(st.value)


def pgb_server_wait(srv: Server, job: int, timeout_s: float = -1.0, per_vertex: bool = False):
    """(total, per-vertex numpy array or None, latency seconds)."""
    tot = ctypes.c_uint64()
    lat = ctypes.c_double()
    pv = None
    ptr = None
    if per_vertex:
        pv = np.zeros(srv.n_of.get(job, 0), np.uint64)
        ptr = pv.ctypes.data if pv.size else None
    rc = load().pgb_server_wait(srv, job, timeout_s, ctypes.byref(tot), ptr, ctypes.byref(lat))
    if rc != PGB_E_TIMEOUT:
        srv.n_of.pop(job, None)
        srv.borrowed.pop(job, None)
    _check(rc, "pgb_server_wait")
    return int(tot.value), pv, float(lat.value)


def pgb_server_cancel(srv: Server, job: int):
    _check(load().pgb_server_cancel(srv, job), "pgb_server_cancel")


def pgb_server_stats(srv: Server) -> dict:
    info = ServerInfo()
    _check(load().pgb_server_stats(srv, ctypes.byref(info)), "pgb_server_stats")
    return {k: int(getattr(info, k)) for k, _ in ServerInfo._fields_}


def pgb_server_destroy(srv: Server):
    srv.free()
