"""ORACLE: test infrastructure only.

Plain single-threaded CPU restatement of exact triangle counting over block
triples (PGAbB, arXiv 2209.04541, Section 3.6), used to check the CUDA path.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library and never
imports it; the only shared module is the seeded input generator
(``graphgen``).

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  clean            pinned: hand-built inputs with known cleaned form,
                   symmetric/sorted/unique invariants, networkx-free
                   brute force set construction.
  node_iterator    pinned: O(n^3) brute force, closed forms (K_n, W_n, C_n,
                   grids, stars, trees, K_ab, K_abc, fans), trace(A^3)/6 and
                   diag(A^3)/2 by dense matmul, sum t = 3T, relabel
                   invariance.
  tc_vertex        pinned: equals diag(A^3)/2 and brute force per vertex.
  degree_rank      pinned: permutation, non-decreasing degree, ID ties.
  orient           pinned: each undirected edge exactly once, upward, sorted.
  cuts             pinned: closed form on hand-made prefix sums, monotone,
                   endpoints; uniform rule equals floor(t n / p).
  block_edges      pinned: hand-derived p x p matrices on a 6-vertex graph
                   (both cut rules, empty parts, a vertex on a cut), a dense
                   brute force from the definition of the parts, sums to
                   |E+|, zero below the diagonal.
  triples          pinned: brute-force enumeration count p(p+1)(p+2)/6 for
                   dense blocks, weight order.
  tc_forward       pinned: equals node_iterator and brute force; per-triple
                   counts equal a dense brute force that places each
                   triangle by the definition of the parts, and
                   hand-derived values on a 6-vertex graph.
  tc_forward_mt    pinned: equals tc_forward (total and every t[x]).
  cc_min_label     pinned: networkx connected components (a library
                   routine), closed forms (disjoint cliques, paths,
                   isolated vertices), relabelling.
  k4_count         pinned: brute force over all 4-sets, closed forms (K_n,
                   complete 4-partite K_abcd, tripartite and wheel graphs).
  c4_count         pinned: brute force over all 4-tuples, closed forms
                   (K_ab, grids, K_n, cycles, K_4 minus an edge).
  pagerank         pinned: uniform ranks on regular graphs and the star's
                   fixed point (closed forms), networkx.pagerank on graphs
                   without isolated vertices (a library routine), sum of
                   ranks 1 without isolated vertices, iteration limit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_MT = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_mt = None

CUT_NNZ = 0
CUT_UNIFORM = 1


def build(force: bool = False, out: str | None = None, defines=(), openmp: bool = False,
          src: str | None = None) -> str:
    """Compile the oracle with gcc (-O2): single-threaded, or with OpenMP
    (``openmp``), which only adds ``or_tc_forward_mt``.  ``src`` compiles
    another copy of the source (the tests' planted-mistake checks)."""
    target = out or (_LIB_MT if openmp else _LIB)
    source = src or _SRC
    if (not force and out is None and os.path.exists(target)
            and os.path.getmtime(target) >= os.path.getmtime(source)):
        return target
    tmp = target + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11"] + (["-fopenmp"] if openmp else [])
    cmd += [f"-D{d}" for d in defines] + ["-o", tmp, source]
    subprocess.run(cmd, check=True)
    os.replace(tmp, target)
    return target


def _bind(lib):
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.or_clean.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p, u32p, i64p, u32p]
    lib.or_clean.restype = ctypes.c_int64
    lib.or_tc_node_iterator.argtypes = [ctypes.c_uint32, i64p, u32p, u64p]
    lib.or_tc_node_iterator.restype = ctypes.c_uint64
    lib.or_tc_vertex.argtypes = [ctypes.c_uint32, i64p, u32p, ctypes.c_uint32]
    lib.or_tc_vertex.restype = ctypes.c_uint64
    lib.or_tc_vertex_sample.argtypes = [ctypes.c_uint32, i64p, u32p, ctypes.c_uint64, u32p, u64p]
    lib.or_tc_vertex_sample.restype = None
    lib.or_degree_rank.argtypes = [ctypes.c_uint32, i64p, u32p, u32p]
    lib.or_degree_rank.restype = ctypes.c_int
    lib.or_orient.argtypes = [ctypes.c_uint32, i64p, u32p, u32p, i64p, u32p]
    lib.or_orient.restype = ctypes.c_int64
    lib.or_cuts.argtypes = [ctypes.c_uint32, i64p, ctypes.c_uint32, ctypes.c_int, u32p]
    lib.or_cuts.restype = ctypes.c_int
    lib.or_block_edges.argtypes = [ctypes.c_uint32, i64p, u32p, ctypes.c_uint32, u32p, u64p]
    lib.or_block_edges.restype = ctypes.c_int
    lib.or_triples.argtypes = [ctypes.c_uint32, u64p, u32p, u64p]
    lib.or_triples.restype = ctypes.c_int64
    lib.or_tc_forward.argtypes = [ctypes.c_uint32, i64p, u32p, u64p, ctypes.c_uint32, u32p, u64p]
    lib.or_tc_forward.restype = ctypes.c_uint64
    lib.or_alg_bytes.argtypes = [ctypes.c_uint32, i64p, u32p]
    lib.or_alg_bytes.restype = ctypes.c_uint64
    lib.or_k4_count.argtypes = [ctypes.c_uint32, i64p, u32p]
    lib.or_k4_count.restype = ctypes.c_uint64
    lib.or_c4_count.argtypes = [ctypes.c_uint32, i64p, u32p]
    lib.or_c4_count.restype = ctypes.c_uint64
    lib.or_cc_min_label.argtypes = [ctypes.c_uint32, i64p, u32p, u32p]
    lib.or_cc_min_label.restype = ctypes.c_int64
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.or_pagerank.argtypes = [ctypes.c_uint32, i64p, u32p, ctypes.c_double, ctypes.c_double, ctypes.c_int, f64p,
                                f64p]
    lib.or_pagerank.restype = ctypes.c_int
    if hasattr(lib, "or_tc_forward_mt"):
        lib.or_tc_forward_mt.argtypes = [ctypes.c_uint32, i64p, u32p, u64p, ctypes.c_int, ctypes.c_uint32]
        lib.or_tc_forward_mt.restype = ctypes.c_uint64
        lib.or_num_threads.argtypes = []
        lib.or_num_threads.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load the oracle library (``path`` selects a separately built copy)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(ctypes.CDLL(_LIB))
    return _lib


def load_mt():
    """The OpenMP build (same source compiled with -fopenmp)."""
    global _lib_mt
    with _lock:
        if _lib_mt is None:
            build(openmp=True)
            _lib_mt = _bind(ctypes.CDLL(_LIB_MT))
    return _lib_mt


def num_threads() -> int:
    """Threads the OpenMP build uses by default."""
    return int(load_mt().or_num_threads())


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


class Graph:
    """Cleaned symmetric adjacency (original IDs): ``offs`` int64[n+1], ``adj`` uint32."""

    def __init__(self, n, offs, adj, lib=None):
        self.n, self.offs, self.adj, self.lib = n, offs, adj, lib or load()

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return int(self.offs[-1]) // 2

    def degree(self) -> np.ndarray:
        return np.diff(self.offs)


def clean(src, dst, n: int, lib=None) -> Graph:
    """Section 5.1: undirected, deduplicated, self-loop-free adjacency."""
    lib = lib or load()
    src, dst = _u32(src), _u32(dst)
    m = len(src)
    offs = np.zeros(n + 1, dtype=np.int64)
    adj = np.empty(max(2 * m, 1), dtype=np.uint32)
    got = lib.or_clean(n, m, _p(src, ctypes.c_uint32), _p(dst, ctypes.c_uint32),
                       _p(offs, ctypes.c_int64), _p(adj, ctypes.c_uint32))
    if got < 0:
        raise ValueError("vertex ID out of range" if got == -1 else "out of memory")
    return Graph(n, offs, adj[:got], lib)  # a view: no second copy of a large adjacency


def tc_node_iterator(g: Graph, per_vertex: bool = True):
    """Global count T and per-vertex counts t (original IDs)."""
    t = np.zeros(max(g.n, 1), dtype=np.uint64) if per_vertex else None
    tot = g.lib.or_tc_node_iterator(g.n, _p(g.offs, ctypes.c_int64), _p(g.adj, ctypes.c_uint32),
                                    _p(t, ctypes.c_uint64) if per_vertex else None)
    return int(tot), (t[: g.n] if per_vertex else None)


def tc_vertex(g: Graph, xs) -> np.ndarray:
    """t[x] for each x in ``xs``, computed one vertex at a time."""
    xs = _u32(xs)
    out = np.zeros(len(xs), dtype=np.uint64)
    g.lib.or_tc_vertex_sample(g.n, _p(g.offs, ctypes.c_int64), _p(g.adj, ctypes.c_uint32),
                              len(xs), _p(xs, ctypes.c_uint32), _p(out, ctypes.c_uint64))
    return out


class Oriented:
    """Degree-ordered, upper-oriented CSR in rank space."""

    def __init__(self, n, perm, rank, rowptr, col, lib):
        self.n, self.perm, self.rank, self.rowptr, self.col, self.lib = n, perm, rank, rowptr, col, lib

    @property
    def m(self) -> int:
        return int(self.rowptr[-1])


def orient(g: Graph) -> Oriented:
    """Section 5.4: degree ordering (ties by ID) and upper orientation."""
    lib, n = g.lib, g.n
    perm = np.empty(max(n, 1), dtype=np.uint32)
    rank = np.empty(max(n, 1), dtype=np.uint32)
    lib.or_degree_rank(n, _p(g.offs, ctypes.c_int64), _p(perm, ctypes.c_uint32), _p(rank, ctypes.c_uint32))
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.empty(max(g.m, 1), dtype=np.uint32)
    got = lib.or_orient(n, _p(g.offs, ctypes.c_int64), _p(g.adj, ctypes.c_uint32),
                        _p(rank, ctypes.c_uint32), _p(rowptr, ctypes.c_int64), _p(col, ctypes.c_uint32))
    assert got == g.m
    return Oriented(n, perm[:n], rank[:n], rowptr, col[:got].copy(), lib)


def cuts(o: Oriented, p: int, rule: int = CUT_NNZ) -> np.ndarray:
    c = np.zeros(p + 1, dtype=np.uint32)
    rc = o.lib.or_cuts(o.n, _p(o.rowptr, ctypes.c_int64), p, rule, _p(c, ctypes.c_uint32))
    if rc != 0:
        raise ValueError("p must be >= 1")
    return c


def block_edges(o: Oriented, p: int, c: np.ndarray) -> np.ndarray:
    be = np.zeros(p * p, dtype=np.uint64)
    c = _u32(c)
    o.lib.or_block_edges(o.n, _p(o.rowptr, ctypes.c_int64), _p(o.col, ctypes.c_uint32), p,
                         _p(c, ctypes.c_uint32), _p(be, ctypes.c_uint64))
    return be.reshape(p, p)


def triples(p: int, be: np.ndarray, lib=None):
    """(ijk[T,3], weight[T]) in queue order (weight descending, then i, j, k)."""
    lib = lib or load()
    be = np.ascontiguousarray(be, dtype=np.uint64).reshape(-1)
    cap = max(p * (p + 1) * (p + 2) // 6, 1)
    ijk = np.zeros(3 * cap, dtype=np.uint32)
    w = np.zeros(cap, dtype=np.uint64)
    cnt = lib.or_triples(p, _p(be, ctypes.c_uint64), _p(ijk, ctypes.c_uint32), _p(w, ctypes.c_uint64))
    return ijk[: 3 * cnt].reshape(cnt, 3), w[:cnt]


def tc_forward(o: Oriented, p: int | None = None, c=None, per_vertex: bool = True):
    """(T, t_orig or None, triple_counts[p,p,p] or None) over the oriented graph."""
    n = o.n
    t = np.zeros(max(n, 1), dtype=np.uint64) if per_vertex else None
    tc = None
    cptr = None
    if p is not None:
        tc = np.zeros(p * p * p, dtype=np.uint64)
        c = _u32(c)
        cptr = _p(c, ctypes.c_uint32)
    tot = o.lib.or_tc_forward(n, _p(o.rowptr, ctypes.c_int64), _p(o.col, ctypes.c_uint32),
                              _p(t, ctypes.c_uint64) if per_vertex else None,
                              p or 0, cptr, _p(tc, ctypes.c_uint64) if tc is not None else None)
    t_orig = None
    if per_vertex:
        t_orig = np.zeros(n, dtype=np.uint64)
        t_orig[o.perm] = t[:n]
    return int(tot), t_orig, (tc.reshape(p, p, p) if tc is not None else None)


def tc_forward_mt(o: Oriented, per_vertex: bool = True, threads: int = 0, stride: int = 1):
    """(T, t_orig or None): the forward count with its rows shared among
    OpenMP threads (``threads`` <= 0: OpenMP's default).  With ``stride``
    1 the counts equal ``tc_forward``'s; a larger stride counts only rows
    0, stride, 2 stride, ... (a timing sample)."""
    lib = load_mt()
    n = o.n
    t = np.zeros(max(n, 1), dtype=np.uint64) if per_vertex else None
    tot = lib.or_tc_forward_mt(n, _p(o.rowptr, ctypes.c_int64), _p(o.col, ctypes.c_uint32),
                               _p(t, ctypes.c_uint64) if per_vertex else None, int(threads), int(stride))
    if tot == (1 << 64) - 1:
        raise MemoryError("per-thread counters")
    t_orig = None
    if per_vertex:
        t_orig = np.zeros(n, dtype=np.uint64)
        t_orig[o.perm] = t[:n]
    return int(tot), t_orig


def k4_count(g: Graph) -> int:
    """Number of 4-cliques."""
    return int(g.lib.or_k4_count(g.n, _p(g.offs, ctypes.c_int64), _p(g.adj, ctypes.c_uint32)))


def c4_count(g: Graph) -> int:
    """Number of 4-cycles (butterflies on a bipartite graph)."""
    c = int(g.lib.or_c4_count(g.n, _p(g.offs, ctypes.c_int64), _p(g.adj, ctypes.c_uint32)))
    if c == (1 << 64) - 1:
        raise MemoryError("pair counters")
    return c


def cc_min_label(g: Graph):
    """(labels, components): label[x] = smallest vertex ID in x's component."""
    lab = np.zeros(max(g.n, 1), dtype=np.uint32)
    c = g.lib.or_cc_min_label(g.n, _p(g.offs, ctypes.c_int64), _p(g.adj, ctypes.c_uint32), _p(lab, ctypes.c_uint32))
    if c < 0:
        raise MemoryError("components queue")
    return lab[: g.n], int(c)


def pagerank(g: Graph, damping: float = 0.85, tol: float = 1e-4, max_iter: int = 20):
    """(ranks float64[n], iterations, last L1 change) of the undirected graph."""
    r = np.zeros(max(g.n, 1), dtype=np.float64)
    err = ctypes.c_double()
    it = g.lib.or_pagerank(g.n, _p(g.offs, ctypes.c_int64), _p(g.adj, ctypes.c_uint32), damping, tol, max_iter,
                           _p(r, ctypes.c_double), ctypes.byref(err))
    if it < 0:
        raise MemoryError("rank arrays")
    return r[: g.n], int(it), float(err.value)


def alg_bytes(o: Oriented) -> int:
    return int(o.lib.or_alg_bytes(o.n, _p(o.rowptr, ctypes.c_int64), _p(o.col, ctypes.c_uint32)))
