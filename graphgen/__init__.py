"""Seeded synthetic graph generators (raw edge lists) shared by the oracle and
the CUDA path.

This module is input plumbing only: it holds none of the triangle-counting
arithmetic.  Every function returns ``(src, dst, n)`` with ``src``/``dst``
uint32 numpy arrays of equal length (one raw edge per position) and ``n`` the
vertex count.  Which generators keep duplicates or self-loops is stated per
function; the consumer's ingest step removes them.

The C implementation (``graphgen.c``) draws from one counter-based SplitMix64
stream per generator, so outputs are bit-identical for any thread count.
The workloads stand in for the paper's real-world inputs (PGAbB, Section 5.1:
44 real-world graphs made undirected and deduplicated), which are not
available here.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_HDR = os.path.join(_HERE, "gg_stream.h")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_DEV_SRC = os.path.join(_HERE, "graphgen_dev.cu")
_DEV_LIB = os.path.join(_HERE, "libgraphgen_dev.so")
_lock = threading.Lock()
_lib = None

# relabelling of R-MAT vertex IDs: none, the seeded Fisher-Yates permutation
# (Graph500), or the seeded Feistel bijection (parallel; host and device)
RELABEL = {"none": 0, "shuffle": 1, "feistel": 2}

# R-MAT quadrant probabilities of the Graph500 Kronecker generator.
RMAT_ABC = (0.57, 0.19, 0.19)


def _stale(lib: str, *srcs: str) -> bool:
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(x) for x in srcs)


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` with gcc (OpenMP) if missing or stale."""
    if not force and not _stale(_LIB, _SRC, _HDR):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def build_device(force: bool = False) -> str:
    """Compile ``libgraphgen_dev.so`` (the device generators) with nvcc for
    sm_103a if missing or stale."""
    if not force and not _stale(_DEV_LIB, _DEV_SRC, _HDR):
        return _DEV_LIB
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    tmp = _DEV_LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo", "-shared",
           "-Xcompiler", "-fPIC", "-o", tmp, _DEV_SRC]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _DEV_LIB)
    return _DEV_LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.gg_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                    ctypes.c_int, u32p, u32p]
            lib.gg_rmat.restype = ctypes.c_int
            lib.gg_er_pairs.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.gg_er_pairs.restype = ctypes.c_int
            lib.gg_er_distinct.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p, u32p]
            lib.gg_er_distinct.restype = ctypes.c_int
            lib.gg_grid_count.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
            lib.gg_grid_count.restype = ctypes.c_uint64
            lib.gg_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_uint64, u32p, u32p]
            lib.gg_grid.restype = ctypes.c_int
            lib.gg_rgg.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, u32p, u32p]
            lib.gg_rgg.restype = ctypes.c_int64
            lib.gg_splitmix_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_splitmix_draw.restype = ctypes.c_uint64
            lib.gg_splitmix_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_splitmix_raw.restype = ctypes.c_uint64
            lib.gg_num_threads.restype = ctypes.c_int
            lib.gg_feistel_label.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
            lib.gg_feistel_label.restype = ctypes.c_uint32
            lib.gg_shuffle_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
            lib.gg_shuffle_permutation.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _empty(m: int, pinned_alloc=None):
    if pinned_alloc is not None:
        return pinned_alloc(m), pinned_alloc(m)
    return np.empty(m, dtype=np.uint32), np.empty(m, dtype=np.uint32)


def splitmix_draw(seed: int, c: int) -> int:
    """Draw ``c`` of the SplitMix64 stream keyed by ``seed`` (for tests)."""
    return int(_load().gg_splitmix_draw(seed, c))


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, abc=RMAT_ABC,
         permute: bool = True, out=None, relabel: str = "shuffle"):
    """R-MAT graph: ``edge_factor * 2**scale`` raw edges on ``2**scale`` vertices.

    Quadrant probabilities ``(a, b, c, 1-a-b-c)``; no noise; seeded vertex
    relabelling when ``permute``, by ``relabel``: ``"shuffle"`` (the
    Fisher-Yates permutation) or ``"feistel"`` (the Feistel bijection, which
    the device generator evaluates in parallel).  Duplicates and self-loops
    are kept.  ``out`` may be a pair of preallocated uint32 arrays (e.g.
    pinned).
    """
    n = 1 << scale
    m = edge_factor * n
    src, dst = out if out is not None else _empty(m)
    mode = RELABEL[relabel] if permute else 0
    rc = _load().gg_rmat(scale, m, abc[0], abc[1], abc[2], seed, mode, _ptr(src), _ptr(dst))
    if rc != 0:
        raise ValueError(f"gg_rmat failed ({rc})")
    return src, dst, n


def er_distinct(n: int, m: int, seed: int = 1):
    """Erdos-Renyi G(n, m): ``m`` distinct pairs, no self-loops, random direction."""
    src, dst = _empty(m)
    rc = _load().gg_er_distinct(n, m, seed, _ptr(src), _ptr(dst))
    if rc != 0:
        raise ValueError(f"gg_er_distinct failed ({rc})")
    return src, dst, n


def er_pairs(n: int, m: int, seed: int = 1, out=None):
    """``m`` i.i.d. uniform ordered pairs over ``[0, n)^2`` (duplicates and
    self-loops kept)."""
    src, dst = out if out is not None else _empty(m)
    rc = _load().gg_er_pairs(n, m, seed, _ptr(src), _ptr(dst))
    if rc != 0:
        raise ValueError(f"gg_er_pairs failed ({rc})")
    return src, dst, n


def grid(w: int, h: int, extra: int = 0, seed: int = 1):
    """``w x h`` 4-neighbour grid plus ``extra`` uniform random pairs (no
    self-loops; repeats of grid edges possible)."""
    lib = _load()
    m = int(lib.gg_grid_count(w, h, extra))
    src, dst = _empty(m)
    rc = lib.gg_grid(w, h, extra, seed, _ptr(src), _ptr(dst))
    if rc != 0:
        raise ValueError(f"gg_grid failed ({rc})")
    return src, dst, w * h


def grid_plus_percent(side: int = 4096, percent: float = 1.0, seed: int = 1):
    """Square grid with ``percent``% (of the grid's edge count, rounded) random
    extra edges."""
    base = 2 * side * (side - 1)
    extra = int(round(base * percent / 100.0))
    return grid(side, side, extra, seed)


def rgg(n: int, r: float | None = None, seed: int = 1):
    """Random geometric graph in the unit square; default radius gives an
    expected average degree of about 6 (``r = sqrt(6 / (pi n))``)."""
    if r is None:
        r = math.sqrt(6.0 / (math.pi * max(n, 1)))
    lib = _load()
    cnt = int(lib.gg_rgg(n, r, seed, None, None))
    if cnt < 0:
        raise ValueError(f"gg_rgg failed ({cnt})")
    src, dst = _empty(cnt)
    got = int(lib.gg_rgg(n, r, seed, _ptr(src), _ptr(dst)))
    assert got == cnt
    return src, dst, n


def feistel_label(x: int, bits: int, seed: int) -> int:
    """The Feistel relabelling of ``x`` in ``[0, 2**bits)`` for ``seed``."""
    return int(_load().gg_feistel_label(x, bits, seed))


def shuffle_permutation(n: int, seed: int) -> np.ndarray:
    """The Fisher-Yates relabelling ``rmat`` applies (``relabel="shuffle"``)."""
    perm = np.empty(n, np.uint32)
    _load().gg_shuffle_permutation(n, seed, _ptr(perm))
    return perm


def serve_spec(i: int, max_scale: int):
    """Job i of the serving workload (triangle-count jobs on graphs of mixed
    sizes): the families in equal thirds by i mod 3, R-MAT (scale uniform in
    [10, max_scale], edge factor uniform in [8, 32], Feistel relabelling),
    Erdos-Renyi i.i.d. pairs (n log-uniform in [2^10, 2^max_scale], average
    degree log-uniform in [4, 64]) and random geometric graphs (n
    log-uniform, average degree about 6); parameters drawn from numpy's
    generator seeded by i, graph seed = i.  Returns ("rmat", scale, ef),
    ("er", n, m) or ("rgg", n)."""
    rng = np.random.default_rng(i)
    fam = i % 3
    if fam == 0:
        s = int(rng.integers(10, max_scale + 1))
        ef = int(rng.integers(8, 33))
        return ("rmat", s, ef)
    n = int(round(2.0 ** rng.uniform(10, max_scale)))
    if fam == 1:
        deg = 2.0 ** rng.uniform(2, 6)
        return ("er", n, max(1, int(n * deg / 2)))
    return ("rgg", n)


def serve_job(i: int, max_scale: int):
    """Job i of the serving workload, generated on the host."""
    sp = serve_spec(i, max_scale)
    if sp[0] == "rmat":
        return rmat(sp[1], sp[2], i, relabel="feistel")
    if sp[0] == "er":
        return er_pairs(sp[1], sp[2], i)
    return rgg(sp[1], None, i)


def splitmix_raw(state: int, c: int) -> int:
    """Output ``c`` of plain SplitMix64 started at ``state``."""
    return int(_load().gg_splitmix_raw(state, c))


def num_threads() -> int:
    return int(_load().gg_num_threads())
