"""The seeded generators on the device (``graphgen_dev.cu``): the same raw edge
lists as the host functions of ``graphgen``, edge for edge, written into
uint32 CUDA tensors on a given stream.  Input plumbing only.

Each function returns ``(src, dst, n)`` with ``src``/``dst`` torch uint32
tensors on the current CUDA device.  ``stream`` is a ``torch.cuda.Stream``
(default: the current stream); the tensors are ready once that stream
reaches the point of the call.
"""
from __future__ import annotations

import ctypes
import math
import threading

from . import RMAT_ABC, RELABEL, _DEV_LIB, build_device, serve_spec, shuffle_permutation

_lock = threading.Lock()
_lib = None


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_device()
            lib = ctypes.CDLL(_DEV_LIB)
            vp = ctypes.c_void_p
            lib.ggd_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, ctypes.c_int, vp, vp, vp, vp]
            lib.ggd_rmat.restype = ctypes.c_int
            lib.ggd_er_pairs.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, vp, vp, vp]
            lib.ggd_er_pairs.restype = ctypes.c_int
            lib.ggd_rgg_plan.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, vp,
                                         ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64)]
            lib.ggd_rgg_plan.restype = ctypes.c_int
            lib.ggd_rgg_fill.argtypes = [vp, vp, vp, vp]
            lib.ggd_rgg_fill.restype = ctypes.c_int
            lib.ggd_rgg_free.argtypes = [vp, vp]
            lib.ggd_rgg_free.restype = None
            _lib = lib
    return _lib


def _on(stream):
    """Context that makes ``stream`` current (allocations and copies of the
    call are then ordered on it)."""
    import contextlib

    import torch
    return torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()


def _cur():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _pair(m: int):
    import torch
    return (torch.empty(max(m, 1), dtype=torch.uint32, device="cuda")[:m],
            torch.empty(max(m, 1), dtype=torch.uint32, device="cuda")[:m])


def _p(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed ({rc})")


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, abc=RMAT_ABC, relabel: str = "feistel",
         stream=None):
    """``graphgen.rmat(scale, edge_factor, seed, abc, relabel=relabel)`` on the
    device.  ``"shuffle"`` makes the Fisher-Yates permutation on the host
    (a sequential walk over 2^scale labels) and applies it on the device."""
    import torch
    n = 1 << scale
    m = edge_factor * n
    with _on(stream):
        src, dst = _pair(m)
        perm = None
        if relabel == "shuffle":
            perm = torch.from_numpy(shuffle_permutation(n, seed)).to("cuda")
        _check(_load().ggd_rmat(scale, m, abc[0], abc[1], abc[2], seed, RELABEL[relabel], _p(perm), _p(src),
                                _p(dst), _cur()), "ggd_rmat")
    return src, dst, n


def er_pairs(n: int, m: int, seed: int = 1, stream=None):
    """``graphgen.er_pairs(n, m, seed)`` on the device."""
    with _on(stream):
        src, dst = _pair(m)
        _check(_load().ggd_er_pairs(n, m, seed, _p(src), _p(dst), _cur()), "ggd_er_pairs")
    return src, dst, n


def rgg(n: int, r: float | None = None, seed: int = 1, stream=None):
    """``graphgen.rgg(n, r, seed)`` on the device (same edges, same order).
    Synchronises the stream once, to size the output."""
    if r is None:
        r = math.sqrt(6.0 / (math.pi * max(n, 1)))
    lib = _load()
    with _on(stream):
        plan = ctypes.c_void_p()
        cnt = ctypes.c_int64()
        st = _cur()
        _check(lib.ggd_rgg_plan(n, r, seed, st, ctypes.byref(plan), ctypes.byref(cnt)), "ggd_rgg_plan")
        try:
            src, dst = _pair(int(cnt.value))
            _check(lib.ggd_rgg_fill(plan, _p(src), _p(dst), st), "ggd_rgg_fill")
        finally:
            lib.ggd_rgg_free(plan, st)
    return src, dst, n


def serve_job(i: int, max_scale: int, stream=None):
    """Job i of the serving workload (``graphgen.serve_spec``) generated on
    the device: the same edges as ``graphgen.serve_job``."""
    sp = serve_spec(i, max_scale)
    if sp[0] == "rmat":
        return rmat(sp[1], sp[2], i, relabel="feistel", stream=stream)
    if sp[0] == "er":
        return er_pairs(sp[1], sp[2], i, stream=stream)
    return rgg(sp[1], None, i, stream=stream)
