"""Allocator hooks on the GPU: kernels read rows with aligned 32-byte loads,
so the library takes only 256-byte aligned blocks from a hook.  A hook that
hands out misaligned memory makes the call fail with PGB_E_INVAL before any
kernel runs, and the block goes back to the hook's free function.

Runs in a child process: the hook can only change while no handle is alive,
and the test session's library has the torch allocator installed."""
import os
import subprocess
import sys
import textwrap

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import ctypes, sys
    import numpy as np
    import torch
    from paper_2209_04541_b300 import pgabb as P
    lib = P.load(register_torch_allocator=False)
    raw_alloc = torch._C._cuda_cudaCachingAllocator_raw_alloc
    raw_delete = torch._C._cuda_cudaCachingAllocator_raw_delete
    shift = int(sys.argv[1])
    live = {}
    def _alloc(size, stream, ctx):
        base = raw_alloc(int(size) + 256, int(stream or 0))
        live[base + shift] = base
        return base + shift
    def _free(ptr, size, stream, ctx):
        raw_delete(live.pop(int(ptr)))
    fa, ff = P._ALLOC_FN(_alloc), P._FREE_FN(_free)
    assert lib.pgb_set_allocator(fa, ff, None) == 0
    src = np.array([0, 1, 2, 0], np.uint32)
    dst = np.array([1, 2, 0, 3], np.uint32)
    try:
        g = P.pgb_graph_from_edges(src, dst, 4)
        b = P.pgb_partition(g, 1)
        T, _ = P.pgb_tc_result_get(P.pgb_tc_run(b, P.pgb_tc_opts_default()))
        b.free(); g.free()
        print("ok", T, len(live))
    except P.PgbError as e:
        print("err", e.code, len(live))
""")


@pytest.mark.parametrize("shift", [0, 16])
def test_hook_alignment(shift):
    out = subprocess.run([sys.executable, "-c", CHILD, str(shift)], cwd=ROOT, capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    last = out.stdout.strip().splitlines()[-1].split()
    if shift == 0:
        assert last[0] == "ok" and int(last[1]) == 1
    else:
        # refused before any kernel ran; every block went back to the hook
        assert last[0] == "err" and int(last[1]) == -1 and int(last[2]) == 0
