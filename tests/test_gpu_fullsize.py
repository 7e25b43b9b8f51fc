"""Full-size parity: the CUDA path on the benchmark's own workloads.

Expected values come from the oracle only, written by
``tests/golden/make_golden.py`` into ``tests/golden/full_<name>.txt``: the
exact triangle total, the SHA-256 of all n per-vertex counts (uint64
little-endian, original vertex IDs), and t[x] for a seeded vertex sample by
the oracle's one-vertex count.  The checks are bit-exact (tolerance 0):
total, every per-vertex count (through the digest), every sampled count,
and sum(t) = 3 T.

R-MAT scale 20 (p = 16) runs in the plain one-launch-per-triple mode and in
the persistent mode; R-MAT scale 24 (p = 32) and the 4096 x 4096 grid with
1% extra edges (p = 32) run in the launch configuration bench.py times
(persistent, automatic variant, per-vertex); R-MAT scale 27 (p = 64) runs
resident and with the in-edge index streamed under a 16 GiB budget.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


def digest(t):
    return hashlib.sha256(np.ascontiguousarray(t, dtype="<u8").tobytes()).hexdigest()


def run_full(name, p, mode, variant=P.PGB_VAR_AUTO, stream_budget=None, cache_budget=None):
    want = make_golden.load(name)
    src, dst, n = make_golden.generate(make_golden.WORKLOADS[name])
    assert n == want["n"]
    ds = torch.from_numpy(src).cuda()
    dd = torch.from_numpy(dst).cuda()
    src_keep = (src, dst) if cache_budget is not None else None
    del src, dst
    g = P.pgb_graph_from_edges(ds, dd, n)
    assert P.pgb_graph_info(g)[1] == want["m"]
    b = P.pgb_partition(g, p)
    g.free()
    del ds, dd
    tv = torch.zeros(n, dtype=torch.uint64, device="cuda")
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=mode, variant=variant))
    T, _ = P.pgb_tc_result_get(r, per_vertex=tv)
    assert T == want["T"]
    t = tv.cpu().numpy()
    assert digest(t) == want["t_sha256"], "per-vertex counts differ from the oracle's"
    assert np.array_equal(t[want["x"]], want["t"])
    assert int(t.sum(dtype=np.uint64)) == 3 * T
    if stream_budget is not None:
        # the same graph with the in-edge index streamed under a budget
        P.pgb_blocks_offload(b)
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=mode, variant=variant, device_budget=stream_budget))
        T2, _ = P.pgb_tc_result_get(r, per_vertex=tv)
        assert T2 == T and P.pgb_tc_result_stream(r)[1] > 1
        assert np.array_equal(tv.cpu().numpy(), t)
    b.free()
    del r
    torch.cuda.empty_cache()
    if cache_budget is not None:
        # a fresh partition with the columns offloaded too (block cache tier)
        b2 = P.pgb_partition(P.pgb_graph_from_edges(torch.from_numpy(src_keep[0]).cuda(),
                                                    torch.from_numpy(src_keep[1]).cuda(), n), p)
        P.pgb_blocks_offload_columns(b2, cache_budget[1])
        r = P.pgb_tc_run(b2, P.pgb_tc_opts_default(device_budget=cache_budget[0]))
        T3, _ = P.pgb_tc_result_get(r, per_vertex=tv)
        assert T3 == T and P.pgb_tc_result_stream(r, slice_loads=True)[2] > 0
        assert digest(tv.cpu().numpy()) == want["t_sha256"]
        b2.free()
        del r
        torch.cuda.empty_cache()


@pytest.mark.parametrize("mode", [P.PGB_MODE_PLAIN, P.PGB_MODE_PERSISTENT])
def test_rmat20_p16_full_size(mode):
    run_full("rmat20", 16, mode)


def test_rmat24_p32_full_size_bench_configuration():
    run_full("rmat24", 32, P.PGB_MODE_PERSISTENT)


def test_rmat24_p32_full_size_bsearch_variant():
    run_full("rmat24", 32, P.PGB_MODE_PERSISTENT, P.PGB_VAR_BSEARCH)


@pytest.mark.parametrize("mode", [P.PGB_MODE_PLAIN, P.PGB_MODE_PERSISTENT])
def test_grid4096_p32_full_size(mode):
    """The 4096 x 4096 grid with 1% uniform extra edges at full size."""
    run_full("grid4096", 32, mode)


def test_rmat27_p64_full_size_and_streamed():
    """R-MAT scale 27 (2.1 G edges, the autotuned 512-thread shape): the
    oracle's total and every per-vertex count, resident; with the columns
    offloaded too under a 4 GiB budget (block cache tier, 45 row ranges);
    and with the in-edge index streamed under a 16 GiB budget."""
    run_full("rmat27", 64, P.PGB_MODE_PERSISTENT, stream_budget=16 << 30, cache_budget=(4 << 30, 45))
