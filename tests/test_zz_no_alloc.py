"""The allocation-free entry point against the regular one.

pgb_tc_count_oriented_noalloc exists for callers that may not allocate
device memory while counting (a host framework that owns all device memory,
or a latency-critical loop that cannot take cudaMalloc's synchronisation).
It keeps its working memory in one fixed device array inside the library, so
these checks call it twice in a row (the second call must not see the
first call's leftovers), then on a smaller graph, and compare every count
bit-exactly (integer counts, tolerance 0) with pgb_tc_run on the same graph.
They also check that the call makes no allocation through the library's
allocator (which the binding points at torch's caching allocator).

This file is collected last so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402


def _regular(src, dst, n, p):
    ds = torch.from_numpy(src).cuda()
    dd = torch.from_numpy(dst).cuda()
    g = P.pgb_graph_from_edges(ds, dd, n)
    b = P.pgb_partition(g, p)
    T, t = P.pgb_tc_result_get(P.pgb_tc_run(b))
    rowptr = torch.from_numpy(P.pgb_blocks_export(b, P.PGB_EXPORT_ROWPTR).astype(np.uint32)).cuda()
    col = torch.from_numpy(P.pgb_blocks_export(b, P.PGB_EXPORT_COL)).cuda()
    perm = torch.from_numpy(P.pgb_blocks_export(b, P.PGB_EXPORT_PERM)).cuda()
    return T, t, rowptr, col, perm


def _allocations():
    return torch.cuda.memory_stats().get("allocation.all.allocated", 0)


def _noalloc(n, rowptr, col, perm, per_vertex=True):
    total = torch.full((1,), 987654321, dtype=torch.uint64, device="cuda")
    pv = torch.full((n,), 7, dtype=torch.uint64, device="cuda") if per_vertex else None
    torch.cuda.synchronize()
    before = _allocations()
    P.pgb_tc_count_oriented_noalloc(n, col.numel(), rowptr, col, perm, total, pv)
    after = _allocations()
    assert after == before, "the no-allocation entry point allocated through the library allocator"
    return int(total.item()), (pv.cpu().numpy() if per_vertex else None)


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    src, dst, n = graphgen.rmat(16, 16, 3)
    T, t, rowptr, col, perm = _regular(src, dst, n, 4)
    assert T > 0
    for _ in range(2):
        got_T, got_t = _noalloc(n, rowptr, col, perm)
        assert got_T == T
        assert np.array_equal(got_t, t)
    # rank-indexed output and global-only output
    got_T, got_rank = _noalloc(n, rowptr, col, None)
    assert got_T == T
    assert np.array_equal(got_rank, t[perm.cpu().numpy()])
    assert _noalloc(n, rowptr, col, perm, per_vertex=False)[0] == T
    # a smaller graph right after a larger one
    src2, dst2, n2 = graphgen.er_distinct(4096, 65536, 1)
    T2, t2, rowptr2, col2, perm2 = _regular(src2, dst2, n2, 4)
    for _ in range(2):
        got_T, got_t = _noalloc(n2, rowptr2, col2, perm2)
        assert got_T == T2
        assert np.array_equal(got_t, t2)


def test_noalloc_rejects_sizes_beyond_its_limit():
    n = P.PGB_NOALLOC_MAX_VERTICES + 1
    rowptr = torch.zeros(n + 1, dtype=torch.uint32, device="cuda")
    total = torch.zeros(1, dtype=torch.uint64, device="cuda")
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_count_oriented_noalloc(n, 0, rowptr, None, None, total, None)
    assert ei.value.code == P.PGB_E_INVAL
    assert "limit" in str(ei.value)


def test_noalloc_reports_malformed_columns():
    # rowptr = [0, 1, 1]: one edge 0 -> 5 with column out of range for n = 2
    rowptr = torch.tensor([0, 1, 1], dtype=torch.uint32, device="cuda")
    col = torch.tensor([5], dtype=torch.uint32, device="cuda")
    total = torch.zeros(1, dtype=torch.uint64, device="cuda")
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_count_oriented_noalloc(2, 1, rowptr, col, None, total, None)
    assert ei.value.code == P.PGB_E_INVAL
