"""The allocation-free entry point against the regular one.

pgb_tc_count_oriented_noalloc exists for callers that may not allocate
device memory while counting (a host framework that owns all device memory,
or a latency-critical loop that cannot take cudaMalloc's synchronisation).
It keeps its working memory in one fixed device array inside the library, so
these checks call it twice in a row (the second call must not see the
first call's leftovers), then on a smaller graph, and compare every count
bit-exactly (integer counts, tolerance 0) with pgb_tc_run on the same graph
and with the oracle.  They also check that the call makes no allocation
through the library's allocator (which the binding points at torch's caching
allocator), and that each broken input rule is reported and leaves nothing
behind for the next call.

This file is collected last so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import graphgen
import oracle

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


def _oracle_counts(src, dst, n):
    T, t, _ = oracle.tc_forward(oracle.orient(oracle.clean(src, dst, n)))
    return T, t


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    src, dst, n = graphgen.rmat(16, 16, 3)
    T, t, rowptr, col, perm = _regular(src, dst, n, 4)
    oT, ot = _oracle_counts(src, dst, n)
    assert T == oT > 0 and np.array_equal(t, ot)
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
    oT2, ot2 = _oracle_counts(src2, dst2, n2)
    assert T2 == oT2 and np.array_equal(t2, ot2)
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


# (name, n, rowptr, col, perm, message fragment): each breaks one input rule;
# every read the kernels make stays inside rowptr[0..n] and col[0..m).
MALFORMED = [
    ("column_out_of_range", 2, [0, 1, 1], [5], None, "out of range"),
    ("rowptr0_not_zero", 2, [1, 1, 1], [1], None, "out of range"),
    ("rowptr_n_not_m", 2, [0, 1, 1], [1, 1], None, "out of range"),
    ("rowptr_decreasing", 3, [0, 2, 1, 2], [1, 2], None, "not strictly ascending"),
    ("column_not_above_row", 3, [0, 1, 2, 2], [1, 0], None, "not strictly ascending"),
    ("row_descending", 3, [0, 2, 2, 2], [2, 1], None, "not strictly ascending"),
    ("row_repeated_column", 3, [0, 2, 2, 2], [1, 1], None, "not strictly ascending"),
    ("perm_out_of_range", 3, [0, 2, 3, 3], [1, 2, 2], [0, 1, 7], "out of range"),
    ("perm_repeated_vertex", 3, [0, 2, 3, 3], [1, 2, 2], [0, 0, 2], "two ranks"),
]


@pytest.mark.parametrize("case", MALFORMED, ids=lambda c: c[0])
def test_noalloc_reports_each_broken_rule_then_counts_cleanly(case):
    _, n, rp, cl, pm, why = case
    rowptr = torch.tensor(rp, dtype=torch.uint32, device="cuda")
    col = torch.tensor(cl, dtype=torch.uint32, device="cuda")
    perm = torch.tensor(pm, dtype=torch.uint32, device="cuda") if pm is not None else None
    total = torch.zeros(1, dtype=torch.uint64, device="cuda")
    pv = torch.zeros(n, dtype=torch.uint64, device="cuda")
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_count_oriented_noalloc(n, len(cl), rowptr, col, perm, total, pv)
    assert ei.value.code == P.PGB_E_INVAL
    assert why in str(ei.value)
    # K4 right after: the error word, the counters and the perm bitmap start clean
    k4_rowptr = torch.tensor([0, 3, 5, 6, 6], dtype=torch.uint32, device="cuda")
    k4_col = torch.tensor([1, 2, 3, 2, 3, 3], dtype=torch.uint32, device="cuda")
    k4_perm = torch.tensor([3, 1, 0, 2], dtype=torch.uint32, device="cuda")
    for _ in range(2):
        got_T, got_t = _noalloc(4, k4_rowptr, k4_col, k4_perm)
        assert got_T == 4 and got_t.tolist() == [3, 3, 3, 3]
