"""Streaming tier (Section 4.4 asynchronous block copies; the host-DRAM case
of Section 1): after pgb_blocks_offload the in-edge index lives in pinned host
memory and runs copy it to the device in chunks under a device budget.

Counts are exact integers, so every comparison with the oracle and with the
resident run is bit-exact.  Budgets are chosen so that the index is cut into
several chunks (more than the two slots, so the slots are reused)."""
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import golden_files, load_golden, messy_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb  # noqa: E402

P = pgabb
SLOT_BYTES_PER_IN_EDGE = 44  # index entry (12) + one work item bound (32)


def _blocks(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(np.ascontiguousarray(src, np.uint32)).cuda(),
                               torch.from_numpy(np.ascontiguousarray(dst, np.uint32)).cuda(), n)
    return P.pgb_partition(g, p)


def _budget(b, per_vertex, slot_in_edges):
    return P.pgb_blocks_resident_bytes(b, per_vertex) + 2 * slot_in_edges * SLOT_BYTES_PER_IN_EDGE


def _oracle(src, dst, n):
    g = oracle.clean(src, dst, n)
    return oracle.tc_node_iterator(g)


def _streamed(b, per_vertex, budget, threads=0):
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(per_vertex=int(per_vertex), device_budget=budget,
                                              hash_threads=threads))
    T, t = P.pgb_tc_result_get(r, per_vertex=per_vertex)
    nbytes, chunks = P.pgb_tc_result_stream(r)
    assert P.pgb_tc_result_variant(r) == P.PGB_VAR_HASH
    return T, t, nbytes, chunks


@pytest.mark.parametrize("per_vertex", [True, False])
def test_rmat_streamed_matches_oracle_and_resident(per_vertex):
    src, dst, n = graphgen.rmat(16, 16, 21)
    oT, ot = _oracle(src, dst, n)
    b = _blocks(src, dst, n, 8)
    m = P.pgb_blocks_info(b)["m"]
    rT, rt = P.pgb_tc_result_get(P.pgb_tc_run(b, P.pgb_tc_opts_default(per_vertex=int(per_vertex))),
                                 per_vertex=per_vertex)
    assert rT == oT
    P.pgb_blocks_offload(b)
    T, t, nbytes, chunks = _streamed(b, per_vertex, _budget(b, per_vertex, m // 7))
    assert T == oT == rT
    if per_vertex:
        assert np.array_equal(t, ot) and np.array_equal(t, rt)
    assert chunks >= 7
    # every in-edge's index entry crosses the host link exactly once
    assert nbytes >= 12 * m
    # default budget: one chunk of 1 GiB slots
    T1, t1, nb1, c1 = _streamed(b, per_vertex, 0)
    assert T1 == oT and c1 == 1 and nb1 >= 12 * m
    if per_vertex:
        assert np.array_equal(t1, ot)


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_tiny_slots_many_chunks(threads):
    """Slots of 4096 in-edges, the largest work item: hundreds of chunks."""
    src, dst, n = graphgen.rmat(14, 16, 5)
    oT, ot = _oracle(src, dst, n)
    b = _blocks(src, dst, n, 4)
    P.pgb_blocks_offload(b)
    T, t, _, chunks = _streamed(b, True, _budget(b, True, 4096), threads)
    assert chunks > 20
    assert T == oT and np.array_equal(t, ot)


@pytest.mark.parametrize("path", golden_files(), ids=lambda x: x.split("/")[-1])
def test_golden_fixtures_streamed(path):
    src, dst, n, T, t = load_golden(path)
    for p in sorted({1, 2, n}):
        b = _blocks(src, dst, n, p)
        P.pgb_blocks_offload(b)
        gT, gt, _, _ = _streamed(b, True, _budget(b, True, 4096))
        assert gT == T and np.array_equal(gt, t)


@pytest.mark.parametrize("seed", range(6))
def test_random_messy_streamed(seed):
    rng = np.random.default_rng(7000 + seed)
    n = int(rng.integers(2, 3000))
    m = int(rng.integers(0, 20 * n))
    src, dst = messy_random(n, m, rng)
    oT, ot = _oracle(src, dst, n)
    b = _blocks(src, dst, n, int(rng.integers(1, min(n, 16) + 1)))
    P.pgb_blocks_offload(b)
    T, t, _, _ = _streamed(b, True, _budget(b, True, 4096))
    assert T == oT and np.array_equal(t, ot)


def test_empty_and_edgeless():
    e = np.zeros(0, np.uint32)
    for n in (0, 5):
        b = _blocks(e, e, n, 1)
        P.pgb_blocks_offload(b)
        T, t, nbytes, chunks = _streamed(b, True, 0)
        assert T == 0 and nbytes == 0 and chunks == 0
        assert t.shape == (n,) and not t.any()


def test_offloaded_state_rules():
    src, dst, n = graphgen.rmat(12, 8, 3)
    oT, _ = _oracle(src, dst, n)
    b = _blocks(src, dst, n, 4)
    col_before = P.pgb_blocks_export(b, P.PGB_EXPORT_COL)
    P.pgb_blocks_offload(b)
    P.pgb_blocks_offload(b)  # second call is a no-op
    # the partition's exports still work
    assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_COL), col_before)
    # only the persistent hash path reads a streamed index
    for kw in (dict(mode=P.PGB_MODE_PLAIN), dict(variant=P.PGB_VAR_BSEARCH), dict(variant=P.PGB_VAR_MERGE)):
        with pytest.raises(P.PgbError) as ei:
            P.pgb_tc_run(b, P.pgb_tc_opts_default(**kw))
        assert ei.value.code == P.PGB_E_STATE
    # a budget at or below the resident arrays can never fit
    floor = P.pgb_blocks_resident_bytes(b, True)
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_run(b, P.pgb_tc_opts_default(device_budget=floor))
    assert ei.value.code == P.PGB_E_BUDGET
    # slots smaller than one work item cannot fit either
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_run(b, P.pgb_tc_opts_default(device_budget=floor + 2 * 16 * SLOT_BYTES_PER_IN_EDGE))
    assert ei.value.code == P.PGB_E_BUDGET
    # and the handle still counts afterwards
    assert _streamed(b, True, 0)[0] == oT
    assert P.pgb_blocks_resident_bytes(b, False) < floor


def _induced_top_triangles(src, dst, n, K):
    """Oracle: triangles of the subgraph the K highest ranks induce."""
    g = oracle.clean(src, dst, n)
    o = oracle.orient(g)
    top = np.zeros(n, bool)
    top[o.perm[n - K:]] = True
    s_ = np.repeat(np.arange(n, dtype=np.uint32), np.diff(g.offs).astype(np.int64))
    d_ = g.adj.astype(np.uint32)
    keep = top[s_] & top[d_] & (s_ < d_)
    return oracle.tc_node_iterator(oracle.clean(s_[keep], d_[keep], n), False)[0]


@pytest.mark.parametrize("per_vertex", [True, False])
def test_index_tier_with_dense_top_block(per_vertex):
    """The index tier with the dense top block: its bytes come out of the
    budget, the streamed launches skip its in-edges, and the counts still
    equal the oracle's; the block's own count is the induced subgraph's."""
    src, dst, n = graphgen.rmat(16, 16, 21)
    oT, ot = _oracle(src, dst, n)
    b = _blocks(src, dst, n, 8)
    m = P.pgb_blocks_info(b)["m"]
    P.pgb_blocks_offload(b)
    budget = _budget(b, per_vertex, m // 7) + (256 << 20)
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(per_vertex=int(per_vertex), device_budget=budget, dense_core=2048))
    T, t = P.pgb_tc_result_get(r, per_vertex=per_vertex)
    d = P.pgb_tc_result_dense_core(r)
    assert T == oT and d["ranks"] == 2048 and d["ms"] > 0
    if per_vertex:
        assert np.array_equal(t, ot)
    assert d["triangles"] == _induced_top_triangles(src, dst, n, 2048)
    assert P.pgb_tc_result_stream(r)[1] >= 1
