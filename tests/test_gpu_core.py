"""The dense top block (pgb_tc_opts.dense_core): the triangles among the K
highest ranks are counted from a dense GEMM of the block's adjacency, the
intersection kernels skip the in-edges whose tail is in the block, and the
run's total and per-vertex counts still equal the oracle's bit for bit.  The
block's own count equals the oracle's count on the subgraph the top K ranks
induce (ranks from the oracle's degree order)."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402


def induced_top_triangles(g, K):
    """Oracle: triangles of the subgraph induced by the K highest ranks."""
    o = oracle.orient(g)
    top = np.zeros(g.n, bool)
    top[o.perm[g.n - K:]] = True
    src = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.offs).astype(np.int64))
    dst = g.adj.astype(np.uint32)
    keep = top[src] & top[dst] & (src < dst)
    sub = oracle.clean(src[keep], dst[keep], g.n)
    return oracle.tc_node_iterator(sub, False)[0]


def run(src, dst, n, p, **kw):
    b = P.pgb_partition(P.pgb_graph_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n), p)
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(**kw))
    T, t = P.pgb_tc_result_get(r, per_vertex=bool(kw.get("per_vertex", 1)))
    d = P.pgb_tc_result_dense_core(r)
    return T, t, (d["ranks"], d["triangles"])


CASES = [
    ("rmat12", lambda: graphgen.rmat(12, 16, 7), 4),
    ("rmat13_ef24", lambda: graphgen.rmat(13, 24, 3), 8),
    ("rmat15", lambda: graphgen.rmat(15, 16, 1), 16),
    ("er", lambda: graphgen.er_distinct(5000, 80000, 2), 4),
    ("grid", lambda: graphgen.grid_plus_percent(96, 1.0, 4), 4),
]


@pytest.mark.parametrize("name,make,p", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("K", [256, 1000, 2304, 4096])
def test_dense_block_matches_oracle(name, make, p, K):
    src, dst, n = make()
    g = oracle.clean(src, dst, n)
    T_ref, t_ref = oracle.tc_node_iterator(g)
    T, t, (ranks, tc) = run(src, dst, n, p, dense_core=K)
    want_k = min((K + 255) // 256 * 256, n)
    assert ranks == want_k
    assert T == T_ref and np.array_equal(t, t_ref)
    assert tc == induced_top_triangles(g, ranks)


@pytest.mark.parametrize("variant", ["BSEARCH", "MERGE", "HASH"])
def test_dense_block_with_each_kernel(variant):
    src, dst, n = graphgen.rmat(13, 16, 11)
    g = oracle.clean(src, dst, n)
    T_ref, t_ref = oracle.tc_node_iterator(g)
    T, t, (ranks, _) = run(src, dst, n, 8, dense_core=2048, variant=getattr(P, "PGB_VAR_" + variant))
    assert ranks == 2048 and T == T_ref and np.array_equal(t, t_ref)


def test_whole_graph_as_one_dense_block():
    """K = n: the GEMM counts every triangle, the kernels skip every in-edge."""
    src, dst, n = graphgen.rmat(11, 16, 5)
    g = oracle.clean(src, dst, n)
    T_ref, t_ref = oracle.tc_node_iterator(g)
    T, t, (ranks, tc) = run(src, dst, n, 4, dense_core=n)
    assert ranks == n and tc == T_ref and T == T_ref and np.array_equal(t, t_ref)


def test_dense_block_off_totals_only_and_graph_replay():
    src, dst, n = graphgen.rmat(14, 16, 2)
    g = oracle.clean(src, dst, n)
    T_ref, t_ref = oracle.tc_node_iterator(g)
    T, _, (ranks, tc) = run(src, dst, n, 8, dense_core=-1)
    assert ranks == 0 and tc == 0 and T == T_ref
    b = P.pgb_partition(P.pgb_graph_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n), 8)
    for kw in (dict(dense_core=3072, per_vertex=0), dict(dense_core=3072, use_graph=1),
               dict(dense_core=3072, use_graph=1)):
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(**kw))
        pv = bool(kw.get("per_vertex", 1))
        T, t = P.pgb_tc_result_get(r, per_vertex=pv)
        assert T == T_ref
        if pv:
            assert np.array_equal(t, t_ref)
        d = P.pgb_tc_result_dense_core(r)
        assert d["ranks"] == 3072 and (d["ms"] == -1.0) == bool(kw.get("use_graph"))


def test_autotuner_leaves_small_and_flat_graphs_alone():
    """Below 2048 vertices, or without a dense top (a grid), no block."""
    for src, dst, n in (graphgen.rmat(10, 16, 1), graphgen.grid_plus_percent(128, 1.0, 1)):
        T, t, (ranks, _) = run(src, dst, n, 4)
        assert ranks == 0
        assert T == oracle.tc_node_iterator(oracle.clean(src, dst, n), False)[0]


@pytest.mark.parametrize("n,m,seed", [(1001, 30000, 3), (777, 60000, 5)])
def test_dense_block_of_unaligned_size(n, m, seed):
    """K = n not a multiple of 8 (leading dimensions cuBLAS cannot tile with
    aligned tensor-core loads): still exact."""
    src, dst, _ = graphgen.er_distinct(n, m, seed)
    g = oracle.clean(src, dst, n)
    T_ref, t_ref = oracle.tc_node_iterator(g)
    T, t, (ranks, tc) = run(src, dst, n, 4, dense_core=n)
    assert ranks == n and tc == T_ref and T == T_ref and np.array_equal(t, t_ref)
