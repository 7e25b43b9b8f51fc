"""HYBRID mode: the host kernel beside the GPU (PGAbB Section 4.4), against
the oracle.

The head parts are ordered by estimated work (lookups plus in-edges); the
host takes the lightest ones while their summed estimate stays within the
cut-off share, the GPU counts the rest in the same run.  Every count is
compared bit-exactly (tolerance 0) with the oracle at several cut-offs, from
nothing on the host to everything on the host, and the parts the host took
are checked against the rule.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402


def union(*graphs):
    srcs, dsts, base = [], [], 0
    for s, d, n in graphs:
        srcs.append(s.astype(np.uint32) + np.uint32(base))
        dsts.append(d.astype(np.uint32) + np.uint32(base))
        base += n
    return np.concatenate(srcs), np.concatenate(dsts), base


GRAPHS = {
    "rmat16": lambda: graphgen.rmat(16, 16, 31),
    "grid_u_rmat14": lambda: union(graphgen.grid_plus_percent(200, 1.0, 3), graphgen.rmat(14, 16, 4)),
}


@pytest.fixture(scope="module", params=sorted(GRAPHS))
def graph(request):
    src, dst, n = GRAPHS[request.param]()
    T, t = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    g = P.pgb_graph_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    b = P.pgb_partition(g, 16)
    return b, T, t


def expected_host_parts(b, share_ppm):
    probes = P.pgb_blocks_export(b, P.PGB_EXPORT_PART_PROBES).astype(np.int64)
    in_edges = P.pgb_blocks_export(b, P.PGB_EXPORT_BLOCK_EDGES).sum(axis=0).astype(np.int64)
    est = probes + in_edges
    order = sorted(range(len(est)), key=lambda j: (est[j], -j))
    cap = est.sum() * share_ppm / 1e6
    host, acc = np.zeros(len(est), dtype=bool), 0
    for j in order:
        if est[j] == 0:
            continue
        if acc + est[j] > cap:
            break
        acc += est[j]
        host[j] = True
    return host


@pytest.mark.parametrize("share", [0, 2000, 150000, 600000, 1000000])
@pytest.mark.parametrize("per_vertex", [True, False])
def test_hybrid_counts_match_oracle_at_every_cutoff(graph, share, per_vertex):
    b, T, t = graph
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_HYBRID, host_share_ppm=share,
                                              per_vertex=int(per_vertex)))
    gT, gt = P.pgb_tc_result_get(r, per_vertex=per_vertex)
    assert gT == T
    if per_vertex:
        assert np.array_equal(gt, t)
    parts = P.pgb_tc_result_part_variants(r)
    want = expected_host_parts(b, share if share else 1000)
    assert np.array_equal(parts == P.PGB_VAR_HOST, want)
    h = P.pgb_tc_result_hybrid(r)
    assert h["host_parts"] == int(want.sum())
    if share == 1000000:
        assert (parts[P.pgb_blocks_export(b, P.PGB_EXPORT_BLOCK_EDGES).sum(axis=0) > 0] == P.PGB_VAR_HOST).all()


@pytest.mark.parametrize("threads", [1, 3])
def test_hybrid_thread_counts(graph, threads):
    b, T, t = graph
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_HYBRID, host_share_ppm=400000,
                                              host_threads=threads))
    gT, gt = P.pgb_tc_result_get(r)
    assert gT == T and np.array_equal(gt, t)
    assert P.pgb_tc_result_hybrid(r)["host_threads"] <= threads


def test_hybrid_cancel_and_states(graph):
    b, T, t = graph
    tok = P.pgb_cancel_create()
    try:
        P.pgb_cancel_set(tok)
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_HYBRID, host_share_ppm=500000, cancel=tok))
        with pytest.raises(P.PgbError) as ei:
            P.pgb_tc_result_get(r)
        assert ei.value.code == P.PGB_E_CANCELLED
        P.pgb_cancel_reset(tok)
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_HYBRID, host_share_ppm=500000, cancel=tok))
        gT, gt = P.pgb_tc_result_get(r)
        assert gT == T and np.array_equal(gt, t)
    finally:
        tok.free()
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_HYBRID, use_graph=1))
    assert ei.value.code == P.PGB_E_STATE
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_HYBRID, host_share_ppm=2000000))
    assert ei.value.code == P.PGB_E_INVAL


@pytest.mark.parametrize("share", [1000, 1000000])
@pytest.mark.parametrize("per_vertex", [True, False])
def test_hybrid_with_dense_top_block(graph, share, per_vertex):
    """The dense top block in HYBRID runs: with every part on the host
    (share 10^6) the host kernel must skip the block's in-edges, or the
    block's triangles would be counted twice."""
    b, T, t = graph
    assert P.pgb_blocks_info(b)["n"] > 2048
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_HYBRID, host_share_ppm=share, dense_core=2048,
                                              per_vertex=int(per_vertex)))
    gT, gt = P.pgb_tc_result_get(r, per_vertex=per_vertex)
    d = P.pgb_tc_result_dense_core(r)
    assert d["ranks"] == 2048 and d["triangles"] > 0 and gT == T
    if per_vertex:
        assert np.array_equal(gt, t)
