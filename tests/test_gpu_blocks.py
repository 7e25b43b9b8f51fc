"""Block storage formats and the Hilbert launch order (Section 4.3.1/4.3.2),
against the oracle.

Each block A_ij exported as CSR, COO and CCOO (block-local IDs) must hold
exactly the oriented edges of the oracle's graph with tail in V_i and head
in V_j, rows ascending and columns ascending within a row; the autotuned
format must be the one with the fewest bytes.  A plain run launched along
the Hilbert curve must give the same total, per-vertex and per-triple
counts as the queue order.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402


def build(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    return P.pgb_partition(g, p)


def oracle_block(o, c, i, j):
    """(local rows, local columns) of the oracle's block A_ij, CSR order."""
    rows, cols = [], []
    for u in range(int(c[i]), int(c[i + 1])):
        for v in o.col[o.rowptr[u]:o.rowptr[u + 1]].tolist():
            if c[j] <= v < c[j + 1]:
                rows.append(u - int(c[i]))
                cols.append(v - int(c[j]))
    return np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64)


@pytest.mark.parametrize("graph", ["rmat12", "grid64"])
def test_block_exports_match_oracle(graph):
    src, dst, n = graphgen.rmat(12, 8, 2) if graph == "rmat12" else graphgen.grid_plus_percent(64, 3.0, 1)
    p = 6
    o = oracle.orient(oracle.clean(src, dst, n))
    c = oracle.cuts(o, p)
    b = build(src, dst, n, p)
    formats_seen = set()
    for i in range(p):
        for j in range(p):
            rows, cols = oracle_block(o, c, i, j)
            info = P.pgb_blocks_block_info(b, i, j)
            nr = int(c[i + 1] - c[i])
            assert info["rows"] == nr and info["cols"] == int(c[j + 1] - c[j]) and info["nnz"] == len(rows)
            nonempty = len(np.unique(rows))
            assert info["nonempty_rows"] == nonempty
            sizes = {P.PGB_FMT_CSR: 4 * (nr + 1 + len(rows)), P.PGB_FMT_COO: 8 * len(rows),
                     P.PGB_FMT_CCOO: 4 * (2 * nonempty + 1 + len(rows))}
            assert (info["bytes_csr"], info["bytes_coo"], info["bytes_ccoo"]) == tuple(sizes[f] for f in range(3))
            assert sizes[info["format"]] == min(sizes.values())
            formats_seen.add(info["format"])
            ptr, col = P.pgb_blocks_export_block(b, i, j, P.PGB_FMT_CSR)
            assert np.array_equal(np.repeat(np.arange(nr), np.diff(ptr.astype(np.int64))), rows)
            assert np.array_equal(col, cols) and ptr[0] == 0 and ptr[-1] == len(rows)
            r2, c2 = P.pgb_blocks_export_block(b, i, j, P.PGB_FMT_COO)
            assert np.array_equal(r2, rows) and np.array_equal(c2, cols)
            nzr, off, c3 = P.pgb_blocks_export_block(b, i, j, P.PGB_FMT_CCOO)
            assert np.array_equal(nzr, np.unique(rows)) and np.array_equal(c3, cols)
            assert np.array_equal(np.repeat(nzr, np.diff(off.astype(np.int64))), rows)
    assert formats_seen, "at least one block"
    with pytest.raises(P.PgbError):
        P.pgb_blocks_block_info(b, p, 0)


def test_hilbert_launch_order_keeps_every_count():
    src, dst, n = graphgen.rmat(14, 16, 6)
    T, t = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = build(src, dst, n, 12)
    res = {}
    for order in (P.PGB_ORDER_WEIGHT, P.PGB_ORDER_HILBERT):
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(mode=P.PGB_MODE_PLAIN, per_triple=1, order=order))
        gT, gt = P.pgb_tc_result_get(r)
        assert gT == T and np.array_equal(gt, t)
        res[order] = P.pgb_tc_result_triples(r)
    assert np.array_equal(res[P.PGB_ORDER_WEIGHT], res[P.PGB_ORDER_HILBERT])
