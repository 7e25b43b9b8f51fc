"""Per-part autotuning of the persistent run, against the oracle.

The autotuner picks, per head part V_j, the middle-vertex hash kernel or
the edge-wise binary-search kernel from that part's lookups per oriented
edge; the triangles whose middle vertex lies in V_j are counted by the
chosen kernel alone, so the split is exact.  These checks pin the per-part
statistic (an integer) against its definition evaluated on the oracle's
oriented graph, check that each part's choice follows the rule, and compare
every count bit-exactly (tolerance 0) with the oracle on graphs whose parts
disagree: the disjoint union of a grid (short lists) and an R-MAT graph
(long lists), the shape of a serve batch.
"""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402

HASH_MIN_LOOKUPS_PER_EDGE = 32


def union(*graphs):
    """Disjoint union of raw edge lists: graph k's IDs shift by the vertex
    counts of the graphs before it."""
    srcs, dsts, base = [], [], 0
    for s, d, n in graphs:
        srcs.append(s.astype(np.uint32) + np.uint32(base))
        dsts.append(d.astype(np.uint32) + np.uint32(base))
        base += n
    return np.concatenate(srcs), np.concatenate(dsts), base


def part_probes_by_definition(o, cuts):
    """Sum over oriented edges (u, v) with v in part j of the entries of u's
    row after v, from the oracle's oriented graph."""
    p = len(cuts) - 1
    rows = np.repeat(np.arange(o.n, dtype=np.int64), np.diff(o.rowptr))
    after = o.rowptr[rows + 1] - (np.arange(o.m, dtype=np.int64) + 1)
    part = np.searchsorted(np.asarray(cuts, dtype=np.int64), o.col.astype(np.int64), side="right") - 1
    out = np.zeros(p, dtype=np.uint64)
    np.add.at(out, part, after.astype(np.uint64))
    return out


def expected_choice(block_edges, part_probes):
    p = len(part_probes)
    edges = block_edges.sum(axis=0)  # column sums: edges whose head lies in part j
    hash_part = (edges == 0) | (part_probes >= HASH_MIN_LOOKUPS_PER_EDGE * edges)
    if hash_part.all():
        return P.PGB_VAR_HASH, np.full(p, P.PGB_VAR_HASH)
    if not (hash_part & (edges > 0)).any():
        return P.PGB_VAR_BSEARCH, np.full(p, P.PGB_VAR_BSEARCH)
    return P.PGB_VAR_MIXED, np.where(hash_part, P.PGB_VAR_HASH, P.PGB_VAR_BSEARCH)


def build(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    return P.pgb_partition(g, p)


def run(b, **kw):
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(**kw))
    T, t = P.pgb_tc_result_get(r, per_vertex=kw.get("per_vertex", 1) != 0)
    return T, t, P.pgb_tc_result_variant(r), P.pgb_tc_result_part_variants(r)


CASES = {
    "grid128": lambda: graphgen.grid_plus_percent(128, 1.0, 4),
    "rmat16": lambda: graphgen.rmat(16, 16, 8),
    "grid256_u_rmat14": lambda: union(graphgen.grid_plus_percent(256, 1.0, 2), graphgen.rmat(14, 16, 3)),
    "rgg_u_rmat13_u_er": lambda: union(graphgen.rgg(20000, None, 5), graphgen.rmat(13, 24, 6),
                                       graphgen.er_pairs(4000, 60000, 7)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("p", [8, 16])
def test_per_part_choice_follows_the_rule_and_counts_match(name, p):
    src, dst, n = CASES[name]()
    o = oracle.orient(oracle.clean(src, dst, n))
    oT, ot, _ = oracle.tc_forward(o)
    b = build(src, dst, n, p)
    cuts = P.pgb_blocks_export(b, P.PGB_EXPORT_CUTS)
    assert np.array_equal(cuts, oracle.cuts(o, p))
    probes = P.pgb_blocks_export(b, P.PGB_EXPORT_PART_PROBES)
    assert np.array_equal(probes, part_probes_by_definition(o, cuts))
    be = P.pgb_blocks_export(b, P.PGB_EXPORT_BLOCK_EDGES)
    want_var, want_parts = expected_choice(be, probes)
    T, t, var, parts = run(b)
    assert var == want_var
    assert np.array_equal(parts, want_parts)
    assert T == oT and np.array_equal(t, ot)
    if name == "grid128":
        assert var == P.PGB_VAR_BSEARCH
    if name.startswith("grid256_u") and p == 16:
        # parts 13-14 hold the R-MAT graph's middle ranks (about 30 lookups
        # per edge and more), the others the grid and the hubs (fewer)
        assert var == P.PGB_VAR_MIXED, "the union's flat and skewed parts should choose differently"


@pytest.mark.parametrize("threads", [0, 128, 256, 512])
def test_mixed_run_equals_single_kernel_runs(threads):
    """On the union, the per-part run, the all-hash run and the
    all-binary-search run give the oracle's counts, with and without
    per-vertex counts and with graph replay."""
    src, dst, n = union(graphgen.grid_plus_percent(300, 1.0, 9), graphgen.rmat(15, 16, 11),
                        graphgen.grid_plus_percent(64, 5.0, 12))
    oT, ot = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = build(src, dst, n, 16)
    for kw in (dict(), dict(variant=P.PGB_VAR_HASH), dict(variant=P.PGB_VAR_BSEARCH)):
        T, t, var, _ = run(b, hash_threads=threads, **kw)
        assert T == oT and np.array_equal(t, ot), kw
        if not kw:
            assert var == P.PGB_VAR_MIXED
        T2, _, _, _ = run(b, hash_threads=threads, per_vertex=0, **kw)
        assert T2 == oT
    for _ in range(3):  # a captured MIXED plan replayed
        T, t, var, _ = run(b, hash_threads=threads, use_graph=1)
        assert var == P.PGB_VAR_MIXED and T == oT and np.array_equal(t, ot)
