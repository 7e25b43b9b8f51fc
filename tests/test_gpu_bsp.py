"""Single-block bulk-synchronous kernels (Shiloach-Vishkin components and
PageRank) on the block store, against the oracle.

Component labels (the smallest original ID of each component) are unique,
so they are compared bit-exactly.  PageRank is double precision on both
sides with a different summation order: a rank is a sum of at most deg(v)
terms, so reordering moves it by at most about deg(v) * 2^-52 relative per
iteration, and the contraction (d = 0.85) keeps that from growing over 20
iterations; with degrees below 10^4 here the bound is under 1e-10, and the
test allows rtol 1e-9.  The iteration counts must agree.
"""
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import complete, edges_to_arrays, messy_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402

RTOL = 1e-9


def blocks(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(np.ascontiguousarray(src, np.uint32)).cuda(),
                               torch.from_numpy(np.ascontiguousarray(dst, np.uint32)).cuda(), n)
    return P.pgb_partition(g, p)


def cases():
    out = []
    for seed in range(6):
        rng = np.random.default_rng(1500 + seed)
        n = int(rng.integers(2, 3000))
        src, dst = messy_random(n, int(rng.integers(0, 2 * n)), rng)
        out.append((f"messy{seed}", src, dst, n, int(rng.integers(1, min(n, 16) + 1))))
    s, d, n = graphgen.rmat(14, 4, 7)  # sparse: many components and isolated vertices
    out.append(("rmat14_ef4", s, d, n, 8))
    s, d, n = graphgen.rmat(15, 16, 8)
    out.append(("rmat15", s, d, n, 16))
    s, d, n = graphgen.grid_plus_percent(100, 0.5, 9)
    out.append(("grid100", s, d, n, 8))
    edges = [(5 + a, 5 + b) for a, b in complete(5)] + complete(4)
    s, d = edges_to_arrays(edges)
    out.append(("cliques", s, d, 20, 3))
    return out


@pytest.mark.parametrize("case", cases(), ids=lambda c: c[0])
def test_components_match_oracle(case):
    _, src, dst, n, p = case
    want, comps = oracle.cc_min_label(oracle.clean(src, dst, n))
    b = blocks(src, dst, n, p)
    lab, it, got_comps = P.pgb_cc_run(b)
    assert np.array_equal(lab, want)
    assert got_comps == comps and it >= 1
    dev = torch.zeros(n, dtype=torch.uint32, device="cuda")
    P.pgb_cc_run(b, labels=dev)
    assert np.array_equal(dev.cpu().numpy(), want)


@pytest.mark.parametrize("case", cases(), ids=lambda c: c[0])
def test_pagerank_matches_oracle(case):
    _, src, dst, n, p = case
    g = oracle.clean(src, dst, n)
    want, it, err = oracle.pagerank(g)
    b = blocks(src, dst, n, p)
    got, git, gerr = P.pgb_pagerank_run(b)
    assert git == it
    assert np.allclose(got, want, rtol=RTOL, atol=0)
    assert abs(gerr - err) <= 1e-9 * max(err, 1e-300) + 1e-15
    # a tighter tolerance and more iterations, into a device tensor
    want2, it2, _ = oracle.pagerank(g, tol=1e-10, max_iter=60)
    dev = torch.zeros(n, dtype=torch.float64, device="cuda")
    _, git2, _ = P.pgb_pagerank_run(b, P.pgb_pagerank_opts_default(tol=1e-10, max_iter=60), ranks=dev)
    assert git2 == it2
    assert np.allclose(dev.cpu().numpy(), want2, rtol=RTOL, atol=0)


def test_bsp_edge_cases():
    e = np.zeros(0, np.uint32)
    b = blocks(e, e, 5, 2)
    lab, _, comps = P.pgb_cc_run(b)
    assert lab.tolist() == [0, 1, 2, 3, 4] and comps == 5
    r, it, _ = P.pgb_pagerank_run(b)
    want, wit, _ = oracle.pagerank(oracle.clean(e, e, 5))
    assert np.allclose(r, 0.15 / 5, rtol=1e-15) and np.allclose(want, 0.15 / 5, rtol=1e-15) and it == wit == 2
    src, dst, n = graphgen.rmat(10, 8, 3)
    b = blocks(src, dst, n, 4)
    P.pgb_blocks_offload(b)
    with pytest.raises(P.PgbError) as ei:
        P.pgb_cc_run(b)
    assert ei.value.code == P.PGB_E_STATE
    with pytest.raises(P.PgbError) as ei:
        P.pgb_pagerank_run(blocks(src, dst, n, 4), P.pgb_pagerank_opts_default(damping=1.5))
    assert ei.value.code == P.PGB_E_INVAL
