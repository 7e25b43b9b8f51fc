"""Pins for the oracle's single-block bulk-synchronous computations
(connected components, PageRank): each check ties the oracle to something
other than itself -- networkx (a library routine), closed forms, invariants.
The paper prints no component labels or ranks for any graph."""
import networkx as nx
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import complete, cycle, edges_to_arrays, grid2d, messy_random, star


def nx_graph(src, dst, n):
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((int(a), int(b)) for a, b in zip(src, dst) if a != b)
    return G


# ------------------------------------------------------------ components

@pytest.mark.parametrize("seed", range(10))
def test_cc_matches_networkx(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(1, 300))
    src, dst = messy_random(n, int(rng.integers(0, n + 1)), rng)
    lab, comps = oracle.cc_min_label(oracle.clean(src, dst, n))
    want = np.zeros(n, dtype=np.uint32)
    parts = list(nx.connected_components(nx_graph(src, dst, n)))
    for comp in parts:
        want[list(comp)] = min(comp)
    assert comps == len(parts)
    assert np.array_equal(lab, want)


def test_cc_closed_forms():
    # three disjoint cliques on IDs {5..9}, {0..3}, {12..14}; 4, 10, 11 isolated
    edges = [(5 + a, 5 + b) for a, b in complete(5)] + complete(4) + [(12 + a, 12 + b) for a, b in complete(3)]
    lab, comps = oracle.cc_min_label(oracle.clean(*edges_to_arrays(edges), 15))
    assert comps == 6
    assert lab.tolist() == [0, 0, 0, 0, 4, 5, 5, 5, 5, 5, 10, 11, 12, 12, 12]
    # a path listed from its far end: one component labelled 0
    n = 50
    lab, comps = oracle.cc_min_label(oracle.clean(*edges_to_arrays([(n - 1 - i, n - 2 - i) for i in range(n - 1)]), n))
    assert comps == 1 and not lab.any()


def test_cc_relabel_invariance():
    src, dst, n = graphgen.rmat(11, 4, 3)
    lab, comps = oracle.cc_min_label(oracle.clean(src, dst, n))
    perm = np.random.default_rng(4).permutation(n).astype(np.uint32)
    lab2, comps2 = oracle.cc_min_label(oracle.clean(perm[src], perm[dst], n))
    assert comps2 == comps
    # the same partition into components, each labelled by its smallest ID
    for c in np.unique(lab):
        members = np.flatnonzero(lab == c)
        new = perm[members]
        assert len(np.unique(lab2[new])) == 1 and lab2[new[0]] == new.min()


# -------------------------------------------------------------- PageRank

@pytest.mark.parametrize("graph", ["cycle", "complete", "grid_torus"])
def test_pagerank_uniform_on_regular_graphs(graph):
    if graph == "cycle":
        edges, n = cycle(37), 37
    elif graph == "complete":
        edges, n = complete(12), 12
    else:
        w = 9
        edges = [(r * w + c, r * w + (c + 1) % w) for r in range(w) for c in range(w)]
        edges += [(r * w + c, ((r + 1) % w) * w + c) for r in range(w) for c in range(w)]
        n = w * w
    r, it, err = oracle.pagerank(oracle.clean(*edges_to_arrays(edges), n))
    assert np.allclose(r, 1.0 / n, rtol=1e-13, atol=0)
    assert it == 1 and err < 1e-13


def test_pagerank_star_fixed_point():
    k, d = 9, 0.85
    n = k + 1
    a = (1 - d) / n
    centre = a * (1 + d * k) / (1 - d * d)
    leaf = a + d * centre / k
    r, it, err = oracle.pagerank(oracle.clean(*edges_to_arrays(star(k)), n), tol=1e-15, max_iter=10000)
    assert abs(r[0] - centre) < 1e-13 and np.allclose(r[1:], leaf, rtol=0, atol=1e-13)
    assert err < 1e-13  # the change stalls at the rounding level


@pytest.mark.parametrize("seed", range(6))
def test_pagerank_matches_networkx_without_isolated_vertices(seed):
    rng = np.random.default_rng(900 + seed)
    src, dst, n = graphgen.rmat(9, 8, 50 + seed)
    g = oracle.clean(src, dst, n)
    keep = np.flatnonzero(g.degree() > 0)
    # the subgraph on the vertices with edges, relabelled 0..k-1
    remap = np.full(n, -1, dtype=np.int64)
    remap[keep] = np.arange(len(keep))
    s2, d2 = remap[src], remap[dst]
    ok = (s2 >= 0) & (d2 >= 0) & (s2 != d2)
    s2, d2 = s2[ok].astype(np.uint32), d2[ok].astype(np.uint32)
    k = len(keep)
    r, it, err = oracle.pagerank(oracle.clean(s2, d2, k), tol=1e-14, max_iter=10000)
    want = nx.pagerank(nx_graph(s2, d2, k), alpha=0.85, tol=1e-14, max_iter=10000)
    assert np.allclose(r, [want[i] for i in range(k)], rtol=1e-8, atol=1e-12)
    assert abs(r.sum() - 1.0) < 1e-12


def test_pagerank_limit_and_isolated_vertices():
    src, dst = edges_to_arrays(grid2d(6, 5))
    n = 40  # vertices 30..39 isolated: they keep the base rank (1 - d) / n
    r, it, err = oracle.pagerank(oracle.clean(src, dst, n), tol=0.0, max_iter=7)
    assert it == 7 and err > 0
    assert np.allclose(r[30:], 0.15 / n, rtol=1e-15, atol=0)
    r1, it1, _ = oracle.pagerank(oracle.clean(src, dst, n), tol=1e-4, max_iter=20)
    assert 1 <= it1 <= 20
