"""Pins for the oracle's other multi-block pattern counts (Section 3.2:
k-clique finding and butterfly counting): 4-cliques and 4-cycles, checked
against brute force over all vertex sets and against closed forms."""
import itertools
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
from _graphs import (complete, complete_bipartite, complete_tripartite, cycle, dense_adjacency, edges_to_arrays,
                     grid2d, messy_random, wheel)


def graph(edges, n):
    return oracle.clean(*edges_to_arrays(edges), n)


def brute(src, dst, n):
    A = dense_adjacency(src, dst, n)
    k4 = sum(1 for q in itertools.combinations(range(n), 4) if all(A[a, b] for a, b in itertools.combinations(q, 2)))
    c4 = 0
    for q in itertools.combinations(range(n), 4):
        a, b, c, d = q
        # the three distinct 4-cycles on a 4-set
        for x, y, z, w in ((a, b, c, d), (a, b, d, c), (a, c, b, d)):
            c4 += A[x, y] and A[y, z] and A[z, w] and A[w, x]
    return k4, c4


@pytest.mark.parametrize("seed", range(12))
def test_brute_force(seed):
    rng = np.random.default_rng(3100 + seed)
    n = int(rng.integers(1, 16))
    src, dst = messy_random(n, int(rng.integers(0, 3 * n + 1)), rng)
    g = oracle.clean(src, dst, n)
    assert (oracle.k4_count(g), oracle.c4_count(g)) == brute(src, dst, n)


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_dense(seed):
    rng = np.random.default_rng(3200 + seed)
    n = 14
    keep = rng.random((n, n)) < 0.7
    s, d = np.nonzero(np.triu(keep, 1))
    s, d = s.astype(np.uint32), d.astype(np.uint32)
    g = oracle.clean(s, d, n)
    assert (oracle.k4_count(g), oracle.c4_count(g)) == brute(s, d, n)


@pytest.mark.parametrize("n", [4, 5, 9, 20])
def test_complete(n):
    g = graph(complete(n), n)
    assert oracle.k4_count(g) == comb(n, 4)
    assert oracle.c4_count(g) == 3 * comb(n, 4)


def test_closed_forms():
    # complete 4-partite K_{a,b,c,d}: one 4-clique per choice of one vertex per part
    parts = [3, 4, 2, 5]
    offs = np.cumsum([0] + parts)
    edges = [(x, y) for i in range(4) for j in range(i + 1, 4)
             for x in range(offs[i], offs[i + 1]) for y in range(offs[j], offs[j + 1])]
    assert oracle.k4_count(graph(edges, offs[-1])) == 3 * 4 * 2 * 5
    assert oracle.k4_count(graph(complete_tripartite(3, 4, 5), 12)) == 0
    assert oracle.k4_count(graph(wheel(9), 9)) == 0
    # K_{a,b}: a pair of each side closes one butterfly
    for a, b in ((2, 2), (3, 5), (6, 7)):
        assert oracle.c4_count(graph(complete_bipartite(a, b), a + b)) == comb(a, 2) * comb(b, 2)
    # a w x h grid has one 4-cycle per unit square
    for w, h in ((2, 2), (5, 4), (13, 9)):
        assert oracle.c4_count(graph(grid2d(w, h), w * h)) == (w - 1) * (h - 1)
    assert oracle.c4_count(graph(cycle(4), 4)) == 1
    assert oracle.c4_count(graph(cycle(7), 7)) == 0
    assert oracle.c4_count(graph([(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)], 4)) == 1  # K_4 minus an edge


def test_relabel_invariance():
    src, dst, n = graphgen.rmat(8, 8, 5)
    g = oracle.clean(src, dst, n)
    perm = np.random.default_rng(1).permutation(n).astype(np.uint32)
    g2 = oracle.clean(perm[src], perm[dst], n)
    assert oracle.k4_count(g2) == oracle.k4_count(g)
    assert oracle.c4_count(g2) == oracle.c4_count(g)
