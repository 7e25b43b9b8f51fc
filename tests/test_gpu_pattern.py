"""4-clique and 4-cycle (butterfly) counts on the block store, against the
oracle; integer counts, compared bit-exactly (tolerance 0)."""
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
from _graphs import complete, complete_bipartite, edges_to_arrays, grid2d, messy_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402


def blocks(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(np.ascontiguousarray(src, np.uint32)).cuda(),
                               torch.from_numpy(np.ascontiguousarray(dst, np.uint32)).cuda(), n)
    return P.pgb_partition(g, p)


def bipartite(a, b, m, seed):
    """m random edges between parts [0, a) and [a, a + b) (repeats allowed)."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, a, m).astype(np.uint32), (a + rng.integers(0, b, m)).astype(np.uint32), a + b)


def cases():
    out = []
    for seed in range(6):
        rng = np.random.default_rng(4100 + seed)
        n = int(rng.integers(2, 600))
        src, dst = messy_random(n, int(rng.integers(0, 8 * n)), rng)
        out.append((f"messy{seed}", src, dst, n, int(rng.integers(1, min(n, 8) + 1))))
    for scale, ef in ((12, 16), (14, 8)):
        s, d, n = graphgen.rmat(scale, ef, scale)
        out.append((f"rmat{scale}", s, d, n, 8))
    s, d, n = bipartite(3000, 500, 40000, 3)
    out.append(("bipartite", s, d, n, 8))
    s, d, n = graphgen.grid_plus_percent(64, 2.0, 5)
    out.append(("grid64", s, d, n, 4))
    return out


@pytest.mark.parametrize("case", cases(), ids=lambda c: c[0])
def test_counts_match_oracle(case):
    _, src, dst, n, p = case
    g = oracle.clean(src, dst, n)
    b = blocks(src, dst, n, p)
    assert P.pgb_k4_count(b) == oracle.k4_count(g)
    assert P.pgb_c4_count(b) == oracle.c4_count(g)


def test_closed_forms_on_gpu():
    for k in (4, 7, 40):
        b = blocks(*edges_to_arrays(complete(k)), k, 3)
        assert P.pgb_k4_count(b) == comb(k, 4)
        assert P.pgb_c4_count(b) == 3 * comb(k, 4)
    b = blocks(*edges_to_arrays(complete_bipartite(30, 45)), 75, 4)
    assert P.pgb_c4_count(b) == comb(30, 2) * comb(45, 2)
    assert P.pgb_k4_count(b) == 0
    b = blocks(*edges_to_arrays(grid2d(50, 31)), 50 * 31, 6)
    assert P.pgb_c4_count(b) == 49 * 30
    e = np.zeros(0, np.uint32)
    b = blocks(e, e, 9, 2)
    assert P.pgb_k4_count(b) == 0 and P.pgb_c4_count(b) == 0
