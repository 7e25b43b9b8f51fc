"""Pins for the oracle: each check ties the oracle to something other than
itself (hand-derived fixtures, brute force over all triples, closed forms,
dense matrix powers, invariants).  The paper prints no triangle counts for
any graph, so no value here comes from the paper; all come from mathematics.
"""
import os
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
from _graphs import (brute_force, complete, complete_bipartite, complete_tripartite, cube_counts,
                     cycle, edges_to_arrays, fan, golden_files, grid2d, load_golden, messy_random,
                     random_tree, star, wheel)


def count(src, dst, n):
    g = oracle.clean(src, dst, n)
    T, t = oracle.tc_node_iterator(g)
    o = oracle.orient(g)
    T2, t2, _ = oracle.tc_forward(o)
    assert T2 == T and np.array_equal(t2, t), "forward and node-iterator disagree"
    return T, t


# ---------------------------------------------------------------- fixtures

@pytest.mark.parametrize("path", golden_files(), ids=lambda p: p.split("/")[-1])
def test_golden_fixture(path):
    src, dst, n, T, t = load_golden(path)
    got_T, got_t = count(src, dst, n)
    assert got_T == T
    assert np.array_equal(got_t, t)


# ------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(24))
def test_brute_force_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 48))
    m = int(rng.integers(0, 4 * n + 1))
    src, dst = messy_random(n, m, rng)
    T, t = count(src, dst, n)
    bT, bt = brute_force(src, dst, n)
    assert T == bT
    assert np.array_equal(t, bt)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_dense(seed):
    rng = np.random.default_rng(100 + seed)
    n = 30
    keep = rng.random((n, n)) < 0.6
    src, dst = np.nonzero(np.triu(keep, 1))
    src, dst = src.astype(np.uint32), dst.astype(np.uint32)
    T, t = count(src, dst, n)
    bT, bt = brute_force(src, dst, n)
    assert (T, t.tolist()) == (bT, bt.tolist())


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", [3, 4, 5, 9, 17, 40])
def test_complete_graph(n):
    T, t = count(*edges_to_arrays(complete(n)), n)
    assert T == comb(n, 3)
    assert np.all(t == comb(n - 1, 2))


@pytest.mark.parametrize("n", [5, 6, 11, 50])
def test_wheel(n):
    T, t = count(*edges_to_arrays(wheel(n)), n)
    assert T == n - 1
    assert t[0] == n - 1 and np.all(t[1:] == 2)


@pytest.mark.parametrize("n", [4, 5, 12, 101])
def test_cycle(n):
    T, t = count(*edges_to_arrays(cycle(n)), n)
    assert T == 0 and not t.any()


def test_triangle_cycle():
    T, t = count(*edges_to_arrays(cycle(3)), 3)
    assert T == 1 and np.all(t == 1)


@pytest.mark.parametrize("k", [2, 3, 10, 40])
def test_fan(k):
    T, t = count(*edges_to_arrays(fan(k)), k + 1)
    assert T == k - 1
    assert t[0] == k - 1
    assert t[1] == 1 and t[k] == 1
    assert np.all(t[2:k] == 2)


@pytest.mark.parametrize("w,h", [(2, 2), (5, 7), (32, 32)])
def test_grid(w, h):
    T, t = count(*edges_to_arrays(grid2d(w, h)), w * h)
    assert T == 0


@pytest.mark.parametrize("k", [1, 5, 60])
def test_star(k):
    T, _ = count(*edges_to_arrays(star(k)), k + 1)
    assert T == 0


def test_tree():
    rng = np.random.default_rng(7)
    T, _ = count(*edges_to_arrays(random_tree(200, rng)), 200)
    assert T == 0


@pytest.mark.parametrize("a,b", [(1, 1), (3, 4), (10, 12)])
def test_complete_bipartite(a, b):
    T, _ = count(*edges_to_arrays(complete_bipartite(a, b)), a + b)
    assert T == 0


@pytest.mark.parametrize("a,b,c", [(1, 1, 1), (2, 2, 2), (3, 4, 5), (7, 1, 9)])
def test_complete_tripartite(a, b, c):
    T, t = count(*edges_to_arrays(complete_tripartite(a, b, c)), a + b + c)
    assert T == a * b * c
    assert np.all(t[:a] == b * c)
    assert np.all(t[a:a + b] == a * c)
    assert np.all(t[a + b:] == a * b)


def test_empty_and_edgeless():
    e = np.zeros(0, dtype=np.uint32)
    assert count(e, e, 0)[0] == 0
    T, t = count(e, e, 9)
    assert T == 0 and len(t) == 9 and not t.any()
    loops = np.arange(5, dtype=np.uint32)
    T, t = count(loops, loops, 5)
    assert T == 0


def test_out_of_range_id_rejected():
    with pytest.raises(ValueError):
        oracle.clean(np.array([0, 5], np.uint32), np.array([1, 1], np.uint32), 5)


# ------------------------------------------------- matrix-power pins (n <= 2048)

@pytest.mark.parametrize("gen", ["er", "rmat", "er_dense"])
def test_cube_trace_and_diagonal(gen):
    if gen == "er":
        src, dst, n = graphgen.er_distinct(2048, 40000, 11)
    elif gen == "rmat":
        src, dst, n = graphgen.rmat(11, 16, 3)
    else:
        src, dst, n = graphgen.er_distinct(300, 20000, 5)
    T, t = count(src, dst, n)
    cT, ct = cube_counts(src, dst, n)
    assert T == cT
    assert np.array_equal(t, ct)


def test_config_er_small_sanity_band():
    """ER G(4096, 65536): expected count C(n,3) q^3 ~ 5461 (q = m / C(n,2)).
    A sanity band, not a pin; the pins are the other tests."""
    src, dst, n = graphgen.er_distinct(4096, 65536, 1)
    g = oracle.clean(src, dst, n)
    assert g.m == 65536
    T, t = oracle.tc_node_iterator(g)
    q = 65536 / comb(4096, 2)
    mu = comb(4096, 3) * q ** 3
    assert abs(T - mu) < 6 * np.sqrt(mu) + 50
    assert int(t.sum()) == 3 * T


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(4))
def test_sum_per_vertex_is_three_T(seed):
    src, dst, n = graphgen.rmat(10, 8, seed)
    T, t = count(src, dst, n)
    assert int(t.sum()) == 3 * T


@pytest.mark.parametrize("seed", range(3))
def test_relabel_invariance(seed):
    rng = np.random.default_rng(seed)
    src, dst, n = graphgen.rmat(9, 12, 40 + seed)
    T, t = count(src, dst, n)
    perm = rng.permutation(n).astype(np.uint32)
    T2, t2 = count(perm[src], perm[dst], n)
    assert T2 == T
    assert np.array_equal(t2[perm], t)


def test_tc_vertex_matches_node_iterator_and_cube():
    src, dst, n = graphgen.rmat(10, 16, 9)
    g = oracle.clean(src, dst, n)
    _, t = oracle.tc_node_iterator(g)
    xs = np.arange(n, dtype=np.uint32)
    assert np.array_equal(oracle.tc_vertex(g, xs), t)
    _, ct = cube_counts(src, dst, n)
    assert np.array_equal(oracle.tc_vertex(g, xs), ct)


# ------------------------------------------------------------- clean pins

def test_clean_structure():
    rng = np.random.default_rng(3)
    n = 60
    src, dst = messy_random(n, 500, rng)
    g = oracle.clean(src, dst, n)
    want = set()
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            want.add((a, b))
            want.add((b, a))
    got = set()
    for v in range(n):
        row = g.adj[g.offs[v]:g.offs[v + 1]].tolist()
        assert row == sorted(set(row)), "rows sorted, no repeats"
        assert v not in row, "no self-loops"
        got.update((v, x) for x in row)
    assert got == want
    assert g.m == len(want) // 2


# --------------------------------------------------- degree order + orient

def test_degree_rank_and_orientation():
    src, dst, n = graphgen.rmat(10, 8, 21)
    g = oracle.clean(src, dst, n)
    o = oracle.orient(g)
    deg = g.degree()
    assert sorted(o.perm.tolist()) == list(range(n))
    assert np.array_equal(o.rank[o.perm], np.arange(n))
    keys = [(int(deg[v]), int(v)) for v in o.perm]
    assert keys == sorted(keys), "ascending degree, ties by original ID"
    seen = set()
    for r in range(n):
        row = o.col[o.rowptr[r]:o.rowptr[r + 1]].tolist()
        assert row == sorted(set(row))
        assert all(x > r for x in row), "edges point up in rank"
        for x in row:
            a, b = int(o.perm[r]), int(o.perm[x])
            seen.add((min(a, b), max(a, b)))
    assert o.m == g.m
    want = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist()) if a != b}
    assert seen == want


# ------------------------------------------------------- partition pins

def test_cuts_closed_forms():
    # Hand-made oriented graph on 6 vertices with out-degrees 4,0,2,2,0,0:
    # prefix P = [0,4,4,6,8,8,8], M = 8.
    rowptr = np.array([0, 4, 4, 6, 8, 8, 8], dtype=np.int64)
    col = np.array([1, 2, 3, 4, 3, 4, 4, 5], dtype=np.uint32)
    o = oracle.Oriented(6, np.arange(6, dtype=np.uint32), np.arange(6, dtype=np.uint32),
                        rowptr, col, oracle.load())
    # p=2: least r with 2*P[r] >= 8 -> P[r] >= 4 -> r = 1.
    assert oracle.cuts(o, 2).tolist() == [0, 1, 6]
    # p=4: thresholds P*4 >= 8, 16, 24 -> P >= 2, 4, 6 -> r = 1, 1, 3.
    assert oracle.cuts(o, 4).tolist() == [0, 1, 1, 3, 6]
    assert oracle.cuts(o, 1).tolist() == [0, 6]
    assert oracle.cuts(o, 4, oracle.CUT_UNIFORM).tolist() == [0, 1, 3, 4, 6]
    assert oracle.cuts(o, 6, oracle.CUT_UNIFORM).tolist() == [0, 1, 2, 3, 4, 5, 6]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 16])
@pytest.mark.parametrize("rule", [oracle.CUT_NNZ, oracle.CUT_UNIFORM])
def test_partition_invariance(p, rule):
    src, dst, n = graphgen.rmat(11, 16, 5)
    g = oracle.clean(src, dst, n)
    T, _ = oracle.tc_node_iterator(g, per_vertex=False)
    o = oracle.orient(g)
    c = oracle.cuts(o, p, rule)
    assert c[0] == 0 and c[-1] == n and np.all(np.diff(c.astype(np.int64)) >= 0)
    be = oracle.block_edges(o, p, c)
    assert int(be.sum()) == o.m
    assert not np.tril(be, -1).any(), "upper orientation leaves i > j blocks empty"
    T2, _, tc = oracle.tc_forward(o, p, c, per_vertex=False)
    assert T2 == T
    assert int(tc.sum()) == T
    # a triangle u < v < w has part(u) <= part(v) <= part(w)
    i, j, k = np.nonzero(tc)
    assert np.all(i <= j) and np.all(j <= k)
    # every triple with a triangle is in the queue; the queue has no triple with an empty block
    ijk, w = oracle.triples(p, be)
    queued = {tuple(x) for x in ijk.tolist()}
    assert {(a, b, c_) for a, b, c_ in zip(i.tolist(), j.tolist(), k.tolist())} <= queued
    for (a, b, c_), wt in zip(ijk.tolist(), w.tolist()):
        assert be[a, b] and be[a, c_] and be[b, c_]
        assert wt == be[a, b] + be[a, c_] + be[b, c_]


def test_triples_enumeration_and_order():
    p = 5
    be = np.ones((p, p), dtype=np.uint64)
    ijk, w = oracle.triples(p, be)
    assert len(ijk) == p * (p + 1) * (p + 2) // 6  # all i <= j <= k
    assert np.all(w == 3)
    assert [tuple(x) for x in ijk.tolist()] == sorted(tuple(x) for x in ijk.tolist())
    rng = np.random.default_rng(0)
    be = np.triu(rng.integers(0, 4, size=(p, p))).astype(np.uint64)
    ijk, w = oracle.triples(p, be)
    assert np.all(np.diff(w.astype(np.int64)) <= 0), "decreasing weight"
    brute = [(i, j, k) for i in range(p) for j in range(i, p) for k in range(j, p)
             if be[i, j] and be[i, k] and be[j, k]]
    assert sorted(tuple(x) for x in ijk.tolist()) == brute


def test_alg_bytes_small():
    # path 0-1-2 plus triangle edge 0-2: oriented by degree (all degree 2,
    # ties by ID) gives rows 0:{1,2}, 1:{2}; indeg = [0,1,2], outdeg = [2,1,0]
    src, dst = edges_to_arrays([(0, 1), (1, 2), (0, 2)])
    o = oracle.orient(oracle.clean(src, dst, 3))
    assert o.rowptr.tolist() == [0, 2, 3, 3]
    assert oracle.alg_bytes(o) == 4 * 3 + 4 * (0 * 2 + 1 * 1 + 2 * 0) + 8 * 4


# --------------------------------------------------------- generator pins

def test_splitmix_published_sequence():
    # SplitMix64 from state 1234567: the published first outputs.
    assert [graphgen.splitmix_raw(1234567, c) for c in range(3)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423]


@pytest.mark.parametrize("bits", [1, 2, 3, 7, 10, 13])
def test_feistel_relabelling_is_a_bijection(bits):
    for seed in (1, 2, 99):
        lab = [graphgen.feistel_label(x, bits, seed) for x in range(1 << bits)]
        assert sorted(lab) == list(range(1 << bits))
    if bits >= 7:  # a seeded shuffle, not the identity, and seed-dependent
        assert lab != list(range(1 << bits))
        assert lab != [graphgen.feistel_label(x, bits, 1) for x in range(1 << bits)]


def test_rmat_relabellings_compose_with_the_unrelabelled_graph():
    """Relabelled R-MAT = the unrelabelled edges mapped through the stated
    bijection (Fisher-Yates permutation or Feistel labels), edge by edge."""
    scale, ef, seed = 11, 8, 6
    s0, d0, n = graphgen.rmat(scale, ef, seed, relabel="none")
    perm = graphgen.shuffle_permutation(n, seed)
    assert sorted(perm.tolist()) == list(range(n))
    s1, d1, _ = graphgen.rmat(scale, ef, seed, relabel="shuffle")
    assert np.array_equal(s1, perm[s0]) and np.array_equal(d1, perm[d0])
    assert np.array_equal(s1, graphgen.rmat(scale, ef, seed)[0])  # the default relabelling
    lab = np.array([graphgen.feistel_label(x, scale, seed) for x in range(n)], np.uint32)
    s2, d2, _ = graphgen.rmat(scale, ef, seed, relabel="feistel")
    assert np.array_equal(s2, lab[s0]) and np.array_equal(d2, lab[d0])


def test_serving_mix_spec():
    """The serving workload's job parameters: families in thirds, stated
    ranges, deterministic per job index."""
    specs = [graphgen.serve_spec(i, 22) for i in range(3000)]
    assert specs == [graphgen.serve_spec(i, 22) for i in range(3000)]
    assert all(sp[0] == ("rmat", "er", "rgg")[i % 3] for i, sp in enumerate(specs))
    rm = [sp for sp in specs if sp[0] == "rmat"]
    assert {sp[1] for sp in rm} == set(range(10, 23)) and {sp[2] for sp in rm} == set(range(8, 33))
    er = [sp for sp in specs if sp[0] == "er"]
    assert all(1 << 10 <= sp[1] <= 1 << 22 and 2 * sp[1] <= 2 * sp[2] + 2 <= 64 * sp[1] + 2 for sp in er)
    assert all(1 << 10 <= sp[1] <= 1 << 22 for sp in specs if sp[0] == "rgg")
    fam, scale, ef = graphgen.serve_spec(0, 12)
    src, dst, n = graphgen.serve_job(0, 12)
    assert fam == "rmat" and n == 1 << scale and len(src) == ef << scale


def test_generators_deterministic_and_shaped():
    a = graphgen.rmat(12, 16, 4)
    b = graphgen.rmat(12, 16, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = graphgen.rmat(12, 16, 5)
    assert not np.array_equal(a[0], c[0])
    assert a[2] == 4096 and len(a[0]) == 16 * 4096
    src, dst, n = graphgen.grid(5, 4, 3, 1)
    assert len(src) == 4 * 4 + 5 * 3 + 3 and n == 20
    assert np.all(src[-3:] != dst[-3:])
    src, dst, n = graphgen.er_distinct(100, 1000, 2)
    keys = {(min(a, b), max(a, b)) for a, b in zip(src.tolist(), dst.tolist())}
    assert len(keys) == 1000 and all(a != b for a, b in keys)
    src, dst, n = graphgen.rgg(5000, None, 3)
    assert np.all(src < dst)
    assert 4.0 < 2 * len(src) / n < 8.0  # average degree near 6


def test_grid_extra_percent_count():
    src, dst, n = graphgen.grid_plus_percent(64, 1.0, 2)
    base = 2 * 64 * 63
    assert len(src) == base + round(base / 100)
    g = oracle.clean(src, dst, n)
    T, _ = oracle.tc_node_iterator(g, per_vertex=False)
    gb = oracle.clean(src[:base], dst[:base], n)
    assert oracle.tc_node_iterator(gb, per_vertex=False)[0] == 0
    assert T >= 0


# ------------------------------------------- block attribution pins
# The p x p block sizes (Section 4.3: A_ij holds the oriented edges whose
# tail lies in part i and head in part j) and the per-triple counts
# (Section 3.6 block-list composition: a triangle a < b < c in rank order
# belongs to the triple (part a, part b, part c)) are fixed here by values
# derived by hand and by a brute force that places every edge and triangle
# from the definition of the parts: part t = the rank range [c_t, c_t+1).

# The oriented 6-vertex graph of test_cuts_closed_forms: edges 0->1, 0->2,
# 0->3, 0->4, 2->3, 2->4, 3->4, 3->5; its triangles are 023, 024, 034, 234.
HAND_ROWPTR = np.array([0, 4, 4, 6, 8, 8, 8], dtype=np.int64)
HAND_COL = np.array([1, 2, 3, 4, 3, 4, 4, 5], dtype=np.uint32)

# (p, rule) -> (cuts, nonzero block sizes {(i, j): count}, nonzero triple counts)
HAND_PARTITIONS = {
    # parts {0}, {1..5}: vertex 1 sits exactly on the cut c_1 = 1
    (2, oracle.CUT_NNZ): ([0, 1, 6], {(0, 1): 4, (1, 1): 4}, {(0, 1, 1): 3, (1, 1, 1): 1}),
    # parts {0}, {} (empty), {1, 2}, {3, 4, 5}: vertex 1 on the double cut c_1 = c_2 = 1
    (4, oracle.CUT_NNZ): ([0, 1, 1, 3, 6], {(0, 2): 2, (0, 3): 2, (2, 3): 2, (3, 3): 2},
                          {(0, 2, 3): 2, (0, 3, 3): 1, (2, 3, 3): 1}),
    # parts {0, 1, 2}, {3, 4, 5}
    (2, oracle.CUT_UNIFORM): ([0, 3, 6], {(0, 0): 2, (0, 1): 4, (1, 1): 2}, {(0, 0, 1): 2, (0, 1, 1): 2}),
    # parts {0}, {1, 2}, {3}, {4, 5}
    (4, oracle.CUT_UNIFORM): ([0, 1, 3, 4, 6], {(0, 1): 2, (0, 2): 1, (0, 3): 1, (1, 2): 1, (1, 3): 1,
                                                (2, 3): 2},
                              {(0, 1, 2): 1, (0, 1, 3): 1, (0, 2, 3): 1, (1, 2, 3): 1}),
}


def hand_attribution(lib, p, rule):
    o = oracle.Oriented(6, np.arange(6, dtype=np.uint32), np.arange(6, dtype=np.uint32),
                        HAND_ROWPTR, HAND_COL, lib)
    c = oracle.cuts(o, p, rule)
    be = oracle.block_edges(o, p, c)
    T, t, tc = oracle.tc_forward(o, p, c, per_vertex=True)
    return c, be, T, t, tc


def dense_from(entries, shape):
    out = np.zeros(shape, dtype=np.uint64)
    for idx, v in entries.items():
        out[idx] = v
    return out


@pytest.mark.parametrize("p,rule", sorted(HAND_PARTITIONS))
def test_block_edges_and_triples_hand_derived(p, rule):
    want_cuts, want_be, want_tc = HAND_PARTITIONS[(p, rule)]
    c, be, T, t, tc = hand_attribution(oracle.load(), p, rule)
    assert c.tolist() == want_cuts
    assert np.array_equal(be, dense_from(want_be, (p, p)))
    assert np.array_equal(tc, dense_from(want_tc, (p, p, p)))
    assert T == 4
    assert t.tolist() == [3, 0, 3, 3, 3, 0]  # 0: 023 024 034; 2: 023 024 234; 3: 023 034 234; 4: 024 034 234


def part_by_definition(cuts, r):
    """The unique t with c_t <= r < c_t+1."""
    hits = [t for t in range(len(cuts) - 1) if cuts[t] <= r < cuts[t + 1]]
    assert len(hits) == 1
    return hits[0]


def attribution_by_definition(src, dst, n, rank, cuts):
    """Block sizes and per-triple counts from the definitions alone: every
    undirected edge {a, b} is the oriented edge from the lower to the higher
    rank; every triangle is placed by the parts of its three ranks in
    ascending order."""
    p = len(cuts) - 1
    part = [part_by_definition(cuts, r) for r in range(n)]
    adj = np.zeros((n, n), dtype=bool)
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            adj[rank[a], rank[b]] = adj[rank[b], rank[a]] = True
    be = np.zeros((p, p), dtype=np.uint64)
    for x in range(n):
        for y in range(x + 1, n):
            if adj[x, y]:
                be[part[x], part[y]] += 1
    tc = np.zeros((p, p, p), dtype=np.uint64)
    for x in range(n):
        for y in range(x + 1, n):
            if not adj[x, y]:
                continue
            for z in range(y + 1, n):
                if adj[x, z] and adj[y, z]:
                    tc[part[x], part[y], part[z]] += 1
    return be, tc


def attribution_cases():
    """(name, src, dst, n, cut list or rule) cases: random dense graphs under
    both rules, a hub-heavy graph whose nnz cuts repeat (empty parts), and
    hand-set cuts with empty parts and vertices exactly on cuts."""
    cases = []
    for seed in range(3):
        rng = np.random.default_rng(500 + seed)
        n = int(rng.integers(18, 34))
        keep = rng.random((n, n)) < rng.uniform(0.25, 0.6)
        s, d = np.nonzero(np.triu(keep, 1))
        cases.append((f"dense{seed}", s.astype(np.uint32), d.astype(np.uint32), n))
    # a star plus a clique: one vertex of high degree, so nnz cuts pile up
    edges = [(0, k) for k in range(1, 20)] + complete(6)
    s, d = edges_to_arrays(edges)
    cases.append(("star_clique", s, d, 20))
    return cases


@pytest.mark.parametrize("case", attribution_cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("p", [2, 3, 4, 7])
@pytest.mark.parametrize("rule", [oracle.CUT_NNZ, oracle.CUT_UNIFORM, "hand"])
def test_block_attribution_brute_force(case, p, rule):
    _, src, dst, n = case
    o = oracle.orient(oracle.clean(src, dst, n))
    if rule == "hand":
        # empty parts (repeated cuts) and cuts at both ends of the rank range
        inner = sorted(np.random.default_rng(p).choice(np.arange(0, n + 1), size=p - 1).tolist())
        inner[0] = 0
        c = np.array([0] + inner + [n], dtype=np.uint32)
    else:
        c = oracle.cuts(o, p, rule)
    be = oracle.block_edges(o, p, c)
    _, _, tc = oracle.tc_forward(o, p, c, per_vertex=False)
    want_be, want_tc = attribution_by_definition(src, dst, n, o.rank, c.tolist())
    assert np.array_equal(be, want_be)
    assert np.array_equal(tc, want_tc)


def test_planted_cut_boundary_mistake_is_caught(tmp_path):
    """A copy of the oracle with the part lookup shifted by one at a cut
    boundary (a vertex exactly on c_t+1 kept in part t) must fail the pins
    above: the hand-derived matrices and the brute force."""
    src_text = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    good, bad = "cuts[t + 1] <= r", "cuts[t + 1] < r"
    assert src_text.count(good) == 1
    mutated = tmp_path / "oracle_mutated.c"
    mutated.write_text(src_text.replace(good, bad))
    lib = oracle.load(oracle.build(out=str(tmp_path / "liboracle_mutated.so"), src=str(mutated)))
    failures = 0
    for (p, rule), (want_cuts, want_be, want_tc) in HAND_PARTITIONS.items():
        c, be, _, _, tc = hand_attribution(lib, p, rule)
        if not (np.array_equal(be, dense_from(want_be, (p, p)))
                and np.array_equal(tc, dense_from(want_tc, (p, p, p)))):
            failures += 1
    assert failures == len(HAND_PARTITIONS), "every hand case has a vertex on a cut"
    _, src, dst, n = attribution_cases()[0]
    g = oracle.clean(src, dst, n, lib=lib)
    o = oracle.orient(g)
    c = oracle.cuts(o, 4)
    want_be, _ = attribution_by_definition(src, dst, n, o.rank, c.tolist())
    assert not np.array_equal(oracle.block_edges(o, 4, c), want_be)


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_forward_mt_equals_forward(threads):
    src, dst, n = graphgen.rmat(12, 16, 9)
    o = oracle.orient(oracle.clean(src, dst, n))
    T, t, _ = oracle.tc_forward(o)
    T2, t2 = oracle.tc_forward_mt(o, threads=threads)
    assert T2 == T and np.array_equal(t2, t)
    # a row sample counts exactly the triangles whose lowest-ranked vertex
    # is a sampled row
    T3, t3 = oracle.tc_forward_mt(o, threads=threads, stride=5)
    assert int(t3.sum(dtype=np.uint64)) == 3 * T3 and 0 < T3 < T
    assert T3 == sum(_row_count(o, u) for u in range(0, n, 5))


def _row_count(o, u):
    """Triangles u < v < w found from row u, by set intersection in Python."""
    row = o.col[o.rowptr[u]:o.rowptr[u + 1]].tolist()
    s = set(row)
    cnt = 0
    for v in row:
        cnt += len(s.intersection(o.col[o.rowptr[v]:o.rowptr[v + 1]].tolist()))
    return cnt
