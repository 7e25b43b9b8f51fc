"""Block cache tier: after pgb_blocks_offload_columns the columns and a
tail-block-major in-edge index live in pinned host memory; runs keep a cache
of column slices (one per row block) on the device, as many as the budget
allows, and count pieces of block pairs (Section 4.4 copies of a task's
blocks, with eviction).

Counts are exact integers: every comparison with the oracle and the resident
run is bit-exact.  Budgets from two slices (constant eviction) to all of them
(each slice copied once) must give the same counts."""
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import golden_files, load_golden, messy_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb  # noqa: E402

P = pgabb


def _blocks(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(np.ascontiguousarray(src, np.uint32)).cuda(),
                               torch.from_numpy(np.ascontiguousarray(dst, np.uint32)).cuda(), n)
    return P.pgb_partition(g, p)


def _oracle(src, dst, n):
    return oracle.tc_node_iterator(oracle.clean(src, dst, n))


def _run(b, per_vertex=True, budget=0, threads=0):
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(per_vertex=int(per_vertex), device_budget=budget,
                                              hash_threads=threads))
    T, t = P.pgb_tc_result_get(r, per_vertex=per_vertex)
    nbytes, pieces, loads = P.pgb_tc_result_stream(r, slice_loads=True)
    assert P.pgb_tc_result_variant(r) == P.PGB_VAR_HASH
    return T, t, nbytes, pieces, loads


@pytest.mark.parametrize("per_vertex", [True, False])
def test_rmat_cache_sizes_match_oracle(per_vertex):
    src, dst, n = graphgen.rmat(16, 16, 31)
    oT, ot = _oracle(src, dst, n)
    p = 8
    b = _blocks(src, dst, n, p)
    m = P.pgb_blocks_info(b)["m"]
    col = P.pgb_blocks_export(b, P.PGB_EXPORT_COL)
    floor_before = P.pgb_blocks_resident_bytes(b, per_vertex)
    P.pgb_blocks_offload_columns(b)
    assert P.pgb_blocks_resident_bytes(b, per_vertex) < floor_before
    assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_COL), col)
    loads_by_size = {}
    for slices in (2, 3, 5, p):
        budget = P.pgb_blocks_cache_budget(b, slices, per_vertex)
        T, t, nbytes, pieces, loads = _run(b, per_vertex, budget)
        assert T == oT
        if per_vertex:
            assert np.array_equal(t, ot)
        # every in-edge crosses the link once; every slice at least once
        assert nbytes >= 12 * m + 4 * m
        assert pieces >= 1
        loads_by_size[slices] = loads
    # a full cache copies each slice once; small caches evict and reload
    assert loads_by_size[p] == p
    assert loads_by_size[2] > p
    assert min(loads_by_size.values()) == p
    # no budget: a full cache
    T, t, _, _, loads = _run(b, per_vertex, 0)
    assert T == oT and loads == p


@pytest.mark.parametrize("path", golden_files(), ids=lambda x: x.split("/")[-1])
def test_golden_fixtures_column_tier(path):
    src, dst, n, T, t = load_golden(path)
    for p in sorted({1, 2, 3, n}):
        if p > n:
            continue
        b = _blocks(src, dst, n, p)
        P.pgb_blocks_offload_columns(b)
        gT, gt, _, _, _ = _run(b, True, P.pgb_blocks_cache_budget(b, 2))
        assert gT == T and np.array_equal(gt, t)


@pytest.mark.parametrize("seed", range(6))
def test_random_messy_column_tier(seed):
    rng = np.random.default_rng(9100 + seed)
    n = int(rng.integers(2, 3000))
    m = int(rng.integers(0, 20 * n))
    src, dst = messy_random(n, m, rng)
    oT, ot = _oracle(src, dst, n)
    p = int(rng.integers(1, min(n, 12) + 1))
    b = _blocks(src, dst, n, p)
    P.pgb_blocks_offload_columns(b)
    T, t, _, _, _ = _run(b, True, P.pgb_blocks_cache_budget(b, 2))
    assert T == oT and np.array_equal(t, ot)


def test_heavy_heads_and_key_slices_column_tier():
    """K_1500 plus a fringe: heads with more than 1024 higher neighbours
    (key-range slices) and pieces that cut inside one head's in-edges."""
    from math import comb
    k = 1500
    a, bb = np.triu_indices(k, 1)
    rng = np.random.default_rng(5)
    fs, fd = rng.integers(0, 4000, 20000), rng.integers(0, 4000, 20000)
    src = np.concatenate([a, fs]).astype(np.uint32)
    dst = np.concatenate([bb, fd]).astype(np.uint32)
    n = 4000
    oT, ot = _oracle(src, dst, n)
    assert oT >= comb(k, 3)
    for p in (1, 4, 9):
        b = _blocks(src, dst, n, p)
        P.pgb_blocks_offload_columns(b)
        for threads in (128, 256, 512):
            T, t, _, _, _ = _run(b, True, P.pgb_blocks_cache_budget(b, 2), threads)
            assert T == oT and np.array_equal(t, ot)


@pytest.mark.parametrize("slices", [1, 3, 17, 100000])
def test_slice_counts_column_tier(slices):
    """Row ranges coarser or finer than the partition's blocks (capped at n
    and at 1024): the same counts, fewer pieces when coarser."""
    src, dst, n = graphgen.rmat(15, 16, 41)
    oT, ot = _oracle(src, dst, n)
    if slices > 1024:
        b = _blocks(src, dst, n, 8)
        with pytest.raises(P.PgbError) as ei:
            P.pgb_blocks_offload_columns(b, slices)
        assert ei.value.code == P.PGB_E_INVAL
        return
    b = _blocks(src, dst, n, 8)
    P.pgb_blocks_offload_columns(b, slices)
    T, t, _, pieces, loads = _run(b, True, P.pgb_blocks_cache_budget(b, 2))
    assert T == oT and np.array_equal(t, ot)
    assert pieces >= 1
    if slices == 1:
        assert loads == 1


def test_empty_and_edgeless_column_tier():
    e = np.zeros(0, np.uint32)
    for n in (0, 6):
        b = _blocks(e, e, n, 1)
        P.pgb_blocks_offload_columns(b)
        T, t, nbytes, pieces, loads = _run(b, True, 0)
        assert T == 0 and pieces == 0 and loads == 0
        assert t.shape == (n,) and not t.any()


def test_column_tier_state_rules():
    src, dst, n = graphgen.rmat(12, 8, 3)
    oT, _ = _oracle(src, dst, n)
    b = _blocks(src, dst, n, 4)
    P.pgb_blocks_offload(b)
    with pytest.raises(P.PgbError) as ei:
        P.pgb_blocks_offload_columns(b)
    assert ei.value.code == P.PGB_E_STATE
    with pytest.raises(P.PgbError) as ei:
        P.pgb_blocks_cache_budget(b, 2)
    assert ei.value.code == P.PGB_E_STATE
    b = _blocks(src, dst, n, 4)
    P.pgb_blocks_offload_columns(b)
    P.pgb_blocks_offload_columns(b)  # a second call is a no-op
    P.pgb_blocks_offload(b)          # and so is the index offload
    for kw in (dict(mode=P.PGB_MODE_PLAIN), dict(variant=P.PGB_VAR_BSEARCH), dict(variant=P.PGB_VAR_MERGE)):
        with pytest.raises(P.PgbError) as ei:
            P.pgb_tc_run(b, P.pgb_tc_opts_default(**kw))
        assert ei.value.code == P.PGB_E_STATE
    two = P.pgb_blocks_cache_budget(b, 2)
    assert P.pgb_blocks_cache_budget(b, 3) > two
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_run(b, P.pgb_tc_opts_default(device_budget=two - 1))
    assert ei.value.code == P.PGB_E_BUDGET
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_run(b, P.pgb_tc_opts_default(device_budget=P.pgb_blocks_resident_bytes(b, True)))
    assert ei.value.code == P.PGB_E_BUDGET
    assert _run(b, True, two)[0] == oT
