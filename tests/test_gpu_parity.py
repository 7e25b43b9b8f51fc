"""Parity of the CUDA path (through the C ABI) with the oracle.

Every count is an exact integer, so every comparison is bit-exact
(tolerance 0): global totals, per-vertex counts in original IDs, per-triple
counts, and the intermediate arrays (cleaned graph, degree rank, oriented
CSR, cuts, block sizes, queue).  Sizes span many 32-edge warp steps and
ragged tails; edge cases cover empty inputs, self-loops only, p = 1, p = n,
empty parts and both cut rules.
"""
from math import comb

import numpy as np
import pytest

import graphgen
import oracle
from _graphs import golden_files, load_golden, messy_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb  # noqa: E402

P = pgabb


def gpu_count(src, dst, n, p, rule=P.PGB_CUT_NNZ, mode=P.PGB_MODE_PERSISTENT, per_vertex=True,
              device=True, chunk=0, order=P.PGB_ORDER_WEIGHT, per_triple=False, variant=P.PGB_VAR_AUTO,
              hash_threads=0):
    if device:
        s = torch.from_numpy(np.ascontiguousarray(src, np.uint32)).cuda()
        d = torch.from_numpy(np.ascontiguousarray(dst, np.uint32)).cuda()
    else:
        s, d = np.ascontiguousarray(src, np.uint32), np.ascontiguousarray(dst, np.uint32)
    g = P.pgb_graph_from_edges(s, d, n)
    b = P.pgb_partition(g, p, rule)
    opts = P.pgb_tc_opts_default(mode=mode, per_vertex=int(per_vertex), chunk_edges=chunk, order=order,
                                 per_triple=int(per_triple), variant=variant, hash_threads=hash_threads)
    r = P.pgb_tc_run(b, opts)
    T, t = P.pgb_tc_result_get(r, per_vertex=per_vertex)
    tri = P.pgb_tc_result_triples(r) if per_triple else None
    return T, t, tri, g, b


def oracle_count(src, dst, n):
    g = oracle.clean(src, dst, n)
    T, t = oracle.tc_node_iterator(g)
    return T, t, g


MODES = [P.PGB_MODE_PERSISTENT, P.PGB_MODE_PLAIN]


@pytest.mark.parametrize("path", golden_files(), ids=lambda x: x.split("/")[-1])
@pytest.mark.parametrize("mode", MODES)
def test_golden_fixtures(path, mode):
    src, dst, n, T, t = load_golden(path)
    for p in range(1, n + 1):
        gT, gt, _, _, _ = gpu_count(src, dst, n, p, mode=mode)
        assert gT == T
        assert np.array_equal(gt, t)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("mode", MODES)
def test_random_messy_graphs(seed, mode):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 400))
    m = int(rng.integers(0, 12 * n))
    src, dst = messy_random(n, m, rng)
    T, t, _ = oracle_count(src, dst, n)
    p = int(rng.integers(1, min(n, 20) + 1))
    rule = int(rng.integers(0, 2))
    gT, gt, _, _, _ = gpu_count(src, dst, n, p, rule=rule, mode=mode, device=bool(seed % 2))
    assert gT == T
    assert np.array_equal(gt, t)


def test_edge_cases():
    e = np.zeros(0, np.uint32)
    for mode in MODES:
        assert gpu_count(e, e, 0, 1, mode=mode)[0] == 0
        T, t, _, _, _ = gpu_count(e, e, 7, 3, mode=mode)
        assert T == 0 and len(t) == 7 and not t.any()
        loops = np.arange(9, dtype=np.uint32)
        T, t, _, _, _ = gpu_count(loops, loops, 9, 9, mode=mode)
        assert T == 0 and not t.any()
        tri_s, tri_d = np.array([0, 1, 2, 2, 1], np.uint32), np.array([1, 2, 0, 0, 1], np.uint32)
        T, t, _, _, _ = gpu_count(tri_s, tri_d, 3, 3, mode=mode)
        assert T == 1 and t.tolist() == [1, 1, 1]


def test_invalid_inputs_rejected():
    s = torch.tensor([0, 5], dtype=torch.uint32, device="cuda")
    d = torch.tensor([1, 2], dtype=torch.uint32, device="cuda")
    with pytest.raises(P.PgbError) as ei:
        P.pgb_graph_from_edges(s, d, 5)
    assert ei.value.code == P.PGB_E_INVAL
    g = P.pgb_graph_from_edges(s, d, 6)
    with pytest.raises(P.PgbError):
        P.pgb_partition(g, 0)
    with pytest.raises(P.PgbError):
        P.pgb_partition(g, 7)
    b = P.pgb_partition(g, 2)
    r = P.pgb_tc_run(b, P.pgb_tc_opts_default(per_vertex=0))
    with pytest.raises(P.PgbError) as ei:
        P.pgb_tc_result_get(r, per_vertex=True)
    assert ei.value.code == P.PGB_E_STATE
    assert P.pgb_tc_result_get(r, per_vertex=None)[0] == 0


def test_er_config_intermediates_and_counts():
    """ER G(4096, 65536), p = 4: every intermediate array and count."""
    src, dst, n = graphgen.er_distinct(4096, 65536, 1)
    og = oracle.clean(src, dst, n)
    oT, ot = oracle.tc_node_iterator(og)
    oo = oracle.orient(og)
    for rule in (P.PGB_CUT_NNZ, P.PGB_CUT_UNIFORM):
        oc = oracle.cuts(oo, 4, rule)
        obe = oracle.block_edges(oo, 4, oc)
        oijk, ow = oracle.triples(4, obe)
        _, _, otc = oracle.tc_forward(oo, 4, oc, per_vertex=False)
        gT, gt, tri, g, b = gpu_count(src, dst, n, 4, rule=rule, mode=P.PGB_MODE_PLAIN, per_triple=True)
        assert gT == oT and np.array_equal(gt, ot)
        a_, b_, deg = P.pgb_graph_export(g)
        assert np.array_equal(deg, og.degree().astype(np.uint32))
        assert len(a_) == og.m and np.all(a_ < b_)
        keys = a_.astype(np.uint64) << np.uint64(32) | b_.astype(np.uint64)
        assert np.all(np.diff(keys.astype(np.int64)) > 0)
        assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_PERM), oo.perm)
        assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_ROWPTR), oo.rowptr)
        assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_COL), oo.col)
        assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_CUTS), oc)
        assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_BLOCK_EDGES), obe)
        assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_TRIPLES), oijk)
        assert np.array_equal(P.pgb_blocks_export(b, P.PGB_EXPORT_WEIGHTS), ow)
        want = np.array([otc[i, j, k] for i, j, k in oijk.tolist()], np.uint64)
        assert np.array_equal(tri, want)
        assert int(otc.sum()) == oT
        info = P.pgb_blocks_info(b)
        assert info["alg_bytes"] == oracle.alg_bytes(oo)
        gT2, gt2, _, _, _ = gpu_count(src, dst, n, 4, rule=rule, mode=P.PGB_MODE_PERSISTENT)
        assert gT2 == oT and np.array_equal(gt2, ot)


@pytest.mark.parametrize("scale,p", [(12, 1), (13, 5), (14, 16), (15, 32)])
@pytest.mark.parametrize("mode", MODES)
def test_rmat_medium(scale, p, mode):
    src, dst, n = graphgen.rmat(scale, 16, scale)
    og = oracle.clean(src, dst, n)
    oT, ot = oracle.tc_node_iterator(og)
    for chunk in ([0, 32, 96] if mode == P.PGB_MODE_PERSISTENT else [0]):
        gT, gt, _, _, _ = gpu_count(src, dst, n, p, mode=mode, chunk=chunk)
        assert gT == oT
        assert np.array_equal(gt, ot)


@pytest.mark.parametrize("order", [P.PGB_ORDER_WEIGHT, P.PGB_ORDER_LOCALITY])
def test_grid_and_rgg(order):
    src, dst, n = graphgen.grid_plus_percent(256, 1.0, 3)
    oT, ot, _ = oracle_count(src, dst, n)
    gT, gt, _, _, _ = gpu_count(src, dst, n, 8, order=order)
    assert gT == oT and np.array_equal(gt, ot)
    src, dst, n = graphgen.rgg(50000, None, 4)
    oT, ot, _ = oracle_count(src, dst, n)
    gT, gt, _, _, _ = gpu_count(src, dst, n, 8, order=order)
    assert gT == oT and np.array_equal(gt, ot)


def test_repeatable_and_global_only_matches():
    src, dst, n = graphgen.rmat(14, 16, 77)
    a = gpu_count(src, dst, n, 8)
    b = gpu_count(src, dst, n, 8)
    c = gpu_count(src, dst, n, 8, per_vertex=False)
    assert a[0] == b[0] == c[0]
    assert np.array_equal(a[1], b[1])
    assert int(a[1].sum()) == 3 * a[0]


def test_count_edges_one_call_host_and_device():
    src, dst, n = graphgen.rmat(13, 16, 5)
    oT, ot, _ = oracle_count(src, dst, n)
    T, t = P.pgb_tc_count_edges(src, dst, n, 8)
    assert T == oT and np.array_equal(t, ot)
    ds = torch.from_numpy(src).cuda()
    dd = torch.from_numpy(dst).cuda()
    T, t = P.pgb_tc_count_edges(ds, dd, n, 8)
    assert T == oT and np.array_equal(t.cpu().numpy(), ot)


def test_from_csr_matches_edges():
    src, dst, n = graphgen.rmat(12, 8, 2)
    og = oracle.clean(src, dst, n)
    oT, ot = oracle.tc_node_iterator(og)
    g = P.pgb_graph_from_csr(n, og.offs, og.adj)
    b = P.pgb_partition(g, 4)
    T, t = P.pgb_tc_result_get(P.pgb_tc_run(b))
    assert T == oT and np.array_equal(t, ot)


VARIANTS = [P.PGB_VAR_BSEARCH, P.PGB_VAR_MERGE, P.PGB_VAR_HASH]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("per_vertex", [True, False])
def test_persistent_variants_rmat(variant, per_vertex):
    src, dst, n = graphgen.rmat(15, 16, 21)
    og = oracle.clean(src, dst, n)
    oT, ot = oracle.tc_node_iterator(og)
    gT, gt, _, _, _ = gpu_count(src, dst, n, 8, variant=variant, per_vertex=per_vertex)
    assert gT == oT
    if per_vertex:
        assert np.array_equal(gt, ot)


@pytest.mark.parametrize("variant", VARIANTS)
def test_persistent_variants_messy(variant):
    for seed in range(6):
        rng = np.random.default_rng(500 + seed)
        n = int(rng.integers(2, 3000))
        src, dst = messy_random(n, int(rng.integers(0, 20 * n)), rng)
        T, t, _ = oracle_count(src, dst, n)
        gT, gt, _, _, _ = gpu_count(src, dst, n, int(rng.integers(1, 9)), variant=variant)
        assert gT == T and np.array_equal(gt, t)


def test_hash_splits_heavy_middle_vertices():
    """K_2100 plus 300 vertices each joined to clique vertices 0, 1, 2.

    In degree order the clique's low members have more than 1024 higher
    neighbours (the hash kernel's table capacity: their tables are split into
    key-range slices), and with 256 in-edges per work item the high members'
    in-edges are split into chunks.  Closed form: C(2100, 3) clique triangles
    plus 3 per extra vertex; t = C(2099, 2) on clique vertices, + 2 * 300 on
    0, 1, 2, and 3 on each extra vertex."""
    from math import comb
    k, extra = 2100, 300
    a, b = np.triu_indices(k, 1)
    xs = np.repeat(np.arange(k, k + extra), 3)
    ys = np.tile(np.array([0, 1, 2]), extra)
    src = np.concatenate([a, xs]).astype(np.uint32)
    dst = np.concatenate([b, ys]).astype(np.uint32)
    n = k + extra
    want_t = np.full(n, comb(k - 1, 2), dtype=np.uint64)
    want_t[:3] += 2 * extra
    want_t[k:] = 3
    for variant in VARIANTS:
        for p in (1, 5):
            for chunk in (0, 256):
                gT, gt, _, _, _ = gpu_count(src, dst, n, p, variant=variant, chunk=chunk)
                assert gT == comb(k, 3) + 3 * extra
                assert np.array_equal(gt, want_t)


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_hash_cta_shapes(threads):
    """Every CTA shape of the hash kernel (the autotuner picks the wider
    shapes only for graphs of many vertices, so they are forced here)."""
    for path in golden_files():
        src, dst, n, T, t = load_golden(path)
        for p in sorted({1, 2, n}):
            gT, gt, _, _, _ = gpu_count(src, dst, n, p, variant=P.PGB_VAR_HASH, hash_threads=threads)
            assert gT == T and np.array_equal(gt, t)
    for seed in range(3):
        rng = np.random.default_rng(800 + seed)
        n = int(rng.integers(2, 3000))
        src, dst = messy_random(n, int(rng.integers(0, 20 * n)), rng)
        T, t, _ = oracle_count(src, dst, n)
        gT, gt, _, _, _ = gpu_count(src, dst, n, int(rng.integers(1, 9)), variant=P.PGB_VAR_HASH,
                                    hash_threads=threads)
        assert gT == T and np.array_equal(gt, t)
    src, dst, n = graphgen.rmat(15, 16, 21)
    oT, ot = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    for pv in (True, False):
        gT, gt, _, _, _ = gpu_count(src, dst, n, 8, variant=P.PGB_VAR_HASH, hash_threads=threads, per_vertex=pv)
        assert gT == oT
        if pv:
            assert np.array_equal(gt, ot)
    # K_2600: 2,599 keys per list, more than one table of the two smaller
    # shapes holds (key slices) and within one of the 512-thread shape
    k = 2600
    a, b = np.triu_indices(k, 1)
    gT, gt, _, _, _ = gpu_count(a.astype(np.uint32), b.astype(np.uint32), k, 3, variant=P.PGB_VAR_HASH,
                                hash_threads=threads)
    assert gT == comb(k, 3) and np.all(gt == comb(k - 1, 2))
    with pytest.raises(P.PgbError) as ei:
        gpu_count(src, dst, n, 8, variant=P.PGB_VAR_HASH, hash_threads=192)
    assert ei.value.code == P.PGB_E_INVAL


def test_plain_mode_rejects_hash():
    src, dst, n = graphgen.rmat(8, 8, 1)
    with pytest.raises(P.PgbError) as ei:
        gpu_count(src, dst, n, 2, mode=P.PGB_MODE_PLAIN, variant=P.PGB_VAR_HASH)
    assert ei.value.code == P.PGB_E_INVAL


@pytest.mark.parametrize("path", golden_files(), ids=lambda x: x.split("/")[-1])
def test_plain_merge_golden(path):
    """PLAIN mode with the merge variant: one launch per triple, every p."""
    src, dst, n, T, t = load_golden(path)
    for p in range(1, n + 1):
        gT, gt, _, _, _ = gpu_count(src, dst, n, p, mode=P.PGB_MODE_PLAIN, variant=P.PGB_VAR_MERGE)
        assert gT == T and np.array_equal(gt, t)


def test_merge_long_balanced_lists():
    """Lists far longer than one 32-entry chunk on both sides, with ragged
    tails: K_200 (every edge's lists overlap in up to 198 entries) plus a
    sparse random fringe; per-triple counts equal the binary-search ones."""
    from math import comb
    k = 200
    a, b = np.triu_indices(k, 1)
    rng = np.random.default_rng(77)
    fs = rng.integers(0, 600, 3000)
    fd = rng.integers(0, 600, 3000)
    src = np.concatenate([a, fs]).astype(np.uint32)
    dst = np.concatenate([b, fd]).astype(np.uint32)
    n = 600
    T, t, _ = oracle_count(src, dst, n)
    assert T >= comb(k, 3)
    for mode in MODES:
        for p in (1, 3, 7):
            gT, gt, tri, _, _ = gpu_count(src, dst, n, p, mode=mode, variant=P.PGB_VAR_MERGE,
                                          per_triple=mode == P.PGB_MODE_PLAIN)
            assert gT == T and np.array_equal(gt, t)
            if mode == P.PGB_MODE_PLAIN:
                _, _, tri_b, _, _ = gpu_count(src, dst, n, p, mode=mode, variant=P.PGB_VAR_BSEARCH,
                                              per_triple=True)
                assert np.array_equal(tri, tri_b)

