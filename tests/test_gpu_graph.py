"""CUDA-graph replay of a run (use_graph = 1): the run's device work is
captured once per setting on the blocks handle and replayed.  Counts are
exact integers: every replay must equal the oracle and the uncaptured run
bit for bit, including per-triple counts of PLAIN mode."""
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import golden_files, load_golden

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb  # noqa: E402

P = pgabb

SETTINGS = [
    dict(mode=P.PGB_MODE_PLAIN),
    dict(mode=P.PGB_MODE_PLAIN, per_triple=1),
    dict(mode=P.PGB_MODE_PERSISTENT, variant=P.PGB_VAR_BSEARCH),
    dict(mode=P.PGB_MODE_PLAIN, variant=P.PGB_VAR_MERGE, per_triple=1),
    dict(mode=P.PGB_MODE_PERSISTENT, variant=P.PGB_VAR_MERGE),
    dict(mode=P.PGB_MODE_PERSISTENT, variant=P.PGB_VAR_HASH),
    dict(mode=P.PGB_MODE_PERSISTENT, variant=P.PGB_VAR_HASH, hash_threads=256),
    dict(mode=P.PGB_MODE_PERSISTENT, variant=P.PGB_VAR_HASH, hash_threads=512),
    dict(mode=P.PGB_MODE_PERSISTENT, variant=P.PGB_VAR_AUTO, per_vertex=0),
]


def _blocks(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(np.ascontiguousarray(src, np.uint32)).cuda(),
                               torch.from_numpy(np.ascontiguousarray(dst, np.uint32)).cuda(), n)
    return P.pgb_partition(g, p)


def _get(b, stream=None, **kw):
    o = P.pgb_tc_opts_default(**kw)
    r = P.pgb_tc_run(b, o, stream)
    T, t = P.pgb_tc_result_get(r, per_vertex=bool(o.per_vertex))
    tri = P.pgb_tc_result_triples(r) if kw.get("per_triple") else None
    return T, t, tri


@pytest.mark.parametrize("kw", SETTINGS, ids=lambda d: "-".join(f"{k}{v}" for k, v in d.items()))
def test_rmat_replays_match_oracle(kw):
    src, dst, n = graphgen.rmat(14, 16, 9)
    oT, ot = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = _blocks(src, dst, n, 8)
    T0, t0, tri0 = _get(b, **kw)
    assert T0 == oT
    for _ in range(3):
        T, t, tri = _get(b, use_graph=1, **kw)
        assert T == oT
        if kw.get("per_vertex", 1):
            assert np.array_equal(t, ot) and np.array_equal(t, t0)
        if tri0 is not None:
            assert np.array_equal(tri, tri0) and int(tri.sum()) == oT


@pytest.mark.parametrize("path", golden_files(), ids=lambda x: x.split("/")[-1])
def test_golden_fixtures_replayed(path):
    src, dst, n, T, t = load_golden(path)
    for p in sorted({1, 2, n}):
        b = _blocks(src, dst, n, p)
        for kw in SETTINGS:
            for _ in range(2):
                gT, gt, _ = _get(b, use_graph=1, **kw)
                assert gT == T
                if kw.get("per_vertex", 1):
                    assert np.array_equal(gt, t)


def test_replay_launch_count_and_result_isolation():
    """A replay launches the same kernels as the uncaptured run; results of
    earlier replays survive later ones (outputs are copied per result)."""
    src, dst, n = graphgen.rmat(13, 8, 2)
    oT, ot = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = _blocks(src, dst, n, 6)
    for kw in SETTINGS:
        o_plain = P.pgb_tc_opts_default(**kw)
        o_graph = P.pgb_tc_opts_default(use_graph=1, **kw)
        l0 = P.pgb_kernel_launches()
        P.pgb_tc_result_get(P.pgb_tc_run(b, o_plain), per_vertex=False)
        uncaptured = P.pgb_kernel_launches() - l0
        P.pgb_tc_result_get(P.pgb_tc_run(b, o_graph), per_vertex=False)  # capture + first replay
        l1 = P.pgb_kernel_launches()
        r1 = P.pgb_tc_run(b, o_graph)
        r2 = P.pgb_tc_run(b, o_graph)
        replayed = (P.pgb_kernel_launches() - l1) / 2
        # the uncaptured run also builds work items on the device
        assert 0 < replayed <= uncaptured
        for r in (r1, r2):
            T, t = P.pgb_tc_result_get(r, per_vertex=bool(o_graph.per_vertex))
            assert T == oT
            if o_graph.per_vertex:
                assert np.array_equal(t, ot)


def test_replays_on_two_streams():
    src, dst, n = graphgen.rmat(13, 16, 4)
    oT, ot = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = _blocks(src, dst, n, 4)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    rs = [P.pgb_tc_run(b, P.pgb_tc_opts_default(use_graph=1), s) for s in (s1, s2, s1, s2)]
    for r in rs:
        T, t = P.pgb_tc_result_get(r)
        assert T == oT and np.array_equal(t, ot)


def test_empty_graph_replay():
    e = np.zeros(0, np.uint32)
    for n in (0, 9):
        b = _blocks(e, e, n, 1)
        for kw in SETTINGS:
            T, t, tri = _get(b, use_graph=1, **kw)
            assert T == 0
            if kw.get("per_vertex", 1):
                assert t.shape == (n,) and not t.any()


def test_graph_flag_ignored_after_offload():
    src, dst, n = graphgen.rmat(12, 16, 6)
    oT, ot = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = _blocks(src, dst, n, 4)
    assert _get(b, use_graph=1)[0] == oT  # leaves a captured plan behind
    P.pgb_blocks_offload(b)
    T, t, _ = _get(b, use_graph=1)
    assert T == oT and np.array_equal(t, ot)
