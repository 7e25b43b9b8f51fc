"""Host edge lists of 2^26 pairs or more are ingested in chunks: each chunk is
sorted while the next one is copied, then the sorted runs are merged.  The
cleaned graph (pairs and degrees), the counts and the error on a bad vertex
ID must be those of the device-input path."""
import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402


def both_paths(src, dst, n):
    """The cleaned graph from host arrays (pinned) and from device arrays."""
    hs = torch.from_numpy(src).pin_memory()
    hd = torch.from_numpy(dst).pin_memory()
    g_host = P.pgb_graph_from_edges(hs, hd, n)
    g_dev = P.pgb_graph_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    return g_host, g_dev


@pytest.mark.parametrize("scale,ef,seed", [(22, 16, 3), (21, 40, 8)])
def test_chunked_host_ingest_equals_device_ingest(scale, ef, seed):
    """2^26 pairs (two chunks) and 2^21 x 40 = 83.9 M pairs (a ragged third
    chunk): the same cleaned pairs, degrees, and per-vertex counts."""
    src, dst, n = graphgen.rmat(scale, ef, seed)
    assert len(src) >= 1 << 26
    g_host, g_dev = both_paths(src, dst, n)
    a1, b1, d1 = P.pgb_graph_export(g_host)
    a2, b2, d2 = P.pgb_graph_export(g_dev)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2) and np.array_equal(d1, d2)
    T = []
    for g in (g_host, g_dev):
        r = P.pgb_tc_run(P.pgb_partition(g, 16), P.pgb_tc_opts_default())
        T.append(P.pgb_tc_result_get(r))
    assert T[0][0] == T[1][0] and np.array_equal(T[0][1], T[1][1])
    torch.cuda.empty_cache()


def test_chunked_host_ingest_matches_oracle_and_counts_end_to_end():
    """pgb_tc_count_edges from pinned host arrays (the end-to-end path) on a
    2^26-pair graph with self-loops and repeats: the oracle's counts."""
    rng = np.random.default_rng(5)
    n = 1 << 20
    src, dst, _ = graphgen.er_pairs(n, 1 << 26, 9)
    loops = rng.choice(len(src), 1000, replace=False)
    src[loops] = dst[loops]  # self-loops
    src[-5000:] = dst[:5000]  # repeats of early pairs, reversed, in the last chunk
    dst[-5000:] = src[:5000]
    g = oracle.clean(src, dst, n)
    T_ref, t_ref = oracle.tc_node_iterator(g)
    hs = torch.from_numpy(src).pin_memory()
    hd = torch.from_numpy(dst).pin_memory()
    out = torch.zeros(n, dtype=torch.uint64, pin_memory=True)
    T, _ = P.pgb_tc_count_edges(hs, hd, n, 8, P.PGB_CUT_NNZ, P.pgb_tc_opts_default(), per_vertex=out)
    assert T == T_ref and np.array_equal(out.numpy(), t_ref)


def test_chunked_host_ingest_rejects_bad_ids():
    src, dst, n = graphgen.er_pairs(1 << 20, 1 << 26, 4)
    dst[(1 << 25) + 17] = n  # in the second chunk
    with pytest.raises(P.PgbError) as ei:
        P.pgb_graph_from_edges(torch.from_numpy(src).pin_memory(), torch.from_numpy(dst).pin_memory(), n)
    assert ei.value.code == P.PGB_E_INVAL
    # the library stays usable
    ok = (dst[:1000] % n).astype(np.uint32)
    g = P.pgb_graph_from_edges(torch.from_numpy(src[:1000].copy()).pin_memory(), torch.from_numpy(ok).pin_memory(), n)
    assert P.pgb_graph_info(g)[0] == n
