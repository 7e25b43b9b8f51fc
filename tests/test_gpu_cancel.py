"""Stop requests through a cancel token, against the oracle.

A run given a cancel token reads it from its kernels (the persistent
kernels every 64 work fetches, a plain per-triple launch at entry) and,
when it is set, skips the rest of its work; pgb_tc_result_get then fails
with PGB_E_CANCELLED.  Nothing here waits without a limit, faults or traps:
the stop is a flag the kernels read.  After every stopped run the same
partition, with the token reset, must count exactly what the oracle counts
(tolerance 0).
"""
import time

import numpy as np
import pytest

import graphgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402

SETTINGS = {
    "plain": dict(mode=P.PGB_MODE_PLAIN),
    "bsearch": dict(variant=P.PGB_VAR_BSEARCH),
    "hash": dict(variant=P.PGB_VAR_HASH),
    "auto": dict(),
    "hash+graph": dict(variant=P.PGB_VAR_HASH, use_graph=1),
    "plain+graph": dict(mode=P.PGB_MODE_PLAIN, use_graph=1),
}


def build(src, dst, n, p):
    g = P.pgb_graph_from_edges(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    return P.pgb_partition(g, p)


@pytest.fixture(scope="module")
def rmat17():
    src, dst, n = graphgen.rmat(17, 16, 21)
    T, t, _ = oracle.tc_forward(oracle.orient(oracle.clean(src, dst, n)))
    return build(src, dst, n, 16), T, t


@pytest.mark.parametrize("name", sorted(SETTINGS))
def test_token_set_before_the_run_cancels_it_and_a_reset_run_is_exact(rmat17, name):
    b, T, t = rmat17
    tok = P.pgb_cancel_create()
    try:
        P.pgb_cancel_set(tok)
        assert P.pgb_cancel_is_set(tok)
        for _ in range(2):  # graph settings: the capture run, then a replay
            r = P.pgb_tc_run(b, P.pgb_tc_opts_default(cancel=tok, **SETTINGS[name]))
            with pytest.raises(P.PgbError) as ei:
                P.pgb_tc_result_get(r)
            assert ei.value.code == P.PGB_E_CANCELLED
            r.free()
        P.pgb_cancel_reset(tok)
        for _ in range(2):
            r = P.pgb_tc_run(b, P.pgb_tc_opts_default(cancel=tok, **SETTINGS[name]))
            gT, gt = P.pgb_tc_result_get(r)
            assert gT == T and np.array_equal(gt, t)
    finally:
        tok.free()


def test_cancelled_run_stops_early():
    """R-MAT scale 21 with the hash kernel: a run whose token is set stops
    after about one work item per CTA, far below the full kernel time."""
    src, dst, n = graphgen.rmat(21, 16, 4)
    b = build(src, dst, n, 32)
    del src, dst
    tok = P.pgb_cancel_create()
    try:
        full = []
        for _ in range(3):
            r = P.pgb_tc_run(b, P.pgb_tc_opts_default(cancel=tok, variant=P.PGB_VAR_HASH))
            T, _ = P.pgb_tc_result_get(r)
            full.append(P.pgb_tc_result_kernel_ms(r))
        P.pgb_cancel_set(tok)
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(cancel=tok, variant=P.PGB_VAR_HASH))
        with pytest.raises(P.PgbError):
            P.pgb_tc_result_get(r)
        stopped = P.pgb_tc_result_kernel_ms(r)
        assert stopped < 0.5 * min(full), (stopped, full)
        P.pgb_cancel_reset(tok)
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(cancel=tok, variant=P.PGB_VAR_HASH))
        assert P.pgb_tc_result_get(r)[0] == T
    finally:
        tok.free()


def test_cancel_while_plain_launches_run():
    """Plain mode queues one launch per block triple; a token set while they
    run stops the launches that have not started.  The run either stops
    (PGB_E_CANCELLED, sooner than a full run) or, if it already finished,
    returns the exact counts; the next run is exact."""
    src, dst, n = graphgen.rmat(18, 16, 6)
    T, t = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = build(src, dst, n, 32)
    tok = P.pgb_cancel_create()
    try:
        opts = P.pgb_tc_opts_default(cancel=tok, mode=P.PGB_MODE_PLAIN)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = P.pgb_tc_run(b, opts)
        P.pgb_tc_result_get(r)
        full_s = time.perf_counter() - t0
        outcomes = []
        for delay in (0.0, 0.1, 0.3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = P.pgb_tc_run(b, opts)
            time.sleep(delay * full_s)
            P.pgb_cancel_set(tok)
            try:
                gT, gt = P.pgb_tc_result_get(r)
                assert gT == T and np.array_equal(gt, t)
                outcomes.append("done")
            except P.PgbError as e:
                assert e.code == P.PGB_E_CANCELLED
                assert time.perf_counter() - t0 < full_s + 0.5
                outcomes.append("cancelled")
            P.pgb_cancel_reset(tok)
        assert "cancelled" in outcomes
        gT, gt = P.pgb_tc_result_get(P.pgb_tc_run(b, opts))
        assert gT == T and np.array_equal(gt, t)
    finally:
        tok.free()


def test_streamed_run_cancels():
    src, dst, n = graphgen.rmat(16, 16, 2)
    T, t = oracle.tc_node_iterator(oracle.clean(src, dst, n))
    b = build(src, dst, n, 8)
    P.pgb_blocks_offload(b)
    tok = P.pgb_cancel_create()
    try:
        budget = P.pgb_blocks_resident_bytes(b, True) + (4 << 20)
        P.pgb_cancel_set(tok)
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(cancel=tok, device_budget=budget, chunk_edges=1024))
        with pytest.raises(P.PgbError) as ei:
            P.pgb_tc_result_get(r)
        assert ei.value.code == P.PGB_E_CANCELLED
        P.pgb_cancel_reset(tok)
        r = P.pgb_tc_run(b, P.pgb_tc_opts_default(cancel=tok, device_budget=budget, chunk_edges=1024))
        gT, gt = P.pgb_tc_result_get(r)
        assert gT == T and np.array_equal(gt, t)
        assert P.pgb_tc_result_stream(r)[1] > 1
    finally:
        tok.free()


def test_server_cancel_of_a_running_job():
    """SERIAL mode: a job cancelled while it runs ends as cancelled (its
    batch is stopped through the thread's token), and the jobs after it are
    exact."""
    big = graphgen.rmat(20, 16, 3)
    small = graphgen.rmat(12, 16, 5)
    sT, st = oracle.tc_node_iterator(oracle.clean(*small))
    srv = P.pgb_server_create(P.pgb_server_opts_default(mode=P.PGB_SERVE_SERIAL, per_vertex=1))
    try:
        j = P.pgb_server_submit(srv, *big)
        deadline = time.perf_counter() + 30
        while P.pgb_server_poll(srv, j) == P.PGB_JOB_QUEUED and time.perf_counter() < deadline:
            time.sleep(0.0005)
        P.pgb_server_cancel(srv, j)
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_wait(srv, j, 60.0)
        assert ei.value.code == P.PGB_E_CANCELLED
        for _ in range(3):
            k = P.pgb_server_submit(srv, *small)
            gT, gt, _ = P.pgb_server_wait(srv, k, 60.0, per_vertex=True)
            assert gT == sT and np.array_equal(gt, st)
    finally:
        P.pgb_server_destroy(srv)
