"""Serve loop on the GPU: each job's counts are exact (bit-identical to the
oracle) whether it runs alone (SERIAL, one job at a time) or interleaved with
other jobs in shared persistent launches (BATCHED, continuous batching), and
the admission, cancel and timeout paths behave as the header states."""
import numpy as np
import pytest

import graphgen
import oracle
from _graphs import messy_random

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2209_04541_b300 import pgabb as P  # noqa: E402


def job_mix(seed=0):
    rng = np.random.default_rng(seed)
    jobs = []
    for s in (6, 8, 10, 12, 13):
        jobs.append(graphgen.rmat(s, int(rng.integers(8, 33)), int(rng.integers(1, 1000))))
    for n in (50, 1000, 5000):
        m = int(n * rng.integers(2, 33) // 2)
        jobs.append(graphgen.er_pairs(n, m, int(rng.integers(1, 1000))))
    jobs.append(graphgen.rgg(20000, None, 3))
    jobs.append(graphgen.grid_plus_percent(64, 1.0, 2))
    src, dst = messy_random(300, 4000, rng)
    jobs.append((src, dst, 300))
    e = np.zeros(0, np.uint32)
    jobs.append((e, e, 0))           # empty graph
    jobs.append((e, e, 17))          # isolated vertices only
    loops = np.arange(9, dtype=np.uint32)
    jobs.append((loops, loops, 9))   # self-loops only
    return jobs


def expected(jobs):
    out = []
    for src, dst, n in jobs:
        g = oracle.clean(src, dst, n)
        out.append(oracle.tc_node_iterator(g))
    return out


def run_server(jobs, mode, **kw):
    srv = P.pgb_server_create(P.pgb_server_opts_default(mode=mode, **kw))
    try:
        ids = [P.pgb_server_submit(srv, s, d, n) for s, d, n in jobs]
        res = [P.pgb_server_wait(srv, j, 120.0, per_vertex=True) for j in ids]
        stats = P.pgb_server_stats(srv)
    finally:
        P.pgb_server_destroy(srv)
    return res, stats


def test_serve_alone_and_mixed_match_oracle():
    jobs = job_mix()
    want = expected(jobs)
    batched, st_b = run_server(jobs, P.PGB_SERVE_BATCHED, max_inflight=4, max_batch_jobs=64)
    serial, st_s = run_server(jobs, P.PGB_SERVE_SERIAL)
    assert st_b["done"] == len(jobs) and st_s["done"] == len(jobs)
    # a job spread over several launches counts once per launch
    assert st_b["jobs_in_batches"] >= len(jobs)
    for (T, t), (bT, bt, blat), (sT, st, slat) in zip(want, batched, serial):
        assert bT == T and sT == T
        assert np.array_equal(bt, t) and np.array_equal(st, t)
        assert blat > 0 and slat > 0
    # a single job submitted alone gives the same answer as in the mix
    alone, _ = run_server(jobs[4:5], P.PGB_SERVE_BATCHED)
    assert alone[0][0] == want[4][0] and np.array_equal(alone[0][1], want[4][1])


def test_serve_mixed_batches_share_launches():
    jobs = [graphgen.rmat(10, 16, s) for s in range(24)]
    want = expected(jobs)
    srv = P.pgb_server_create(P.pgb_server_opts_default(max_inflight=2, max_batch_jobs=16))
    try:
        P.pgb_server_pause(srv, True)
        ids = [P.pgb_server_submit(srv, s, d, n) for s, d, n in jobs]
        P.pgb_server_pause(srv, False)
        res = [P.pgb_server_wait(srv, j, 120.0, per_vertex=True) for j in ids]
        st = P.pgb_server_stats(srv)
    finally:
        P.pgb_server_destroy(srv)
    assert st["done"] == len(jobs)
    assert st["batches"] == 2, "24 queued jobs at 16 per batch make two batches"
    for (T, t), (bT, bt, _) in zip(want, res):
        assert bT == T and np.array_equal(bt, t)


@pytest.mark.parametrize("batch_edges", [1, 60000, 0])
def test_serve_batch_caps_match_oracle(batch_edges):
    """Batch caps from one job per batch (every job is larger than one edge)
    to everything in one batch; totals and per-vertex counts stay exact."""
    jobs = [graphgen.rmat(14, 16, 3), graphgen.rmat(9, 8, 4), graphgen.er_pairs(3000, 40000, 5),
            graphgen.rgg(5000, None, 6), graphgen.rmat(12, 32, 7)]
    want = expected(jobs)
    srv = P.pgb_server_create(P.pgb_server_opts_default(mode=P.PGB_SERVE_BATCHED, max_inflight=1,
                                                        batch_edges=batch_edges))
    try:
        P.pgb_server_pause(srv, True)
        ids = [P.pgb_server_submit(srv, s, d, n) for s, d, n in jobs]
        P.pgb_server_pause(srv, False)
        res = [P.pgb_server_wait(srv, j, 120.0, per_vertex=True) for j in ids]
        st = P.pgb_server_stats(srv)
    finally:
        P.pgb_server_destroy(srv)
    assert st["done"] == len(jobs)
    if batch_edges == 1:
        assert st["batches"] == len(jobs)
    if batch_edges == 0:
        assert st["batches"] == 1
    for (T, t), (bT, bt, _) in zip(want, res):
        assert bT == T and np.array_equal(bt, t)


def test_serve_bad_job_fails_alone_in_a_batch():
    """A job with an endpoint >= n fails; the jobs batched with it do not."""
    jobs = [graphgen.rmat(10, 16, 1), (np.array([0, 7, 1], np.uint32), np.array([1, 2, 2], np.uint32), 5),
            graphgen.rmat(9, 16, 2)]
    srv = P.pgb_server_create(P.pgb_server_opts_default(max_inflight=1))
    try:
        P.pgb_server_pause(srv, True)
        ids = [P.pgb_server_submit(srv, s, d, n) for s, d, n in jobs]
        P.pgb_server_pause(srv, False)
        for k in (0, 2):
            T, t, _ = P.pgb_server_wait(srv, ids[k], 120.0, per_vertex=True)
            oT, ot = oracle.tc_node_iterator(oracle.clean(*jobs[k]))
            assert T == oT and np.array_equal(t, ot)
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_wait(srv, ids[1], 60.0)
        assert ei.value.code == P.PGB_E_INVAL
        assert P.pgb_server_stats(srv)["batches"] == 1
    finally:
        P.pgb_server_destroy(srv)


def test_serve_budget_cancel_timeout_and_failures():
    big = graphgen.rmat(17, 16, 5)
    small = graphgen.rmat(8, 8, 6)
    est_big = P.pgb_server_job_bytes(len(big[0]), big[2])
    srv = P.pgb_server_create(P.pgb_server_opts_default(budget_bytes=est_big + (1 << 20), max_inflight=2))
    try:
        # a job that can never fit the budget is refused at submit
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_submit(srv, *graphgen.rmat(19, 16, 1)[:2], 1 << 19)
        assert ei.value.code == P.PGB_E_BUDGET
        # with admission held, jobs stay queued: a bounded wait times out and
        # a queued job can be cancelled
        P.pgb_server_pause(srv, True)
        j1 = P.pgb_server_submit(srv, big[0], big[1], big[2])
        j2 = P.pgb_server_submit(srv, big[0], big[1], big[2])
        assert P.pgb_server_poll(srv, j1) == P.PGB_JOB_QUEUED
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_wait(srv, j1, 0.05)
        assert ei.value.code == P.PGB_E_TIMEOUT
        P.pgb_server_cancel(srv, j2)
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_wait(srv, j2, 60.0)
        assert ei.value.code == P.PGB_E_CANCELLED
        P.pgb_server_pause(srv, False)
        T1, _, _ = P.pgb_server_wait(srv, j1, 120.0)
        assert T1 == oracle.tc_node_iterator(oracle.clean(*big), per_vertex=False)[0]
        # a job with a vertex ID >= n fails; the server keeps serving
        bad = P.pgb_server_submit(srv, np.array([0, 7], np.uint32), np.array([1, 2], np.uint32), 5)
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_wait(srv, bad, 60.0)
        assert ei.value.code == P.PGB_E_INVAL
        ok = P.pgb_server_submit(srv, *small)
        assert P.pgb_server_wait(srv, ok, 60.0)[0] == oracle.tc_node_iterator(oracle.clean(*small), False)[0]
        st = P.pgb_server_stats(srv)
        assert st["cancelled"] == 1 and st["failed"] == 1 and st["bytes_in_use"] == 0
    finally:
        P.pgb_server_destroy(srv)


def test_serve_without_per_vertex():
    srv = P.pgb_server_create(P.pgb_server_opts_default(per_vertex=0))
    try:
        g = graphgen.rmat(9, 8, 3)
        j = P.pgb_server_submit(srv, *g)
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_wait(srv, j, 60.0, per_vertex=True)
        assert ei.value.code == P.PGB_E_STATE
        j = P.pgb_server_submit(srv, *g)
        assert P.pgb_server_wait(srv, j, 60.0)[0] == oracle.tc_node_iterator(oracle.clean(*g), False)[0]
    finally:
        P.pgb_server_destroy(srv)


def test_serve_benchmark_mix_sample_matches_oracle():
    """A seeded sample of the benchmark's own serving workload (10,000 jobs,
    scales up to 16; job i seeded by i, as bench.py makes it): every sampled
    job, counted in one batched mix, equals the oracle's counts."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    idx = sorted(np.random.default_rng(2027).choice(10000, size=24, replace=False).tolist())
    jobs = [bench.serve_job(i, 16) for i in idx]
    want = expected(jobs)
    res, stats = run_server(jobs, P.PGB_SERVE_BATCHED)
    assert stats["batches"] < len(jobs)
    for (T, t), (gT, gt, _) in zip(want, res):
        assert gT == T and np.array_equal(gt, t)


def test_serve_device_inputs_match_host_inputs():
    """Jobs submitted as device arrays (copied and held on the device while
    queued, or borrowed in place) or as borrowed host arrays (pinned and
    pageable) give the counts of the same jobs submitted from host memory, in
    both modes."""
    jobs = job_mix(5)
    want = expected(jobs)
    for mode in (P.PGB_SERVE_BATCHED, P.PGB_SERVE_SERIAL):
        srv = P.pgb_server_create(P.pgb_server_opts_default(mode=mode, max_inflight=2))
        try:
            ids = []
            for k, (s, d, n) in enumerate(jobs):
                kind = k % 5  # host copied, device copied, device borrowed, pinned and pageable host borrowed
                if kind in (1, 2):
                    s = torch.from_numpy(np.ascontiguousarray(s)).cuda()
                    d = torch.from_numpy(np.ascontiguousarray(d)).cuda()
                    torch.cuda.synchronize()
                elif kind == 3:
                    s = torch.from_numpy(np.ascontiguousarray(s)).pin_memory()
                    d = torch.from_numpy(np.ascontiguousarray(d)).pin_memory()
                elif kind == 4:
                    s, d = np.array(s, np.uint32), np.array(d, np.uint32)
                ids.append(P.pgb_server_submit(srv, s, d, n, borrow=kind >= 2))
                del s, d
            torch.cuda.synchronize()
            res = [P.pgb_server_wait(srv, j, 120.0, per_vertex=True) for j in ids]
        finally:
            P.pgb_server_destroy(srv)
        for (T, t), (gT, gt, _) in zip(want, res):
            assert gT == T and np.array_equal(gt, t)


def test_serve_device_inputs_cancel_and_destroy_while_queued():
    """Queued device jobs can be cancelled, and a server destroyed with device
    jobs still queued releases them; the next server counts normally."""
    g = graphgen.rmat(10, 16, 4)
    T = oracle.tc_node_iterator(oracle.clean(*g), False)[0]
    ds, dd = torch.from_numpy(g[0]).cuda(), torch.from_numpy(g[1]).cuda()
    srv = P.pgb_server_create(P.pgb_server_opts_default())
    try:
        P.pgb_server_pause(srv, True)
        ids = [P.pgb_server_submit(srv, ds, dd, g[2]) for _ in range(4)]
        P.pgb_server_cancel(srv, ids[1])
        with pytest.raises(P.PgbError) as ei:
            P.pgb_server_wait(srv, ids[1], 10.0)
        assert ei.value.code == P.PGB_E_CANCELLED
        P.pgb_server_pause(srv, False)
        assert P.pgb_server_wait(srv, ids[0], 60.0)[0] == T
    finally:
        P.pgb_server_destroy(srv)  # ids[2], ids[3] may still be queued
    srv = P.pgb_server_create(P.pgb_server_opts_default())
    try:
        assert P.pgb_server_wait(srv, P.pgb_server_submit(srv, ds, dd, g[2]), 60.0)[0] == T
        # borrowed inputs: a cancelled queued job, then a destroy with jobs queued
        P.pgb_server_pause(srv, True)
        ids = [P.pgb_server_submit(srv, ds, dd, g[2], borrow=True) for _ in range(3)]
        assert len(srv.borrowed) == 3
        P.pgb_server_cancel(srv, ids[0])
        with pytest.raises(P.PgbError):
            P.pgb_server_wait(srv, ids[0], 10.0)
        assert len(srv.borrowed) == 2
        P.pgb_server_pause(srv, False)
        assert P.pgb_server_wait(srv, ids[1], 60.0)[0] == T
    finally:
        P.pgb_server_destroy(srv)
    assert not srv.borrowed


def test_serve_full_size_mix_sample_matches_oracle_goldens():
    """A sample of the serving workload at its stated size (scales up to 22:
    the largest R-MAT, ER and RGG job of the first 10,000 plus seeded random
    jobs), generated on the device and submitted from device memory as the
    full-size bench does, counted in batched mixes: each job's total and
    per-vertex counts equal the oracle's stored values."""
    import hashlib
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_golden
    from graphgen import device as gd

    sample = make_golden.load_serve()
    assert len(sample) >= 12
    srv = P.pgb_server_create(P.pgb_server_opts_default(mode=P.PGB_SERVE_BATCHED, max_inflight=2))
    try:
        ids = []
        for job, spec, n, raw, m, T, sha in sample:
            assert graphgen.serve_spec(job, 22) == spec
            s, d, gn = gd.serve_job(job, 22)
            assert gn == n and s.numel() == raw
            torch.cuda.synchronize()
            ids.append(P.pgb_server_submit(srv, s, d, n, borrow=len(ids) % 2 == 1))
            del s, d
        for (job, spec, n, raw, m, T, sha), j in zip(sample, ids):
            gT, gt, _ = P.pgb_server_wait(srv, j, 600.0, per_vertex=True)
            assert gT == T, (job, spec)
            assert hashlib.sha256(np.ascontiguousarray(gt, dtype="<u8").tobytes()).hexdigest() == sha, (job, spec)
    finally:
        P.pgb_server_destroy(srv)
    torch.cuda.empty_cache()


def test_bench_staged_serve_client_matches_oracle():
    """bench.py's full-size serve client (jobs made on the device in
    segments, staged in pinned host memory or in device memory, submitted
    from there in a closed loop or at timed arrivals) on a small mix with a
    staging buffer of 2^18 words (one of the largest jobs, 2^12 x 32 raw
    edges, takes 2^18), so that it runs in many segments: every total equals the
    oracle's on the host-generated job, in both modes."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    count, scale = 40, 12
    want = [oracle.tc_node_iterator(oracle.clean(*graphgen.serve_job(i, scale)), False)[0] for i in range(count)]
    arrivals = np.cumsum(np.full(count, 0.002))
    for where in ("host", "device"):
        words = 1 << 18
        buf = (torch.empty(words, dtype=torch.uint32, pin_memory=True) if where == "host"
               else torch.empty(words, dtype=torch.uint32, device="cuda"))
        for mode in (P.PGB_SERVE_SERIAL, P.PGB_SERVE_BATCHED):
            tot, lat, span, st, raw, client = bench.run_serve_staged(count, scale, mode, None, buf)
            assert tot == want and span > 0 and all(x > 0 for x in lat)
            assert client["segments"] >= 8
        tot, *_ = bench.run_serve_staged(count, scale, P.PGB_SERVE_BATCHED, arrivals, buf)
        assert tot == want
    with pytest.raises(ValueError):  # a job larger than the buffer
        bench.run_serve_staged(count, scale, P.PGB_SERVE_BATCHED, None, torch.empty(1000, dtype=torch.uint32,
                                                                                     pin_memory=True))
