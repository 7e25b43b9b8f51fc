#!/usr/bin/env python3
"""Benchmark of exact block-triple triangle counting on one B300 per rank.

One step is the whole hot path on one synthetic graph whose raw edge list is
already resident in HBM: ingest (undirected, deduplicated, self-loops
dropped), degree order and orientation, p x p partition, block-triple queue,
the counting kernel with global and per-vertex counts, and the reduction.
The metric is unique undirected edges per second of step time (PGAbB
Section 5.4 counts triangles after degree ordering; here ordering and
partitioning are inside the timed step).

``value``: device-resident throughput, CUDA events on the launching stream.
``e2e``:   the same through the one-call C ABI entry with pinned host
           buffers (host-to-device copy of the raw edges and device-to-host
           copy of the total and per-vertex counts inside the timed call).
``roofline``: the counting kernel's own algorithmic bytes over its device
           time, against the measured HBM copy bandwidth.  For the
           middle-vertex kernel that is 4 probes + 12 |E+| (every looked-up
           entry of the tails' rows plus the in-edge index); for the
           edge-wise kernels 4|E+| + 4 sum_v indeg(v) outdeg(v) + 8(n+1).
           The second formula is also given for the middle-vertex kernel,
           as ``edgewise_bound``: it charges a re-read of v's list per
           in-edge, which that kernel serves from shared memory, so it is a
           bound for the edge-wise method, not a bandwidth fraction; so is
           ``merge_bytes``, both lists read per oriented edge.
``cpu_baseline``: the oracle on the same workload: its clean, degree order
           and orientation single-threaded in full, and its forward count
           on a stride sample of the rows with every host core (OpenMP
           build), scaled to the whole graph; the single-core figure beside.

With ``--impl reference`` the oracle itself is the measured arm (rank 0
only).  Under torchrun each rank runs an independent replica (the path
needs no exchange between replicas): ``value`` is the summed edges of all
ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen  # noqa: E402

WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, ef=16, p=32, seed=1,
                   desc="R-MAT scale 24, edge factor 16 (a,b,c,d = .57,.19,.19,.05), seeded relabel; p=32"),
    "rmat23": dict(kind="rmat", scale=23, ef=16, p=32, seed=1,
                   desc="R-MAT scale 23, edge factor 16 (a,b,c,d = .57,.19,.19,.05), seeded relabel; p=32"),
    "rmat22": dict(kind="rmat", scale=22, ef=16, p=32, seed=1,
                   desc="R-MAT scale 22, edge factor 16 (a,b,c,d = .57,.19,.19,.05), seeded relabel; p=32"),
    "rmat20": dict(kind="rmat", scale=20, ef=16, p=16, seed=1,
                   desc="R-MAT scale 20, edge factor 16 (a,b,c,d = .57,.19,.19,.05), seeded relabel; p=16"),
    "grid4096": dict(kind="grid", side=4096, pct=1.0, p=32, seed=1,
                     desc="4096x4096 4-neighbour grid + 1% uniform random extra edges; p=32"),
    "er4096": dict(kind="er", n=4096, m=65536, p=4, seed=1,
                   desc="Erdos-Renyi G(n=4096, m=65536) distinct pairs; p=4"),
    "rgg22": dict(kind="rgg", n=1 << 22, p=32, seed=1,
                  desc="random geometric graph, n=2^22, average degree about 6; p=32"),
    "er22": dict(kind="erp", n=1 << 22, m=32 << 22, p=32, seed=1,
                 desc="Erdos-Renyi, n=2^22, 2^27 uniform pairs (average degree about 64); p=32"),
    "rmat25": dict(kind="rmat", scale=25, ef=16, p=64, seed=1,
                   desc="R-MAT scale 25, edge factor 16 (a,b,c,d = .57,.19,.19,.05), seeded relabel; p=64"),
    "rmat26": dict(kind="rmat", scale=26, ef=16, p=64, seed=1,
                   desc="R-MAT scale 26, edge factor 16 (a,b,c,d = .57,.19,.19,.05), seeded relabel; p=64"),
    "rmat27": dict(kind="rmat", scale=27, ef=16, p=64, seed=1,
                   desc="R-MAT scale 27, edge factor 16 (a,b,c,d = .57,.19,.19,.05), seeded relabel; p=64"),
    "grid4096_u_rmat22": dict(kind="union", members=("grid4096", "rmat22"), p=32, seed=1,
                              desc="disjoint union of the 4096x4096 grid + 1% and R-MAT scale 22 ef16 (the shape "
                                   "of a serve batch: flat and skewed graphs in one partition); p=32"),
}

# Reference arm: the oracle's whole pipeline per step at a size it finishes
# in about a second single-threaded.
REF_SAMPLE = dict(kind="rmat", scale=17, ef=16, p=8, seed=1)


def generate(w, out=None):
    if w["kind"] == "union":
        srcs, dsts, base = [], [], 0
        for name in w["members"]:
            s_, d_, n_ = generate(WORKLOADS[name])
            srcs.append(s_ + np.uint32(base))
            dsts.append(d_ + np.uint32(base))
            base += n_
        return np.concatenate(srcs), np.concatenate(dsts), base
    if w["kind"] == "rmat":
        if w["scale"] >= 16 and _cuda_ok():
            return rmat_on_device(w, out)
        return graphgen.rmat(w["scale"], w["ef"], w["seed"], out=out)
    if w["kind"] == "grid":
        return graphgen.grid_plus_percent(w["side"], w["pct"], w["seed"])
    if w["kind"] == "er":
        return graphgen.er_distinct(w["n"], w["m"], w["seed"])
    if w["kind"] == "erp":
        return graphgen.er_pairs(w["n"], w["m"], w["seed"])
    if w["kind"] == "rgg":
        return graphgen.rgg(w["n"], None, w["seed"])
    raise ValueError(w)


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def rmat_on_device(w, out=None):
    """graphgen.rmat(scale, ef, seed) made by the device generator (the same
    edges: the host's Fisher-Yates labels applied on the device) and copied
    to host arrays (`out`, e.g. pinned, or new numpy arrays); the host
    generator takes tens of seconds at scale 27."""
    import torch
    from graphgen import device as gd
    s_d, d_d, n = gd.rmat(w["scale"], w["ef"], w["seed"], relabel="shuffle")
    if out is None:
        out = (np.empty(s_d.numel(), np.uint32), np.empty(d_d.numel(), np.uint32))
    torch.from_numpy(out[0]).copy_(s_d)
    torch.from_numpy(out[1]).copy_(d_d)
    del s_d, d_d
    torch.cuda.empty_cache()
    return out[0], out[1], n


def raw_edge_count(w):
    if w["kind"] == "rmat":
        return w["ef"] << w["scale"]
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return 6400.0, "of fallback"


def measured_tensor_peak():
    """Dense bf16 tensor throughput measured on the B300s, sustained
    (the dense block runs inside a long step), in TFLOP/s; fp16 runs at the
    same nominal rate.  Fallback: the recipe's sustained figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "of measured (bf16 sustained; fp16 same nominal rate)"
    except Exception:
        return 1400.0, "of fallback (bf16 sustained)"


KERNEL_SOURCE = {"k_tc_hash": "tc_hash.cu", "k_tc_persistent": "tc.cu", "k_tc_tuple": "tc.cu"}


def kernel_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes from the committed ncu summary for this kernel
    and workload, or None when absent or taken on an older kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    src = os.path.join(ROOT, "paper_2209_04541_b300", "csrc", KERNEL_SOURCE.get(kernel, "tc.cu"))
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h:
        return None
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return int(m.group(1)) if h.group(1) == cur else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None, interval_ms: int = 200):
        self.gpu_id = gpu_id
        self.interval_ms = interval_ms
        self.proc = None
        self.err = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms",
               str(self.interval_ms)]
        if self.gpu_id:
            cmd.insert(1, f"--id={self.gpu_id}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception as e:  # nvidia-smi missing
            self.err = str(e)
        time.sleep(0.15)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "error": self.err or "no sampler"}
        time.sleep(0.1)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sms, maxes, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sms.append(float(parts[0]))
                maxes.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxes) if maxes else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sms), "reasons": sorted(reasons)}


def aggregate(ms_local: float, units_local: float, dist=None):
    """(max step ms over ranks, summed units over ranks)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local, units_local
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def oracle_pipeline(w):
    """Oracle on one sample: clean -> order/orient -> count (global and
    per-vertex).  Returns (seconds, unique edges, triangles)."""
    import oracle
    src, dst, n = generate(w)
    t0 = time.perf_counter()
    g = oracle.clean(src, dst, n)
    o = oracle.orient(g)
    c = oracle.cuts(o, w["p"])
    oracle.block_edges(o, w["p"], c)
    T, _, _ = oracle.tc_forward(o)
    return time.perf_counter() - t0, g.m, T


def cpu_baseline(src, dst, n, target_s=12.0):
    """The oracle on the benchmark's own graph (a bounded sample of the
    work): clean + degree order + orientation in full (the oracle's
    single-threaded C), then the forward count with per-vertex counts over
    every stride-th row, on all host cores (OpenMP build) and on one core.
    Rows sampled with a stride give 1/stride of the count's work in
    expectation, so the whole count is estimated as stride x the sample's
    time.  Returns the cpu_baseline object (value: all cores)."""
    import oracle
    t0 = time.perf_counter()
    g = oracle.clean(src, dst, n)
    o = oracle.orient(g)
    prep_s = time.perf_counter() - t0
    m = g.m
    del g
    cores = oracle.num_threads()

    def timed(threads, stride):
        t = time.perf_counter()
        oracle.tc_forward_mt(o, per_vertex=True, threads=threads, stride=stride)
        return time.perf_counter() - t

    def sampled(threads, target):
        # fixed cost of a count (per-thread counters, their final sum): one row
        fixed = timed(threads, n + 1)
        stride = 4096
        while True:
            dt = timed(threads, stride)
            est = fixed + stride * max(dt - fixed, 0.0)
            if dt - fixed >= 0.25 * target or stride == 1:
                return stride, dt, est
            stride = max(1, min(stride // 2, int((est - fixed) / target) or 1))

    s_all, dt_all, est_all = sampled(cores, target_s)
    s_one, dt_one, est_one = sampled(1, target_s / 2)
    del o
    return {"value": m / (prep_s + est_all), "unit": "edges/s", "cores": cores, "kind": "oracle",
            "single_core_value": m / (prep_s + est_one),
            "sample": f"oracle on the benchmark's R-MAT graph itself ({m} unique edges): clean + degree order + "
                      f"orientation in full, single-threaded C, {prep_s:.1f} s; forward count with per-vertex "
                      f"counts over every {s_all}th row on {cores} cores (OpenMP build) in {dt_all:.2f} s, "
                      f"x{s_all} = {est_all:.1f} s estimated for all rows; single core: every {s_one}th row in "
                      f"{dt_one:.2f} s, x{s_one} = {est_one:.1f} s",
            "prep_s": prep_s, "count_s_all_cores": est_all, "count_s_single_core": est_one}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    w = REF_SAMPLE
    times = []
    m = T = 0
    for i in range(args.warmup + args.steps):
        secs, m, T = oracle_pipeline(w)
        if i >= args.warmup:
            times.append(secs)
    ms = 1e3 * statistics.mean(times)
    value = m / (ms / 1e3)
    sample = (f"oracle (single-threaded C) clean+order+orient+partition+count per step on R-MAT scale "
              f"{w['scale']} ef{w['ef']} p={w['p']} ({m} unique edges, {T} triangles), a bounded sample of "
              f"the {args.workload} workload family")
    line = {"impl": "reference", "metric": "TC edges/s", "value": value, "unit": "edges/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "sample": f"rmat_s{w['scale']}"},
            "cpu_baseline": {"value": value, "unit": "edges/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serve_job(i: int, max_scale: int):
    """Job i of the serving workload (graphgen.serve_spec), generated on the
    host: (src, dst, n) numpy arrays."""
    return graphgen.serve_job(i, max_scale)


def serve_job_device(i: int, max_scale: int, stream=None):
    """Job i generated on the device (the same edges as serve_job): (src,
    dst, n) with uint32 CUDA tensors written on `stream`."""
    from graphgen import device as gd
    return gd.serve_job(i, max_scale, stream)


def serve_jobs(count: int, max_scale: int):
    """The first `count` jobs of the serving workload."""
    return [serve_job(i, max_scale) for i in range(count)]


def run_serve(jobs, mode, arrivals=None, **kw):
    """Submit the jobs (all at once, or at the given arrival offsets in
    seconds) and wait for all; returns (totals, latencies s, makespan s)."""
    from paper_2209_04541_b300 import pgabb as P
    srv = P.pgb_server_create(P.pgb_server_opts_default(mode=mode, per_vertex=1, **kw))
    try:
        ids = []
        t0 = time.perf_counter()
        for k, (s, d, n) in enumerate(jobs):
            if arrivals is not None:
                delay = t0 + arrivals[k] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            ids.append(P.pgb_server_submit(srv, s, d, n))
        out = [P.pgb_server_wait(srv, j, 600.0) for j in ids]
        t1 = time.perf_counter()
        stats = P.pgb_server_stats(srv)
    finally:
        P.pgb_server_destroy(srv)
    return [o[0] for o in out], [o[2] for o in out], t1 - t0, stats


def serve_bench(args):
    from paper_2209_04541_b300 import pgabb as P
    jobs = serve_jobs(args.serve_jobs, args.serve_max_scale)
    edges = int(sum(len(j[0]) for j in jobs))
    run_serve(jobs[:8], P.PGB_SERVE_BATCHED)  # warm-up
    res = {}
    tot_s, _, span_s, _ = run_serve(jobs, P.PGB_SERVE_SERIAL)
    tot_b, _, span_b, st_b = run_serve(jobs, P.PGB_SERVE_BATCHED)
    assert tot_s == tot_b, "serial and batched counts differ"
    cap_s, cap_b = len(jobs) / span_s, len(jobs) / span_b
    sweep = {}
    for factor in (0.5, 0.8, 0.95):
        rate = factor * cap_s
        rng = np.random.default_rng(12345)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(jobs)))
        res = {}
        for name, mode in (("serial", P.PGB_SERVE_SERIAL), ("batched", P.PGB_SERVE_BATCHED)):
            tot, lat, span, st = run_serve(jobs, mode, arrivals)
            assert tot == tot_s
            lat_ms = np.array(lat) * 1e3
            res[name] = {"jobs_s": len(jobs) / span, "p50_ms": float(np.percentile(lat_ms, 50)),
                         "p99_ms": float(np.percentile(lat_ms, 99)), "launches": st["batches"]}
        sweep[f"{factor:.2f}"] = {"rate_jobs_s": rate, **res}
    return {"metric": "serve jobs/s and p50/p99 latency", "jobs": len(jobs), "raw_edges": edges,
            "mix": f"thirds of R-MAT (scale 10-{args.serve_max_scale}, ef 8-32, Feistel relabelling), ER (n "
                   f"2^10-2^{args.serve_max_scale} "
                   "log-uniform, avg degree 4-64 log-uniform), RGG (avg degree 6); seed = job index; per-vertex on",
            "capacity_jobs_s": {"serial": cap_s, "batched": cap_b},
            "poisson_rate_jobs_s": sweep["0.80"]["rate_jobs_s"],
            "poisson": {k: sweep["0.80"][k] for k in ("serial", "batched")},
            "poisson_sweep_by_fraction_of_serial_capacity": sweep,
            "batched_launches_closed_loop": st_b["batches"]}


def run_serve_staged(count, max_scale, mode, arrivals=None, buf=None, stream=None, inflight=1):
    """The serving workload from a staging buffer: the jobs are generated on
    the device in segments, each copied into `buf` (a uint32 tensor: pinned
    host memory, or device memory) while the server is idle and outside the
    timed region, until the next job would not fit; then the segment's jobs
    are submitted as borrowed slices of `buf` (all at once, or at their
    arrival offsets in seconds, restarted at each segment), so that each
    job's latency includes the server's copy of its edges from `buf`.  Only
    the serving is timed: the makespan is the sum over segments of (last
    completion - segment start).  Totals only.  Returns (totals, latencies
    s, makespan s, stats, raw edges, client dict: submissions later than
    1 ms past their arrival, segments, staging seconds, seconds in submit
    calls).  `inflight`: the server's batch threads (BATCHED mode), so that
    one batch's copy and graph build overlap another's counting."""
    import queue
    import threading

    import torch
    from paper_2209_04541_b300 import pgabb as P
    import collections

    cap = int(buf.numel())
    stream = stream or torch.cuda.Stream()
    copy_stream = torch.cuda.Stream()
    srv = P.pgb_server_create(P.pgb_server_opts_default(mode=mode, per_vertex=0, max_inflight=inflight))
    totals, lats = [0] * count, [0.0] * count
    span = 0.0
    raw = late = segments = 0
    t_stage = t_sub = 0.0
    carry = None
    pending = []
    th = q = None
    try:
        k = 0
        while k < count:
            ts = time.perf_counter()
            seg, pos = [], 0
            flight, flight_edges = collections.deque(), 0  # copies not yet known to be done
            while k + len(seg) < count:
                s, d, n = carry if carry is not None else serve_job_device(k + len(seg), max_scale, stream)
                carry = None
                m = int(s.numel())
                if pos + 2 * m > cap:
                    if not seg:
                        raise ValueError(f"job {k} ({m} raw edges) does not fit the staging buffer of {cap} words")
                    carry = (s, d, n)
                    break
                # the copy overlaps the next job's generation; at most 2^28
                # raw edges of generated arrays wait for their copies
                copy_stream.wait_stream(stream)
                with torch.cuda.stream(copy_stream):
                    buf[pos:pos + m].copy_(s, non_blocking=True)
                    buf[pos + m:pos + 2 * m].copy_(d, non_blocking=True)
                s.record_stream(copy_stream)
                d.record_stream(copy_stream)
                ev = torch.cuda.Event()
                ev.record(copy_stream)
                flight.append((ev, m))
                flight_edges += m
                while flight_edges > 1 << 28:
                    e, mm = flight.popleft()
                    e.synchronize()
                    flight_edges -= mm
                seg.append((pos, m, n))
                pos += 2 * m
                del s, d
            copy_stream.synchronize()
            stream.synchronize()
            t_stage += time.perf_counter() - ts
            q = queue.Queue()
            err = []

            def waiter(todo=len(seg)):
                try:
                    for _ in range(todo):
                        j, jid = q.get()
                        if jid is None:
                            return
                        totals[j], _, lats[j] = P.pgb_server_wait(srv, jid, 900.0)
                except BaseException as exc:  # handed to the caller
                    err.append(exc)

            th = threading.Thread(target=waiter, daemon=True)
            th.start()
            base = arrivals[k - 1] if arrivals is not None and k else 0.0
            subs = []
            t0 = time.perf_counter()
            for o, (pos, m, n) in enumerate(seg):
                if err:
                    break
                if arrivals is not None:
                    due = t0 + arrivals[k + o] - base
                    delay = due - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                tsub = time.perf_counter()
                if arrivals is not None and tsub - due > 1e-3:
                    late += 1
                jid = P.pgb_server_submit(srv, buf[pos:pos + m], buf[pos + m:pos + 2 * m], n, borrow=True)
                t_sub += time.perf_counter() - tsub
                subs.append(tsub)
                pending.append(jid)
                q.put((k + o, jid))
            th.join()
            th = None
            if err:
                raise err[0]
            pending.clear()
            span += max(subs[o] + lats[k + o] for o in range(len(seg))) - t0
            raw += sum(m for _, m, _ in seg)
            k += len(seg)
            segments += 1
        stats = P.pgb_server_stats(srv)
    finally:
        if th is not None:  # an error while submitting: let the waiter return before the server goes
            for jid in pending:
                try:
                    P.pgb_server_cancel(srv, jid)
                except Exception:
                    pass
            q.put((None, None))
            th.join()
        P.pgb_server_destroy(srv)
    client = {"late_submissions": late, "segments": segments, "staging_s": round(t_stage, 3),
              "submit_s": round(t_sub, 3)}
    return totals, lats, span, stats, raw, client


def serve_bench_device(args):
    """The serving workload at its stated size (R-MAT scales up to 22, ER and
    RGG n up to 2^22).  The whole mix (tens of G raw edges) fits neither host
    nor device memory, so it is served in segments: each segment's jobs are
    made on the device and staged (untimed, server idle) in pinned host
    memory (by default; each job's host-to-device copy is then inside its
    latency) or in device memory, then served (timed).  Capacity (closed
    loop) and Poisson loads at the given fractions of the one-at-a-time
    capacity (0.8 by default), for both modes; totals only."""
    import torch
    from paper_2209_04541_b300 import pgabb as P
    J, S = args.serve_jobs, args.serve_max_scale
    loads = [float(x) for x in args.serve_loads.split(",")]
    words = args.serve_stage_words
    if args.serve_input == "host":
        buf = torch.empty(words, dtype=torch.uint32, pin_memory=True)
    else:
        buf = torch.empty(words, dtype=torch.uint32, device="cuda")
    k = args.serve_inflight
    run = lambda mode, arrivals=None: run_serve_staged(J, S, mode, arrivals, buf, inflight=k)  # noqa: E731
    run_serve_staged(24, S, P.PGB_SERVE_BATCHED, None, buf, inflight=k)  # warm-up
    tot_s, _, span_s, _, raw, cl_s = run(P.PGB_SERVE_SERIAL)
    tot_b, _, span_b, st_b, _, cl_b = run(P.PGB_SERVE_BATCHED)
    assert tot_s == tot_b, "serial and batched counts differ"
    cap_s, cap_b = J / span_s, J / span_b
    sweep = {}
    for factor in loads:
        rate = factor * cap_s
        rng = np.random.default_rng(12345)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=J))
        res = {}
        for name, mode in (("serial", P.PGB_SERVE_SERIAL), ("batched", P.PGB_SERVE_BATCHED)):
            tot, lat, span, st, _, client = run(mode, arrivals)
            assert tot == tot_s
            lat_ms = np.array(lat) * 1e3
            res[name] = {"jobs_s": J / span, "p50_ms": float(np.percentile(lat_ms, 50)),
                         "p99_ms": float(np.percentile(lat_ms, 99)), "launches": st["batches"],
                         "client": client}
        sweep[f"{factor:.2f}"] = {"rate_jobs_s": rate, **res}
    del buf
    torch.cuda.empty_cache()
    head = sweep.get("0.80") or sweep[f"{loads[0]:.2f}"]
    where = "pinned host memory" if args.serve_input == "host" else "device memory"
    out = {"metric": "serve jobs/s and p50/p99 latency", "jobs": J, "raw_edges": raw,
           "triangles": int(sum(tot_s)),
           "mix": f"thirds of R-MAT (scale 10-{S}, ef 8-32, Feistel relabelling), ER (n 2^10-2^{S} log-uniform, "
                  "avg degree 4-64 log-uniform), RGG (avg degree 6); seed = job index; made on the device in "
                  f"segments of up to {words} words, staged in {where} while the server is idle (untimed), "
                  "then submitted from there as borrowed arrays (the server's copy inside each job's "
                  "latency); makespan = sum of the segments' serving times; totals only",
           "inputs": args.serve_input,
           "batched_threads": k,
           "capacity_jobs_s": {"serial": cap_s, "batched": cap_b},
           "capacity_edges_s": {"serial": raw / span_s, "batched": raw / span_b},
           "capacity_client": {"serial": cl_s, "batched": cl_b},
           "poisson_rate_jobs_s": head["rate_jobs_s"],
           "poisson": {k: head[k] for k in ("serial", "batched")},
           "batched_launches_closed_loop": st_b["batches"]}
    if len(sweep) > 1:
        out["poisson_sweep_by_fraction_of_serial_capacity"] = sweep
    return out


def serve_summary(serve):
    """The serve figures that matter, compact, for the end of the line."""
    if not serve or "error" in serve:
        return serve
    p = serve["poisson"]
    return {"jobs": serve["jobs"], "capacity_jobs_s": serve["capacity_jobs_s"],
            "at_0.8x_serial_capacity": {k: {"jobs_s": round(p[k]["jobs_s"], 1), "p50_ms": round(p[k]["p50_ms"], 2),
                                            "p99_ms": round(p[k]["p99_ms"], 2)} for k in ("serial", "batched")}}


def h2d_gbs(torch, nbytes=1 << 30, reps=5):
    """Pinned host-to-device copy bandwidth of this GPU's host link."""
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d.copy_(h, non_blocking=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        d.copy_(h, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    return nbytes * reps / (e0.elapsed_time(e1) / 1e3) / 1e9


def bsp_rows(P, torch, b, info, n, stream, reps=3):
    """Single-block bulk-synchronous kernels on the same partition:
    Shiloach-Vishkin components (hook rounds until none hooks) and PageRank
    (the paper's damping 0.85, tolerance 1e-4, at most 20 iterations),
    outputs in device tensors, wall time per call (each call synchronises)."""
    m = info["m"]
    lab = torch.zeros(n, dtype=torch.uint32, device="cuda")
    ranks = torch.zeros(n, dtype=torch.float64, device="cuda")
    cc, pr = [], []
    for i in range(1 + reps):
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, it_cc, comps = P.pgb_cc_run(b, labels=lab, stream=stream)
        t1 = time.perf_counter()
        _, it_pr, err = P.pgb_pagerank_run(b, ranks=ranks, stream=stream)
        t2 = time.perf_counter()
        if i:
            cc.append(t1 - t)
            pr.append(t2 - t1)
    cc_s, pr_s = statistics.median(cc), statistics.median(pr)
    # PageRank bytes per iteration: offsets and both neighbour lists once,
    # one 8-byte rank/degree read per neighbour entry, two 8-byte writes per
    # vertex (the reads are random: a bound, not the traffic)
    pr_bytes = 16 * (n + 1) + 8 * m + 16 * m + 16 * n
    return {"cc": {"wall_ms": 1e3 * cc_s, "hook_rounds": it_cc, "components": comps,
                   "edges_s_per_round": m * it_cc / cc_s},
            "pagerank": {"wall_ms": 1e3 * pr_s, "iterations": it_pr, "last_l1_change": err,
                         "ms_per_iteration": 1e3 * pr_s / max(it_pr, 1),
                         "bytes_per_iteration": pr_bytes,
                         "achieved_gbs": pr_bytes * it_pr / pr_s / 1e9}}


def tiers_bench(args):
    """The runtime tiers on one partition each of R-MAT s24 and the grid
    (count phase only, the partition built once): launch per block triple
    versus the persistent autotuned kernel, each with and without CUDA-graph
    replay, and the hybrid scheduler (host threads on the lightest parts) at
    three cut-offs.  Per-vertex counts on, written to a device tensor."""
    import torch
    from paper_2209_04541_b300 import pgabb as P
    out = {}
    for name in args.tiers_workloads.split(","):
        w = dict(WORKLOADS[name])
        s_np, d_np, n = generate(w)
        stream = torch.cuda.current_stream()
        g = P.pgb_graph_from_edges(torch.from_numpy(s_np).cuda(), torch.from_numpy(d_np).cuda(), n, stream)
        del s_np, d_np
        b = P.pgb_partition(g, w["p"], P.PGB_CUT_NNZ, stream)
        g.free()
        info = P.pgb_blocks_info(b)
        tv = torch.zeros(n, dtype=torch.uint64, device="cuda")
        rows = {}
        T0 = None
        settings = [("plain", dict(mode=P.PGB_MODE_PLAIN)),
                    ("plain+graph", dict(mode=P.PGB_MODE_PLAIN, use_graph=1)),
                    ("persistent-auto", dict()),
                    ("persistent-auto+graph", dict(use_graph=1))]
        # HYBRID (host kernel on the lightest parts, under a cut-off share of
        # the estimated work), beside the GPU-only rows, never instead of them
        settings += [(f"hybrid-{ppm / 1e4:g}%", dict(mode=P.PGB_MODE_HYBRID, host_share_ppm=ppm))
                     for ppm in (100, 1000, 10000)]
        for label, kw in settings:
            o = P.pgb_tc_opts_default(**kw)
            walls, kms, hms = [], [], []
            for i in range(2 + args.tiers_steps):
                torch.cuda.synchronize()
                t = time.perf_counter()
                r = P.pgb_tc_run(b, o, stream)
                T, _ = P.pgb_tc_result_get(r, per_vertex=tv)
                wall = time.perf_counter() - t
                if i >= 2:
                    walls.append(wall)
                    kms.append(P.pgb_tc_result_kernel_ms(r))
                    hms.append(P.pgb_tc_result_hybrid(r))
                var = P.pgb_tc_result_variant(r)
                r.free()
                T0 = T if T0 is None else T0
                assert T == T0, "tiers disagree"
            wall = statistics.median(walls)
            rows[label] = {"edges_s": info["m"] / wall, "wall_ms": 1e3 * wall,
                           "device_ms": statistics.median(kms),
                           "kernel": "k_tc_hash" if var == P.PGB_VAR_HASH else
                                     ("k_tc_tuple" if "plain" in label else
                                      ("k_tc_hash+k_tc_persistent" if var == P.PGB_VAR_MIXED else "k_tc_persistent"))}
            if label.startswith("hybrid"):
                rows[label].update({"host_ms": statistics.median(h["host_ms"] for h in hms),
                                    "host_parts": hms[-1]["host_parts"], "host_threads": hms[-1]["host_threads"],
                                    "host_in_edges": hms[-1]["host_in_edges"]})
        bsp = bsp_rows(P, torch, b, info, n, stream)
        b.free()
        del tv
        torch.cuda.empty_cache()
        out[name] = {"workload": w["desc"], "unique_edges": info["m"], "triples": info["triples"],
                     "triangles": T0, "tiers": rows, "bsp": bsp}
    return {"metric": "count-phase edges/s by runtime tier", "steps": args.tiers_steps,
            "note": "device_ms: CUDA events around the counting launches (a replayed graph: the whole graph)",
            "workloads": out}


def autotune_bench(args):
    """Per-part autotuning on a graph whose parts disagree: the count phase
    (partition built once) with the per-part choice (AUTO), with the hash
    kernel for every part, and with the edge-wise kernel for every part.
    Per-vertex counts on, written to a device tensor; counts must agree."""
    import torch
    from paper_2209_04541_b300 import pgabb as P
    w = dict(WORKLOADS[args.autotune_workload])
    s_np, d_np, n = generate(w)
    stream = torch.cuda.current_stream()
    g = P.pgb_graph_from_edges(torch.from_numpy(s_np).cuda(), torch.from_numpy(d_np).cuda(), n, stream)
    del s_np, d_np
    b = P.pgb_partition(g, w["p"], P.PGB_CUT_NNZ, stream)
    g.free()
    info = P.pgb_blocks_info(b)
    tv = torch.zeros(n, dtype=torch.uint64, device="cuda")
    rows, T0 = {}, None
    names = {P.PGB_VAR_HASH: "hash", P.PGB_VAR_BSEARCH: "bsearch", P.PGB_VAR_MIXED: "mixed"}
    for label, var in (("auto", P.PGB_VAR_AUTO), ("hash", P.PGB_VAR_HASH), ("bsearch", P.PGB_VAR_BSEARCH)):
        o = P.pgb_tc_opts_default(variant=var)
        kms = []
        for i in range(2 + args.tiers_steps):
            r = P.pgb_tc_run(b, o, stream)
            T, _ = P.pgb_tc_result_get(r, per_vertex=tv)
            if i >= 2:
                kms.append(P.pgb_tc_result_kernel_ms(r))
            used = P.pgb_tc_result_variant(r)
            parts = P.pgb_tc_result_part_variants(r)
            r.free()
            T0 = T if T0 is None else T0
            assert T == T0, "variants disagree"
        rows[label] = {"kernel_ms": statistics.median(kms), "edges_s": info["m"] / (statistics.median(kms) / 1e3),
                       "variant_used": names.get(used, used),
                       "hash_parts": int((parts == P.PGB_VAR_HASH).sum()), "parts": int(len(parts))}
    b.free()
    del tv
    torch.cuda.empty_cache()
    best_single = min(rows["hash"]["kernel_ms"], rows["bsearch"]["kernel_ms"])
    return {"metric": "count-phase kernel ms by variant choice", "workload": w["desc"], "unique_edges": info["m"],
            "triangles": T0, "lookups_per_edge": info["probes"] / max(info["m"], 1), "choices": rows,
            "auto_vs_best_single_choice": best_single / rows["auto"]["kernel_ms"]}


def pattern_bench(args):
    """The other multi-block patterns on one partition: 4-cliques and 4-cycles
    (wall time per call, each call synchronises), counts equal across
    repeats."""
    import torch
    from paper_2209_04541_b300 import pgabb as P
    w = dict(WORKLOADS[args.pattern_workload])
    s_np, d_np, n = generate(w)
    stream = torch.cuda.current_stream()
    g = P.pgb_graph_from_edges(torch.from_numpy(s_np).cuda(), torch.from_numpy(d_np).cuda(), n, stream)
    del s_np, d_np
    b = P.pgb_partition(g, w["p"], P.PGB_CUT_NNZ, stream)
    g.free()
    info = P.pgb_blocks_info(b)
    out = {"workload": w["desc"], "unique_edges": info["m"]}
    for name, fn in (("k4", P.pgb_k4_count), ("c4", P.pgb_c4_count)):
        times, vals = [], set()
        for i in range(3):
            torch.cuda.synchronize()
            t = time.perf_counter()
            vals.add(fn(b, stream))
            if i:
                times.append(time.perf_counter() - t)
        assert len(vals) == 1, f"{name} counts differ between calls"
        wall = statistics.median(times)
        out[name] = {"count": vals.pop(), "wall_ms": 1e3 * wall, "edges_s": info["m"] / wall}
    b.free()
    torch.cuda.empty_cache()
    return out


def stream_bench(args):
    """The streaming tiers against the same graph fully resident: the in-edge
    index in pinned host memory (budget --stream-budget-gb), and the block
    cache with the columns offloaded too (budget --cache-budget-gb)."""
    import torch
    from paper_2209_04541_b300 import pgabb as P
    w = dict(WORKLOADS[args.stream_workload])
    mraw = raw_edge_count(w)
    hs = torch.empty(mraw, dtype=torch.uint32, pin_memory=True)
    hd = torch.empty(mraw, dtype=torch.uint32, pin_memory=True)
    _, _, n_raw = generate(w, out=(hs.numpy(), hd.numpy()))

    def build():
        stream = torch.cuda.current_stream()
        t0 = time.perf_counter()
        g = P.pgb_graph_from_edges(hs.cuda(), hd.cuda(), n_raw, stream)
        b = P.pgb_partition(g, w["p"], P.PGB_CUT_NNZ, stream)
        g.free()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        return b, n_raw, time.perf_counter() - t0

    def timed(b, opts, reps):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t = time.perf_counter()
            r = P.pgb_tc_run(b, opts)
            T, tv = P.pgb_tc_result_get(r, per_vertex=True)
            wall = time.perf_counter() - t
            out.append((T, tv, wall, P.pgb_tc_result_kernel_ms(r), P.pgb_tc_result_stream(r, slice_loads=True),
                        P.pgb_tc_result_dense_core(r)["ranks"]))
            r.free()
        return out

    reps = max(3, args.stream_steps)
    b, n, prep_s = build()
    info = P.pgb_blocks_info(b)
    m = info["m"]
    res = timed(b, P.pgb_tc_opts_default(), 1 + reps)[1:]
    T, tv_res = res[0][0], res[0][1]
    assert int(tv_res.sum(dtype=np.uint64)) == 3 * T
    link = h2d_gbs(torch)

    def summary(runs, budget, floor):
        for x in runs:
            assert x[0] == T and np.array_equal(x[1], tv_res), "streamed counts differ from resident counts"
        kms = statistics.median(x[3] for x in runs)
        wall = statistics.median(x[2] for x in runs)
        nbytes, chunks, loads = runs[0][4]
        return {"device_budget_bytes": budget, "resident_floor_bytes": floor, "chunks": chunks,
                "slice_loads": loads, "streamed_bytes": nbytes, "value": m / wall, "unit": "edges/s",
                "wall_ms": 1e3 * wall, "kernel_ms": kms, "link_gbs": nbytes / (kms / 1e3) / 1e9,
                "link_frac": nbytes / (kms / 1e3) / 1e9 / link, "dense_core_ranks": runs[0][5]}

    out = {"metric": "streamed TC edges/s", "workload": w["desc"], "n": n, "unique_edges": m, "triangles": T,
           "resident_graph_bytes": 4 * m + 12 * m + 4 * m + 12 * (n + 1), "steps": reps, "preprocess_s": prep_s,
           "h2d_peak_gbs": link,
           "resident": {"value": m / statistics.median(x[2] for x in res), "unit": "edges/s",
                        "wall_ms": 1e3 * statistics.median(x[2] for x in res),
                        "kernel_ms": statistics.median(x[3] for x in res), "dense_core_ranks": res[0][5]},
           "check": "streamed totals and per-vertex counts equal the resident run's; sum t = 3T"}
    # tier 1: the in-edge index streamed, columns resident
    budget = int(args.stream_budget_gb * (1 << 30))
    P.pgb_blocks_offload(b)
    out["index"] = summary(timed(b, P.pgb_tc_opts_default(device_budget=budget), 1 + reps)[1:], budget,
                           P.pgb_blocks_resident_bytes(b, True))
    b.free()
    torch.cuda.empty_cache()
    # tier 2: the block cache (columns offloaded too), from a fresh partition
    if args.cache_budget_gb > 0:
        b, _, _ = build()
        budget = int(args.cache_budget_gb * (1 << 30))
        # row ranges sized so that about five slices fit the budget beside the
        # resident arrays (24 bytes per vertex) and the piece slots
        avail = budget - 24 * n - (128 << 20)
        slices = info["p"] if avail <= 0 else min(info["p"], max(2, -(-20 * m // avail)))
        t0 = time.perf_counter()
        P.pgb_blocks_offload_columns(b, slices)
        off_s = time.perf_counter() - t0
        torch.cuda.empty_cache()
        two = P.pgb_blocks_cache_budget(b, 2)
        if budget < two:
            out["cache"] = {"error": f"budget below two slices ({two} bytes)"}
        else:
            c = summary(timed(b, P.pgb_tc_opts_default(device_budget=budget), 1 + reps)[1:], budget,
                        P.pgb_blocks_resident_bytes(b, True))
            c["offload_s"] = off_s
            c["slices"] = slices
            c["slices_in_cache"] = sum(1 for k in range(1, slices + 1)
                                       if P.pgb_blocks_cache_budget(b, k) <= budget)
            out["cache"] = c
        b.free()
        torch.cuda.empty_cache()
    del hs, hd
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rmat24")
    ap.add_argument("--mode", choices=["persistent", "plain"], default="persistent")
    ap.add_argument("--order", choices=["weight", "locality"], default="weight")
    ap.add_argument("--variant", choices=["auto", "bsearch", "merge", "hash"], default="auto")
    ap.add_argument("--chunk", type=int, default=0,
                    help="pgb_tc_opts.chunk_edges: edges per chunk of the binary-search kernel AND in-edges per item "
                         "of the hash kernel (0 = each kernel's own default)")
    ap.add_argument("--per-vertex", type=int, default=1)
    ap.add_argument("--hash-threads", type=int, default=0, choices=[0, 128, 256, 512],
                    help="CTA shape of the hash kernel (0 = autotuned)")
    ap.add_argument("--p", type=int, default=0, help="override the workload's p")
    ap.add_argument("--dense-core", type=int, default=0,
                    help="dense top block of the degree order: 0 autotuned, -1 none, K > 0 that many ranks")
    ap.add_argument("--hash-min-lookups", type=int, default=0,
                    help="per-part autotuner threshold, lookups per edge (0 = the library's 32)")
    ap.add_argument("--clock-interval-ms", type=int, default=200,
                    help="nvidia-smi sampling interval during the timed steps (each sample briefly holds the driver)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-jobs", type=int, default=10000)
    ap.add_argument("--serve-mix", choices=["full", "small"], default="full",
                    help="full: the serving mix at its stated size (scales up to 22, jobs made on the device in "
                         "segments, staged (see --serve-input), totals only); small: host-generated "
                         "jobs up to scale 16, submitted from host memory, per-vertex counts on")
    ap.add_argument("--serve-input", choices=["host", "device"], default="host",
                    help="full mix: where the jobs are staged before they are submitted: pinned host memory "
                         "(each job's host-to-device copy inside its latency) or device memory")
    ap.add_argument("--serve-stage-words", type=int, default=1 << 33,
                    help="full mix: staging buffer in uint32 words (2 per raw edge; a segment is the jobs that "
                         "fit)")
    ap.add_argument("--serve-inflight", type=int, default=6,
                    help="full mix: the server's batch threads in BATCHED mode")
    ap.add_argument("--serve-loads", default="0.8",
                    help="full mix: comma-separated Poisson loads, as fractions of the one-at-a-time capacity")
    ap.add_argument("--serve-max-scale", type=int, default=0,
                    help="largest R-MAT scale and log2 n of the mix (0: 22 for the full mix, 16 for the small one)")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-tiers", action="store_true")
    ap.add_argument("--tiers-workloads", default="rmat24,grid4096")
    ap.add_argument("--tiers-steps", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-patterns", action="store_true")
    ap.add_argument("--pattern-workload", choices=sorted(WORKLOADS), default="rmat20")
    ap.add_argument("--autotune-workload", choices=sorted(WORKLOADS), default="grid4096_u_rmat22")
    ap.add_argument("--stream-workload", choices=["rmat24", "rmat22", "rmat27"], default="rmat27",
                    help="streamed graph (default: R-MAT s27, p=64, the out-of-core configuration)")
    ap.add_argument("--stream-budget-gb", type=float, default=16.0, help="index tier device budget")
    ap.add_argument("--stream-steps", type=int, default=3)
    ap.add_argument("--cache-budget-gb", type=float, default=4.0,
                    help="block cache tier budget (0 = skip the tier)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.serve_jobs < 1 or args.serve_inflight < 1 or args.serve_stage_words < 2:
        ap.error("--serve-jobs and --serve-inflight must be >= 1, --serve-stage-words >= 2")
    try:
        loads = [float(x) for x in args.serve_loads.split(",")]
    except ValueError:
        loads = []
    if not loads or not all(0.0 < x < 10.0 for x in loads):
        ap.error("--serve-loads takes comma-separated positive fractions, e.g. 0.5,0.8,0.95")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2209_04541_b300 import pgabb as P

    wall = {}  # seconds of wall clock per section of this run
    t_sec = time.perf_counter()
    w = dict(WORKLOADS[args.workload])
    if args.p:
        w["p"] = args.p
    mraw = raw_edge_count(w)
    if mraw is not None:
        hs = torch.empty(mraw, dtype=torch.uint32, pin_memory=True)
        hd = torch.empty(mraw, dtype=torch.uint32, pin_memory=True)
        _, _, n = generate(w, out=(hs.numpy(), hd.numpy()))
    else:
        s_np, d_np, n = generate(w)
        hs = torch.from_numpy(s_np).pin_memory()
        hd = torch.from_numpy(d_np).pin_memory()
    mraw = hs.numel()
    stream = torch.cuda.current_stream()
    ds, dd = hs.cuda(non_blocking=True), hd.cuda(non_blocking=True)
    tv = torch.zeros(n, dtype=torch.uint64, device="cuda")
    P.load()
    mode = P.PGB_MODE_PERSISTENT if args.mode == "persistent" else P.PGB_MODE_PLAIN
    variant = {"auto": P.PGB_VAR_AUTO, "bsearch": P.PGB_VAR_BSEARCH, "merge": P.PGB_VAR_MERGE,
               "hash": P.PGB_VAR_HASH}[args.variant]
    opts = P.pgb_tc_opts_default(mode=mode, per_vertex=args.per_vertex, chunk_edges=args.chunk, variant=variant,
                                 hash_threads=args.hash_threads, hash_min_lookups=args.hash_min_lookups,
                                 dense_core=args.dense_core,
                                 order=P.PGB_ORDER_WEIGHT if args.order == "weight" else P.PGB_ORDER_LOCALITY)
    info = {}
    dense_ms = []

    def step():
        g = P.pgb_graph_from_edges(ds, dd, n, stream)
        b = P.pgb_partition(g, w["p"], P.PGB_CUT_NNZ, stream)
        g.free()
        r = P.pgb_tc_run(b, opts, stream)
        T, _ = P.pgb_tc_result_get(r, per_vertex=tv if args.per_vertex else None)
        kms = P.pgb_tc_result_kernel_ms(r)
        dc = P.pgb_tc_result_dense_core(r)
        dense_ms.append(dc["ms"] if dc["ranks"] else 0.0)
        if not info:
            info["dense"] = dc
            info.update(P.pgb_blocks_info(b))
            info["variant_used"] = P.pgb_tc_result_variant(r)
            pv_ = P.pgb_tc_result_part_variants(r)
            info["parts_by_kernel"] = {"hash": int((pv_ == P.PGB_VAR_HASH).sum()),
                                       "edgewise": int(((pv_ == P.PGB_VAR_BSEARCH) | (pv_ == P.PGB_VAR_MERGE)).sum())}
            # sum_u outdeg(u)^2 from the oriented offsets (first warm-up step only)
            outdeg = np.diff(P.pgb_blocks_export(b, P.PGB_EXPORT_ROWPTR)).astype(np.uint64)
            info["sum_outdeg_sq"] = int((outdeg * outdeg).sum())
        r.free()
        b.free()
        return T, kms

    for _ in range(args.warmup):
        T, _ = step()
    torch.cuda.synchronize()
    if dist.is_initialized():
        dist.barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid, args.clock_interval_ms)
    sampler.start()
    l0 = P.pgb_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kms_all = []
    dense_ms.clear()
    e0.record(stream)
    for _ in range(args.steps):
        T2, kms = step()
        kms_all.append(kms)
        assert T2 == T, "counts differ between steps"
    e1.record(stream)
    torch.cuda.synchronize()
    launches = P.pgb_kernel_launches() - l0
    clocks = sampler.stop()
    if dist.is_initialized():
        dist.barrier()
    torch.cuda.synchronize()
    ms_local = e0.elapsed_time(e1) / args.steps
    m_u = info["m"]
    ms, units = aggregate(ms_local, float(m_u), dist)
    value = units / (ms / 1e3)

    kernel_ms = statistics.mean(kms_all)
    peak, peak_note = measured_peaks()
    if mode == P.PGB_MODE_PLAIN:
        kname = "k_tc_tuple"
    elif info["variant_used"] == P.PGB_VAR_HASH:
        kname = "k_tc_hash"
    elif info["variant_used"] == P.PGB_VAR_MIXED:
        # per-part choice: the hash kernel counts most parts (by lookups),
        # the edge-wise kernel the flat ones; kernel_ms covers both launches
        kname = "k_tc_hash"
    else:
        kname = "k_tc_persistent"
    dense = info["dense"]
    dense_mean = statistics.mean(dense_ms) if dense["ranks"] else 0.0
    # the intersection kernels' own time: the count phase less the dense block's
    sparse_ms = kernel_ms - dense_mean
    ew_achieved = info["alg_bytes"] / (kernel_ms / 1e3) / 1e9
    if kname == "k_tc_hash":
        # bytes this kernel must stream: every looked-up entry of the tails'
        # rows (4 per probe; less the lookups left to the dense block), one
        # 8-byte in-edge descriptor per edge, and each head's list (4 per edge)
        kb = 4 * (info["probes"] - dense["lookups_skipped"]) + 12 * info["m"]
        bytes_rule = "4 (probes - dense-block lookups) + 12|E+| (looked-up tail-row entries, in-edge index, head lists)"
    else:
        kb = info["alg_bytes"]
        bytes_rule = "4|E+| + 4 sum_v indeg(v) outdeg(v) + 8(n+1)"
    achieved = kb / (sparse_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_note, "alg_bytes": kb, "alg_bytes_rule": bytes_rule,
                "kernel_ms": sparse_ms, "count_phase_ms": kernel_ms,
                "traffic": kernel_traffic(kname, args.workload)}
    if dense["ranks"]:
        tf_peak = measured_tensor_peak()
        tflops = dense["gemm_flop"] / (dense_mean / 1e3) / 1e12
        roofline["dense_block"] = {
            "bound": "tensor", "ranks": dense["ranks"], "triangles": dense["triangles"],
            "lookups_taken_from_kernels": dense["lookups_skipped"], "ms": dense_mean,
            "achieved": tflops, "unit": "TFLOP/s", "peak": tf_peak[0], "peak_source": tf_peak[1],
            "frac": tflops / tf_peak[0] if tf_peak[0] else None,
            "note": "fp16 0/1 GEMM strips of the top block (fp16 rate = bf16 rate), fill and masked reduction "
                    "inside the timed ms"}
    if kname == "k_tc_hash":
        roofline["edgewise_bound"] = {
            "note": "4|E+| + 4 sum_v indeg(v) outdeg(v) + 8(n+1): the edge-wise method's bytes, which re-read "
                    "v's list per in-edge; this kernel holds that list in shared memory, so this is not a "
                    "bandwidth fraction",
            "alg_bytes": info["alg_bytes"], "achieved": ew_achieved, "ratio_to_peak": ew_achieved / peak}
        # the per-edge merge's bytes: both partial lists read for every
        # oriented edge (u, v), 4 sum_u outdeg(u)^2 + 4 sum_v indeg(v) outdeg(v)
        mb = 4 * (info["sum_outdeg_sq"] + info["wedges"])
        roofline["merge_bytes"] = {
            "note": "4 sum over oriented edges (u,v) of (outdeg(u) + outdeg(v)): both lists read per edge, as a "
                    "merge would; not a bandwidth fraction for this kernel",
            "bytes": mb, "achieved": mb / (kernel_ms / 1e3) / 1e9, "ratio_to_peak": mb / (kernel_ms / 1e3) / 1e9 / peak}

    wall["headline"] = round(time.perf_counter() - t_sec, 1)
    t_sec = time.perf_counter()
    e2e = None
    if not args.no_e2e:
        hout = torch.zeros(n, dtype=torch.uint64, pin_memory=True)
        times = []
        for i in range(2 + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Te, _ = P.pgb_tc_count_edges(hs, hd, n, w["p"], P.PGB_CUT_NNZ, opts, stream,
                                         per_vertex=hout if args.per_vertex else None)
            t1 = time.perf_counter()
            assert Te == T
            if i >= 2:
                times.append(t1 - t0)
        e_ms, e_units = aggregate(1e3 * statistics.mean(times), float(m_u), dist)
        e2e = {"value": e_units / (e_ms / 1e3), "unit": "edges/s", "ms_per_step": e_ms,
               "h2d_bytes_per_step": 8 * mraw, "d2h_bytes_per_step": 8 + (8 * n if args.per_vertex else 0)}

    wall["e2e"] = round(time.perf_counter() - t_sec, 1)
    t_sec = time.perf_counter()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(hs.numpy(), hd.numpy(), n)
        except Exception as exc:  # reported, not hidden
            cpu = {"error": f"{type(exc).__name__}: {exc}"}

    wall["cpu_baseline"] = round(time.perf_counter() - t_sec, 1)
    t_sec = time.perf_counter()
    serve = None
    del ds, dd, tv
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_serve:
        try:
            if not args.serve_max_scale:
                args.serve_max_scale = 22 if args.serve_mix == "full" else 16
            if args.serve_mix == "full":
                serve = serve_bench_device(args)
            else:
                serve = serve_bench(args)
        except Exception as exc:  # reported, not hidden: the TC line stands on its own
            serve = {"error": f"{type(exc).__name__}: {exc}"}
    wall["serve"] = round(time.perf_counter() - t_sec, 1)
    t_sec = time.perf_counter()
    tiers = None
    if rank == 0 and not args.no_tiers:
        try:
            tiers = tiers_bench(args)
        except Exception as exc:  # reported, not hidden
            tiers = {"error": f"{type(exc).__name__}: {exc}"}
    wall["tiers"] = round(time.perf_counter() - t_sec, 1)
    t_sec = time.perf_counter()
    autotune = None
    if rank == 0 and not args.no_autotune:
        try:
            autotune = autotune_bench(args)
        except Exception as exc:  # reported, not hidden
            autotune = {"error": f"{type(exc).__name__}: {exc}"}
    wall["autotune"] = round(time.perf_counter() - t_sec, 1)
    t_sec = time.perf_counter()
    patterns = None
    if rank == 0 and not args.no_patterns:
        try:
            patterns = pattern_bench(args)
        except Exception as exc:  # reported, not hidden
            patterns = {"error": f"{type(exc).__name__}: {exc}"}
    wall["patterns"] = round(time.perf_counter() - t_sec, 1)
    t_sec = time.perf_counter()
    streamed = None
    if rank == 0 and not args.no_stream:
        try:
            streamed = stream_bench(args)
        except Exception as exc:  # reported, not hidden
            streamed = {"error": f"{type(exc).__name__}: {exc}"}

    wall["stream"] = round(time.perf_counter() - t_sec, 1)
    if rank == 0:
        line = {"metric": "TC edges/s", "value": value, "unit": "edges/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": w["desc"], "name": args.workload, "p": w["p"], "mode": args.mode,
                           "variant": args.variant, "kernel": kname,
                           "variant_used": {P.PGB_VAR_HASH: "hash", P.PGB_VAR_BSEARCH: "bsearch",
                                            P.PGB_VAR_MERGE: "merge", P.PGB_VAR_MIXED: "mixed (per part)"}.get(
                                                info["variant_used"], info["variant_used"]),
                           "parts_by_kernel": info["parts_by_kernel"],
                           "order": args.order, "per_vertex": bool(args.per_vertex), "n": n,
                           "raw_edges": mraw, "unique_edges": m_u, "triangles": T,
                           "wedges": info["wedges"], "probes": info["probes"], "triples": info["triples"],
                           "parallelism": f"replicas x{world}",
                           "l2": "inputs larger than L2 (raw edge list %.2f GB, oriented graph %.2f GB)"
                                 % (8 * mraw / 1e9, 8 * m_u / 1e9)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "gpu_launches_per_step": launches / args.steps,
                "clocks": clocks, "serve": serve, "tiers": tiers, "autotune": autotune, "patterns": patterns,
                "stream": streamed}
        line["serve_summary"] = serve_summary(serve)
        line["section_wall_s"] = wall
        print(json.dumps(line), flush=True)
    if dist.is_initialized():
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
