"""Multi-rank host paths of bench.py on CPU (gloo, world size 2).

Under torchrun every rank runs an independent replica of the whole path (the
block tuples shard with no data exchange); bench.py then takes the slowest
rank's step time and the summed work of all ranks.  These tests run that
aggregation, and the reference arm's rank split, in two gloo processes."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank        # rank 1 is the slow one
    units_local = 1000.0 * (rank + 1)
    ms, units = bench.aggregate(ms_local, units_local, dist)
    dist.barrier()
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_aggregate_takes_max_time_and_sum_of_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in got:
        assert ms == 15.0
        assert units == 3000.0


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(7.0, 11.0, None) == (7.0, 11.0)


def test_reference_arm_runs_on_rank0_only(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "REF_SAMPLE", dict(kind="rmat", scale=10, ef=8, p=2, seed=1))
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    # rank 1 exits 0 without work or output
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--gpus", "2"], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == ""
    # rank 0 prints one JSON line describing the oracle arm
    args = type("A", (), dict(steps=1, warmup=3, gpus=2, workload="rmat24"))()
    import io
    import contextlib
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args, 0, 2) == 0
    line = json.loads(buf.getvalue().strip())
    assert line["impl"] == "reference" and line["unit"] == "edges/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.parametrize("bad", [["--warmup", "1"], ["--serve-jobs", "0"], ["--serve-inflight", "0"],
                                 ["--serve-loads", "0.8,x"], ["--serve-loads", "0"], ["--serve-stage-words", "1"]])
def test_bench_rejects_bad_arguments(bad):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference"] + bad,
                         capture_output=True, text=True, timeout=120)
    assert out.returncode != 0
