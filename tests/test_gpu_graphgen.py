"""The device generators write the host generators' graphs edge for edge (same
arrays, same order): R-MAT under each relabelling, i.i.d. ER pairs and
random geometric graphs, from tiny and ragged sizes up to the largest jobs
of the serving workload at scale 22.  These are input plumbing; equality
with the host arrays is what lets oracle values of host-generated graphs
stand for device-generated ones."""
import numpy as np
import pytest

import graphgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from graphgen import device as gd  # noqa: E402


def same(host, dev):
    hs, hd, hn = host
    ds, dd, dn = dev
    assert hn == dn
    assert ds.numel() == len(hs) and dd.numel() == len(hd)
    assert torch.equal(ds, torch.from_numpy(hs).cuda()), "src differs"
    assert torch.equal(dd, torch.from_numpy(hd).cuda()), "dst differs"


@pytest.mark.parametrize("relabel", ["none", "shuffle", "feistel"])
@pytest.mark.parametrize("scale,ef,seed", [(1, 4, 2), (2, 3, 9), (5, 16, 1), (12, 8, 77), (17, 20, 5)])
def test_rmat_device_equals_host(scale, ef, seed, relabel):
    same(graphgen.rmat(scale, ef, seed, relabel=relabel), gd.rmat(scale, ef, seed, relabel=relabel))


@pytest.mark.parametrize("n,m,seed", [(1, 5, 1), (7, 0, 2), (1000, 12345, 3), ((1 << 20) + 7, 3_000_001, 4)])
def test_er_pairs_device_equals_host(n, m, seed):
    same(graphgen.er_pairs(n, m, seed), gd.er_pairs(n, m, seed))


@pytest.mark.parametrize("n,r,seed", [(1, None, 1), (2, 2.0, 1), (50, 0.3, 7), (1000, None, 2), (65537, None, 3),
                                      (300000, 0.004, 11), (1 << 20, None, 5)])
def test_rgg_device_equals_host(n, r, seed):
    same(graphgen.rgg(n, r, seed), gd.rgg(n, r, seed))


def test_rgg_device_on_a_side_stream():
    s = torch.cuda.Stream()
    dev = gd.rgg(20000, None, 9, stream=s)
    s.synchronize()
    same(graphgen.rgg(20000, None, 9), dev)


@pytest.mark.parametrize("job", [93, 5530, 6656])
def test_largest_serving_jobs_device_equal_host(job):
    """The largest R-MAT (scale 22, ef 32), ER and RGG jobs of the serving
    workload at scales up to 22."""
    same(graphgen.serve_job(job, 22), gd.serve_job(job, 22))
    torch.cuda.empty_cache()


def test_bench_rmat24_made_on_device_equals_host():
    """The benchmark's R-MAT s24 input, made by the device generator with
    the host's Fisher-Yates labels (bench.py does so from scale 16 up),
    equals the host generator's edge list."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    w = bench.WORKLOADS["rmat24"]
    hs, hd, n = graphgen.rmat(w["scale"], w["ef"], w["seed"])
    ds, dd, dn = bench.rmat_on_device(w)
    assert dn == n and np.array_equal(ds, hs) and np.array_equal(dd, hd)
