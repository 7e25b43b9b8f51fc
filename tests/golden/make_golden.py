#!/usr/bin/env python3
"""Write expected values for full-size parity tests, using only the oracle.

For each large synthetic workload this script generates the raw edge list
(seeded, ``graphgen``), cleans it and counts with the oracle (plain C):
- the exact triangle total T and the per-vertex counts t[x] of every vertex
  by the oracle's forward count (its OpenMP build, whose counts equal the
  single-threaded build's, a pinned property); t is stored as the SHA-256
  of its n uint64 values, little-endian, in original vertex ID order;
- t[x] for a seeded sample of vertices by the oracle's one-vertex count (the
  number of edges among the neighbours of x), an independent second route.
The sample holds the highest-degree vertices plus uniformly drawn ones.
Nothing here touches the CUDA library.

    python tests/golden/make_golden.py rmat20 rmat24 grid4096 rmat27

writes ``tests/golden/full_<name>.txt``.  ``serve22`` writes
``tests/golden/full_serve22_sample.txt``: for a sample of the serving workload at
scales up to 22 (``graphgen.serve_spec``; the largest job of each family
plus seeded random jobs) each job's T and the SHA-256 of its per-vertex
counts, by the same oracle count.
"""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = {
    "rmat20": dict(kind="rmat", scale=20, ef=16, seed=1),
    "rmat24": dict(kind="rmat", scale=24, ef=16, seed=1),
    # the one-vertex count on the hubs of scale 27 takes too long: its sample
    # holds vertices of degree >= 2 and degree-quantile vertices below the
    # top 0.01%
    "rmat27": dict(kind="rmat", scale=27, ef=16, seed=1, hub_sample=False),
    "grid4096": dict(kind="grid", side=4096, pct=1.0, seed=1),
}


def digest(t) -> str:
    """SHA-256 of per-vertex counts as n uint64 little-endian values."""
    return hashlib.sha256(np.ascontiguousarray(t, dtype="<u8").tobytes()).hexdigest()


def generate(w):
    if w["kind"] == "grid":
        return graphgen.grid_plus_percent(w["side"], w["pct"], w["seed"])
    return graphgen.rmat(w["scale"], w["ef"], w["seed"])


def describe(w):
    if w["kind"] == "grid":
        return [f"# {w['side']}x{w['side']} 4-neighbour grid + {w['pct']}% uniform random extra edges, "
                f"seed {w['seed']} (graphgen.grid_plus_percent).\n"]
    return [f"# R-MAT scale {w['scale']}, edge factor {w['ef']}, a,b,c = .57,.19,.19, seed {w['seed']},\n",
            "# seeded relabel (graphgen.rmat).\n"]
N_TOP = 8
N_RANDOM = 192


def make(name):
    w = WORKLOADS[name]
    t0 = time.time()
    src, dst, n = generate(w)
    g = oracle.clean(src, dst, n)
    del src, dst
    deg = g.degree()
    rng = np.random.default_rng(12345)
    if not w.get("hub_sample", True):
        order = np.argsort(deg, kind="stable")
        live = np.flatnonzero(deg >= 2)
        quant = order[(np.array([0.9, 0.99, 0.999, 0.9995, 0.9999]) * n).astype(np.int64)]
        xs = np.unique(np.concatenate([quant, rng.choice(live, size=N_RANDOM, replace=False)])).astype(np.uint32)
    else:
        top = np.argsort(-deg, kind="stable")[:N_TOP]
        rand = rng.choice(n, size=N_RANDOM, replace=False)
        xs = np.unique(np.concatenate([top, rand])).astype(np.uint32)
    tx = oracle.tc_vertex(g, xs)
    m = g.m
    o = oracle.orient(g)
    del g
    T, t = oracle.tc_forward_mt(o, per_vertex=True)
    del o
    assert np.array_equal(t[xs], tx), "forward count and one-vertex count disagree"
    assert int(t.sum(dtype=np.uint64)) == 3 * T
    path = os.path.join(HERE, f"full_{name}.txt")
    with open(path, "w") as f:
        for line in describe(w):
            f.write(line)
        f.write("# Values from the oracle only (tests/golden/make_golden.py): T = oracle forward count;\n")
        f.write("# t_sha256 = SHA-256 of all n per-vertex counts (uint64 little-endian, original IDs) from the\n")
        f.write("# same count; x lines: t[x] by the oracle's one-vertex count (the number of triangles\n")
        f.write("# containing x, PGAbB Section 3.6 definition).\n")
        f.write(f"n {n}\nm {m}\nT {T}\nt_sha256 {digest(t)}\n")
        for x, c in zip(xs.tolist(), tx.tolist()):
            f.write(f"x {x} {c}\n")
    print(f"{name}: n={n} m={m} T={T} sample={len(xs)} in {time.time() - t0:.0f} s -> {path}", flush=True)


def load(name):
    path = os.path.join(HERE, f"full_{name}.txt")
    out = {"x": [], "t": []}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tag, *rest = line.split()
            if tag == "x":
                out["x"].append(int(rest[0]))
                out["t"].append(int(rest[1]))
            elif tag == "t_sha256":
                out[tag] = rest[0]
            else:
                out[tag] = int(rest[0])
    out["x"] = np.array(out["x"], dtype=np.int64)
    out["t"] = np.array(out["t"], dtype=np.uint64)
    return out


SERVE_MAX_SCALE = 22
SERVE_JOBS = 10000
SERVE_RANDOM = 9


def serve_sample():
    """Job indices of the serving sample: the largest job of each family (by
    raw edges; RGG by n) among the first SERVE_JOBS, then seeded random ones."""
    specs = [graphgen.serve_spec(i, SERVE_MAX_SCALE) for i in range(SERVE_JOBS)]

    def size(sp):
        return sp[2] << sp[1] if sp[0] == "rmat" else (sp[2] if sp[0] == "er" else sp[1])

    big = [max((i for i, sp in enumerate(specs) if sp[0] == fam), key=lambda i: size(specs[i]))
           for fam in ("rmat", "er", "rgg")]
    rand = np.random.default_rng(2028).choice(SERVE_JOBS, size=SERVE_RANDOM, replace=False).tolist()
    return sorted(set(big + rand))


def make_serve():
    path = os.path.join(HERE, "full_serve22_sample.txt")
    lines = []
    for i in serve_sample():
        t0 = time.time()
        sp = graphgen.serve_spec(i, SERVE_MAX_SCALE)
        src, dst, n = graphgen.serve_job(i, SERVE_MAX_SCALE)
        raw = len(src)
        g = oracle.clean(src, dst, n)
        del src, dst
        m = g.m
        o = oracle.orient(g)
        del g
        T, t = oracle.tc_forward_mt(o, per_vertex=True)
        del o
        assert int(t.sum(dtype=np.uint64)) == 3 * T
        lines.append(f"job {i} {' '.join(map(str, sp))} n {n} raw {raw} m {m} T {T} t_sha256 {digest(t)}\n")
        print(lines[-1].strip(), f"({time.time() - t0:.0f} s)", flush=True)
    with open(path, "w") as f:
        f.write(f"# Sample of the serving workload at scales up to {SERVE_MAX_SCALE} (graphgen.serve_spec /\n")
        f.write("# graphgen.serve_job, job i seeded by i): the largest R-MAT, ER and RGG job among the first\n")
        f.write(f"# {SERVE_JOBS} plus {SERVE_RANDOM} seeded random jobs.  Values from the oracle only\n")
        f.write("# (tests/golden/make_golden.py serve22): T = oracle forward count of the cleaned graph;\n")
        f.write("# t_sha256 = SHA-256 of its n per-vertex counts (uint64 little-endian, original IDs).\n")
        for line in lines:
            f.write(line)
    print(f"-> {path}")


def load_serve():
    """[(job, spec tuple, n, raw, m, T, t_sha256)] from full_serve22_sample.txt."""
    out = []
    with open(os.path.join(HERE, "full_serve22_sample.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = line.split()
            k = w.index("n")
            spec = tuple([w[2]] + [int(x) for x in w[3:k]])
            kv = dict(zip(w[k::2], w[k + 1::2]))
            out.append((int(w[1]), spec, int(kv["n"]), int(kv["raw"]), int(kv["m"]), int(kv["T"]), kv["t_sha256"]))
    return out


if __name__ == "__main__":
    for name in sys.argv[1:] or ["rmat20"]:
        if name == "serve22":
            make_serve()
        else:
            make(name)
