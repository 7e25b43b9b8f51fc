#!/usr/bin/env python3
"""Write expected values for full-size parity tests, using only the oracle.

For each large synthetic workload this script generates the raw edge list
(seeded, ``graphgen``), cleans it and counts with the oracle (plain C,
single-threaded): the exact triangle total by the oracle's forward count,
and t[x] for a seeded sample of vertices by the oracle's one-vertex count
(the number of edges among the neighbours of x).  The sample holds the
highest-degree vertices plus uniformly drawn ones.  Nothing here touches the
CUDA library.

    python tests/golden/make_golden.py rmat20 rmat24 rmat27

writes ``tests/golden/full_<name>.txt``.
"""
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
    "rmat20": dict(scale=20, ef=16, seed=1),
    "rmat24": dict(scale=24, ef=16, seed=1),
    # too large for the oracle's total (hours single-threaded) and for its
    # one-vertex count on the hubs: a sample of vertices of degree >= 2 and
    # of degree-quantile vertices below the top 0.01%
    "rmat27": dict(scale=27, ef=16, seed=1, sample_only=True),
}
N_TOP = 8
N_RANDOM = 192


def make(name):
    w = WORKLOADS[name]
    t0 = time.time()
    src, dst, n = graphgen.rmat(w["scale"], w["ef"], w["seed"])
    g = oracle.clean(src, dst, n)
    del src, dst
    deg = g.degree()
    rng = np.random.default_rng(12345)
    if w.get("sample_only"):
        T = None
        order = np.argsort(deg, kind="stable")
        live = np.flatnonzero(deg >= 2)
        quant = order[(np.array([0.9, 0.99, 0.999, 0.9995, 0.9999]) * n).astype(np.int64)]
        xs = np.unique(np.concatenate([quant, rng.choice(live, size=N_RANDOM, replace=False)])).astype(np.uint32)
    else:
        o = oracle.orient(g)
        T, _, _ = oracle.tc_forward(o, per_vertex=False)
        del o
        top = np.argsort(-deg, kind="stable")[:N_TOP]
        rand = rng.choice(n, size=N_RANDOM, replace=False)
        xs = np.unique(np.concatenate([top, rand])).astype(np.uint32)
    tx = oracle.tc_vertex(g, xs)
    path = os.path.join(HERE, f"full_{name}.txt")
    with open(path, "w") as f:
        f.write(f"# R-MAT scale {w['scale']}, edge factor {w['ef']}, a,b,c = .57,.19,.19, seed {w['seed']},\n")
        f.write("# seeded relabel (graphgen.rmat).  Values from the oracle only (tests/golden/make_golden.py):\n")
        f.write("# T (when present) = oracle forward count; t[x] = oracle one-vertex count for the listed x (the\n")
        f.write("# number of triangles containing x, PGAbB Section 3.6 definition).\n")
        f.write(f"n {n}\nm {g.m}\n")
        if T is not None:
            f.write(f"T {T}\n")
        for x, c in zip(xs.tolist(), tx.tolist()):
            f.write(f"x {x} {c}\n")
    print(f"{name}: n={n} m={g.m} T={T} sample={len(xs)} in {time.time() - t0:.0f} s -> {path}")


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
            else:
                out[tag] = int(rest[0])
    out["x"] = np.array(out["x"], dtype=np.int64)
    out["t"] = np.array(out["t"], dtype=np.uint64)
    return out


if __name__ == "__main__":
    for name in sys.argv[1:] or ["rmat20"]:
        make(name)
