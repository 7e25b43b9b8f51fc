"""Test helpers: small hand-built graph families, golden-fixture loading and
brute-force counts.  No triangle-counting code from the library or the
oracle lives here; the brute force below is the definition itself (three
mutually adjacent vertices) evaluated over all vertex triples."""
from __future__ import annotations

import glob
import itertools
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(path):
    n, edges, T, t = None, [], None, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, *rest = line.split()
            if tag == "n":
                n = int(rest[0])
            elif tag == "e":
                edges.append((int(rest[0]), int(rest[1])))
            elif tag == "T":
                T = int(rest[0])
            elif tag == "t":
                t = np.array([int(x) for x in rest], dtype=np.uint64)
    src = np.array([a for a, _ in edges], dtype=np.uint32)
    dst = np.array([b for _, b in edges], dtype=np.uint32)
    return src, dst, n, T, t


def golden_files():
    """Small hand-derived fixtures (the oracle-written full-size files,
    ``full_*.txt``, have their own loader)."""
    return sorted(p for p in glob.glob(os.path.join(GOLDEN_DIR, "*.txt"))
                  if not os.path.basename(p).startswith("full_"))


def edges_to_arrays(edges):
    src = np.array([a for a, _ in edges], dtype=np.uint32)
    dst = np.array([b for _, b in edges], dtype=np.uint32)
    return src, dst


def complete(n):
    return [(a, b) for a in range(n) for b in range(a + 1, n)]


def cycle(n):
    return [(i, (i + 1) % n) for i in range(n)]


def wheel(n):
    """Hub 0 plus an (n-1)-cycle on 1..n-1."""
    rim = [(1 + i, 1 + (i + 1) % (n - 1)) for i in range(n - 1)]
    return rim + [(0, i) for i in range(1, n)]


def fan(k):
    """Hub 0 joined to every vertex of the path 1..k."""
    return [(i, i + 1) for i in range(1, k)] + [(0, i) for i in range(1, k + 1)]


def star(k):
    return [(0, i) for i in range(1, k + 1)]


def grid2d(w, h):
    out = []
    for y in range(h):
        for x in range(w):
            v = y * w + x
            if x + 1 < w:
                out.append((v, v + 1))
            if y + 1 < h:
                out.append((v, v + w))
    return out


def complete_bipartite(a, b):
    return [(i, a + j) for i in range(a) for j in range(b)]


def complete_tripartite(a, b, c):
    parts = [list(range(a)), list(range(a, a + b)), list(range(a + b, a + b + c))]
    out = []
    for p, q in itertools.combinations(range(3), 2):
        out += [(x, y) for x in parts[p] for y in parts[q]]
    return out


def random_tree(n, rng):
    return [(i, int(rng.integers(0, i))) for i in range(1, n)]


def dense_adjacency(src, dst, n):
    A = np.zeros((n, n), dtype=np.int64)
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            A[a, b] = 1
            A[b, a] = 1
    return A


def brute_force(src, dst, n):
    """T and t by checking every vertex triple a < b < c."""
    A = dense_adjacency(src, dst, n)
    T = 0
    t = np.zeros(n, dtype=np.uint64)
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[b, c] and A[a, c]:
            T += 1
            t[a] += 1
            t[b] += 1
            t[c] += 1
    return T, t


def cube_counts(src, dst, n):
    """T = trace(A^3) / 6 and t = diag(A^3) / 2 via a float64 matmul.

    Entries of A^3 are at most n^2 < 2^53 for the sizes used, so the float64
    products and sums are exact integers.
    """
    A = dense_adjacency(src, dst, n).astype(np.float64)
    A3 = (A @ A) @ A
    d = np.rint(np.diag(A3)).astype(np.int64)
    assert np.all(d % 2 == 0)
    T6 = int(d.sum())
    assert T6 % 6 == 0
    return T6 // 6, (d // 2).astype(np.uint64)


def messy_random(n, m, rng):
    """Random multigraph edge list with self-loops, repeats and both directions."""
    src = rng.integers(0, n, size=m).astype(np.uint32)
    dst = rng.integers(0, n, size=m).astype(np.uint32)
    if m > 4:
        k = m // 4
        src[:k], dst[:k] = dst[m - k:].copy(), src[m - k:].copy()
    return src, dst
