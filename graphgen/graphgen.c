/*
 * Seeded synthetic graph generators (raw undirected edge lists).
 *
 * This module is shared input plumbing: both the CPU oracle and the CUDA
 * path consume its output, and it holds none of the triangle-counting
 * arithmetic.  Every generator writes raw (src, dst) pairs of uint32 vertex
 * IDs; duplicates, self-loops and both directions may appear where stated,
 * and are removed by whoever ingests the list.
 *
 * Randomness: one counter-based stream built on SplitMix64 (Steele, Lea and
 * Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).
 * Draw c of the stream keyed by `seed` is
 *     mix(key + (c + 1) * 0x9E3779B97F4A7C15),   key = mix(seed),
 * where mix() is SplitMix64's output function.  Because each draw depends
 * only on (seed, c), the parallel generators are bit-identical for any
 * thread count.  The stream, the R-MAT edge step and the Feistel
 * relabelling live in gg_stream.h, which the device generators
 * (graphgen_dev.cu) include too.
 *
 * Workloads (synthetic stand-ins for the paper's real-world datasets, which
 * are not available; the paper's own synthetic graph is a Kronecker graph):
 *   - R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with a seeded vertex
 *     relabelling, as in Graph500;
 *   - Erdos-Renyi G(n, m) with m distinct pairs, or m i.i.d. pairs;
 *   - a W x H 4-neighbour grid plus k uniform random extra edges;
 *   - a random geometric graph in the unit square.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "gg_stream.h"

uint64_t gg_splitmix_draw(uint64_t seed, uint64_t c) { return gg_draw(gg_mix(seed), c); }

/* Output c of plain SplitMix64 started at `state` (for checking against the
 * published sequence). */
uint64_t gg_splitmix_raw(uint64_t state, uint64_t c) { return gg_draw(state, c); }

/* Seeded permutation of [0, n) by Fisher-Yates, stream key mix(seed ^ tag). */
static void gg_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
    uint64_t key = gg_mix(seed ^ 0x5045524D5554ULL);
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n; i > 1; --i) {
        uint32_t j = gg_below((uint32_t)(gg_draw(key, i) >> 32), i);
        uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
    }
}

/*
 * R-MAT: m edges on n = 2^scale vertices.  Edge e descends `scale` levels;
 * at each level one 32-bit uniform picks a quadrant with probabilities
 * (a, b, c, 1-a-b-c) (top-left, top-right, bottom-left, bottom-right),
 * setting one bit of src (row) and dst (column), most significant first.
 * No noise.  Relabelling of both endpoints: permute = 0 none, 1 a seeded
 * Fisher-Yates permutation (as Graph500), 2 the seeded Feistel bijection of
 * gg_stream.h (evaluated per endpoint, so it parallelises).  Duplicates and
 * self-loops are kept.
 */
int gg_rmat(uint32_t scale, uint64_t m, double a, double b, double c, uint64_t seed,
            int permute, uint32_t* src, uint32_t* dst) {
    if (scale == 0 || scale > 31 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    if (permute < 0 || permute > 2) return -1;
    const uint64_t key = gg_mix(seed);
    uint64_t ta, tb, tc;
    gg_rmat_thresholds(a, b, c, &ta, &tb, &tc);
    const uint64_t fkey = gg_mix(seed ^ GG_TAG_FEISTEL);
    int64_t mm = (int64_t)m;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < mm; ++e) {
        uint32_t s, d;
        gg_rmat_edge(key, scale, (uint64_t)e, ta, tb, tc, &s, &d);
        if (permute == 2) {
            s = gg_feistel(s, scale, fkey);
            d = gg_feistel(d, scale, fkey);
        }
        src[e] = s; dst[e] = d;
    }
    if (permute == 1) {
        uint32_t n = 1u << scale;
        uint32_t* perm = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
        if (!perm) return -2;
        gg_permutation(n, seed, perm);
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < mm; ++e) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
        free(perm);
    }
    return 0;
}

/* The Fisher-Yates relabelling gg_rmat applies for `seed` (permute = 1),
 * for a device generator to apply. */
void gg_shuffle_permutation(uint32_t n, uint64_t seed, uint32_t* perm) { gg_permutation(n, seed, perm); }

/* The Feistel relabelling of x in [0, 2^bits) for seed (for checks). */
uint32_t gg_feistel_label(uint32_t x, uint32_t bits, uint64_t seed) {
    return gg_feistel(x, bits, gg_mix(seed ^ GG_TAG_FEISTEL));
}

/*
 * Erdos-Renyi, i.i.d. pairs: m uniform ordered pairs over [0, n)^2.
 * Self-loops and duplicates are kept (the ingest removes them).
 */
int gg_er_pairs(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
    if (n == 0) return -1;
    const uint64_t key = gg_mix(seed ^ 0x4552ULL);
    int64_t mm = (int64_t)m;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < mm; ++e) {
        uint64_t x = gg_draw(key, (uint64_t)e);
        src[e] = gg_below((uint32_t)(x >> 32), n);
        dst[e] = gg_below((uint32_t)x, n);
    }
    return 0;
}

/*
 * Erdos-Renyi G(n, m): m distinct unordered pairs {a, b}, a != b, drawn
 * uniformly (self-loops and repeats are rejected and redrawn).  Pairs are
 * written in the order drawn, the draw's first endpoint as src, so each
 * pair's direction is random.
 */
int gg_er_distinct(uint32_t n, uint64_t m, uint64_t seed, uint32_t* src, uint32_t* dst) {
    if (n < 2) return m == 0 ? 0 : -1;
    if (m > (uint64_t)n * (n - 1) / 2) return -1;
    const uint64_t key = gg_mix(seed ^ 0x4552444953ULL);
    uint64_t cap = 1;
    while (cap < 2 * m + 16) cap <<= 1;
    uint64_t* table = (uint64_t*)malloc(cap * sizeof(uint64_t));
    if (!table) return -2;
    memset(table, 0xFF, cap * sizeof(uint64_t));
    uint64_t got = 0, c = 0;
    while (got < m) {
        uint64_t x = gg_draw(key, c++);
        uint32_t a = gg_below((uint32_t)(x >> 32), n);
        uint32_t b = gg_below((uint32_t)x, n);
        if (a == b) continue;
        uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
        uint64_t k = (lo << 32) | hi;
        uint64_t h = gg_mix(k) & (cap - 1);
        int dup = 0;
        while (table[h] != ~0ULL) {
            if (table[h] == k) { dup = 1; break; }
            h = (h + 1) & (cap - 1);
        }
        if (dup) continue;
        table[h] = k;
        src[got] = a; dst[got] = b;
        ++got;
    }
    free(table);
    return 0;
}

/* Number of edges gg_grid writes: grid edges plus `extra`. */
uint64_t gg_grid_count(uint32_t w, uint32_t h, uint64_t extra) {
    return (uint64_t)(w - 1) * h + (uint64_t)w * (h - 1) + extra;
}

/*
 * W x H 4-neighbour grid (vertex y*W + x; edges to the right and below),
 * followed by `extra` uniform random pairs with self-loops redrawn
 * (repeats of existing edges are possible and removed at ingest).
 */
int gg_grid(uint32_t w, uint32_t h, uint64_t extra, uint64_t seed, uint32_t* src, uint32_t* dst) {
    if (w == 0 || h == 0) return -1;
    uint64_t n64 = (uint64_t)w * h;
    if (n64 > 0xFFFFFFFFULL) return -1;
    uint32_t n = (uint32_t)n64;
    uint64_t horiz = (uint64_t)(w - 1) * h;
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < (int64_t)h; ++y) {
        for (uint32_t x = 0; x + 1 < w; ++x) {
            uint64_t e = (uint64_t)y * (w - 1) + x;
            src[e] = (uint32_t)y * w + x; dst[e] = (uint32_t)y * w + x + 1;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < (int64_t)h - 1; ++y) {
        for (uint32_t x = 0; x < w; ++x) {
            uint64_t e = horiz + (uint64_t)y * w + x;
            src[e] = (uint32_t)y * w + x; dst[e] = (uint32_t)(y + 1) * w + x;
        }
    }
    uint64_t base = horiz + (uint64_t)w * (h - 1);
    const uint64_t key = gg_mix(seed ^ 0x47524944ULL);
    uint64_t c = 0;
    for (uint64_t e = 0; e < extra; ++e) {
        uint32_t a, b;
        do {
            uint64_t x = gg_draw(key, c++);
            a = gg_below((uint32_t)(x >> 32), n);
            b = gg_below((uint32_t)x, n);
        } while (a == b);
        src[base + e] = a; dst[base + e] = b;
    }
    return 0;
}

/*
 * Random geometric graph: n points uniform in [0,1)^2 (coordinates from one
 * draw each: x = hi32 / 2^32, y = lo32 / 2^32); {a, b} is an edge when the
 * Euclidean distance is below r.  Each edge is written once with a < b.
 * Call with src == dst == NULL to get the count; the second call with
 * arrays of that length fills them (same order every time).
 */
int64_t gg_rgg(uint32_t n, double r, uint64_t seed, uint32_t* src, uint32_t* dst) {
    if (n == 0) return 0;
    if (!(r > 0.0)) return -1;
    const uint64_t key = gg_mix(seed ^ 0x524747ULL);
    double* px = (double*)malloc((size_t)n * sizeof(double));
    double* py = (double*)malloc((size_t)n * sizeof(double));
    uint32_t g = (uint32_t)floor(1.0 / r);
    if (g < 1) g = 1;
    if (g > 65536) g = 65536;
    uint64_t ncell = (uint64_t)g * g;
    uint32_t* cnt = (uint32_t*)calloc(ncell + 1, sizeof(uint32_t));
    uint32_t* order = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* cell = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    if (!px || !py || !cnt || !order || !cell) {
        free(px); free(py); free(cnt); free(order); free(cell);
        return -2;
    }
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t x = gg_draw(key, i);
        px[i] = (double)(uint32_t)(x >> 32) * (1.0 / 4294967296.0);
        py[i] = (double)(uint32_t)x * (1.0 / 4294967296.0);
        uint32_t cx = (uint32_t)(px[i] * g), cy = (uint32_t)(py[i] * g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        cell[i] = cy * g + cx;
        cnt[cell[i] + 1]++;
    }
    for (uint64_t k = 0; k < ncell; ++k) cnt[k + 1] += cnt[k];
    uint32_t* pos = (uint32_t*)malloc((size_t)(ncell + 1) * sizeof(uint32_t));
    memcpy(pos, cnt, (size_t)(ncell + 1) * sizeof(uint32_t));
    for (uint32_t i = 0; i < n; ++i) order[pos[cell[i]]++] = i;
    free(pos);
    const double r2 = r * r;
    int64_t out = 0;
    for (uint32_t a = 0; a < n; ++a) {
        int64_t cx = cell[a] % g, cy = cell[a] / g;
        for (int64_t dy = -1; dy <= 1; ++dy) {
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t nx = cx + dx, ny = cy + dy;
                if (nx < 0 || ny < 0 || nx >= g || ny >= g) continue;
                uint64_t k = (uint64_t)ny * g + nx;
                for (uint32_t t = cnt[k]; t < cnt[k + 1]; ++t) {
                    uint32_t b = order[t];
                    if (b <= a) continue;
                    double ddx = px[a] - px[b], ddy = py[a] - py[b];
                    if (ddx * ddx + ddy * ddy < r2) {
                        if (src) { src[out] = a; dst[out] = b; }
                        ++out;
                    }
                }
            }
        }
    }
    free(px); free(py); free(cnt); free(order); free(cell);
    return out;
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
