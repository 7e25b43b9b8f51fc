/*
 * ORACLE (test infrastructure only).
 *
 * A plain, slow, single-threaded CPU restatement of what the block-triple
 * triangle-counting path computes.  Only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Counts are exact integers (uint64).  Functions, each with the passage of
 * PGAbB (arXiv 2209.04541) it follows:
 *
 *   or_clean              Section 5.1: graphs are made undirected and
 *                         duplicate edges are removed; self-loops dropped.
 *   or_tc_node_iterator   Section 3.6: a triangle is a mutually connected
 *                         triple; count common neighbours of each edge's
 *                         endpoints by list intersection.  Original IDs.
 *   or_tc_vertex          the per-vertex count t[x] = number of triangles
 *                         containing x, for one x at a time.
 *   or_degree_rank        Section 5.4: degree-based vertex ordering
 *                         (ascending degree, ties by original ID).
 *   or_orient             Section 5.4: triangle counting needs half the
 *                         edges (keep u->v when rank(u) < rank(v)).
 *   or_cuts               Section 4.3: symmetric rectilinear p x p cuts
 *                         (nnz-balanced or uniform contiguous rank ranges).
 *   or_block_edges        Section 3.1 / 4.3: edges of block A_ij.
 *   or_triples            Section 3.6 block-list composition; Section 4.4
 *                         default weight (edges in the block-list), sorted
 *                         in decreasing weight.
 *   or_tc_forward         Section 3.6 kernel summed over all block triples:
 *                         for each oriented edge (u,v), count common
 *                         out-neighbours; per-vertex and per-triple counts.
 *   or_tc_vertex_sample   or_tc_vertex over a list of vertices.
 *   or_tc_forward_mt      or_tc_forward with its rows shared among OpenMP
 *                         threads (only in the -fopenmp build); same counts.
 *   or_cc_min_label       Section 3.4 (Shiloach-Vishkin solves connected
 *                         components): each vertex labelled with the
 *                         smallest vertex ID of its component.
 *   or_pagerank           Section 5.2.1: PageRank on the undirected graph,
 *                         damping d, L1 error tolerance, iteration limit.
 *   or_k4_count           Section 3.2 multi-block pattern mode, k-clique
 *                         finding with k = 4: sets of four mutually
 *                         adjacent vertices.
 *   or_c4_count           Section 3.2, butterfly counting: cycles of four
 *                         distinct vertices (on a bipartite graph, the
 *                         butterflies).
 *
 * The plain build (no -fopenmp) is single-threaded and is the reference;
 * the OpenMP build differs only in or_tc_forward_mt.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- clean */

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Symmetric adjacency of the simple undirected graph given by m raw pairs:
 * each pair (a, b) with a != b contributes b to N(a) and a to N(b); lists
 * are sorted and repeated entries removed.  offs has n+1 entries; adj must
 * hold 2m entries.  Returns the number of adjacency entries (twice the
 * number of undirected edges), or -1 if an ID is >= n.
 */
int64_t or_clean(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                 int64_t* offs, uint32_t* adj) {
    for (uint64_t e = 0; e < m; ++e)
        if (src[e] >= n || dst[e] >= n) return -1;
    int64_t* fill = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!fill) return -2;
    for (uint64_t e = 0; e < m; ++e) {
        if (src[e] == dst[e]) continue;
        fill[src[e] + 1]++;
        fill[dst[e] + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) fill[v + 1] += fill[v];
    int64_t* pos = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!pos) { free(fill); return -2; }
    memcpy(pos, fill, ((size_t)n + 1) * sizeof(int64_t));
    for (uint64_t e = 0; e < m; ++e) {
        uint32_t a = src[e], b = dst[e];
        if (a == b) continue;
        adj[pos[a]++] = b;
        adj[pos[b]++] = a;
    }
    free(pos);
    int64_t out = 0;
    offs[0] = 0;
    for (uint32_t v = 0; v < n; ++v) {
        int64_t lo = fill[v], hi = fill[v + 1];
        qsort(adj + lo, (size_t)(hi - lo), sizeof(uint32_t), cmp_u32);
        for (int64_t t = lo; t < hi; ++t) {
            if (t > lo && adj[t] == adj[t - 1]) continue;
            adj[out++] = adj[t];
        }
        offs[v + 1] = out;
    }
    free(fill);
    return out;
}

/* -------------------------------------------------------- node iterator */

/*
 * Node iterator over original IDs: every triangle {u < v < w} is found once,
 * at u, from the edge (u, v), as a common neighbour w > v of u and v
 * (sorted-list merge).  Adds 1 to t[u], t[v], t[w] per triangle when t is
 * not NULL (t must be zeroed by the caller).  Returns the triangle count.
 */
uint64_t or_tc_node_iterator(uint32_t n, const int64_t* offs, const uint32_t* adj, uint64_t* t) {
    uint64_t total = 0;
    for (uint32_t u = 0; u < n; ++u) {
        for (int64_t e = offs[u]; e < offs[u + 1]; ++e) {
            uint32_t v = adj[e];
            if (v <= u) continue;
            int64_t p = e + 1, pe = offs[u + 1];     /* N(u), entries > v */
            int64_t q = offs[v], qe = offs[v + 1];   /* N(v) */
            while (q < qe && adj[q] <= v) ++q;       /* entries > v */
            while (p < pe && q < qe) {
                if (adj[p] < adj[q]) ++p;
                else if (adj[p] > adj[q]) ++q;
                else {
                    uint32_t w = adj[p];
                    ++total;
                    if (t) { t[u]++; t[v]++; t[w]++; }
                    ++p; ++q;
                }
            }
        }
    }
    return total;
}

static int contains(const uint32_t* a, int64_t len, uint32_t x) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < len && a[lo] == x;
}

/*
 * t[x] for one vertex: the number of edges {a, b} with both ends in N(x),
 * i.e. the number of pairs a < b of neighbours of x with b in N(a).
 * Each such pair is one triangle {x, a, b}.  The shorter of N(a) and N(x)
 * is scanned and each entry looked up in the other.
 */
uint64_t or_tc_vertex(uint32_t n, const int64_t* offs, const uint32_t* adj, uint32_t x) {
    if (x >= n) return 0;
    const uint32_t* nx = adj + offs[x];
    int64_t dx = offs[x + 1] - offs[x];
    uint64_t cnt = 0;
    for (int64_t i = 0; i < dx; ++i) {
        uint32_t a = nx[i];
        const uint32_t* na = adj + offs[a];
        int64_t da = offs[a + 1] - offs[a];
        if (da <= dx) {
            for (int64_t j = 0; j < da; ++j)
                if (na[j] > a && contains(nx, dx, na[j])) ++cnt;
        } else {
            for (int64_t j = i + 1; j < dx; ++j)     /* nx[j] > a */
                if (contains(na, da, nx[j])) ++cnt;
        }
    }
    return cnt;
}

void or_tc_vertex_sample(uint32_t n, const int64_t* offs, const uint32_t* adj,
                         uint64_t k, const uint32_t* xs, uint64_t* out) {
    for (uint64_t i = 0; i < k; ++i) out[i] = or_tc_vertex(n, offs, adj, xs[i]);
}

/* ----------------------------------------------------- degree ordering */

static const int64_t* g_offs_for_cmp;

static int cmp_deg_id(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    int64_t dx = g_offs_for_cmp[x + 1] - g_offs_for_cmp[x];
    int64_t dy = g_offs_for_cmp[y + 1] - g_offs_for_cmp[y];
    if (dx != dy) return dx < dy ? -1 : 1;
    return (x > y) - (x < y);
}

/*
 * Degree order: vertices sorted by (degree ascending, original ID
 * ascending).  perm[r] = the vertex of rank r; rank[v] = rank of v.
 */
int or_degree_rank(uint32_t n, const int64_t* offs, uint32_t* perm, uint32_t* rank) {
    for (uint32_t v = 0; v < n; ++v) perm[v] = v;
    g_offs_for_cmp = offs;
    qsort(perm, n, sizeof(uint32_t), cmp_deg_id);
    g_offs_for_cmp = NULL;
    for (uint32_t r = 0; r < n; ++r) rank[perm[r]] = r;
    return 0;
}

/*
 * Upper orientation in rank space: row r lists rank(y) for every neighbour
 * y of perm[r] with rank(y) > r, ascending.  rowptr has n+1 entries; col
 * must hold offs[n] / 2 entries.  Returns the number of oriented edges.
 */
int64_t or_orient(uint32_t n, const int64_t* offs, const uint32_t* adj, const uint32_t* rank,
                  int64_t* rowptr, uint32_t* col) {
    uint32_t* perm = (uint32_t*)malloc((size_t)n * sizeof(uint32_t) + 1);
    if (!perm) return -2;
    for (uint32_t v = 0; v < n; ++v) perm[rank[v]] = v;
    int64_t out = 0;
    rowptr[0] = 0;
    for (uint32_t r = 0; r < n; ++r) {
        uint32_t x = perm[r];
        int64_t start = out;
        for (int64_t e = offs[x]; e < offs[x + 1]; ++e) {
            uint32_t ry = rank[adj[e]];
            if (ry > r) col[out++] = ry;
        }
        qsort(col + start, (size_t)(out - start), sizeof(uint32_t), cmp_u32);
        rowptr[r + 1] = out;
    }
    free(perm);
    return out;
}

/* ------------------------------------------------------------ partition */

/*
 * Cut points c[0..p] of the rank order, c[0] = 0, c[p] = n.
 *   rule 0 (nnz-balanced): c[t] = least r with rowptr[r] * p >= t * M,
 *                          M = rowptr[n] (oriented edges), 0 < t < p.
 *   rule 1 (uniform):      c[t] = floor(t * n / p).
 * Part t is the rank range [c[t], c[t+1]) (possibly empty).
 */
int or_cuts(uint32_t n, const int64_t* rowptr, uint32_t p, int rule, uint32_t* cuts) {
    if (p == 0) return -1;
    uint64_t M = (uint64_t)rowptr[n];
    cuts[0] = 0;
    for (uint32_t t = 1; t < p; ++t) {
        if (rule == 1) {
            cuts[t] = (uint32_t)(((uint64_t)t * n) / p);
        } else {
            uint32_t r = 0;
            while (r < n && (uint64_t)rowptr[r] * p < (uint64_t)t * M) ++r;
            cuts[t] = r;
        }
    }
    cuts[p] = n;
    return 0;
}

static uint32_t part_of(uint32_t p, const uint32_t* cuts, uint32_t r) {
    uint32_t t = 0;
    while (t + 1 < p && cuts[t + 1] <= r) ++t;
    return t;
}

/* be[i*p + j] = number of oriented edges (u, v) with u in part i, v in part j. */
int or_block_edges(uint32_t n, const int64_t* rowptr, const uint32_t* col, uint32_t p,
                   const uint32_t* cuts, uint64_t* be) {
    memset(be, 0, (size_t)p * p * sizeof(uint64_t));
    for (uint32_t u = 0; u < n; ++u) {
        uint32_t i = part_of(p, cuts, u);
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e)
            be[(size_t)i * p + part_of(p, cuts, col[e])]++;
    }
    return 0;
}

/*
 * Block triples (i, j, k), i <= j <= k, whose blocks A_ij, A_ik, A_jk are
 * all non-empty; weight = be[ij] + be[ik] + be[jk] (the edges of the three
 * list entries).  Sorted by weight descending, then (i, j, k) ascending.
 * ijk gets 3 entries per triple; returns the number of triples.
 */
typedef struct { uint32_t i, j, k; uint64_t w; } or_triple;

static int cmp_triple(const void* a, const void* b) {
    const or_triple* x = (const or_triple*)a;
    const or_triple* y = (const or_triple*)b;
    if (x->w != y->w) return x->w > y->w ? -1 : 1;
    if (x->i != y->i) return x->i < y->i ? -1 : 1;
    if (x->j != y->j) return x->j < y->j ? -1 : 1;
    if (x->k != y->k) return x->k < y->k ? -1 : 1;
    return 0;
}

int64_t or_triples(uint32_t p, const uint64_t* be, uint32_t* ijk, uint64_t* weight) {
    uint64_t cap = (uint64_t)p * (p + 1) * (p + 2) / 6;
    or_triple* tl = (or_triple*)malloc((size_t)(cap ? cap : 1) * sizeof(or_triple));
    if (!tl) return -2;
    int64_t cnt = 0;
    for (uint32_t i = 0; i < p; ++i)
        for (uint32_t j = i; j < p; ++j)
            for (uint32_t k = j; k < p; ++k) {
                uint64_t a = be[(size_t)i * p + j], b = be[(size_t)i * p + k], c = be[(size_t)j * p + k];
                if (a == 0 || b == 0 || c == 0) continue;
                tl[cnt].i = i; tl[cnt].j = j; tl[cnt].k = k; tl[cnt].w = a + b + c;
                ++cnt;
            }
    qsort(tl, (size_t)cnt, sizeof(or_triple), cmp_triple);
    for (int64_t t = 0; t < cnt; ++t) {
        ijk[3 * t] = tl[t].i; ijk[3 * t + 1] = tl[t].j; ijk[3 * t + 2] = tl[t].k;
        weight[t] = tl[t].w;
    }
    free(tl);
    return cnt;
}

/* ------------------------------------------------------ forward count */

/*
 * Rows [u0, u1) of the forward count below: for each oriented edge (u, v)
 * with u in the range, every common out-neighbour w of u and v closes the
 * triangle u < v < w.
 */
static uint64_t forward_rows(uint32_t u0, uint32_t u1, const int64_t* rowptr, const uint32_t* col,
                             uint64_t* t_rank, uint32_t p, const uint32_t* cuts, uint64_t* tc) {
    uint64_t total = 0;
    for (uint32_t u = u0; u < u1; ++u) {
        uint32_t i = tc ? part_of(p, cuts, u) : 0;
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            uint32_t v = col[e];
            uint32_t j = tc ? part_of(p, cuts, v) : 0;
            int64_t a = e + 1, ae = rowptr[u + 1];
            int64_t b = rowptr[v], bend = rowptr[v + 1];
            while (a < ae && b < bend) {
                if (col[a] < col[b]) ++a;
                else if (col[a] > col[b]) ++b;
                else {
                    uint32_t w = col[a];
                    ++total;
                    if (t_rank) { t_rank[u]++; t_rank[v]++; t_rank[w]++; }
                    if (tc) tc[((size_t)i * p + j) * p + part_of(p, cuts, w)]++;
                    ++a; ++b;
                }
            }
        }
    }
    return total;
}

/*
 * Over the oriented graph (rank space): for each oriented edge (u, v),
 * every common out-neighbour w of u and v closes the triangle u < v < w,
 * found exactly once.  Optional outputs (each may be NULL; callers zero
 * them): t_rank[x] per-vertex counts in rank space; tc[(i*p + j)*p + k]
 * per block triple, where i, j, k are the parts of u, v, w (needs p, cuts).
 * Returns the triangle count.
 */
uint64_t or_tc_forward(uint32_t n, const int64_t* rowptr, const uint32_t* col,
                       uint64_t* t_rank, uint32_t p, const uint32_t* cuts, uint64_t* tc) {
    return forward_rows(0, n, rowptr, col, t_rank, p, cuts, tc);
}

#ifdef _OPENMP
#include <omp.h>
/*
 * The same forward count with its rows shared among OpenMP threads (only
 * in the build compiled with -fopenmp).  Rows u = 0, stride, 2 stride, ...
 * are counted (stride 1: every row, the whole count; a larger stride counts
 * a sample of the rows, for timing).  Each thread counts its rows into a
 * private t array of n entries; the arrays are added into t_rank at the
 * end, so with stride 1 the result equals or_tc_forward's.  threads <= 0
 * uses OpenMP's default.  Returns the triangle count of the counted rows,
 * or UINT64_MAX if a private array cannot be allocated.
 */
uint64_t or_tc_forward_mt(uint32_t n, const int64_t* rowptr, const uint32_t* col, uint64_t* t_rank,
                          int threads, uint32_t stride) {
    int nt = threads > 0 ? threads : omp_get_max_threads();
    int64_t step = stride ? (int64_t)stride : 1;
    uint64_t** priv = (uint64_t**)calloc((size_t)nt, sizeof(uint64_t*));
    if (!priv) return UINT64_MAX;
    int fail = 0;
    if (t_rank)
        for (int k = 0; k < nt; ++k)
            if (!(priv[k] = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t)))) fail = 1;
    uint64_t total = 0;
    if (!fail) {
#pragma omp parallel for num_threads(nt) schedule(dynamic, 64) reduction(+ : total)
        for (int64_t u = 0; u < (int64_t)n; u += step)
            total += forward_rows((uint32_t)u, (uint32_t)u + 1, rowptr, col,
                                  t_rank ? priv[omp_get_thread_num()] : NULL, 0, NULL, NULL);
        if (t_rank) {
#pragma omp parallel for num_threads(nt) schedule(static)
            for (int64_t v = 0; v < (int64_t)n; ++v)
                for (int k = 0; k < nt; ++k) t_rank[v] += priv[k][v];
        }
    }
    for (int k = 0; k < nt; ++k) free(priv[k]);
    free(priv);
    return fail ? UINT64_MAX : total;
}

int or_num_threads(void) { return omp_get_max_threads(); }
#endif

/* 4*|E+| + 4*sum_v indeg(v)*outdeg(v) + 8*(n+1): the bytes of the oriented
 * CSR that the edge-wise intersection reads when nothing is reused. */
uint64_t or_alg_bytes(uint32_t n, const int64_t* rowptr, const uint32_t* col) {
    uint64_t* indeg = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!indeg) return 0;
    uint64_t m = (uint64_t)rowptr[n];
    for (uint64_t e = 0; e < m; ++e) indeg[col[e]]++;
    uint64_t wedge = 0;
    for (uint32_t v = 0; v < n; ++v) wedge += indeg[v] * (uint64_t)(rowptr[v + 1] - rowptr[v]);
    free(indeg);
    return 4 * m + 4 * wedge + 8 * ((uint64_t)n + 1);
}

/* ------------------------------------------------ connected components */

/*
 * label[x] = the smallest vertex ID of x's connected component.  Vertices
 * are visited in ascending ID order; each one not yet labelled starts a
 * breadth-first search that labels everything it reaches with the start's
 * ID (the first vertex of a component met in ascending order is its
 * smallest).  Returns the number of components, or -2 without memory.
 */
int64_t or_cc_min_label(uint32_t n, const int64_t* offs, const uint32_t* adj, uint32_t* label) {
    uint32_t* queue = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!queue) return -2;
    for (uint32_t v = 0; v < n; ++v) label[v] = UINT32_MAX;
    int64_t comps = 0;
    for (uint32_t s = 0; s < n; ++s) {
        if (label[s] != UINT32_MAX) continue;
        ++comps;
        size_t head = 0, tail = 0;
        label[s] = s;
        queue[tail++] = s;
        while (head < tail) {
            uint32_t x = queue[head++];
            for (int64_t e = offs[x]; e < offs[x + 1]; ++e) {
                uint32_t y = adj[e];
                if (label[y] == UINT32_MAX) {
                    label[y] = s;
                    queue[tail++] = y;
                }
            }
        }
    }
    free(queue);
    return comps;
}

/* ------------------------------------------------------------ PageRank */

/*
 * PageRank of the undirected graph (every edge counts in both directions),
 * in double precision:
 *   r_0(v)     = 1 / n
 *   r_t+1(v)   = (1 - d) / n + d * sum over neighbours u of r_t(u) / deg(u)
 * (a vertex of degree 0 passes nothing on).  After each iteration the L1
 * change sum_v |r_t+1(v) - r_t(v)| is compared with tol; the iteration
 * stops at the first change below tol, or after max_iter iterations.
 * rank gets r for the last iteration made; returns the iterations made
 * (*err: the last change), or -2 without memory.
 */
int or_pagerank(uint32_t n, const int64_t* offs, const uint32_t* adj, double d, double tol, int max_iter,
                double* rank, double* err) {
    double* cur = (double*)malloc(((size_t)n + 1) * sizeof(double));
    double* nxt = (double*)malloc(((size_t)n + 1) * sizeof(double));
    if (!cur || !nxt) { free(cur); free(nxt); return -2; }
    for (uint32_t v = 0; v < n; ++v) cur[v] = 1.0 / n;
    int it = 0;
    double change = 0.0;
    while (it < max_iter) {
        change = 0.0;
        for (uint32_t v = 0; v < n; ++v) {
            double sum = 0.0;
            for (int64_t e = offs[v]; e < offs[v + 1]; ++e) {
                uint32_t u = adj[e];
                sum += cur[u] / (double)(offs[u + 1] - offs[u]);
            }
            nxt[v] = (1.0 - d) / n + d * sum;
            change += fabs(nxt[v] - cur[v]);
        }
        double* t = cur; cur = nxt; nxt = t;
        ++it;
        if (change < tol) break;
    }
    for (uint32_t v = 0; v < n; ++v) rank[v] = cur[v];
    if (err) *err = change;
    free(cur);
    free(nxt);
    return it;
}

/* ----------------------------------------------------------- 4-cliques */

/*
 * Number of 4-cliques {u < v < w < x} (original IDs, every pair adjacent):
 * for each edge (u, v) with u < v, the common neighbours above v, and for
 * each such w the common neighbours of u, v and w above w.  Membership by
 * binary search in the sorted adjacency lists.
 */
uint64_t or_k4_count(uint32_t n, const int64_t* offs, const uint32_t* adj) {
    uint64_t total = 0;
    for (uint32_t u = 0; u < n; ++u) {
        const uint32_t* nu = adj + offs[u];
        int64_t du = offs[u + 1] - offs[u];
        for (int64_t i = 0; i < du; ++i) {
            uint32_t v = nu[i];
            if (v <= u) continue;
            const uint32_t* nv = adj + offs[v];
            int64_t dv = offs[v + 1] - offs[v];
            for (int64_t j = i + 1; j < du; ++j) {
                uint32_t w = nu[j];              /* w > v, adjacent to u */
                if (!contains(nv, dv, w)) continue;
                const uint32_t* nw = adj + offs[w];
                int64_t dw = offs[w + 1] - offs[w];
                for (int64_t k = j + 1; k < du; ++k) {
                    uint32_t x = nu[k];          /* x > w, adjacent to u */
                    if (contains(nv, dv, x) && contains(nw, dw, x)) ++total;
                }
            }
        }
    }
    return total;
}

/* ------------------------------------------------------------ 4-cycles */

/*
 * Number of cycles a - w - b - y - a on four distinct vertices (as
 * subgraphs).  A 4-cycle has two pairs of opposite vertices, and the pair
 * {a, b} with c common neighbours closes C(c, 2) cycles; so the count is
 * half the sum over unordered pairs a < b of C(c_ab, 2).  For each a the
 * common-neighbour counts of every b > a are gathered in a dense array
 * through the paths a - w - b, then cleared.  Returns UINT64_MAX without
 * memory.
 */
uint64_t or_c4_count(uint32_t n, const int64_t* offs, const uint32_t* adj) {
    uint64_t* cnt = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!cnt) return UINT64_MAX;
    uint64_t pairs = 0;
    for (uint32_t a = 0; a < n; ++a) {
        for (int64_t e = offs[a]; e < offs[a + 1]; ++e) {
            uint32_t w = adj[e];
            for (int64_t f = offs[w]; f < offs[w + 1]; ++f)
                if (adj[f] > a) cnt[adj[f]]++;
        }
        for (int64_t e = offs[a]; e < offs[a + 1]; ++e) {
            uint32_t w = adj[e];
            for (int64_t f = offs[w]; f < offs[w + 1]; ++f) {
                uint32_t b = adj[f];
                if (b > a && cnt[b]) {
                    pairs += cnt[b] * (cnt[b] - 1) / 2;
                    cnt[b] = 0;
                }
            }
        }
    }
    free(cnt);
    return pairs / 2;
}
