/*
 * pgabb.h - C ABI of the B300 block-triple triangle-counting library.
 *
 * The library implements the data-parallel hot path of PGAbB's block-based
 * model (Yasar et al., arXiv 2209.04541) for triangle counting:
 *
 *   load an undirected graph            (Section 5.1 preprocessing)
 *   degree-order and orient it          (Section 5.4: degree ordering;
 *                                        "only half of the edges")
 *   partition it into p x p blocks      (Section 4.3: symmetric
 *                                        rectilinear 2D partition,
 *                                        row-major block IDs)
 *   build the block-triple queue        (Section 3.6 block-list
 *                                        composition; Section 4.4 weights,
 *                                        decreasing order)
 *   run the device kernel per triple    (Section 3.6, Listing 5:
 *                                        per edge of the first block,
 *                                        intersect partial lists)
 *   reduce                              (Section 3.3 reduce_dev)
 *
 * Conventions for every call:
 *   - Return value: PGB_OK (0) or a negative PGB_E_* code.  On error the
 *     thread-local message from pgb_last_error() says what failed and no
 *     output handle is written.  No C++ exception crosses this ABI.
 *   - `mem` says where caller pointers live: PGB_MEM_HOST (pageable or
 *     pinned host memory) or PGB_MEM_DEVICE (device memory of the current
 *     CUDA device).  Host inputs are copied to the device inside the call.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     ordered on it; calls that must return sizes or values to the host
 *     synchronise it.
 *   - Input arrays are borrowed for the duration of the call only.  Handles
 *     (pgb_graph, pgb_blocks, pgb_tc_result) are owned by the library and
 *     released with their *_free call; device memory behind them comes from
 *     the allocator set by pgb_set_allocator (default: cudaMallocAsync on
 *     the handle's stream).
 *   - Vertex IDs are uint32 and must be < n; counts are uint64 and exact.
 */
#ifndef PGABB_H
#define PGABB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status codes */
#define PGB_OK           0
#define PGB_E_INVAL     -1  /* bad argument: NULL pointer, ID >= n, p == 0, ... */
#define PGB_E_NOMEM     -2  /* host or device allocation failed */
#define PGB_E_OVERFLOW  -3  /* a size exceeds the supported range (e.g. >= 2^32 oriented edges) */
#define PGB_E_CUDA      -4  /* a CUDA runtime call or kernel failed */
#define PGB_E_BUDGET    -5  /* the request can never fit the device budget */
#define PGB_E_TIMEOUT   -6  /* a bounded device wait gave up */
#define PGB_E_CANCELLED -7  /* the job was cancelled */
#define PGB_E_STATE     -8  /* handle used in the wrong state */

/* ----------------------------------------------------------- memory kinds */
#define PGB_MEM_HOST   0
#define PGB_MEM_DEVICE 1

/* ------------------------------------------------------------- cut rules */
/* Section 4.3 asks for contiguous symmetric cuts but fixes no rule.
 * PGB_CUT_NNZ: c[t] = least rank r with rowptr[r] * p >= t * |E+| (the
 *              oriented out-degree prefix split into p equal shares).
 * PGB_CUT_UNIFORM: c[t] = floor(t * n / p). */
#define PGB_CUT_NNZ     0
#define PGB_CUT_UNIFORM 1

/* ------------------------------------------------------------- run modes */
/* PGB_MODE_PLAIN: one kernel launch per block triple (i, j, k), each
 *   counting the triangles u < v < w with u in V_i, v in V_j, w in V_k:
 *   the block-list (A_ij, A_ik, A_jk) of Section 3.6 exactly.
 * PGB_MODE_PERSISTENT: persistent kernels drain device queues of work: the
 *   edge-wise kernel takes block columns (A_*j with third range [c_j, n):
 *   the tuples (A_ij, A_i[j..p-1], A_j[j..p-1]) of every i <= j) in chunks
 *   of edges; the hash kernel takes middle-vertex work items.
 * PGB_MODE_HYBRID: Section 4.4's scheduler with host threads beside the GPU.
 *   The head parts (tasks) are ordered by estimated work (lookups plus
 *   in-edges); the host kernel takes the lightest parts while their summed
 *   estimate stays within host_share_ppm / 10^6 of the total (the cut-off:
 *   the host never takes a heavier part), on host_threads threads; the
 *   device counts the other parts as in PERSISTENT mode, at the same time.
 *   Needs resident blocks and use_graph = 0 (else PGB_E_STATE). */
#define PGB_MODE_PLAIN      0
#define PGB_MODE_PERSISTENT 1
#define PGB_MODE_HYBRID     2

/* ------------------------------------------------- intersection variants */
/* Section 3.6 lets the intersection run over sorted lists or a hash map.
 * Every variant returns the same integers; the choice only changes speed.
 * PGB_VAR_AUTO:    chosen by the autotuner (below).
 * PGB_VAR_BSEARCH: each element of the shorter list is binary-searched in
 *                  the longer one; work is flattened across a warp.
 * PGB_VAR_MERGE:   warp-cooperative merge: the warp takes one edge at a
 *                  time and walks both lists in 32-entry chunks; each lane
 *                  finds its entry of one chunk in the other chunk with a
 *                  5-step shuffle search, and the chunk with the smaller
 *                  last entry advances.  Suits long lists of similar length.
 * PGB_VAR_HASH:    middle-vertex form: the partial list of each middle
 *                  vertex v is held in shared memory (a bitmap over its
 *                  third-vertex rank range when that range is at most
 *                  131,072 ranks, else a hash table) and the lists of v's
 *                  in-neighbours after v are streamed through it.
 * PLAIN mode runs PGB_VAR_BSEARCH or PGB_VAR_MERGE (PGB_VAR_HASH gives
 * PGB_E_INVAL).
 * Autotuner (PGB_VAR_AUTO): PLAIN mode runs PGB_VAR_BSEARCH.  PERSISTENT
 * mode chooses per column block j (the head part V_j): the tuples
 * (A_ij, A_ik, A_jk) of one j count exactly the triangles whose middle
 * vertex lies in V_j, so each part can take its own kernel.  A part runs
 * PGB_VAR_HASH when its oriented edges average at least 32 lookups
 * (pgb_tc_opts.hash_min_lookups)
 * (PGB_EXPORT_PART_PROBES[j] >= 32 * sum_i |A_ij|: long lists, skewed
 * degrees) and PGB_VAR_BSEARCH otherwise (short lists); when the parts
 * differ, one hash launch over the hash parts' work items and one edge-wise
 * launch over the other parts' tuples add into the same counts
 * (PGB_VAR_MIXED).  Within the hash form the bitmap or table, and the split
 * of heavy middle vertices into in-edge chunks and key-range slices, are
 * chosen per work item from its rank range, list length and in-degree.
 * PGB_VAR_MIXED is a result value only (pgb_tc_result_variant), and so is
 * PGB_VAR_HOST (pgb_tc_result_part_variants: a part the HYBRID host kernel
 * counted).
 * Dense top block (pgb_tc_opts.dense_core): the K highest ranks of the degree
 * order, where the hubs sit, form a dense diagonal block.  Its triangles
 * (all three vertices among those ranks) are counted from its 0/1 adjacency
 * A as sum_y A[x][y] (A A)[x][y] / 2 per vertex, the product a dense fp16
 * GEMM with fp32 accumulation (exact: integers below 2^24); the intersection
 * kernels skip the in-edges whose tail is in the block.  The autotuner takes
 * the K (a multiple of 2048, at most 32,768) whose saved lookups outweigh
 * the GEMM's time by the most, or none. */
#define PGB_VAR_AUTO    0
#define PGB_VAR_BSEARCH 1
#define PGB_VAR_MERGE   2
#define PGB_VAR_HASH    3
#define PGB_VAR_MIXED   4
#define PGB_VAR_HOST    5

/* Queue order of block tuples (Section 4.4 sorts by decreasing weight). */
#define PGB_ORDER_WEIGHT   0  /* decreasing weight (Section 4.4) */
#define PGB_ORDER_LOCALITY 1  /* by column block j, then decreasing weight */
#define PGB_ORDER_HILBERT  2  /* PLAIN launches: by the Hilbert-curve index of
                                 block (i, j) (Section 4.3.1 allows any
                                 space-filling curve for the block IDs), then
                                 k; PERSISTENT runs treat it as WEIGHT */

typedef struct pgb_graph pgb_graph;
typedef struct pgb_blocks pgb_blocks;
typedef struct pgb_tc_result pgb_tc_result;

/* ------------------------------------------------------------- allocator */
/* Device allocator hooks.  alloc returns device memory usable on `stream`,
 * aligned to 256 bytes as cudaMalloc's is (NULL on failure; a misaligned
 * block is freed again and the call fails with PGB_E_INVAL); free releases
 * memory obtained from alloc.  Set before
 * any handle exists; passing NULLs restores the default (cudaMallocAsync /
 * cudaFreeAsync).  Returns PGB_E_STATE while handles are alive. */
typedef void* (*pgb_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pgb_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
int pgb_set_allocator(pgb_alloc_fn alloc, pgb_free_fn free_fn, void* ctx);

/* ----------------------------------------------------------------- load */
/* Section 5.1 (graphs made undirected, duplicate edges removed); self-loops
 * are dropped.  src/dst: m raw pairs (any direction, repeats allowed),
 * IDs < n.  Produces the cleaned simple undirected graph (kept on the
 * device as sorted canonical pairs a < b plus vertex degrees).
 * Errors: PGB_E_INVAL (NULL with m > 0, ID >= n, out == NULL),
 * PGB_E_NOMEM, PGB_E_OVERFLOW (n > 2^32 - 1 cannot happen; m >= 2^32
 * unique edges), PGB_E_CUDA. */
int pgb_graph_from_edges(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                         int mem, void* stream, pgb_graph** out);

/* Same, from a CSR adjacency: offs int64[n+1] (non-decreasing, offs[0] = 0),
 * cols uint32[offs[n]]; row v lists neighbours of v (either direction, any
 * order, repeats allowed). */
int pgb_graph_from_csr(uint32_t n, const int64_t* offs, const uint32_t* cols, int mem, void* stream,
                       pgb_graph** out);

/* n and the number of undirected edges after cleaning. */
int pgb_graph_info(const pgb_graph* g, uint32_t* n, uint64_t* m_undirected);

/* Copy the cleaned graph out: a[e] < b[e], sorted by (a, b), m_undirected
 * entries each (either may be NULL); deg gets n degrees (may be NULL). */
int pgb_graph_export(const pgb_graph* g, uint32_t* a, uint32_t* b, uint32_t* deg, int mem,
                     void* stream);

void pgb_graph_free(pgb_graph* g);

/* ------------------------------------------------------------ partition */
/* Section 5.4 degree ordering + orientation, then the Section 4.3 p x p
 * symmetric partition and the Section 3.6 / 4.4 block-triple queue.
 *   rank:  vertices sorted by (degree ascending, original ID ascending);
 *   E+:    u -> v for every edge with rank(u) < rank(v), rows sorted;
 *   cuts:  c[0] = 0 <= c[1] <= ... <= c[p] = n by `cut_rule`;
 *   A_ij:  oriented edges with rank(u) in [c_i, c_i+1), rank(v) in
 *          [c_j, c_j+1); only i <= j can be non-empty;
 *   queue: triples i <= j <= k with A_ij, A_ik, A_jk non-empty, weight
 *          |A_ij| + |A_ik| + |A_jk|, decreasing weight, ties by (i, j, k).
 * Errors: PGB_E_INVAL (p == 0, p > 1024, p > n when n > 0, bad rule),
 * PGB_E_NOMEM, PGB_E_OVERFLOW, PGB_E_CUDA.  The graph may be freed after. */
int pgb_partition(const pgb_graph* g, uint32_t p, int cut_rule, void* stream, pgb_blocks** out);

typedef struct {
    uint32_t n;            /* vertices */
    uint32_t p;            /* parts per dimension */
    uint64_t m;            /* oriented edges |E+| = undirected edges */
    uint64_t nonempty_blocks;
    uint64_t triples;      /* queue length */
    uint64_t wedges;       /* sum over v of indeg(v) * outdeg(v) in E+ */
    uint64_t alg_bytes;    /* 4|E+| + 4 * wedges + 8 (n + 1) */
    uint32_t max_outdeg;
    uint32_t reserved;
    uint64_t probes;       /* sum over edges (u, v) of the entries of u's row
                              after v: the lookups of the middle-vertex variant */
} pgb_blocks_stats;

int pgb_blocks_info(const pgb_blocks* b, pgb_blocks_stats* out);

/* Export one array of the partition (host or device destination):
 *   PGB_EXPORT_PERM       uint32[n]   vertex of each rank
 *   PGB_EXPORT_ROWPTR     int64[n+1]  oriented CSR offsets (rank space)
 *   PGB_EXPORT_COL        uint32[m]   oriented CSR columns (rank space)
 *   PGB_EXPORT_CUTS       uint32[p+1]
 *   PGB_EXPORT_BLOCK_EDGES uint64[p*p] |A_ij| row-major
 *   PGB_EXPORT_TRIPLES    uint32[3*T] queue (i, j, k) in order
 *   PGB_EXPORT_WEIGHTS    uint64[T]   queue weights
 *   PGB_EXPORT_PART_PROBES uint64[p]  per head part j: the sum over oriented
 *                                     edges (u, v) with v in V_j of the
 *                                     entries of u's row after v (the
 *                                     autotuner's per-part statistic) */
#define PGB_EXPORT_PERM        0
#define PGB_EXPORT_ROWPTR      1
#define PGB_EXPORT_COL         2
#define PGB_EXPORT_CUTS        3
#define PGB_EXPORT_BLOCK_EDGES 4
#define PGB_EXPORT_TRIPLES     5
#define PGB_EXPORT_WEIGHTS     6
#define PGB_EXPORT_PART_PROBES 7
int pgb_blocks_export(const pgb_blocks* b, int what, void* dst, int mem, void* stream);

void pgb_blocks_free(pgb_blocks* b);

/* Streaming tier (Section 4.4: the scheduler copies a task's blocks to the
 * device asynchronously while other tasks compute; Section 1: graphs that fit
 * in host DRAM but not in device memory).  Moves the in-edge index -- for
 * every oriented edge, grouped by head v, the range of the tail's row after
 * v (8 bytes) and the tail (4 bytes), 12 bytes per edge -- into pinned host
 * memory owned by `b`, and frees it and the edge-wise kernels' arrays (row
 * index, block edge index) on the device.  What stays resident is what the
 * counting kernel reads at random: row offsets, columns, in-edge offsets and
 * the rank permutation (about 4|E+| + 12n bytes).  Later runs on `b` stream
 * the index in chunks (see device_budget) and must use PGB_MODE_PERSISTENT
 * with PGB_VAR_AUTO or PGB_VAR_HASH (else PGB_E_STATE).  Synchronises
 * `stream`.  Calling it twice is a no-op.  Errors: PGB_E_INVAL (NULL),
 * PGB_E_NOMEM (pinned allocation), PGB_E_CUDA. */
int pgb_blocks_offload(pgb_blocks* b, void* stream);

/* Block cache tier (Section 4.4's copies of a task's blocks, with eviction):
 * moves the columns to pinned host memory as well, so that the device keeps
 * only the row offsets, the rank permutation and the cuts (about 8 bytes per
 * vertex; runs add 16 per vertex of counters).  The ranks are cut into
 * `slices` row ranges of about equal edges (0 = the partition's p; at most
 * 1024, and at most n); the columns of one range form one contiguous slice.
 * Fewer, larger slices mean fewer pieces and fewer table rebuilds, but a
 * budget must hold at least two of them.  The in-edge index is re-sorted by
 * (tail range, head, tail) into pinned host memory and cut into pieces of at
 * most 2^21 in-edges of one range pair (tail range i, head range j); each
 * piece's work items are built here, once.  A run keeps a
 * cache of column slices on the device, as many as device_budget allows
 * (at least two), evicting the least recently used slice that the current
 * pieces do not need; it counts the pieces head-block group by head-block
 * group so that the group's slices stay while the tail slices pass through,
 * and overlaps the copies (side stream) with the counting launches.  Call it
 * on resident blocks (PGB_E_STATE after pgb_blocks_offload); afterwards the
 * blocks behave as offloaded (PERSISTENT + hash only; chunk_edges ignored).
 * Needs about 36 bytes per edge of device memory while it builds the index.
 * Synchronises `stream`.  Errors: PGB_E_INVAL, PGB_E_STATE, PGB_E_NOMEM,
 * PGB_E_CUDA. */
int pgb_blocks_offload_columns(pgb_blocks* b, uint32_t slices, void* stream);

/* After pgb_blocks_offload_columns: the smallest device_budget whose column
 * cache holds `slices` slices (capped at p) for runs with the given
 * per_vertex setting.  Queries the current device.  Errors: PGB_E_INVAL
 * (NULL), PGB_E_STATE (columns not offloaded). */
int pgb_blocks_cache_budget(const pgb_blocks* b, int per_vertex, uint32_t slices, uint64_t* budget);

/* The device bytes a streamed run on `b` holds besides its two stream slots:
 * 4(n+1) + 4(m+8) + 4(n+1) + 4n + 4(p+1) for the resident arrays, 16n for the
 * per-vertex counters when per_vertex != 0, and 16 MiB for the launches'
 * partial sums.  A device_budget must exceed it; the rest is split into two
 * slots of 44 bytes per in-edge (index entry plus one work item bound).
 * After pgb_blocks_offload_columns: 4(n+1) + 4n + 4(p+1), 16n for the
 * counters, and 16 MiB; a budget must also cover two piece slots and at
 * least two column slices (PGB_E_BUDGET otherwise).
 * Errors: PGB_E_INVAL (NULL). */
int pgb_blocks_resident_bytes(const pgb_blocks* b, int per_vertex, uint64_t* bytes);

/* --------------------------------------------------------------- cancel */
/* A cancel token stops runs that are already on the device (the paper's
 * scheduler controls its tasks from the host, Section 4.4; a stop request is
 * this library's form of that control).  The token is one word of pinned
 * host memory mapped into the device's address space.  A run given the
 * token (pgb_tc_opts.cancel) reads it from its kernels: the persistent
 * kernels every 64 work fetches, a plain per-triple launch at entry.  A
 * kernel that finds it set skips the rest of its work (every CTA stops
 * after its current work item) and marks the run, and pgb_tc_result_get
 * then fails with PGB_E_CANCELLED.  A run that finished before it looked at
 * the token is complete and returns its counts.  No wait on the token is
 * unbounded: a kernel only reads it.  One token may serve many runs; set it
 * from any thread, reset it before reusing it.  Free it only after the runs
 * that use it have been fetched or freed.
 * Errors: PGB_E_INVAL (NULL), PGB_E_CUDA (pinned mapped allocation). */
typedef struct pgb_cancel pgb_cancel;
int pgb_cancel_create(pgb_cancel** out);
int pgb_cancel_set(pgb_cancel* c);
int pgb_cancel_reset(pgb_cancel* c);
int pgb_cancel_is_set(const pgb_cancel* c, int* set);
void pgb_cancel_free(pgb_cancel* c);

/* ------------------------------------------------------------------ run */
typedef struct {
    int32_t mode;          /* PGB_MODE_* (default PGB_MODE_PERSISTENT) */
    int32_t variant;       /* PGB_VAR_* (default PGB_VAR_AUTO) */
    int32_t per_vertex;    /* also count t[x] per vertex (default 1) */
    int32_t per_triple;    /* PLAIN mode: keep one count per queued triple */
    int32_t use_graph;     /* capture the launches in a CUDA graph (default 0) */
    int32_t order;         /* PGB_ORDER_* (default PGB_ORDER_WEIGHT) */
    uint64_t device_budget;/* offloaded blocks only: device bytes the run may
                              hold (resident arrays, counters, and two stream
                              slots that get the rest); 0 = 1 GiB slots.  A
                              budget below the resident arrays, or one whose
                              slots cannot hold the largest work item, gives
                              PGB_E_BUDGET.  Ignored for resident blocks. */
    uint32_t chunk_edges;  /* PERSISTENT: binary-search variant: edges per
                              dequeued chunk (0 = 64); hash variant: in-edges
                              per work item (0 = 16,384 for resident blocks,
                              4,096 for offloaded ones; larger than 65,535
                              counts as 65,535).  A per-part run uses both
                              kernels, and a value set here applies to both:
                              leave it 0 unless one variant is forced */
    uint32_t hash_threads; /* hash variant: threads per CTA, 128 (8 CTAs per
                              SM, bitmaps over fewer than 131,072 ranks), 256
                              (4 per SM, 262,144 ranks) or 512 (2 per SM,
                              524,288 ranks); 0 = autotuned by vertex count:
                              128 below 2^24 vertices, 256 below 2^26, else
                              512 (128 always for column-offloaded blocks) */
    pgb_cancel* cancel;    /* stop token read by the run's kernels, or NULL */
    uint32_t host_threads; /* HYBRID: host threads (0 = all hardware threads) */
    uint32_t host_share_ppm;/* HYBRID: cut-off, the host's share of the estimated
                              work in parts per million (0 = 1000, i.e. 0.1%;
                              at most 10^6: everything on the host) */
    uint32_t hash_min_lookups; /* AUTO: a head part takes the hash kernel at
                              this many lookups per edge or more (0 = 32) */
    int32_t dense_core;    /* PERSISTENT, resident blocks: the top block of
                              the degree order counted densely on the tensor
                              cores (below).  0: autotuned with PGB_VAR_AUTO,
                              none otherwise; > 0: that many top ranks
                              (rounded up to a multiple of 256, at most n);
                              < 0: none.  HYBRID runs take it too (the
                              host kernel skips its in-edges); streamed runs
                              of the index tier when it fits in half the
                              device budget; PLAIN runs and the column tier
                              never. */
} pgb_tc_opts;

void pgb_tc_opts_default(pgb_tc_opts* o);

/* Section 3.6 device kernel over every queued block tuple, then the
 * Section 3.3 reduction.  Enqueued on `stream`; the result handle is
 * ready when pgb_tc_result_get returns.  Errors: PGB_E_INVAL (bad opts),
 * PGB_E_BUDGET, PGB_E_NOMEM, PGB_E_CUDA. */
int pgb_tc_run(const pgb_blocks* b, const pgb_tc_opts* opts, void* stream, pgb_tc_result** out);

/* Wait for the run and fetch results (Section 3.3: the reduce_dev result of
 * the kernel, n_t in Listing 5, and its per-vertex form).  total: global
 * triangle count (may be NULL).  per_vertex: n uint64 counts t[x] indexed by ORIGINAL vertex ID
 * (may be NULL; PGB_E_STATE if the run had per_vertex = 0).  Fails with
 * PGB_E_CANCELLED, writing nothing, when a kernel of the run stopped early
 * on its cancel token. */
int pgb_tc_result_get(pgb_tc_result* r, uint64_t* total, uint64_t* per_vertex, int mem);

/* PLAIN mode with per_triple = 1: counts[t] for queue entry t (T entries). */
int pgb_tc_result_triples(pgb_tc_result* r, uint64_t* counts, int mem);

/* The dense top block of a run (pgb_tc_opts.dense_core). */
typedef struct {
    uint32_t ranks;            /* the block's ranks (0: no block) */
    uint32_t reserved;
    uint64_t triangles;        /* triangles with all three vertices in the block */
    uint64_t lookups_skipped;  /* lookups the intersection kernels left to the block
                                  (exact when ranks is a multiple of 1024, else 0) */
    double gemm_flop;          /* floating-point operations of its A·A strips */
    float ms;                  /* device time of the dense count (-1: graph replay) */
    float reserved2;
} pgb_dense_core_info;

/* Synchronises the run's stream.  Errors: PGB_E_INVAL. */
int pgb_tc_result_dense_core(pgb_tc_result* r, pgb_dense_core_info* out);

/* The variant that ran (PGB_VAR_BSEARCH, PGB_VAR_MERGE, PGB_VAR_HASH, or
 * PGB_VAR_MIXED when the autotuner chose differently for different parts). */
int pgb_tc_result_variant(pgb_tc_result* r, int* variant);

/* Per-part choice of the run: *p = parts; variants (may be NULL; p entries)
 * gets, for each head part j, the kernel that counted the triangles whose
 * middle vertex lies in V_j (PGB_VAR_HASH, PGB_VAR_BSEARCH, PGB_VAR_MERGE,
 * or PGB_VAR_HOST for the host kernel of a HYBRID run).
 * Errors: PGB_E_INVAL (NULL r or p). */
int pgb_tc_result_part_variants(pgb_tc_result* r, uint32_t* p, int32_t* variants);

/* HYBRID runs: the host kernel's wall time in milliseconds (the host copy of
 * the graph included on the first hybrid run of a partition), the in-edges
 * and parts it counted, and its threads; all 0 for other runs.  Any output
 * pointer may be NULL.  Errors: PGB_E_INVAL (NULL r). */
int pgb_tc_result_hybrid(pgb_tc_result* r, float* host_ms, uint64_t* host_in_edges, uint32_t* host_parts,
                         uint32_t* host_threads);

/* Streamed runs: host-to-device bytes copied (index slices, work items and,
 * for column-offloaded blocks, column slices), the number of chunks (pieces
 * for column-offloaded blocks) and, when slice_loads is not NULL, the column
 * slices copied in (cache misses); all 0 for a run on resident blocks. */
int pgb_tc_result_stream(pgb_tc_result* r, uint64_t* bytes, uint32_t* chunks, uint32_t* slice_loads);

/* Device time of the counting kernels of this run in milliseconds (CUDA
 * events around the launches on the run's stream; for a streamed run this
 * includes the copies it waits for); valid after get. */
int pgb_tc_result_kernel_ms(pgb_tc_result* r, float* ms);

void pgb_tc_result_free(pgb_tc_result* r);

/* One call: load + partition + run + fetch.  per_vertex may be NULL. */
int pgb_tc_count_edges(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t p,
                       int cut_rule, const pgb_tc_opts* opts, int mem, void* stream, uint64_t* total,
                       uint64_t* per_vertex);

/* ---------------------------------------------------------------- serve */
/* A serve loop for triangle-count jobs on graphs of mixed sizes (the paper
 * runs one computation at a time, Section 4.1; serving is this library's
 * extension of the same path).  Jobs are raw edge lists.  Batch threads
 * admit queued jobs in arrival order while the estimated device bytes of
 * admitted jobs stay within budget_bytes.
 *   PGB_SERVE_BATCHED: continuous batching.  Each of `max_inflight` batch
 *     threads takes the queued jobs that fit (up to max_batch_jobs jobs and
 *     batch_edges raw edges; a larger job runs alone) and counts them as ONE
 *     graph, the disjoint union of the jobs: one ingest, one degree order,
 *     one partition and one persistent counting launch whose block tuples
 *     interleave all the jobs'.  A job's per-vertex counts are its slice of
 *     the union's and its total a third of their sum.  Jobs arriving while a
 *     batch runs join the next one; batches of different threads overlap on
 *     the device.
 *   PGB_SERVE_SERIAL: one thread, one job per batch (the baseline).
 * Results are bit-identical to pgb_tc_run on each graph alone.  A job with
 * an endpoint >= n fails alone (PGB_E_INVAL at wait).  The server keeps its
 * own CUDA streams and threads on the device current at create; its threads
 * and queued device inputs take device memory from a stream-ordered memory
 * pool of the server's own (cudaMemPoolCreate), which keeps freed memory
 * mapped for the next batch until pgb_server_destroy; never from hooks set
 * with pgb_set_allocator. */
typedef struct pgb_server pgb_server;

#define PGB_SERVE_BATCHED 0
#define PGB_SERVE_SERIAL  1

#define PGB_JOB_QUEUED    0
#define PGB_JOB_RUNNING   1
#define PGB_JOB_DONE      2
#define PGB_JOB_FAILED    3
#define PGB_JOB_CANCELLED 4

typedef struct {
    uint64_t budget_bytes;    /* HBM admission budget (0 = 64 GiB) */
    uint32_t max_inflight;    /* BATCHED: batch threads (0 = 1, at most 16; the default is 1, best
                                 for small jobs; with large jobs from host memory, more threads
                                 overlap one batch's input copy and build with others' counting);
                                 SERIAL uses 1 */
    uint32_t p;               /* parts per dimension of a batch's graph (0 = 8, capped at n) */
    int32_t mode;             /* PGB_SERVE_* */
    int32_t per_vertex;       /* also return per-vertex counts */
    uint32_t max_batch_jobs;  /* BATCHED: jobs per batch (0 = 256, at most 4096) */
    uint32_t batch_edges;     /* BATCHED: raw edges per batch (0 = 2^27) */
    uint32_t reserved[8];
} pgb_server_opts;

typedef struct {
    uint64_t submitted, done, failed, cancelled, queued;
    uint64_t batches;          /* counting launches (BATCHED mode) */
    uint64_t jobs_in_batches;  /* jobs counted by those launches */
    uint64_t bytes_in_use;     /* estimated device bytes of admitted jobs */
} pgb_server_info;

void pgb_server_opts_default(pgb_server_opts* o);

/* The admission estimate of one job's device bytes (m raw edges, n vertices). */
uint64_t pgb_server_job_bytes(uint64_t m, uint32_t n);

/* Start a server.  Errors: PGB_E_INVAL (bad opts), PGB_E_CUDA. */
int pgb_server_create(const pgb_server_opts* opts, pgb_server** out);

/* Queue one job; src/dst (m raw pairs, IDs < n) are copied before return.
 * Host arrays (mem = PGB_MEM_HOST) are copied into host memory; device
 * arrays (PGB_MEM_DEVICE) into a device buffer of 8 bytes per raw edge that
 * the job holds while queued (outside the admission budget), copied on the
 * legacy default stream: after work the caller queued there, while writes
 * on non-blocking streams must be complete before the call.
 * Errors: PGB_E_BUDGET (the job can never fit the budget), PGB_E_INVAL,
 * PGB_E_STATE (server shutting down), PGB_E_CUDA.  Vertex IDs >= n make the
 * job fail. */
int pgb_server_submit(pgb_server* s, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, int mem,
                      uint64_t* job_id);

/* Queue one job on arrays that the server borrows instead of copying:
 * src/dst (m raw pairs, IDs < n) in device memory of the server's device
 * (mem = PGB_MEM_DEVICE) or in host memory (PGB_MEM_HOST; pinned memory
 * makes the batch's copy asynchronous and at the link's speed).  They must
 * be fully written before the call (a producer stream synchronised) and stay
 * valid and unchanged until pgb_server_wait for the job has returned, or
 * the server is destroyed.  The job's batch copies them to the device on its
 * own stream when it starts (the copy is part of the job's latency); submit
 * itself queues no device work, so it does not wait behind kernels already
 * running.  Errors as pgb_server_submit. */
int pgb_server_submit_borrowed(pgb_server* s, const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                               int mem, uint64_t* job_id);

/* Hold (paused != 0) or resume admission: while held, queued jobs stay
 * queued; jobs already admitted continue. */
int pgb_server_pause(pgb_server* s, int paused);

/* State of a job (PGB_JOB_*). */
int pgb_server_poll(pgb_server* s, uint64_t job_id, int* state);

/* Wait (timeout_s < 0: without limit) and fetch: total, per-vertex counts
 * by original ID into a host array of n (may be NULL), seconds from submit
 * to completion (may be NULL).  A job that ended is forgotten after this
 * call.  Errors: PGB_E_TIMEOUT (not finished; the job stays), PGB_E_CANCELLED,
 * the job's own error if it failed. */
int pgb_server_wait(pgb_server* s, uint64_t job_id, double timeout_s, uint64_t* total, uint64_t* per_vertex,
                    double* latency_s);

/* Cancel: a queued job is dropped at once.  A job already on the device is
 * marked; once every job of its batch is marked (a SERIAL job is alone), the
 * batch's counting kernels are stopped through the batch thread's cancel
 * token.  Either way wait returns PGB_E_CANCELLED for the job. */
int pgb_server_cancel(pgb_server* s, uint64_t job_id);

int pgb_server_stats(pgb_server* s, pgb_server_info* out);

/* Stop: queued jobs are cancelled, batches on the device are stopped through
 * their cancel tokens, threads and streams are released. */
void pgb_server_destroy(pgb_server* s);

/* ------------------------------------------ block layout and storage */
/* Section 4.3.1: blocks get integer IDs, row-major by default, or along a
 * space-filling curve.  pgb_block_order writes the upper blocks (i <= j) of
 * a p x p partition, p(p+1)/2 pairs (i, j) into ij, in row-major or
 * Hilbert-curve order (cell (x = j, y = i) of the 2^k x 2^k grid with
 * 2^k >= p).  pgb_hilbert_index is the curve itself: the position of cell
 * (x, y) in a side x side grid (side a power of two).  Host-only; no GPU
 * needed.  Errors: PGB_E_INVAL. */
#define PGB_LAYOUT_ROWMAJOR 0
#define PGB_LAYOUT_HILBERT  1
int pgb_block_order(uint32_t p, int layout, uint32_t* ij);
int pgb_hilbert_index(uint32_t side, uint32_t x, uint32_t y, uint64_t* d);

/* Section 4.3.2: a block is a subgraph with block-local vertex IDs (rows
 * u - c_i, columns v - c_j), stored as CSR, COO or CCOO.  Inside the library
 * the kernels read blocks as slices of the oriented CSR; these calls
 * materialise one block A_ij for a caller:
 *   PGB_FMT_CSR:  a = offsets uint32[rows + 1], c = columns uint32[nnz]
 *   PGB_FMT_COO:  a = rows uint32[nnz],         c = columns uint32[nnz]
 *   PGB_FMT_CCOO: a = the non-empty rows uint32[nz], d = their offsets
 *                 uint32[nz + 1], c = columns uint32[nnz]
 * (d unused unless CCOO; rows of a row ascending, columns ascending in a
 * row).  pgb_blocks_block_info gives the block's shape, the bytes of each
 * format and `format`: the autotuned choice, the format with the fewest
 * bytes for this block (CCOO when most rows are empty, COO near one edge
 * per non-empty row, CSR otherwise; ties to CSR, then COO).  Both synchronise
 * (block_info on the blocks' own stream).  Errors: PGB_E_INVAL (NULL, i or j
 * >= p, bad format, NULL output for a non-empty block), PGB_E_STATE (columns
 * offloaded), PGB_E_NOMEM, PGB_E_CUDA. */
#define PGB_FMT_CSR  0
#define PGB_FMT_COO  1
#define PGB_FMT_CCOO 2
typedef struct {
    uint32_t rows, cols;      /* |V_i|, |V_j| */
    uint64_t nnz;             /* |A_ij| */
    uint32_t nonempty_rows;
    int32_t format;           /* the autotuned storage format */
    uint64_t bytes_csr, bytes_coo, bytes_ccoo;
} pgb_block_info;
int pgb_blocks_block_info(const pgb_blocks* b, uint32_t i, uint32_t j, pgb_block_info* out);
int pgb_blocks_export_block(const pgb_blocks* b, uint32_t i, uint32_t j, int format, uint32_t* a, uint32_t* c,
                            uint32_t* d, int mem, void* stream);

/* ----------------------------------------- other multi-block patterns */
/* Section 3.2 names k-clique finding and butterfly counting as the other
 * multi-block pattern computations.  Both count on the degree-ordered
 * oriented graph of `b` (resident blocks; PGB_E_STATE after
 * pgb_blocks_offload), synchronise `stream` and write *total (exact).
 *
 * pgb_k4_count: 4-cliques (four mutually adjacent vertices), each found
 *   once from its lowest edge (u, v): common out-neighbours w of u and v,
 *   then common out-neighbours of u, v and w above w.
 * pgb_c4_count: 4-cycles (four distinct vertices a - w - b - y - a, as
 *   subgraphs), each counted once at its highest-ranked vertex; on a
 *   bipartite graph these are its butterflies.  Holds up to 8 GiB of
 *   per-CTA counter arrays (n words each) while it runs.
 * Errors: PGB_E_INVAL (NULL), PGB_E_STATE, PGB_E_NOMEM, PGB_E_CUDA. */
int pgb_k4_count(const pgb_blocks* b, void* stream, uint64_t* total);
int pgb_c4_count(const pgb_blocks* b, void* stream, uint64_t* total);

/* ------------------------------------ single-block bulk-synchronous runs */
/* Section 3.2's single-block bulk-synchronous execution mode on the same
 * block store: each block-list holds one block and every iteration visits
 * every edge.  Both calls need resident blocks (PGB_E_STATE after
 * pgb_blocks_offload), synchronise `stream`, and allocate their working
 * arrays from the library allocator.
 *
 * pgb_cc_run: connected components by Shiloach-Vishkin (Section 3.4):
 *   hook launches over the oriented edges (a root is hooked below the root
 *   of smaller original ID, by compare-and-swap) alternate with link
 *   launches (pointer jumping) until a hook launch hooks nothing.  labels
 *   (n entries, host or device per `mem`) gets, for each ORIGINAL vertex ID,
 *   the smallest original ID in its component; iterations and components
 *   (both may be NULL) get the hook rounds and the number of components. */
int pgb_cc_run(const pgb_blocks* b, void* stream, uint32_t* labels, int mem, uint32_t* iterations,
               uint64_t* components);

/* pgb_pagerank_run: PageRank (Section 5.2.1) of the undirected graph in
 * double precision: r_0 = 1/n, r_t+1(v) = (1 - d)/n + d * sum over
 * neighbours u of r_t(u) / deg(u) (degree-0 vertices pass nothing on);
 * stops after the first iteration whose L1 change is below tol, or after
 * max_iter iterations.  Each vertex pulls over its row and its in-edges (no
 * atomics).  ranks (n entries, host or device) gets r by ORIGINAL vertex ID;
 * iterations and last_change may be NULL.  Defaults (the paper's): damping
 * 0.85, tol 1e-4, max_iter 20.  Errors: PGB_E_INVAL (NULL b or ranks,
 * damping outside [0, 1], negative tol), PGB_E_STATE, PGB_E_NOMEM,
 * PGB_E_CUDA. */
typedef struct {
    double damping;
    double tol;
    uint32_t max_iter;
    uint32_t reserved[3];
} pgb_pagerank_opts;

void pgb_pagerank_opts_default(pgb_pagerank_opts* o);
int pgb_pagerank_run(const pgb_blocks* b, const pgb_pagerank_opts* opts, void* stream, double* ranks, int mem,
                     uint32_t* iterations, double* last_change);

/* ------------------------------------------------- no-allocation count */
/* The paper has no counterpart to this call.  It is for callers that must
 * not allocate device memory while they run: code whose host framework
 * hands out all device memory from its own pool and forbids any other
 * allocation, and latency-critical loops that cannot take the device-wide
 * synchronisation cudaMalloc / cudaFree may cause.  It allocates nothing:
 * no cudaMalloc, no cudaFree, no allocator callback.  Its working memory (a
 * work cursor, per-CTA partial counts, a per-vertex accumulator of
 * PGB_NOALLOC_MAX_VERTICES entries and a bitmap of as many bits, about
 * 8.1 MiB) is one fixed device array inside the library, held on every GPU
 * that loads the library until the process exits.
 *
 * Input: an already degree-ordered, upper-oriented graph in device memory
 * (e.g. from PGB_EXPORT_ROWPTR narrowed to uint32 and PGB_EXPORT_COL):
 *   rowptr uint32[n+1] with rowptr[0] = 0, rowptr[n] = m, non-decreasing;
 *   col    uint32[m] with row u listing its out-neighbours, each > u and
 *          < n, strictly ascending;
 *   perm   uint32[n] rank -> original ID (a permutation of 0..n-1), or NULL
 *          to index output by rank (perm is only read when per_vertex is
 *          not NULL).
 * Output (device memory, written, not accumulated): total uint64[1];
 *   per_vertex uint64[n] or NULL.
 * Counts equal those of pgb_tc_run on the same graph.
 * The call checks every rule above on the device (before it returns, with
 * reads that stay inside the arrays) and fails with PGB_E_INVAL naming the
 * rule that was broken; outputs are then undefined.  It returns after its
 * work on `stream` has finished.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) for that device; make that
 * first call before any stream capture begins.  Every call on a device
 * shares the one array and clears what it needs at the start, so calls
 * whose work overlaps on the GPU (other streams or threads) race and give
 * wrong counts: serialise them.
 * Errors: PGB_E_INVAL (n > PGB_NOALLOC_MAX_VERTICES, NULL pointers, a
 * broken input rule), PGB_E_OVERFLOW (m >= 2^32), PGB_E_CUDA. */
#define PGB_NOALLOC_MAX_VERTICES (1u << 20)
int pgb_tc_count_oriented_noalloc(uint32_t n, uint64_t m, const uint32_t* rowptr, const uint32_t* col,
                                  const uint32_t* perm, unsigned long long* total,
                                  unsigned long long* per_vertex, void* stream);

/* ----------------------------------------------------------------- misc */
const char* pgb_last_error(void);   /* thread-local; never NULL */
const char* pgb_version(void);

/* Number of the library's own CUDA kernels launched by this process so far
 * (calls into library primitives such as CUB radix sorts are not counted). */
uint64_t pgb_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* PGABB_H */
