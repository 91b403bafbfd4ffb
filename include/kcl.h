/*
 * kcl.h — C ABI of the GB300 k-clique listing library (SDegree and BitCol,
 * with Pre-Core and Pre-List), after "Efficient k-clique Listing with Set
 * Intersection Speedup".
 *
 * Problem (Section III-A, Definition 2): given an undirected simple graph
 * G(V, E) and an integer k >= 3, find every k-vertex subset whose vertices
 * are pairwise adjacent.  The library counts them exactly, and in listing
 * mode also writes each one and returns an order-independent checksum.
 *
 * Conventions shared by every call
 *  - Input graph: symmetric CSR.  row_ptr is uint64[n+1] with row_ptr[0] = 0,
 *    col is uint32[row_ptr[n]]; every row strictly ascending (so no duplicate
 *    edges), no self-loops, every id < n, and v in row u iff u in row v.
 *    Anything else is rejected with KCL_EINVAL and nothing is kept.
 *  - Pointers are plain host or device addresses; no framework types cross
 *    this boundary.  `stream` is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream).  Every call is ordered on the graph's stream and
 *    returns only when its results are on the host.
 *  - Ownership: the library copies the input graph into device memory it
 *    owns (freed by kcl_free_graph).  Output buffers (ring, per-root arrays)
 *    belong to the caller.
 *  - Errors never leave the device trapped: device-side checks record a
 *    status word that the call turns into its return code.
 *  - Not thread-safe per graph: calls on one kcl_graph must not overlap.
 *
 * Checksum: for a clique with ids v_1 < ... < v_k (the caller's original
 * ids), H = f(... f(f(G ^ k) ^ v_1) ... ^ v_k) with G = 0x9E3779B97F4A7C15
 * and f the SplitMix64 output finaliser (Steele, Lea & Flood, OOPSLA 2014);
 * the checksum is the sum of H over all cliques mod 2^64.  The paper defines
 * no checksum; this one does not depend on listing order or scheduling.
 */
#ifndef KCL_H
#define KCL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kcl_graph kcl_graph;

typedef enum {
    KCL_OK = 0,
    KCL_EINVAL = 1,     /* bad argument or malformed graph */
    KCL_ENOMEM = 2,     /* device or host allocation failed */
    KCL_EOVERFLOW = 3,  /* the exact count does not fit in 64 bits */
    KCL_ETRUNC = 4,     /* listing: more cliques than ring capacity (wrap = 0) */
    KCL_ETIMEOUT = 5,   /* a bounded device-side wait gave up, or the time limit passed */
    KCL_ECUDA = 6,      /* a CUDA runtime call failed */
    KCL_EABORT = 7,     /* aborted by the caller */
    KCL_ELIMIT = 8,     /* a built-in size limit was exceeded (see kcl_strerror) */
    KCL_ESIZE = 9       /* input larger than the fixed scratch of an allocation-free call */
} kcl_status;

/* Vertex orderings of the two algorithms.
 * KCL_ORDER_DEGREE: SDegree (Algorithm 5, Section VI).  Pre-Core, Pre-List,
 *   then the DAG u -> v iff (d_u, u) < (d_v, v) with degrees of the reduced
 *   graph, and SDegreeList with sorted-list intersections N+_v and C (on
 *   the out-neighbour-reduced lists; dense subproblems may run the same
 *   intersections on bit-rows, see kcl_tuning).
 * KCL_ORDER_COLOR: BitCol (Algorithm 6, Section VII).  Pre-Core, Pre-List,
 *   the degeneracy DAG (bulk peel rounds: eta = (round, id)), then for each
 *   root the subgraph induced by its out-neighbours, greedy colour ordering
 *   (Section VII-A), bitmap encoding (Section VII-C) and BitColList with
 *   colour pruning. */
typedef enum { KCL_ORDER_DEGREE = 0, KCL_ORDER_COLOR = 1 } kcl_ordering;

/* Largest supported k (the paper requires k >= 3, Section III-A). */
#define KCL_MAX_K 32
/* Largest supported out-degree of a root in the oriented graph. */
#define KCL_MAX_OUTDEG 65535

/* Caller-owned device buffer for listed cliques: `capacity` records of k
 * uint32 ids each, ids sorted ascending within a record; record order is
 * unspecified.  wrap = 0: writing stops at capacity and the call returns
 * KCL_ETRUNC (count and checksum still cover every clique).  wrap = 1:
 * records land at (index mod capacity); the ring keeps an arbitrary subset
 * and the call returns KCL_OK. */
typedef struct {
    uint32_t *ids;
    uint64_t capacity;
    int wrap;
} kcl_ring;

/* Copy a graph in and validate it (Section III-A problem input).
 * n: vertex count (0 allowed).  row_ptr/col: CSR as above, host memory if
 * on_device = 0, device memory of the current device if on_device = 1
 * (read in order on `stream`, after the caller's earlier work there).
 * stream: cudaStream_t (void*) used for this graph from now on.
 * out: receives the new graph handle; NULL on error.
 * Returns KCL_EINVAL for a malformed graph, KCL_ENOMEM, KCL_ECUDA. */
kcl_status kcl_load_csr(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                        int on_device, void *stream, kcl_graph **out);

/* Release a graph and all device memory it owns.  NULL is ignored. */
void kcl_free_graph(kcl_graph *g);

/* A second handle on a loaded graph: it shares g's device CSR (g must
 * outlive it) but has its own scratch and stream, so calls on the two
 * handles may run concurrently.  Free it with kcl_free_graph (the CSR stays
 * with g).  Library facility; the paper has none. */
kcl_status kcl_graph_view(const kcl_graph *g, void *stream, kcl_graph **out);

/* Change the stream that later calls on g are ordered on. */
kcl_status kcl_set_stream(kcl_graph *g, void *stream);

uint32_t kcl_num_vertices(const kcl_graph *g);
uint64_t kcl_num_edges(const kcl_graph *g);   /* undirected edges */

/* Count the k-cliques of g (Algorithms 5 and 6 with Pre-Core and Pre-List,
 * Sections V-VII, unless switched off by kcl_set_options).  k in [3,
 * KCL_MAX_K].  *count receives the exact count.
 * KCL_EOVERFLOW if it exceeds 2^64 - 1; KCL_ELIMIT if a root's out-degree
 * exceeds KCL_MAX_OUTDEG. */
kcl_status kcl_count(kcl_graph *g, uint32_t k, kcl_ordering ord, uint64_t *count);

/* List the k-cliques of g into `ring` (device memory, see kcl_ring) and
 * return the exact count, the checksum and the number of records written
 * (min(count, capacity) without wrap; min(count, capacity) with wrap too).
 * The output lines of Algorithms 4, 5 and 6: each clique once, as its
 * original ids sorted ascending. */
kcl_status kcl_list(kcl_graph *g, uint32_t k, kcl_ordering ord, const kcl_ring *ring,
                    uint64_t *count, uint64_t *checksum, uint64_t *written);

/* Per-root counts, for checking against an independent implementation.
 * per_root: device uint64[n], overwritten with the number of k-cliques whose
 * lowest vertex in the ordering eta is that vertex (Theorem 1: each clique is
 * found once, from its eta-first vertex).  Cliques reported by Pre-List are
 * not attributed to a root; *prelist_count receives their number and
 * *count the total. */
kcl_status kcl_count_per_root(kcl_graph *g, uint32_t k, kcl_ordering ord, uint64_t *per_root,
                              uint64_t *count, uint64_t *prelist_count);

/* Per-root counts of the given roots only, for checking large graphs root by
 * root against an independent implementation (whose full count may be out of
 * reach).  The front end runs on the whole graph; then only the roots listed
 * in `roots` (host uint32[n_roots], vertex ids < n; vertices that are not
 * roots under `ord` -- removed by Pre-Core or Pre-List, or d+ < k-1 -- are
 * skipped) are expanded.  per_root: device uint64[n], overwritten as in
 * kcl_count_per_root (zero for every other vertex); *count receives their
 * sum (Pre-List cliques are not included).  Errors: those of kcl_count,
 * KCL_EINVAL for an id >= n. */
kcl_status kcl_count_roots(kcl_graph *g, uint32_t k, kcl_ordering ord, const uint32_t *roots,
                           uint32_t n_roots, uint64_t *per_root, uint64_t *count);

/* Intermediate results of the front end, for stage-by-stage checks.
 * Any pointer may be NULL.  Host buffers of n elements:
 *   alive_core:  1 iff the vertex survives Pre-Core (the (k-1)-core, Alg. 3)
 *   alive_final: 1 iff it also survives Pre-List (Algorithm 4)
 *   outdeg:      out-degree in the DAG of `ord` (0 for removed vertices)
 *   key:         ordering key (reduced degree, or degeneracy peel round)
 * prelist_count: k-cliques reported by Pre-List; max_outdeg: Delta. */
kcl_status kcl_stage_info(kcl_graph *g, uint32_t k, kcl_ordering ord, uint8_t *alive_core,
                          uint8_t *alive_final, uint32_t *outdeg, uint32_t *key,
                          uint64_t *prelist_count, uint32_t *max_outdeg);

/* The colouring BitCol gives one root's subproblem, for checking it against
 * an independent implementation (Section VII-A, Example 6 / Table II): the
 * front end of KCL_ORDER_COLOR runs for k (Pre-Core, Pre-List, degeneracy
 * DAG), then the listing kernels' own subproblem builder colours G_root, the
 * subgraph induced by root's out-neighbours, greedily in (degree in G_root
 * descending, id ascending) order with colours from 1.
 * *outdeg receives d+ of root (0 if it was removed by Pre-Core or Pre-List
 * or has no out-neighbours; nothing else is written then).  nbr and colour:
 * host uint32[capacity]; nbr[i] is the i-th out-neighbour in ascending id,
 * colour[i] its colour.  Errors: KCL_EINVAL (bad argument, root >= n, or
 * capacity < d+), KCL_ELIMIT (d+ above 4096), KCL_ENOMEM, KCL_ECUDA.
 * Allocates its own temporary device scratch; for tests and diagnostics. */
kcl_status kcl_root_colouring(kcl_graph *g, uint32_t k, uint32_t root, uint32_t capacity,
                              uint32_t *nbr, uint32_t *colour, uint32_t *outdeg);

/* Batched counting (the batched form of the workload; the paper has none).
 * A kcl_batch owns device scratch that is reused across calls; create it on
 * the device and stream the batch's graphs live on.
 * kcl_count_batch: gs[i] (loaded graphs, same device), ks[i] in [3,
 *   KCL_MAX_K], ords[i] per graph.  The graphs of each ordering are joined as
 *   one disjoint union on the device, each vertex keeping the k of its graph,
 *   and counted by a single pass of the pipeline (Algorithms 3-6: Pre-Core
 *   and Pre-List with each graph's k, one listing launch per out-degree class
 *   whose persistent CTAs pull the roots of every graph from one queue); each
 *   root's count is attributed to its vertex and summed per graph.  counts:
 *   host uint64[G], receives each graph's exact
 *   k-clique count.  checksums: host uint64[G] or NULL; when given, each
 *   graph's listing checksum (as kcl_list) is computed too.
 * Errors: KCL_EINVAL, KCL_ENOMEM, KCL_ECUDA, KCL_ELIMIT (union beyond 2^32
 *   vertices or edges, or a root above the out-degree limit). */
typedef struct kcl_batch kcl_batch;
kcl_status kcl_batch_create(void *stream, kcl_batch **out);
void kcl_batch_free(kcl_batch *b);
kcl_status kcl_count_batch(kcl_batch *b, kcl_graph *const *gs, const uint32_t *ks,
                           const kcl_ordering *ords, uint32_t G, uint64_t *counts,
                           uint64_t *checksums);
/* Time limit of each pipeline pass of later kcl_count_batch calls on b, as
 * kcl_set_time_limit (0 = none): a pass that exceeds it returns
 * KCL_ETIMEOUT for the whole call. */
kcl_status kcl_batch_set_time_limit(kcl_batch *b, uint64_t ms);

/* Serving loop (a library facility; the paper has none).  Graphs stay
 * resident (the caller's loaded handles, which must outlive the server);
 * `slots` worker threads each own a CUDA stream and scratch, so admitted
 * queries run concurrently and their work overlaps on the device.  A query
 * is admitted while its scratch estimate fits in scratch_budget_bytes (a
 * query larger than the whole budget runs alone).  Continuous batching: a
 * free worker takes the oldest query; queries on graphs with at most
 * small_nnz CSR entries are gathered with the other queued small-graph
 * queries into one batched pass (as kcl_count_batch), and queued copies of
 * the query it takes share its result.  Results are exact: equal to the same
 * query run alone with kcl_count / kcl_list.
 * Times in kcl_server_result are seconds on kcl_server_clock's steady clock
 * (submission, start of the pass that answered it, completion); `batch` is
 * the number of queries that pass answered. */
typedef struct kcl_server kcl_server;
typedef struct {
    uint64_t count;
    uint64_t checksum;   /* list = 1 queries; 0 otherwise */
    double submit_s, start_s, done_s;
    uint32_t batch;
    kcl_status status;
} kcl_server_result;
kcl_status kcl_server_create(uint32_t slots, uint64_t scratch_budget_bytes, uint64_t small_nnz,
                             kcl_server **out);
/* Graphs may be added at any time, also while queries run: a query keeps the
 * handle its id named when it was submitted. */
kcl_status kcl_server_add_graph(kcl_server *s, kcl_graph *g, uint32_t *id);
/* list = 0: count only; list = 1: count + checksum (no ring output). */
kcl_status kcl_server_submit(kcl_server *s, uint32_t graph, uint32_t k, kcl_ordering ord, int list,
                             uint64_t *ticket);
kcl_status kcl_server_poll(kcl_server *s, uint64_t ticket, int *done, kcl_server_result *out);
kcl_status kcl_server_wait(kcl_server *s, uint64_t ticket, kcl_server_result *out);
double kcl_server_clock(const kcl_server *s);
/* Time limit per query of the passes a worker starts from now on, as
 * kcl_set_time_limit (0 = none, the default): a single-query pass gets ms, a
 * batched pass of n gathered small-graph queries n * ms.  The queries of a
 * pass that exceeds its limit finish with status KCL_ETIMEOUT and no count. */
kcl_status kcl_server_set_time_limit(kcl_server *s, uint64_t ms);
/* Finishes queued work, stops the workers and frees the server's scratch. */
void kcl_server_destroy(kcl_server *s);

/* Device time of the stages of the last kcl_count / kcl_list call on g, in
 * milliseconds, measured with CUDA events on the graph's stream when timing
 * is enabled (kcl_enable_timing).  stage ids: 0 Pre-Core, 1 Pre-List,
 * 2 orientation, 3 listing kernels (SDegreeList / subgraph build + BitColList),
 * 4 whole call.  launches[i] = kernel launches in stage i.
 * The listing stage is split by root class: the roots are grouped by their
 * out-degree d+_u (one listing launch per non-empty group), and for c <
 * n_classes group c holds class_roots[c] roots with class_lo[c] <= d+_u <=
 * class_hi[c], listed by one launch that took class_ms[c] milliseconds
 * (0 roots: no launch, class_ms[c] = 0).  Batches leave n_classes = 0. */
#define KCL_NUM_STAGES 5
#define KCL_MAX_CLASSES 16
typedef struct {
    float ms[KCL_NUM_STAGES];
    uint32_t launches[KCL_NUM_STAGES];
    uint32_t n_classes;
    uint32_t class_lo[KCL_MAX_CLASSES];
    uint32_t class_hi[KCL_MAX_CLASSES];
    uint32_t class_roots[KCL_MAX_CLASSES];
    float class_ms[KCL_MAX_CLASSES];
} kcl_timing;
kcl_status kcl_enable_timing(kcl_graph *g, int enable);
kcl_status kcl_last_timing(const kcl_graph *g, kcl_timing *t);
/* The same for a batch: stage times summed over the (k, ordering) groups of
 * the last kcl_count_batch call; *groups receives the number of groups. */
kcl_status kcl_batch_enable_timing(kcl_batch *b, int enable);
kcl_status kcl_batch_last_timing(const kcl_batch *b, kcl_timing *t, uint32_t *groups);

/* Time limit of the listing stage of later kcl_count / kcl_list /
 * kcl_count_per_root calls on g, in milliseconds (0 = none, the default).
 * The paper runs every experiment under a wall-clock limit and reports
 * "exceeds the limit" (Section IX); here the listing kernels stop taking
 * roots and subtrees once the device's global timer passes the limit, and
 * the call returns KCL_ETIMEOUT (its count is then incomplete and not
 * returned).  The front end (Pre-Core, Pre-List, orientation) is not
 * limited. */
kcl_status kcl_set_time_limit(kcl_graph *g, uint64_t ms);

/* Ablation switches (Section IX, the preprocessing and pruning studies): a
 * bitwise OR of
 *   KCL_OPT_NO_PRECORE      skip Pre-Core (Algorithm 3): every vertex stays;
 *   KCL_OPT_NO_PRELIST      skip Pre-List (Algorithm 4): clique components
 *                           are listed by the DFS like any other part;
 *   KCL_OPT_NO_COLOR_PRUNE  BitCol expands every candidate instead of only
 *                           those of colour >= l (Lemma 1).
 * Counts, checksums and listings do not change; only the work does.  A graph
 * starts with 0 (everything on).  Unknown bits: KCL_EINVAL. */
#define KCL_OPT_NO_PRECORE 1u
#define KCL_OPT_NO_PRELIST 2u
#define KCL_OPT_NO_COLOR_PRUNE 4u
kcl_status kcl_set_options(kcl_graph *g, uint32_t flags);
kcl_status kcl_get_options(const kcl_graph *g, uint32_t *flags);

/* Device scratch the graph handle holds now (Section IX's memory study): the
 * per-call workspace (about 74 bytes per vertex and 2 per CSR entry, grown to
 * the largest graph seen) and the listing arena (shared-memory spill of the
 * largest subproblems, sized by k and the largest out-degree), in bytes.
 * The input CSR itself (8 (n+1) + 4 nnz bytes) is not included. */
kcl_status kcl_scratch_bytes(const kcl_graph *g, uint64_t *workspace, uint64_t *arena);

/* Tuning of the listing kernels (a library facility; the paper has no
 * counterpart).  Results never depend on it, only speed does.
 * sdegree_gallop[c] (counting) and sdegree_gallop_list[c] (listing): for the
 *   SDegree launch of out-degree class c (the same classes as kcl_timing's
 *   class split), a leaf (l = 2) intersects by galloping -- each pair
 *   (candidate, later candidate) searched in the candidate's list -- instead
 *   of merging when
 *     pairs * (6 lg + 10) * 10 < (sum of list lengths + pairs) * threshold
 *   (lg = bit length of the mean list length); 0 = always merge (default).
 * sdegree_bitmap[c]: bitmap-versus-list threshold for the CTA-per-root
 *   classes (d+ 129..1024): a root runs SDegreeList on the directed bit-rows
 *   of its reduced subproblem instead of its reduced lists when the rows fit
 *   in shared memory with enough warps and 16 * (list words) > t * (row
 *   words), t = sdegree_bitmap[c] (0 means the default t = 16: lists larger
 *   than rows; 0xFFFFFFFF = lists always).  Both forms compute the same
 *   intersections; only their representation differs.
 * sdegree_cta_warps[c], bitcol_cta_warps[c]: warps per subproblem for the
 *   CTA-per-root classes of each path: how many of the CTA's warps walk the
 *   root's first-level
 *   children (the EdgeParallel units of Section IX-C) after the shared build;
 *   0 = all of them (default), 1 = one warp walks the whole subtree
 *   (NodeParallel), k = at most k warps.
 * sdegree_split[c], bitcol_split[c]: work splitting of heavy roots across
 *   CTAs in the CTA-per-root classes (split depth 1: a root's first-level
 *   children, the edges <u, v> of Section IX-C, are the units).  A CTA that
 *   runs out of roots rebuilds the subproblem of a root still in progress on
 *   another CTA and takes over some of its children when at least t =
 *   split[c] of them are left; 0 = off (default).
 * A graph starts with the defaults; views and batches start with the
 * defaults too. */
typedef struct {
    uint32_t sdegree_gallop[KCL_MAX_CLASSES];
    uint32_t sdegree_gallop_list[KCL_MAX_CLASSES];
    uint32_t sdegree_bitmap[KCL_MAX_CLASSES];
    uint32_t sdegree_cta_warps[KCL_MAX_CLASSES];
    uint32_t bitcol_cta_warps[KCL_MAX_CLASSES];
    uint32_t sdegree_split[KCL_MAX_CLASSES];
    uint32_t bitcol_split[KCL_MAX_CLASSES];
} kcl_tuning;
kcl_status kcl_get_tuning(const kcl_graph *g, kcl_tuning *t);
kcl_status kcl_set_tuning(kcl_graph *g, const kcl_tuning *t);
/* Autotuner: runs kcl_count(g, k, ord) (listing = 0) or kcl_list(g, k, ord,
 * NULL, ...) (listing = 1) once per candidate setting, times every class
 * launch with CUDA events, and keeps for each class the fastest setting (a
 * later candidate must be 2% faster).  For KCL_ORDER_DEGREE it tunes
 * sdegree_bitmap first (candidates 0, 4, 64, 0xFFFFFFFF), then that mode's
 * galloping array (0, 40, 80, 160, 400); for both orderings it then tunes
 * that path's cta_warps array (0, 4, 8) and its split array (0, 2, 8, 32).
 * The tuning
 * is stored in g and copied to *out when out is not NULL.  Timing stays as
 * the caller left it.  Errors: those of kcl_count / kcl_list. */
kcl_status kcl_autotune(kcl_graph *g, uint32_t k, kcl_ordering ord, int listing, kcl_tuning *out);

/* Allocation-free degeneracy ordering (the paper has no counterpart; this is
 * a library facility).  Some callers must not allocate device memory from
 * inside their own loops: a serving loop whose latency budget cannot absorb
 * the device-wide synchronisation that cudaMalloc/cudaFree can cause, or a
 * host program whose device memory is owned by another allocator under a
 * fixed budget.  This call computes the same bulk-peel rounds as the
 * KCL_ORDER_COLOR front end (eta = (round, id); see kcl_stage_info's `key`)
 * without allocating anything: its scratch (peel degrees, two frontiers and a
 * control block, about 12 MiB) is a fixed array that every GPU loading the
 * library holds until the process exits.
 * n: vertices, at most KCL_NOALLOC_MAX_VERTICES (else KCL_ESIZE, nothing run).
 * row_ptr, col: the symmetric CSR graph in device memory (as for
 *   kcl_load_csr; not validated here).
 * alive: device uint8[n], 1 for the vertices to order.
 * degree: device uint32[n], each alive vertex's number of alive neighbours.
 * round_out: device uint32[n] (caller-owned), receives the peel round of each
 *   alive vertex and 0xFFFFFFFF for the others.
 * stream: cudaStream_t as void*.  The call is synchronous: after the launch
 * it copies the kernel's status word to the host and waits for the stream, so
 * it returns when round_out is ready.
 * The first call on a device looks up the scratch array's device address
 * (once per device, with that device current); make that first call before
 * any stream capture.  Every call on a device reuses the same array (the
 * control block is cleared at the start of each call), so calls that overlap
 * on the GPU race and must not be issued concurrently.
 * Errors: KCL_EINVAL (null pointer), KCL_ESIZE, KCL_ECUDA, KCL_ETIMEOUT. */
#define KCL_NOALLOC_MAX_VERTICES (1u << 20)
kcl_status kcl_degeneracy_order_noalloc(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                                        const uint8_t *alive, const uint32_t *degree,
                                        uint32_t *round_out, void *stream);

/* Measured per-SM rates of the instructions the listing kernels are bound by
 * (a measurement facility; the paper has none).  Each probe runs one CTA of
 * 1024 threads per SM with 8 independent dependency chains per thread and
 * times its loop with the SM's cycle counter, so every rate is per SM per SM
 * clock; sm_clock_mhz is the probe's cycles over its CUDA-event time.
 *   popc / lop3 / iadd: 32-bit population count, three-input logic op, add;
 *   bitjoin_words: the BitJoin word of Algorithm 6 as the kernels run it --
 *     a conflict-free 128-bit shared-memory read of a bit-row, a broadcast
 *     128-bit read of the candidate set, AND, POPC and accumulate per word;
 *   lds128_bytes: bytes of conflict-free 128-bit shared-memory loads;
 *   mix64: SplitMix64 rounds h = f(h ^ x) of the listing checksum.
 * Runs for a fraction of a second on `stream` (cudaStream_t as void*) and
 * allocates a few KB of device memory.  Errors: KCL_EINVAL, KCL_ENOMEM,
 * KCL_ECUDA. */
typedef struct {
    uint32_t num_sms;
    double sm_clock_mhz;
    double popc_per_sm_clk;
    double lop3_per_sm_clk;
    double iadd_per_sm_clk;
    double bitjoin_words_per_sm_clk;
    double lds128_bytes_per_sm_clk;
    double mix64_per_sm_clk;
} kcl_int_peaks;
kcl_status kcl_measure_int_peaks(void *stream, kcl_int_peaks *out);

/* Human-readable text for a status. */
const char *kcl_strerror(kcl_status s);

#ifdef __cplusplus
}
#endif

#endif /* KCL_H */
