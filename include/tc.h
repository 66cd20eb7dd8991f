/*
 * tc.h — C ABI of the GB300 exact triangle counter (libtc.so).
 *
 * Method: Wang & Owens, "Fast BFS-Based Triangle Counting on GPUs" (HPEC Graph Challenge 2019).  Triangle counting
 * is posed as matching the query graph Q = K3 in an undirected data graph G (Sec. II-A, Def. 1 and Def. 2) by an
 * all-source breadth-first traversal (Sec. III, Algorithm 1): every source u advances to its neighbours v, every v
 * advances to its neighbours w, and the 2-path u-v-w is kept only when the non-tree (closing) edge u-w exists.  A
 * total order on the vertices — the unique mapping order of Sec. III-A and the duplicate avoidance of Sec. III-C —
 * makes each triangle appear exactly once; this library orders vertices by (number of input pairs at the vertex,
 * id) and traverses only edges that go up in that order.  The answer is the number of matches |M|/|Q| (Algorithm 1, result line).
 *
 * Conventions for every entry point:
 *  - Status: each call returns a tc_status; nothing aborts the process.  tc_last_error() gives a message for the
 *    last failing call on the calling thread.
 *  - Streams: `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.  All device work of
 *    a call is ordered on that stream.
 *  - Ids: vertex ids are int32 in [0, n).  Counts are exact uint64.
 *  - Memory: every device buffer is obtained from the graph's allocator (tc_allocator; when none is given, a
 *    stream-ordered pool that the library keeps per device and that holds on to freed memory) and returned to it;
 *    the graph owns its buffers until tc_free.
 *  - Threads: a tc_graph may be used by one host thread at a time.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define TC_API __attribute__((visibility("default")))
#else
#define TC_API
#endif

typedef enum tc_status {
  TC_OK = 0,
  TC_ERR_INVALID_ARG = 1,  /* null pointer, negative size, bad flag, size above a stated limit */
  TC_ERR_OUT_OF_RANGE = 2, /* an edge endpoint outside [0, n) */
  TC_ERR_NO_MEMORY = 3,    /* the allocator returned NULL */
  TC_ERR_CUDA = 4,         /* a CUDA runtime call failed; see tc_last_error() */
  TC_ERR_TIMEOUT = 5,      /* a bounded device wait gave up */
  TC_ERR_INTERNAL = 6,     /* a device-side consistency check failed */
  TC_ERR_STATE = 7         /* call out of order, e.g. counting before tc_build */
} tc_status;

/* Where a caller's array lives. */
#define TC_PTR_HOST 0x1u
#define TC_PTR_DEVICE 0x2u

/* Device memory provider.  alloc returns a pointer aligned to at least 256 bytes that is usable in stream order
 * on `stream`, or NULL on failure; free releases it in stream order.  ctx is passed back unchanged. */
typedef struct tc_allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} tc_allocator;

typedef struct tc_graph tc_graph; /* opaque */

/* Sizes of a built graph, for reporting. */
typedef struct tc_graph_info {
  int64_t num_vertices;    /* n */
  int64_t num_input_pairs; /* pairs given to tc_load_edges */
  int64_t num_edges;       /* m: distinct undirected edges after dropping self-loops and repeats */
  int64_t csr_entries;     /* column entries of the oriented CSR, rows padded to a multiple of 4 */
  int64_t max_out_degree;  /* largest d+(u) in the orientation of tc_build */
  int64_t num_wedges;      /* W = sum over oriented edges u->v of d+(v): the candidate 2-paths u->v->w */
  int64_t active_sources;  /* sources with d+(u) >= 2 and at least one candidate 2-path */
  int64_t bin_warp;        /* sources handled one warp each */
  int64_t bin_block;       /* sources handled one thread block each */
  int32_t built;           /* 1 after tc_build */
  int32_t count_ctas;      /* CTAs of the fused counting kernel's launch for this graph on the current device (a
                              persistent grid: at most 2 per SM); 0 before tc_build */
  int64_t dense_rows;      /* rows N+(v) also stored as bitmaps over (v, n) (no more words than entries) */
  int64_t dense_wedges;    /* the part of num_wedges through dense rows (tested 128 ids per 16-byte word load) */
  int64_t dense_quads;     /* 16-byte bitmap words that tc_count reads for them: sum of d-(v) * quads(v) */
  int64_t bin_thread;      /* sources handled one lane each (few out-neighbours: each pair tested by a lookup) */
} tc_graph_info;

/*
 * tc_load_edges — take the data graph G (Sec. II-A: "inputs ... one data graph G"; Def. 1).
 *   src, dst     num_edges int32 endpoints; pair i is the undirected edge {src[i], dst[i]} ((u,v) and (v,u) are
 *                the same edge, Def. 1).  Host or device memory as `flags` says (exactly one of TC_PTR_HOST,
 *                TC_PTR_DEVICE).  Read during the call only: the caller keeps ownership and may free or reuse the
 *                arrays once the call returns.
 *   num_edges    >= 0 and < 2^32 - 1.
 *   num_vertices n >= 0; every endpoint must lie in [0, n), else TC_ERR_OUT_OF_RANGE and no graph is returned.
 *   alloc        device memory provider, or NULL for the library's per-device stream-ordered pool.  The
 *                struct is copied; its functions must stay valid until tc_free.
 *   out          receives the new graph handle (set to NULL on failure).
 * Self-loops and repeated pairs are accepted and removed by tc_build (the simple-graph reading of Def. 1).
 * Host arrays that are page-locked and mapped into the device's address space (cudaHostAlloc / pinned tensors)
 * are read by the device directly; other host arrays are copied through a device staging buffer.
 * Synchronises `stream` once (to report out-of-range ids).
 */
TC_API tc_status tc_load_edges(const int32_t* src, const int32_t* dst, int64_t num_edges, int64_t num_vertices,
                               uint32_t flags, const tc_allocator* alloc, void* stream, tc_graph** out);

/*
 * tc_build — the data structure and filtering steps before the traversal (Sec. III-B: CSR storage; Algorithm 1,
 * filtering: NE = degree, Sec. III-A; k-look-ahead pruning, Sec. III-C).  On the device: rank the vertices by
 * (number of input pairs at the vertex, self-loops excluded and repeats included; then id) — a total order that
 * follows the degree (the unique mapping order of Sec. III-A; any total order counts each triangle once, Sec.
 * III-C) — relabel every pair by rank so that it points up the order, sort and de-duplicate the pairs, build the
 * oriented CSR (int64 row offsets, int32 sorted column ids of ranks) and bin the sources u by their
 * candidate-2-path work.  Sources with d+(u) < 2 are dropped (they cannot be the first vertex of a triangle).
 * Frees the edge buffers.  Idempotent: a second call returns TC_OK.  Synchronises `stream`.
 */
TC_API tc_status tc_build(tc_graph* g, void* stream);

/* What tc_build_pruned removed. */
typedef struct tc_prune_stats {
  int64_t rounds;           /* rounds that removed at least one edge */
  int64_t edges_removed;    /* distinct undirected edges removed */
  int64_t vertices_removed; /* vertices that had an edge before pruning and have none after */
  int64_t reserved;
} tc_prune_stats;

/*
 * tc_build_pruned — tc_build with the NE filter applied until it settles (Sec. III-A: NE is the degree, and it is
 * updated after each filtering).  After the repeats are removed, each round drops every edge with an endpoint of
 * degree below 2 in the current graph (such a vertex lies in no triangle, so neither does the edge), until a round
 * removes nothing (the 2-core) or max_rounds rounds ran.  Counts, per-vertex counts and listings are unchanged;
 * tc_graph_get_info describes the pruned graph (num_edges = edges kept).
 *   max_rounds  >= 1: at most that many rounds; 0: until a round removes nothing, at most 65536 rounds (a long
 *               path loses only its two end edges per round); negative: TC_ERR_INVALID_ARG.
 *   stats       host pointer or NULL; zeroed when the graph was already built (nothing is re-run).
 * Each round waits for the GPU once.  Errors as tc_build.
 */
TC_API tc_status tc_build_pruned(tc_graph* g, int32_t max_rounds, tc_prune_stats* stats, void* stream);

/*
 * tc_count — the verification loop of Algorithm 1 for Q = K3, fused: for every source u, every v in N+(u) and
 * every w in N+(v), count the 2-path u->v->w when the closing edge u->w exists (Sec. III-A: the non-tree edge of
 * the triangle's spanning path).  *out_total receives T, the number of triangles (|M|/|Q|).  Requires tc_build
 * (else TC_ERR_STATE).  Blocks until *out_total (host memory) is valid.
 */
TC_API tc_status tc_count(tc_graph* g, uint64_t* out_total, void* stream);

/*
 * tc_count_device — tc_count without the host round trip: writes T to the device word *d_total (8-byte aligned
 * device memory; overwritten, not accumulated) in stream order and returns at once.  No allocation, no
 * synchronisation: the sequence can be captured in a CUDA graph.
 */
TC_API tc_status tc_count_device(tc_graph* g, uint64_t* d_total, void* stream);

/*
 * tc_count_intersect — the same count by the other family of GPU triangle counters: segmented intersection
 * (Sec. II-B: the operator that intersects the neighbour lists of each pair from two frontiers).  Every oriented
 * edge u -> v of the built graph contributes |N+(u) ∩ N+(v)|, one lane per edge, by galloping search over the
 * shorter list.  *out_total receives T (equal to tc_count).  Requires tc_build (else TC_ERR_STATE).  Blocks until
 * *out_total (host memory) is valid.
 */
TC_API tc_status tc_count_intersect(tc_graph* g, uint64_t* out_total, void* stream);

/*
 * tc_count_per_vertex — as tc_count, and also t(x), the number of triangles containing x, for every x in [0, n)
 * (the per-vertex view of the matches M of Algorithm 1).
 *   per_vertex  n uint64 entries, host or device memory as `flags` says (TC_PTR_HOST or TC_PTR_DEVICE);
 *               overwritten.
 *   out_total   host pointer for T, or NULL.
 * Blocks until both outputs are valid.
 */
TC_API tc_status tc_count_per_vertex(tc_graph* g, uint64_t* per_vertex, uint64_t* out_total, uint32_t flags,
                                     void* stream);

/*
 * tc_count_per_vertex_noalloc — tc_count_per_vertex for callers that may not allocate device memory while they
 * run (for example a serving loop that reserves all its memory at start-up, or a host whose device memory belongs
 * to another framework's allocator).  The paper has no counterpart; this is an interface variant only.
 * It allocates nothing: its scratch (the counts in rank space) is a file-scope device array of 2^20 uint64 entries
 * (8 MiB) that every GPU which loads the library holds until the process exits.
 *   d_per_vertex  n uint64 entries of DEVICE memory, overwritten with t(x).
 *   d_total       one uint64 of DEVICE memory, overwritten with T.
 * Graphs with more than 2^20 vertices are rejected with TC_ERR_INVALID_ARG (use tc_count_per_vertex).  The device
 * current at the call must be the one that was current at tc_load_edges (the graph's buffers live there, and the
 * scratch array used is the current device's); otherwise the call returns TC_ERR_INVALID_ARG and launches nothing.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls
 * on a device share the one array, and each call clears the part it uses before counting: calls whose GPU work
 * overlaps (different streams, no ordering between them) race on it and give wrong results.  Asynchronous: the
 * outputs are valid in stream order.
 */
TC_API tc_status tc_count_per_vertex_noalloc(tc_graph* g, uint64_t* d_per_vertex, uint64_t* d_total, void* stream);

/*
 * tc_list_triangles — the matched subgraphs themselves (Sec. II-A: the outputs are the number of matches and the
 * matched node id lists; Algorithm 1 returns M beside the count).  Lists the triangles whose first vertex in the
 * visiting order has rank in [first_source, first_source + num_sources) (ranks run over [0, n); listing every
 * triangle takes first_source = 0, num_sources = n, or several calls over consecutive ranges when the output would
 * not fit in memory).  Each triangle is written once, as three int32 original ids in ascending order.
 *   triples    capacity * 3 int32, host or device memory as `flags` says; the first min(found, capacity) triples
 *              are written, in no particular order.
 *   out_found  host pointer: the number of triangles in the range (it can exceed capacity: list again with more
 *              room or a smaller range).
 * Blocks until the outputs are valid.
 */
TC_API tc_status tc_list_triangles(tc_graph* g, int64_t first_source, int64_t num_sources, int32_t* triples,
                                   int64_t capacity, uint64_t* out_found, uint32_t flags, void* stream);

/* Frontier sizes of one tc_count_unfused call (all counts of slots or matches). */
typedef struct tc_unfused_stats {
  int64_t candidates; /* |c_set|: sources u with d+(u) >= 2 after the NE filter */
  int64_t frontier1;  /* hop-1 advance slots: sum over c_set of d+(u) */
  int64_t partials;   /* hop-1 survivors (u, v) with d+(v) > 0 (the 1-look-ahead) */
  int64_t frontier2;  /* hop-2 advance slots: sum over the partials of d+(v) (the candidate 2-paths) */
  int64_t matches;    /* hop-2 survivors (u, v, w) with u -> w an edge: the triangle count */
  int64_t chunks;     /* hop-2 passes that the byte budget required */
  int64_t peak_bytes; /* largest total of intermediate device buffers held at one time */
  int64_t reserved;
} tc_unfused_stats;

/*
 * tc_count_unfused — the same count by the paper's unfused verification loop (Algorithm 1, Sec. III-A/III-B):
 * a filter of candidate sources by NE, then two rounds of advance (one 32-bit frontier slot per traversed edge,
 * marked kept or masked by the constraint check), compaction of the kept slots (Compute) and their write to the
 * partial results.  Hop 1 extends each source u by its out-neighbours v and keeps those with an out-neighbour
 * (1-look-ahead); hop 2 extends each (u, v) by w in N+(v) and keeps those closed by the edge u -> w.  The result
 * equals tc_count.  It exists to measure what fusion saves: its frontiers hold W slots where tc_count writes none.
 *   out_total        host pointer: T.
 *   max_chunk_bytes  bytes that one hop-2 pass may hold (4 per slot plus 12 per surviving match); the hop-2
 *                    frontier is cut into passes accordingly (at least 4096 and at most 2^31 - 1 slots per pass).
 *                    0: the largest pass.  Negative: TC_ERR_INVALID_ARG.
 *   stats            host pointer or NULL: frontier sizes and the peak bytes held.
 * Memory comes from the graph's allocator (TC_ERR_NO_MEMORY when a frontier does not fit).  Graphs whose hop-1
 * frontier reaches 2^31 - 1 slots are rejected with TC_ERR_INVALID_ARG.  Blocks until the outputs are valid.
 */
TC_API tc_status tc_count_unfused(tc_graph* g, uint64_t* out_total, int64_t max_chunk_bytes,
                                  tc_unfused_stats* stats, void* stream);

/*
 * tc_count_batch — count many built graphs in one persistent launch fed by a device work queue (the traversal of
 * tc_count applied to each graph independently; the batching itself has no counterpart in the paper).
 *   gs          num_graphs built graph handles (host array); the same handle may appear more than once.
 *   out_counts  host array of num_graphs uint64: out_counts[i] = T of gs[i].
 * Blocks until the counts are valid.
 */
TC_API tc_status tc_count_batch(tc_graph* const* gs, int32_t num_graphs, uint64_t* out_counts, void* stream);

/*
 * tc_count_many — count k graphs given as edge lists, ingested, built and counted together as one pipeline: their
 * disjoint union (graph j's ids offset past the vertices of graphs 0..j-1) is built once, and every triangle, found
 * once from its first vertex in the visiting order (Sec. III-A, III-C), is credited to the graph holding that vertex.
 * No triangle spans two graphs, so counts[j] is graph j's own T (Def. 2, Sec. II-A).  The batching itself has no
 * counterpart in the paper: for many small graphs it replaces one launch sequence per graph with one per batch.
 *   srcs, dsts    k pointers to int32 arrays of num_edges[j] pairs each (host or device per flags, all alike; host
 *                 arrays that are page-locked and mapped are read in place, other host arrays are copied first).
 *                 The caller keeps them; they are not needed after the call returns.
 *   num_edges     k pair counts; num_vertices: k vertex counts (graph j's ids in [0, num_vertices[j])).
 *   counts        k uint64 (host), overwritten with each graph's triangle count.
 * The vertices of all k graphs together must fit the int32 id range and their pairs number below 2^32 - 1
 * (TC_ERR_INVALID_ARG otherwise).  An id outside its graph's range gives TC_ERR_OUT_OF_RANGE.  Self-loops and
 * repeated pairs are dropped per graph, as in tc_load_edges.  Device memory comes from the library's pool.
 * Blocks until the counts are valid.
 */
TC_API tc_status tc_count_many(const int32_t* const* srcs, const int32_t* const* dsts, const int64_t* num_edges,
                               const int64_t* num_vertices, int32_t k, uint32_t flags, uint64_t* counts,
                               void* stream);

/*
 * Batch plans — tc_count_batch for a fixed set of graphs counted repeatedly.  tc_batch_plan_create uploads the
 * batch's work table once and captures the launch sequence (zero the counters, the persistent kernel, the copy of
 * the counts to pinned host memory) as a CUDA graph on `stream`; tc_batch_plan_run replays it with one graph launch
 * and copies the counts to out_counts (host, num_graphs entries), blocking until they are valid.  The graphs must
 * stay built and must not be freed while the plan exists.  (No counterpart in the paper.)
 */
typedef struct tc_batch_plan tc_batch_plan; /* opaque */
TC_API tc_status tc_batch_plan_create(tc_graph* const* gs, int32_t num_graphs, void* stream, tc_batch_plan** out);
TC_API tc_status tc_batch_plan_run(tc_batch_plan* p, uint64_t* out_counts, void* stream);
TC_API void tc_batch_plan_free(tc_batch_plan* p); /* NULL is a no-op */

/*
 * Serving loop (no counterpart in the paper; it drives the traversal of tc_count for a stream of requests).
 * A server admits submitted requests by device memory, builds their CSRs concurrently on its own streams, keeps
 * them resident, and counts every graph that is ready whenever the previous launch finishes (continuous batching
 * through tc_count_batch), or one graph per launch when batching is 0.  All waits are host-side.
 */
typedef struct tc_server tc_server; /* opaque */

typedef struct tc_server_config {
  int32_t build_workers;      /* threads that copy and build admitted requests, one stream each (0: 4)           */
  int32_t max_batch;          /* most graphs per counting launch (0: 4096)                                        */
  int32_t batching;           /* 1: continuous batching of the count (each request built alone, ready graphs
                                 counted together); 2: continuous batching of the whole path (the pending requests
                                 that the budget admits ingested, built and counted together, as tc_count_many);
                                 0: one graph per launch                                                          */
  int32_t max_inflight;       /* most admitted, unfinished requests (0: 8192)                                     */
  int64_t hbm_reserve_bytes;  /* device memory never used by admissions (< 0: 8 GiB)                              */
  int64_t hbm_budget_bytes;   /* if > 0, an upper bound on the admission budget                                   */
} tc_server_config;

typedef struct tc_request_result {
  uint64_t id;          /* as returned by tc_server_submit */
  uint64_t triangles;   /* T of the request's graph (valid when status == TC_OK) */
  int32_t status;       /* tc_status of the request */
  int32_t reserved;
  int64_t t_submit_ns;  /* steady-clock timestamps: submitted, admitted, CSR built, count available */
  int64_t t_admit_ns;
  int64_t t_built_ns;
  int64_t t_done_ns;
} tc_request_result;

typedef struct tc_server_stats {
  int64_t submitted, admitted, completed, failed;
  int64_t launches;         /* counting launches (batched or single) */
  int64_t max_batch_seen;   /* most graphs in one launch so far */
  int64_t budget_bytes;     /* admission budget: free device memory at creation minus the reserve */
  int64_t held_bytes;       /* estimated bytes held by admitted, unfinished requests */
  int64_t peak_held_bytes;
  int64_t pending;          /* submitted, not yet admitted */
} tc_server_stats;

/* tc_server_create — start a server on the current device (cfg may be NULL for defaults).  The admission budget is
 * the free device memory now, minus hbm_reserve_bytes.  A request is admitted when its estimated peak footprint
 * fits in what admitted requests leave of the budget (a request alone is always admitted if it fits the budget). */
TC_API tc_status tc_server_create(const tc_server_config* cfg, tc_server** out);

/* tc_server_submit — queue a request: the graph given by num_edges HOST pairs (src[i], dst[i]) on [0, num_vertices)
 * (pinned memory gives the fastest copies).  The arrays must stay valid and unchanged until the request's result
 * has been returned by tc_server_poll.  *id_out (may be NULL) receives the request id.  TC_ERR_NO_MEMORY if the
 * request alone exceeds the budget.  Thread-safe. */
TC_API tc_status tc_server_submit(tc_server* s, const int32_t* src, const int32_t* dst, int64_t num_edges,
                                  int64_t num_vertices, uint64_t* id_out);

/* tc_server_poll — move up to max_results finished requests into out (host array) and set *n_out; waits up to
 * timeout_ms (0: no wait) for at least one.  A failed request has a non-zero status.  Thread-safe. */
TC_API tc_status tc_server_poll(tc_server* s, tc_request_result* out, int32_t max_results, int32_t timeout_ms,
                                int32_t* n_out);

/* tc_server_get_stats — counters of the server so far. */
TC_API tc_status tc_server_get_stats(tc_server* s, tc_server_stats* out);

/* tc_server_destroy — stop the server: requests not yet admitted are dropped, admitted ones finish; results not
 * polled are discarded.  NULL is a no-op. */
TC_API void tc_server_destroy(tc_server* s);

/* tc_graph_get_info — sizes of g (valid fields depend on whether g is built). */
TC_API tc_status tc_graph_get_info(const tc_graph* g, tc_graph_info* info);

/*
 * tc_copy_csr — copy the oriented CSR of a built graph to host memory, for inspection and tests (Sec. III-B: the
 * graph is stored in CSR).  The CSR is in rank space: vertex r is the r-th vertex in the (input-pair count, id)
 * order, and row r holds N+(r), the ranks above r adjacent to it, ascending.  Each row starts at a multiple of 4
 * entries and is padded to a multiple of 4 with the value n.
 *   offsets  n+1 int64 row offsets (host).
 *   cols     csr_entries int32 column entries (host; see tc_graph_info.csr_entries), or NULL.
 *   perm     n int32 (host), or NULL: perm[r] = the original id of rank r.
 * Synchronises `stream`.
 */
TC_API tc_status tc_copy_csr(const tc_graph* g, int64_t* offsets, int32_t* cols, int32_t* perm, void* stream);

/* tc_free — release g and all its device memory (stream-ordered on the last stream g used), then wait for that
 * stream, so the memory is free again when tc_free returns and the next graph's buffers are served from completed
 * frees (measured faster than returning with the frees still queued).  That stream must still exist (not yet
 * destroyed by the caller).  NULL is a no-op. */
TC_API void tc_free(tc_graph* g);

/*
 * Tuning (no counterpart in the paper).  The counting kernel gives a source a whole thread block when its work
 * w(u) (padded second-hop entries) exceeds a threshold, and one warp otherwise; the best threshold depends on the
 * graph's size.  The table maps size classes (by distinct edges m) to thresholds and is consulted by tc_build.
 * It also picks, per graph, between the fused traversal and segmented intersection for tc_count.  Counts never
 * depend on it.  Process-wide; thread-safe.
 */
#define TC_TUNING_MAX_CLASSES 16
typedef struct tc_tuning {
  int32_t num_classes;                                 /* 1..TC_TUNING_MAX_CLASSES */
  int32_t reserved;
  int64_t batch_warp_max_edges;                        /* in tc_count_batch and batch plans, graphs with m at most
                                                          this run every source one warp each: across many graphs
                                                          there is parallelism enough, and a block per source costs
                                                          more than it saves */
  int64_t class_max_edges[TC_TUNING_MAX_CLASSES];      /* ascending; class i holds graphs with m <= class_max_edges[i]
                                                          (the last class also holds every larger graph) */
  int64_t block_min_work[TC_TUNING_MAX_CLASSES];       /* threshold for class i, >= 0 */
  int64_t isect_max_wedges_milli;                      /* tc_count and tc_count_device count a graph with the
                                                          segmented-intersection kernel (tc_count_intersect) when
                                                          1000 * num_wedges <= this * num_edges, i.e. when it has
                                                          few candidate 2-paths per edge; 0: never.  >= 0 */
  int64_t bucket_max_pairs;                            /* tc_build groups the pairs by source in per-source buckets
                                                          sorted on chip for graphs of at most this many input pairs,
                                                          and by a radix sort of all pairs above it (the buckets'
                                                          random accesses stop fitting in L2); 0: always buckets.
                                                          >= 0 */
  int64_t compact_max_pairs;                           /* tc_build of a graph with at most this many input pairs (on
                                                          the bucketed path) synchronises with the host once: buffers
                                                          whose size depends on the data are allocated at bounds
                                                          known from n and the pair count, and every size is read
                                                          back at the end.  Above it, sizes are read as they become
                                                          known (smaller allocations).  0: never.  >= 0 */
  int64_t stage_min_csr_bytes;                         /* tc_count and tc_count_device walk long hop-2 rows through a
                                                          ring of shared memory filled by asynchronous copies
                                                          (cp.async) for graphs whose CSR (8(n+1) + 4 csr_entries
                                                          bytes) is at least this large, i.e. read from DRAM rather
                                                          than L2.  0: never.  >= 0 */
  int64_t tiny_max_pairs;                              /* tc_build of a graph with at most 16384 vertices and at most
                                                          this many input pairs (and fewer than 2^18) on the bucketed
                                                          path runs as one cooperative kernel launch, its steps
                                                          separated by grid-wide barriers, instead of about 25
                                                          launches.  0: never.  >= 0 */
  int64_t vertex_plain_max_edges;                      /* tc_count_per_vertex adds to its per-block counters of the
                                                          top ranks without reading them back for graphs of at most
                                                          this many edges: a source u adds at most d+(u) to one
                                                          counter as the middle vertex and d+(u) as the last, 2m in
                                                          all, so below 2^31 edges no counter reaches 2^32.  Above
                                                          it every add checks its counter.  0 <= this < 2^31 */
} tc_tuning;

/* tc_set_tuning — replace the table (TC_ERR_INVALID_ARG if malformed).  Applies to graphs built afterwards. */
TC_API tc_status tc_set_tuning(const tc_tuning* t);
/* tc_get_tuning — copy the current table (the built-in default until tc_set_tuning is called). */
TC_API tc_status tc_get_tuning(tc_tuning* t);

/* tc_kernel_launches — number of CUDA kernels this library has launched in the process so far (all threads).
 * A diagnostic with no counterpart in the paper: benchmarks difference it around a timed region. */
TC_API uint64_t tc_kernel_launches(void);

/* tc_last_error — message for the last failing call on this thread ("" if none).  Valid until the next call. */
TC_API const char* tc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
