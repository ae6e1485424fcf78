/*
 * bcgpu.h -- C ABI of libbcgpu.so: incremental betweenness centrality on one GPU.
 *
 * The method is Nasre, Pontecorvi and Ramachandran, "Betweenness Centrality --
 * Incremental and Faster" (arXiv 1311.2147).  The library keeps, for every ordered
 * pair (s,t) of a graph G = (V,E) with positive integer edge weights, the distance
 * d(s,t), the shortest-path count sigma_st (Section 2, Eq. 1 and the definition
 * below it) and the dependency delta_s.(t) (Eq. 4), plus the BC vector (Eq. 3), all
 * resident in device memory.  An incremental update -- a new edge, a lower edge
 * weight (Section 1), or both on any subset of the edges incident to one vertex
 * (Section 4) -- is applied by the rank-1 rules of Lemma 2 / Lemma 4 over the whole
 * n x n state, after which the dependencies of the sources whose rows changed are
 * re-accumulated by Brandes' recurrence (Eq. 4, Algorithm 1) over the shortest-path
 * DAG rebuilt from the edges that lie on shortest paths (E*, Section 6).
 *
 * Conventions shared by every call:
 *   * Vertices are 0 .. n-1.  Weights are integers >= 1 (the paper allows positive
 *     reals; integers keep Lemma 2's tie test exact).  A graph is simple: no
 *     self-loops and no repeated edge.
 *   * Undirected graphs are held as G_D (Section 3, "Undirected graphs": each edge
 *     {a,b} is the arcs (a,b) and (b,a)); their BC counts each unordered pair once,
 *     i.e. the G_D sum halved.  Directed BC is the raw Eq. 3 sum.  No normalisation.
 *   * Unreachable pairs: d = INF (the distance type's maximum), sigma = 0, and they
 *     contribute nothing to BC.
 *   * Distances are int32 (BC_DIST_I32) or int64 (BC_DIST_I64); path counts are
 *     uint64 and overflow is detected, never wrapped; dependencies and BC are fp64.
 *   * All pointers passed to these calls are HOST pointers unless a comment says
 *     otherwise.  The caller owns them; the library copies what it needs before the
 *     call returns.  The library owns all device memory of a handle until
 *     bc_destroy.
 *   * Every call returns a bc_status; nothing throws across the ABI.  Calls on one
 *     handle must not overlap (the library does not lock); calls on different
 *     handles are independent.  All work of a handle runs on the CUDA stream given to
 *     bc_init_static (NULL = the legacy default stream).
 *   * Device-side errors (a path count or distance that does not fit its type) are
 *     sticky: they are reported by the call that synchronises, and the handle is
 *     then poisoned -- every later call except bc_destroy / bc_last_error returns
 *     BC_ERR_POISONED.
 *   * A call rejected by host-side validation (BC_ERR_ARG, BC_ERR_NOT_INCREMENTAL)
 *     leaves the state untouched.
 */
#ifndef BCGPU_H
#define BCGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bc_graph bc_graph;   /* opaque handle */

typedef enum bc_status {
    BC_OK = 0,
    BC_ERR_ARG = -1,             /* malformed argument or graph */
    BC_ERR_NOT_INCREMENTAL = -2, /* new weight >= current weight of an existing edge */
    BC_ERR_OVERFLOW = -3,        /* a path count sigma_st needs more than 64 bits */
    BC_ERR_DIST_OVERFLOW = -4,   /* a distance does not fit the distance type */
    BC_ERR_OOM = -5,             /* device or host allocation failed */
    BC_ERR_CUDA = -6,            /* a CUDA runtime call failed (see bc_last_error) */
    BC_ERR_TIMEOUT = -7,         /* a bounded device-side wait gave up */
    BC_ERR_POISONED = -8         /* an earlier device-side error poisoned the handle */
} bc_status;

enum {
    BC_DIRECTED = 1,
    BC_UNDIRECTED = 2,
    BC_DIST_I32 = 16,
    BC_DIST_I64 = 32,
    BC_STATIC_ALL_ARCS = 64      /* bc_init_static: search every arc (no E* pruning) */
};

enum { BC_UPD_EDGE = 0, BC_UPD_VERTEX = 1 };

/* One incremental update of a batch (32 bytes, naturally aligned).
 *   kind == BC_UPD_EDGE:   edge (u, v) gets weight w (a new edge or a lower weight;
 *                          for an undirected graph the edge {u, v}).
 *   kind == BC_UPD_VERTEX: a vertex update of v (Section 4): the k entries
 *                          edges[first .. first + k) of the batch's bc_vedge array.
 */
typedef struct bc_update {
    int32_t kind;
    int32_t u;
    int32_t v;
    int32_t k;
    int64_t w;
    int64_t first;
} bc_update;

/* One edge of a vertex update of v: dir == 0 is the edge (x, v) (in E_i of
 * Section 4), dir == 1 the edge (v, x) (in E_o).  dir is ignored for an undirected
 * graph, where the edge is {v, x}.  16 bytes. */
typedef struct bc_vedge {
    int32_t x;
    int32_t dir;
    int64_t w;
} bc_vedge;

/* Per-handle counters (bc_get_info). */
typedef struct bc_info {
    int32_t n;
    int32_t directed;
    int32_t dist_bytes;          /* 4 or 8 */
    int32_t reserved;
    int64_t m;                   /* arcs of G (G_D for undirected) */
    int64_t estar_arcs;          /* arcs currently held in the E* superset */
    int64_t updates_applied;     /* updates run on the device since init */
    int64_t rows_reaccumulated;  /* sum over updates of the sources re-accumulated */
    int64_t noop_updates;        /* updates that changed no pair */
    int64_t max_rows;            /* largest number of sources of one update */
    int64_t rows_scanned;        /* rows passed through the rank-1 pass (all phases) */
    int64_t pairs_lowered;       /* pairs whose distance dropped (Lemma 2/4 last case) */
    int64_t pairs_tied;          /* pairs that gained tied shortest paths */
    int64_t kernel_launches;     /* kernels enqueued by this handle since init */
    int64_t state_bytes;         /* device bytes owned by the handle */
    double last_init_ms;         /* device time of the static computation in bc_init_static */
    int64_t rows_full;           /* of rows_reaccumulated: rows rebuilt by Algorithm 1 rather than
                                    corrected pair by pair ("pair_updates") */
    int64_t estar_rebuilds;      /* times the E* superset was laid out again (host round trip) */
    int64_t estar_moves;         /* vertex segments of E* moved to the free region instead */
    int64_t pair_rows;           /* rows whose dependencies were corrected pair by pair */
    int64_t pair_targets;        /* (row, changed target) pairs of those corrections */
    int64_t walk_pairs;          /* of pair_targets: pairs whose columns were found by DAG walks
                                    ("pair_walk") */
    int64_t walk_vertices;       /* vertices on their shortest paths (both states) found by the walks */
    int64_t walk_arcs;           /* E* superset arcs the walks examined */
} bc_info;

/*
 * bc_init_static -- build the state of G by a static computation on the device
 * (Brandes' algorithm, Appendix Algorithm 7: all-pairs distances and path counts,
 * the shortest-path DAG of every source from E* as in Section 6 (Algorithm 6 steps
 * 2-4), then Algorithm 1 for every source).  This is also the GPU full-recompute
 * baseline.
 *   out          receives the new handle (NULL on failure).
 *   n            number of vertices (1 .. 32768).
 *   m            number of edges in src/dst/w (undirected: each edge once).
 *   src,dst,w    host arrays of m entries; w in [1, INF-1] of the distance type.
 *   flags        exactly one of BC_DIRECTED / BC_UNDIRECTED, and one of
 *                BC_DIST_I32 / BC_DIST_I64; optionally BC_STATIC_ALL_ARCS.
 *   cuda_stream  a cudaStream_t (NULL = legacy default stream).
 * The all-pairs distances come from one search per source (one CTA each).  By default
 * the searches are restricted to E* as it becomes known (Section 6, Algorithm 6 step
 * 1, whose Hidden Paths algorithm examines only arcs of E*): once the search from a
 * has finished, the arcs (a,b) with w(a,b) > d(a,b) are left out of every later search,
 * and the sources run highest out-degree first.  BC_STATIC_ALL_ARCS searches every
 * arc instead (the same results; kept for comparison).
 * Synchronous.  Returns BC_ERR_ARG for a malformed graph or flags, BC_ERR_OOM when
 * the n x n state does not fit, and the device-side errors above.
 */
int bc_init_static(bc_graph** out, int32_t n, int64_t m, const int32_t* src,
                   const int32_t* dst, const int64_t* w, uint32_t flags, void* cuda_stream);

/*
 * bc_apply_edge_update -- one incremental edge update (u, v, w_new): a new edge, or a
 * lower weight of an existing one (Section 3, Algorithm 3 with Lemma 2; undirected
 * graphs as the two arcs of G_D).  Synchronous.
 *   Rejects u or v out of range, u == v, w_new < 1 or >= INF (BC_ERR_ARG) and
 *   w_new >= current weight (BC_ERR_NOT_INCREMENTAL), leaving the state untouched.
 */
int bc_apply_edge_update(bc_graph* g, int32_t u, int32_t v, int64_t w_new);

/*
 * bc_apply_vertex_update -- one incremental vertex update of v over k incident edges
 * (Section 4: E_i processed first with Algorithm 4 and Lemma 4, then E_o on the
 * reversed graph).  nbr, w_new and dir are host arrays of k entries; dir[i] == 0
 * is the edge (nbr[i], v), 1 is (v, nbr[i]); dir may be NULL for an undirected
 * graph (where it is ignored).  Synchronous.  Rejects an empty or repeated edge set
 * and each edge as bc_apply_edge_update would, leaving the state untouched.
 */
int bc_apply_vertex_update(bc_graph* g, int32_t v, int32_t k, const int32_t* nbr,
                           const int64_t* w_new, const uint8_t* dir);

/*
 * bc_apply_updates -- apply count updates in order, each seeing the state left by
 * the one before (bc_stage_updates + bc_run_staged + bc_synchronize).
 *   ups     host array of count bc_update records.
 *   edges   host array holding every vertex update's edges (may be NULL if none).
 *   n_edges number of entries in edges.
 *   n_done  (optional) receives how many updates were enqueued before the first
 *           rejected one (count when all were valid).
 * Stops at the first invalid update and returns its status; the updates before it
 * are applied.
 */
int bc_apply_updates(bc_graph* g, int32_t count, const bc_update* ups,
                     const bc_vedge* edges, int64_t n_edges, int32_t* n_done);

/*
 * bc_stage_updates -- copy a batch to the handle: the records to host memory owned by
 * the handle and the vertex-update edges to device memory.  Nothing is validated or
 * run yet.  Replaces any batch staged before.  Synchronous (the copy completes).
 */
int bc_stage_updates(bc_graph* g, int32_t count, const bc_update* ups,
                     const bc_vedge* edges, int64_t n_edges);

/*
 * bc_run_staged -- validate the staged updates in order and enqueue the device work of
 * each valid one on the handle's stream.  Does not wait for the device; call
 * bc_synchronize for device-side errors.  Stops at the first invalid update and
 * returns its status (n_done as in bc_apply_updates).
 */
int bc_run_staged(bc_graph* g, int32_t* n_done);

/* bc_synchronize -- wait for the handle's stream and return any device-side error. */
int bc_synchronize(bc_graph* g);

/*
 * bc_query -- non-blocking: BC_OK with *done = 1 when every enqueued update has
 * finished on the device (device-side errors are then reported as by
 * bc_synchronize), *done = 0 while work is still in flight.
 */
int bc_query(bc_graph* g, int32_t* done);

/*
 * bc_get_scores -- BC(v) for every v (Eq. 3), into the host array out[n].
 * Synchronous.  Undirected graphs: halved G_D sums.
 */
int bc_get_scores(bc_graph* g, double* out);

/*
 * bc_get_rows -- copy rows s0 .. s0+count-1 of the state to host arrays of count*n
 * entries each (any of them may be NULL): d widened to int64 (INF -> INT64_MAX),
 * sigma, and delta_s.(t) (0 on the diagonal and for unreachable t).  Synchronous.
 */
int bc_get_rows(bc_graph* g, int32_t s0, int32_t count, int64_t* d_out,
                uint64_t* sigma_out, double* delta_out);

/* bc_get_info -- counters of the handle (synchronous). */
int bc_get_info(bc_graph* g, bc_info* out);

/*
 * bc_get_profile -- device time in ms and kernel launches per kernel class, summed over
 * the updates enqueued while the "profile" option was on (CUDA events recorded around
 * each launch on the handle's stream).  Classes: 0 the rank-1 pass (Lemma 2 / 4),
 * 1 dependency accumulation (Eq. 4 / Algorithm 1), 2 BC row sums, 3 per-vertex passes
 * (Algorithm 4 in both directions, row tests, row write), 4 bookkeeping (compaction,
 * E* writes, flags), 5 pair corrections of the dependency rows ("pair_updates").  ms
 * and launches are host arrays of BC_PROFILE_CLASSES entries (either
 * may be NULL).  reset != 0 clears the sums after reading.  Synchronous.
 */
enum { BC_PROFILE_CLASSES = 6 };
int bc_get_profile(bc_graph* g, double* ms, int64_t* launches, int32_t reset);

/*
 * bc_set_option -- tuning knobs (documented values only):
 *   "full_scan" 0|1: run the rank-1 pass of Lemma 2 / 4 over every row instead of
 *                     only the rows that can change (Section 5 scans all n^2 pairs).
 *   "profile"   0|1: record CUDA events around every launch (see bc_get_profile).
 *   "pair_updates" 0|1 (undirected graphs only, on by default there; BC_ERR_ARG on a
 *                     directed graph): update the dependency row of a source s with
 *                     at most 128 changed pairs (s,t) by adding delta'_st(x) - delta_st(x)
 *                     for those pairs (the pair dependencies of Section 2; pairs whose
 *                     distance and path count did not change keep their shortest paths
 *                     and hence their dependencies) instead of re-running Algorithm 1
 *                     for s.  Off: every changed source is re-accumulated (Section 5).
 *                     The two give the same D and sigma bit for bit and dependencies
 *                     within rounding.
 *   "fused_edges" 0|1 (on by default): an undirected edge update runs one rank-1 pass
 *                     over both directions of the edge, each row's candidate taken from
 *                     the state before the update (Section 3 "Undirected graphs" as one
 *                     pass); 0: the two directed passes one after the other.  Same
 *                     results bit for bit.
 *   "wide_accum" 0|1 (on by default): on graphs of at least 4096 vertices, re-run
 *                     Algorithm 1 for the rows over the target cap in 1024-thread CTAs
 *                     (one source's passes spread over more threads); 0: 256-thread
 *                     CTAs, which share SMs better with other handles' work (the server
 *                     sets 0 for its graphs).  Same results bit for bit.
 *   "pair_walk" 0|1 (undirected graphs only; BC_ERR_ARG on a directed graph): find the
 *                     columns of each changed pair (s,t) -- the vertices on a shortest
 *                     s-t path of the old and of the new state -- by walking DAG(s) of
 *                     Eq. 1 backwards from t over the E* superset, instead of testing
 *                     every column.  Same results bit for bit.  Turning it on allocates
 *                     its scratch (16 bytes per vertex per warp of the walk grid) once;
 *                     BC_ERR_OOM if that fails, BC_ERR_ARG if n is too large for the
 *                     walk's per-warp bit sets (n above ~100k).
 */
int bc_set_option(bc_graph* g, const char* name, int64_t value);

/*
 * Real (fp64) weights.  Section 2 allows positive real weights; Lemma 2 and Lemma 4
 * compare path lengths for equality, so ties must be decided exactly.  A finite
 * double w > 0 is exactly M * 2^e (M an odd integer below 2^53); with E the smallest e
 * over the graph's weights every weight is an integer number of units of 2^E, and so
 * is every path length.  These calls run the state on those integers, so path lengths
 * are the exact sums of the given doubles and two paths tie exactly when those sums
 * are equal (0.1 + 0.2 does not tie with 0.3: as doubles they differ).  BC does not
 * depend on the unit.
 *
 * bc_init_static_f64 -- as bc_init_static with w a host array of m doubles, each
 *   finite and > 0.  BC_ERR_ARG when a weight is not, or when the weights span too
 *   many binary orders of magnitude: n - 1 copies of the largest weight, in units of
 *   the smallest power of two, must fit the distance type (30 bits for BC_DIST_I32,
 *   62 for BC_DIST_I64).
 * bc_apply_edge_update_f64 / bc_apply_vertex_update_f64 -- as bc_apply_edge_update /
 *   bc_apply_vertex_update with double weights, on a handle made by
 *   bc_init_static_f64.  BC_ERR_ARG (state untouched) for a weight that is not a whole
 *   number of the handle's units or exceeds the size bound above.
 * bc_get_weight_unit -- *exp2 = E: the distances of bc_get_rows, and the weights of
 *   bc_get_edges and bc_apply_updates, are integers in units of 2^E (0 for a handle
 *   made by bc_init_static).
 */
int bc_init_static_f64(bc_graph** out, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                       const double* w, uint32_t flags, void* cuda_stream);
int bc_apply_edge_update_f64(bc_graph* g, int32_t u, int32_t v, double w_new);
int bc_apply_vertex_update_f64(bc_graph* g, int32_t v, int32_t k, const int32_t* nbr, const double* w_new,
                               const uint8_t* dir);
int bc_get_weight_unit(bc_graph* g, int32_t* exp2);

/*
 * bc_static_scores_noalloc -- BC(v) of a small graph that is already in device memory,
 * computed without allocating any device memory.  (The paper has no counterpart: this
 * serves callers that cannot call cudaMalloc -- a process whose device memory belongs to
 * a framework's caching allocator, or a serving runtime that reserves HBM at start-up
 * and allows no later allocation, cudaMalloc being able to synchronise the device.)
 * It runs the static computation of bc_init_static with every arc as the E* superset
 * and keeps all scratch in one fixed array inside the library (about 12 MB, held on
 * every GPU that loads the library until the process exits).
 *   n            vertices, 1 .. 512; larger graphs are rejected with BC_ERR_ARG.
 *   arcs         arcs in d_dst / d_w, 0 .. 32768 (BC_ERR_ARG beyond).
 *   d_off        DEVICE int32[n+1]: CSR offsets by tail (arcs of a in [d_off[a], d_off[a+1])).
 *   d_dst, d_w   DEVICE int32 / int64 [arcs]: head and weight of each arc, weight in
 *                [1, INF-1] of the distance type.  An undirected graph is passed as
 *                G_D (both arcs of every edge).  The graph must be simple (repeated
 *                arcs are the caller's to avoid); a bad endpoint, a self-loop or a bad
 *                weight found on the device returns BC_ERR_ARG.
 *   flags        as for bc_init_static.
 *   d_scores     DEVICE double[n]: receives BC (halved G_D sums for undirected).
 *   cuda_stream  stream for all the work (NULL = legacy default stream).
 * Synchronous: it waits for its stream and copies an error word to the host, so it
 * must not be called while its stream (or the legacy stream) is being captured.
 * Calls no cudaMalloc / cudaFree and no allocating library routine.  The first call on
 * a device looks up the device address of the scratch array (cudaGetSymbolAddress)
 * with that device current.  All calls share the one scratch array, which keeps the previous
 * call's contents (the call clears what must start at zero); calls whose work overlaps
 * on the GPU -- from several host threads or on several streams -- race on it.
 */
int bc_static_scores_noalloc(int32_t n, int64_t arcs, const int32_t* d_off, const int32_t* d_dst,
                             const int64_t* d_w, uint32_t flags, double* d_scores, void* cuda_stream);

/*
 * Batches: many graphs updated together.  Round r applies the r-th update of every graph
 * that has one; within a round each phase of the update (Algorithm 4 and Lemma 2 / 4 in
 * both directions, DAG rebuild, Kahn order, Eq. 4, BC) runs as one kernel over the work
 * of all graphs at once, and the rounds are captured once into a CUDA graph that is
 * replayed by one graph launch per call.  Undirected graphs with pair corrections on
 * (option "pair_updates", the default) re-accumulate only their rows over the target
 * cap and correct the others pair by pair with the column test; the DAG walks are not
 * used in batches.  A graph's result is bit-identical to applying the same updates to it
 * alone with the same options (for an undirected graph alone: the column test, i.e. n
 * below the walks' default or "pair_walk" 0; with the walks the dependencies agree
 * within rounding).  The graphs must share the distance type; they stay owned by the
 * caller and must not be used by other calls while a batch call runs.
 */
typedef struct bc_batch bc_batch;

/* bc_batch_create -- group count handles (host array of handles) on a CUDA stream
 * (NULL: the batch creates its own, since the legacy default stream cannot be captured
 * into a CUDA graph).  BC_ERR_ARG for a NULL or poisoned handle or mixed distance types. */
int bc_batch_create(bc_batch** out, int32_t count, bc_graph* const* graphs, void* cuda_stream);

/*
 * bc_batch_apply -- n_updates[g] updates for graph g, concatenated in graph order in
 * ups (host arrays); vertex updates index edges as in bc_apply_updates.  Each graph's
 * updates are validated in order; a graph stops at its first invalid update (the updates
 * before it are applied) and the first such status is returned.  n_done (optional, G
 * entries) receives how many updates each graph applied.  Synchronous; device-side
 * errors poison only the graphs they occur in.
 */
int bc_batch_apply(bc_batch* b, const int32_t* n_updates, const bc_update* ups, const bc_vedge* edges,
                   int64_t n_edges, int32_t* n_done);

/* bc_batch_set_tiles -- launch shape of the batch kernels (what the autotuner varies):
 * tiles[0] CTAs per SM of the per-vertex passes (1..64), tiles[1] of the rank-1 pass,
 * tiles[2] of the BC row sums, tiles[3] cap on accumulation CTAs per SM (0 = as many as
 * fit); with count >= 6 also the rank-1 pass's tile and schedule: tiles[4] 16-byte
 * vectors per thread per work item (1, 2, 4 or 8: the item's column chunk is 256
 * threads x tiles[4] x 16 bytes), tiles[5] 0 = a contiguous block of items per CTA,
 * 1 = items dealt out to the CTAs in turn; with count >= 7 also tiles[6] the threads of an
 * accumulation CTA (512, 256 or 128: one source per CTA either way, more sources in flight
 * per SM with fewer threads; same results bit for bit).  BC_ERR_ARG for a value out of range.
 * The next bc_batch_apply captures a new CUDA graph. */
int bc_batch_set_tiles(bc_batch* b, const int32_t* tiles, int32_t count);

/* bc_batch_last_ms -- device time (CUDA events around the graph launch) of the last apply. */
int bc_batch_last_ms(bc_batch* b, double* ms);

const char* bc_batch_last_error(const bc_batch* b);

/* bc_batch_destroy -- free the batch (not the graphs). */
void bc_batch_destroy(bc_batch* b);

/*
 * bc_get_edges -- the current edges of the graph (undirected: each edge once, a < b),
 * sorted, into host arrays of *m entries.  Call with src = dst = w = NULL to get the
 * count in *m.  Enough to rebuild the state later with bc_init_static.
 */
int bc_get_edges(bc_graph* g, int64_t* m, int32_t* src, int32_t* dst, int64_t* w);

/*
 * Serving.  A server keeps many graphs resident on the device and applies update
 * requests to them as they arrive.  Requests for one graph are applied in arrival
 * order; whenever a graph has nothing on the device, all its queued requests are
 * launched together on its own stream (continuous batching), so requests that arrive
 * while it is busy join its next launch and different graphs' launches overlap.  A
 * graph's device state (about n^2 * (distance bytes + 16) bytes; twice the distance
 * bytes + 24.125 for undirected graphs, which keep the old values of changed pairs for
 * pair corrections) is built only when
 * the budget and the device's free memory leave room; when a graph with queued
 * requests needs room, idle graphs are evicted least-recently-used first and rebuilt
 * from their current edges when needed again.  Results are the same as applying each
 * graph's requests to it alone (same kernels, same order).  Not thread-safe: drive a
 * server from one host thread.
 */
typedef struct bc_server bc_server;

typedef struct bc_result {
    int64_t request_id;
    int32_t graph_id;
    int32_t status;       /* bc_status of the request */
    int64_t latency_ns;   /* submission to the poll that saw it finished */
} bc_result;

/* bc_server_create -- budget: device bytes the server may use for graph states;
 * max_batch: most requests of one graph launched together (<= 0: 64). */
int bc_server_create(bc_server** out, int64_t mem_budget_bytes, int32_t max_batch);

/* bc_server_add_graph -- register a graph (arguments as bc_init_static; host arrays are
 * copied).  It is built on the device now if there is room, otherwise when it first has
 * a request and room can be made.  *graph_id receives its index. */
int bc_server_add_graph(bc_server* s, int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                        const int64_t* w, uint32_t flags, int32_t* graph_id);

/* bc_server_submit -- queue one update for a graph (non-blocking); edges as in
 * bc_apply_updates for a vertex update (copied).  *request_id (optional) receives its id. */
int bc_server_submit(bc_server* s, int32_t graph_id, const bc_update* up, const bc_vedge* edges,
                     int64_t* request_id);

/* bc_server_poll -- non-blocking progress: collect finished launches, admit graphs,
 * launch queued requests of idle graphs; then copy up to max_results finished requests
 * to out (host array) and their number to *n_out. */
int bc_server_poll(bc_server* s, int32_t max_results, bc_result* out, int32_t* n_out);

/* bc_server_pending -- requests still queued, and in flight or not yet collected. */
int bc_server_pending(bc_server* s, int64_t* queued, int64_t* inflight);

/* bc_server_graph -- the handle of a graph (admitting it if needed, waiting for its
 * launch in flight); valid until the next server call. */
int bc_server_graph(bc_server* s, int32_t graph_id, bc_graph** handle);

/* bc_server_stats -- stats[5]: resident graphs, bytes in use, admissions, evictions,
 * launches. */
int bc_server_stats(bc_server* s, int64_t* stats);

void bc_server_destroy(bc_server* s);

/* bc_destroy -- free the handle and its device memory (waits for its stream). */
void bc_destroy(bc_graph* g);

/* bc_last_error -- text of the last error of the handle ("" if none); valid until
 * the next call on the handle.  g may be NULL for errors of a failed bc_init_static. */
const char* bc_last_error(const bc_graph* g);

#ifdef __cplusplus
}
#endif

#endif /* BCGPU_H */
