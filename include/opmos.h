/*
 * opmos.h -- C ABI of the GB300 exact multi-objective shortest-path library.
 *
 * The library computes, for a directed graph G = (V, E, c) with non-negative
 * d-vector arc costs, the cost-unique set of non-dominated start->goal path
 * cost vectors and one path per vector (problem statement, Sec. 3), by the
 * ordered-parallel label-setting search of Sec. 5 (Algorithm 2) on one GPU:
 * each step extracts the window of open labels with the lowest F = g + h in
 * lexicographic order, expands them along their out-arcs (the expansion of
 * Algorithm 1), and merges the candidates into the target nodes' frontiers
 * and the solution set P with dominance checks and pruning (the frontier
 * checks of Algorithm 1, and its goal branch for labels at the goal). The
 * heuristic h is the ideal point: per objective, the shortest distance from
 * each node to the goal (Sec. 4).
 *
 * Conventions (all entry points):
 *   - Every array argument is a HOST pointer. The library copies what it needs;
 *     the caller keeps ownership of its arrays and may free them on return.
 *   - Handles are opaque, owned by the caller, and released by their own
 *     destroy/free call. Graphs and heuristics are immutable after creation.
 *   - Arc costs are uint32, structure of arrays: cost[k*m + e] is the cost of
 *     arc e under objective k. Graphs are CSR: the out-arcs of node u are
 *     e in [rowptr[u], rowptr[u+1]), arc e enters node col[e].
 *   - Cost vectors on output are row-major, count x d, in increasing
 *     lexicographic order (objective 0 first).
 *   - Return value: OPMOS_OK (0) or an OPMOS_ERR_* code. A failed call leaves
 *     no partial result (*out is set to NULL). opmos_last_error() gives a
 *     human-readable message for the calling thread. No C++ exception crosses
 *     this boundary. There is no CPU fallback: without a usable CUDA device
 *     every compute call fails with OPMOS_ERR_CUDA.
 *   - Limits: 1 <= d <= OPMOS_MAX_D; n < 2^31; m < 2^32; the graph must
 *     satisfy 2*(n-1)*max_e c_k(e) < 2^32 for every k (so g and F fit uint32),
 *     else OPMOS_ERR_OVERFLOW.
 */
#ifndef OPMOS_H_
#define OPMOS_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OPMOS_API __attribute__((visibility("default")))
#else
#define OPMOS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define OPMOS_MAX_D 16

enum {
  OPMOS_OK = 0,
  OPMOS_ERR_INVALID_ARG = 1,   /* bad id, bad d, non-monotone rowptr, col >= n, ... */
  OPMOS_ERR_OVERFLOW = 2,      /* cost bound above violated */
  OPMOS_ERR_OUT_OF_MEMORY = 3, /* device or host allocation failed */
  OPMOS_ERR_CAPACITY = 4,      /* a per-query arena (labels, frontiers, open list) filled up */
  OPMOS_ERR_BUDGET = 5,        /* the caller's label budget was exceeded */
  OPMOS_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up, or a search
                                  ran past its time limit (300 s of device time;
                                  OPMOS_TIME_LIMIT_MS in the environment, read at
                                  each call, overrides it) */
  OPMOS_ERR_CUDA = 7,          /* CUDA runtime error or no device */
  OPMOS_PENDING = 8            /* server: ticket not finished yet */
};

typedef struct opmos_graph opmos_graph;
typedef struct opmos_heur opmos_heur;
typedef struct opmos_result opmos_result;
typedef struct opmos_server opmos_server;

/* Search options. Zero in any field selects the library default. */
typedef struct opmos_options {
  uint32_t window;           /* W: target number of labels extracted per step (the NUM_POP of
                                Algorithm 2, Sec. 5). Steps take whole histogram bins of
                                (F[0], F[1]), so a step may take fewer, or more when the lowest
                                bin alone holds more (never more than max(4W, 16384); past that
                                bound which labels of the bin a step takes depends on thread
                                timing, the front does not). Default 1024 (single query), 256
                                (batch). */
  uint32_t lanes_per_label;  /* threads that expand one label's out-arcs: 4, 8, 16 or 32.
                                Default 8. */
  uint32_t tile;             /* frontier growth granule in entries (multiple of 32). Default 32. */
  uint32_t delta;            /* width of one F[0] bucket of the open list. 1 = exact
                                lexicographic-prefix windows. Default 1. */
  uint64_t label_budget;     /* max labels a query may create; exceeding it is
                                OPMOS_ERR_BUDGET. Default: unlimited (arena-bound). */
  uint64_t mem_budget_bytes; /* device arena per query (single) or per batch (batch).
                                Default: 8 GiB single, 160 GiB batch. */
  uint32_t d_used;           /* use only the first d_used objectives (Table 1 order rule,
                                Sec. 6.1). Default: all. */
  uint32_t flags;            /* OPMOS_FLAG_* */
  uint64_t alone_labels;     /* batch: a query that creates more labels than this in its slot of
                                the shared launch leaves it and is solved alone afterwards, on
                                the whole device with the same options but the window
                                alone_window (so with the front and paths opmos_solve gives
                                with that window). Default 1,000,000; UINT64_MAX: never. */
  uint32_t alone_window;     /* batch: the window of the queries solved alone. Default: the
                                window opmos_solve would take from these options. */
  uint32_t reserved;         /* 0 */
  void* stream;              /* cudaStream_t the work is issued on; NULL = default stream. */
} opmos_options;

#define OPMOS_FLAG_NO_PATHS 1u     /* skip path reconstruction (costs only) */
#define OPMOS_FLAG_GRAPH 2u        /* batch: capture each launch (input uploads from pinned staging,
                                      the persistent kernel, result downloads) into a CUDA graph and
                                      replay it; a capture failure is reported as OPMOS_ERR_CUDA */
#define OPMOS_FLAG_FIFO 4u         /* relaxed order: OPEN is a first-in first-out queue and each step
                                      takes its W oldest entries instead of the W lexicographically
                                      lowest F (the FIFO alternative of Sec. 4 and 7.1). The front is
                                      the same; the labels extracted are more. */

/* Counters of one solve (sums over a batch for batch results). Sec. 6.2 lists
 * the paper's counters: extractions, candidate labels, solutions. */
typedef struct opmos_stats {
  uint64_t extracted;      /* labels taken from OPEN and expanded */
  uint64_t dead_skipped;   /* OPEN entries dropped at extraction because pruned (lazy delete) */
  uint64_t goal_pruned;    /* OPEN entries dropped at extraction because P dominates F */
  uint64_t candidates;     /* (label, out-arc) candidates generated */
  uint64_t inserted;       /* labels created (frontier + OPEN inserts), including the start */
  uint64_t pruned;         /* frontier labels removed by a dominating candidate */
  uint64_t steps;          /* window steps */
  uint64_t frontier_cmp;   /* candidate-vs-frontier-entry vector comparisons */
  uint64_t p_cmp;          /* vector comparisons against P */
  uint64_t bytes;          /* algorithmic bytes of the search: per extracted label 8d+12, per
                              candidate 4+8d, per compared frontier or P entry 4d, per
                              inserted label 4d+24, per pruned label 4 */
  uint64_t heuristic_ns;   /* device time of the heuristic kernel(s) */
  uint64_t search_ns;      /* device time of the search kernel(s) */
  uint64_t total_ns;       /* host wall time of the call */
  uint64_t phase_ns[4];    /* device time of the search as seen by the leading thread:
                              [0] window selection and step control, [1] merge of window i
                              overlapped with extraction and expansion of window i+1,
                              [2] end of step (histogram flush, barrier wait), [3] output */
  uint64_t goal_inserted;  /* goal labels accepted into P during the search (before the final
                              removal of dominated members) */
  uint64_t open_scanned;   /* OPEN entries read by the extraction scans, summed over steps
                              (an entry read by two passes of one step counts twice) */
  uint64_t open_rewritten; /* OPEN entries copied forward to the next step's OPEN array */
  uint64_t list_candidates; /* candidates beyond the slots a node has per step (64 in a
                               batch, 128 for a single query), merged from the node's lists */
  uint64_t longest_task_ns[3]; /* summed over steps: the step's longest whole-block merge of a
                                  node with a large frontier, longest one-warp node merge, and
                                  longest extraction work item (the step's critical path) */
  uint64_t heavy_merges;   /* node merges done by one or more whole blocks (a large frontier,
                              or many candidates in the step) */
  uint64_t heavy_max_candidates; /* summed over steps: the most candidates, and the largest */
  uint64_t heavy_max_frontier;   /* frontier, of a node merged by whole blocks in the step */
  uint64_t task_ns[3];     /* summed durations of all block merges (one block each), one-warp
                              merges and extraction items (one warp each) */
} opmos_stats;

/* Fill *opt with the defaults (all fields explicit). */
OPMOS_API void opmos_default_options(opmos_options* opt);

/* Number of usable devices (0 if none) -- never fails. */
OPMOS_API int opmos_device_count(void);

/* Copy a CSR graph to the device (Sec. 3 input G = (V, E, c); Algorithm 1
 * "Input: edge costs C"). rowptr: n+1 entries, rowptr[0] = 0, non-decreasing,
 * rowptr[n] = m. col: m entries < n. cost: d*m entries, SoA as above.
 * The reversed CSR used by the heuristic is built on the host and uploaded
 * with the graph. Errors: INVALID_ARG, OVERFLOW, OUT_OF_MEMORY, CUDA. */
OPMOS_API int opmos_graph_create(uint32_t n, uint64_t m, uint32_t d, const uint64_t* rowptr,
                       const uint32_t* col, const uint32_t* cost, opmos_graph** out);
OPMOS_API void opmos_graph_destroy(opmos_graph* g);

/* Ideal-point heuristic toward goal (Sec. 4; Algorithm 1 "Input: heuristics H"):
 * h[k*n + v] = min over v->goal paths of the summed objective-k cost, or
 * 0xFFFFFFFF if the goal cannot be reached from v. Computed on the device by a
 * bucketed (near/far) reverse single-source shortest-path kernel; the result
 * stays device-resident. d_used = 0 means all objectives. */
OPMOS_API int opmos_heuristic(const opmos_graph* g, uint32_t goal, uint32_t d_used, opmos_heur** out);
/* Copy the heuristic to the host: h_out has d_used*n entries laid out as above. */
OPMOS_API int opmos_heuristic_copy(const opmos_heur* h, uint32_t* h_out);
OPMOS_API void opmos_heuristic_destroy(opmos_heur* h);

/* The heuristic of opmos_heuristic, written into a device buffer the caller
 * owns, with no device memory allocated during the call. The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc while they
 * run (all device memory reserved up front by their own pool allocator, or no
 * tolerance for the allocation and implicit synchronisation it can cause).
 *   h_out_device: device pointer to d_used*n uint32, layout as above
 *     (d_used = 0 means all objectives); stream: cudaStream_t or NULL.
 *   Limit: n <= 262144 nodes, else OPMOS_ERR_CAPACITY (use opmos_heuristic).
 *   Scratch: one fixed array inside the library (about 10.5 MB, held by each
 *     device that loads the library until exit). The first call on a device
 *     looks up its address (cudaGetSymbolAddress) with that device current;
 *     make that first call before any stream capture. Every call reuses the
 *     same array, so calls that overlap on the GPU (other threads, other
 *     streams) race: serialise them. Each call synchronises `stream` (it
 *     reads the kernel's status word back) and returns when the result is
 *     complete.
 *   Speed: the fixed array holds the worklists of 2 thread blocks, so the
 *     d_used single-objective searches run at most 2 at a time (opmos_heuristic
 *     runs all of them at once); for d_used > 2 the call takes up to
 *     ceil(d_used / 2) times as long. Errors: INVALID_ARG, CAPACITY, TIMEOUT, CUDA. */
OPMOS_API int opmos_heuristic_noalloc(const opmos_graph* g, uint32_t goal, uint32_t d_used,
                                      uint32_t* h_out_device, void* stream);

/* One start->goal query (Algorithm 2 semantics, exact result of Sec. 3).
 * heur may be NULL (computed here, its time reported in heuristic_ns); if
 * given it must belong to g and goal. opt may be NULL (defaults).
 * start == goal gives the front {0} with path [start]; an unreachable goal
 * gives OPMOS_OK with count 0. */
OPMOS_API int opmos_solve(const opmos_graph* g, const opmos_heur* heur, uint32_t start, uint32_t goal,
                const opmos_options* opt, opmos_result** out);

/* nq independent queries in one persistent cooperative launch with continuous
 * batching: up to 192 queries run at once in their own arenas (each
 * mem_budget_bytes / 192), all advancing one search step per grid iteration,
 * and a finished query's slot is refilled from the queue at once. A query
 * that outgrows its slot's arena, or creates more than opt->alone_labels
 * labels there, is re-run alone afterwards (the single-query arena and
 * kernel, window opt->alone_window). out receives nq results (each may be
 * NULL) and status[q] each
 * query's own return code; the call returns OPMOS_OK when the batch ran, even
 * if some queries failed. */
OPMOS_API int opmos_solve_batch(const opmos_graph* g, uint32_t nq, const uint32_t* starts,
                      const uint32_t* goals, const opmos_options* opt, opmos_result** out,
                      int* status);

/* Result accessors. */
OPMOS_API uint32_t opmos_result_count(const opmos_result* r);  /* |P| */
OPMOS_API uint32_t opmos_result_d(const opmos_result* r);
/* out: count*d uint32, row-major, lexicographically increasing. */
OPMOS_API int opmos_result_costs(const opmos_result* r, uint32_t* out);
/* Path of solution i (Sec. 3 path pi; reconstructed from parent pointers on
 * the device): nodes[0] = start ... nodes[len-1] = goal, edges[j] = arc id
 * from nodes[j] to nodes[j+1]. *len receives the node count; if it exceeds cap
 * nothing is written and OPMOS_ERR_CAPACITY is returned. Results solved with
 * OPMOS_FLAG_NO_PATHS return OPMOS_ERR_INVALID_ARG. */
OPMOS_API int opmos_result_path(const opmos_result* r, uint32_t i, uint32_t* nodes, uint64_t* edges,
                      uint32_t cap, uint32_t* len);
/* Every path at once, in flat arrays: offsets (count + 1 entries) such that
 * path i's nodes are nodes[offsets[i] .. offsets[i+1]) and its arcs
 * edges[offsets[i] - i .. offsets[i+1] - i - 1). nodes and edges may both be
 * NULL, to read the offsets first: offsets[count] nodes and
 * offsets[count] - count arcs in all. Results solved with
 * OPMOS_FLAG_NO_PATHS return OPMOS_ERR_INVALID_ARG. */
OPMOS_API int opmos_result_paths(const opmos_result* r, uint32_t* offsets, uint32_t* nodes, uint64_t* edges);
OPMOS_API int opmos_result_stats(const opmos_result* r, opmos_stats* out);
OPMOS_API void opmos_result_free(opmos_result* r);

/* Continuous-batching server over device-resident graphs. Queries submitted
 * while others run are admitted as soon as a slot and the device memory
 * budget (opt->mem_budget_bytes, default 64 GiB; one slot = a search arena of
 * 512 MiB, or of what opt->label_budget labels need when that is more, + a
 * 32 MiB result pool) allow; admitted queries run concurrently in
 * one persistent kernel that reads a queue in host-mapped memory, and each
 * result stays in its slot until opmos_server_poll collects it. submit
 * computes the query's heuristic on the SMs the resident kernel leaves free;
 * it fails with OPMOS_ERR_CAPACITY when 2 x slots queries are outstanding.
 * While a server exists, do not call the other compute entry points or
 * device-wide synchronising CUDA calls (cudaFree, cudaDeviceSynchronize) on
 * the same device: they wait for the resident kernel. A query whose arena
 * overflows reports OPMOS_ERR_CAPACITY (no retry). */
OPMOS_API int opmos_server_create(const opmos_graph* const* graphs, uint32_t ngraphs,
                        const opmos_options* opt, opmos_server** out);
/* d = number of leading objectives to use (0 = all). *ticket identifies it. */
OPMOS_API int opmos_server_submit(opmos_server* s, uint32_t graph, uint32_t d, uint32_t start,
                        uint32_t goal, uint64_t* ticket);
/* OPMOS_PENDING until done; then the query's own return code and, on OK, *out. */
OPMOS_API int opmos_server_poll(opmos_server* s, uint64_t ticket, opmos_result** out);
OPMOS_API void opmos_server_destroy(opmos_server* s);

/* Last error message of the calling thread ("" if none). */
OPMOS_API const char* opmos_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* OPMOS_H_ */
