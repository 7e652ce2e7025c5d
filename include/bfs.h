/*
 * bfs.h -- C ABI of the GB300 level-synchronous BFS library (libbfs.so).
 *
 * The operation (Section 2.2 of "Using Graph Properties to Speed-up GPU-based
 * Graph Traversal: A Model-driven Approach", Verstraaten, Varbanescu, de Laat):
 * given a graph and a root vertex, find every vertex reachable from the root
 * and its shortest hop distance. The traversal is level-synchronous (Section
 * 3.1): depths start at "infinity" (written -1 here), the root at 0, and level
 * L expands every vertex at depth L, assigning L + 1 to newly reached
 * vertices, until a level discovers nothing. At every level a binary decision
 * tree (Section 2.1, Section 4.1) over graph and frontier properties chooses
 * the kernel that expands the level; the choice is made on the device, so no
 * host round trip separates levels.
 *
 * Conventions for every entry point:
 *   - Return value: BFS_OK (0) or one of the BFS_ERR_* codes; no exception
 *     crosses this boundary. bfs_status_string() names a code and
 *     bfs_last_error_detail() gives the calling thread's last failure text.
 *   - Vertex ids are int32 in [0, n); the CSR uses int32 offsets and indices
 *     (m < 2^31). Depth is int32, -1 for unreached vertices.
 *   - "device" pointers are CUDA global-memory pointers of the current device;
 *     "host" pointers are ordinary CPU memory.
 *   - Runs are stream-ordered and asynchronous unless stated otherwise.
 *   - A bfs_graph_t may be used from several threads; each run takes its own
 *     workspace from a per-graph pool, so concurrent runs on distinct streams
 *     are safe as long as their depth outputs do not alias.
 */
#ifndef BFS_GB300_H
#define BFS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* bfs_stream_t;

typedef struct bfs_graph* bfs_graph_t;

enum bfs_status {
  BFS_OK = 0,
  BFS_ERR_INVALID_ARG = 1, /* null pointer, negative size, root out of range, bad option */
  BFS_ERR_BAD_GRAPH = 2,   /* CSR malformed: off[0] != 0, off decreasing, off[n] != m, idx out of range */
  BFS_ERR_OOM = 3,         /* a device or host allocation failed */
  BFS_ERR_CUDA = 4,        /* a CUDA runtime call failed; see bfs_last_error_detail() */
  BFS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (reported through a status word) */
  BFS_ERR_BUSY = 6,        /* a queue or pool is full; retry later */
  BFS_ERR_CANCELLED = 7,   /* work was cancelled before it ran */
  BFS_ERR_NOT_FOUND = 8,   /* unknown ticket, graph id or file */
};

/* Variants a level can run. The first BFS_NUM_VARIANTS are the classes the
 * decision tree predicts; the two edge-list kernels of Section 3.1.1 that scan
 * every edge of the graph each level can only be forced (bfs_options). */
enum bfs_variant {
  BFS_VARIANT_TREE = -1,        /* let the decision tree choose per level (default) */
  BFS_VARIANT_PUSH_THREAD = 0,  /* top-down, one thread per frontier vertex (Section 3.1.2, vertex push) */
  BFS_VARIANT_PUSH_WARP = 1,    /* top-down, virtual warp per frontier vertex (Section 3.1.3) */
  BFS_VARIANT_PUSH_CTA = 2,     /* top-down, one CTA per frontier vertex, adjacency staged in shared memory */
  BFS_VARIANT_PUSH_EDGE = 3,    /* top-down, one thread per frontier edge (Section 3.1.1, edge list
                                   restricted to the frontier's edges) */
  BFS_VARIANT_PULL = 4,         /* bottom-up over the visited bitmap, early exit (Section 3.1.2, vertex pull) */
  BFS_NUM_VARIANTS = 5,
  BFS_VARIANT_EDGE_LIST = 5,    /* every edge u->v of the graph, each level: v is reached when u is in the
                                   frontier (Section 3.1.1, edge list); builds a per-edge origin array
                                   (m int32) on first use */
  BFS_VARIANT_REVERSE_EDGE_LIST = 6, /* every edge by destination (the transpose), each level: an unreached v
                                   is reached when its source is in the frontier (Section 3.1.1, reverse
                                   edge list); origin array of the transpose on first use */
  BFS_NUM_FORCED_VARIANTS = 7,
};

/* Flags of bfs_graph_create. */
enum bfs_graph_flags {
  BFS_SYMMETRIC = 1u,       /* caller asserts every edge u->v has v->u; pull then reuses the CSR */
  BFS_INPUT_ON_DEVICE = 2u, /* row_offsets / col_indices are device pointers (else host) */
  BFS_VALIDATE = 4u,        /* accepted for clarity: the CSR is always validated on the device */
};

/* Feature vector layout of the decision tree (Section 4.1 features): graph
 * size; the out-degree 5-number summary (nearest rank, sorted[floor(k (n-1) /
 * 4)]) and floor(256 sd); the level's frontier and discovered counts (also in
 * parts per million of n), the frontier's out-degree sum and the level index;
 * then the in-degree and total-degree (in + out) summaries, Section 4.1's
 * degree distribution of in-, out- or total degree (for a symmetric graph the
 * in-degree summary equals the out-degree one). */
enum bfs_feature {
  BFS_F_N = 0, BFS_F_M = 1, BFS_F_DEG_MIN = 2, BFS_F_DEG_Q1 = 3, BFS_F_DEG_MED = 4, BFS_F_DEG_Q3 = 5,
  BFS_F_DEG_MAX = 6, BFS_F_DEG_SD256 = 7, BFS_F_FRONTIER = 8, BFS_F_FRONTIER_PPM = 9, BFS_F_DISCOVERED = 10,
  BFS_F_DISCOVERED_PPM = 11, BFS_F_FRONTIER_EDGES = 12, BFS_F_LEVEL = 13,
  BFS_F_IN_DEG_MIN = 14, BFS_F_IN_DEG_Q1 = 15, BFS_F_IN_DEG_MED = 16, BFS_F_IN_DEG_Q3 = 17, BFS_F_IN_DEG_MAX = 18,
  BFS_F_IN_DEG_SD256 = 19, BFS_F_TOT_DEG_MIN = 20, BFS_F_TOT_DEG_Q1 = 21, BFS_F_TOT_DEG_MED = 22,
  BFS_F_TOT_DEG_Q3 = 23, BFS_F_TOT_DEG_MAX = 24, BFS_F_TOT_DEG_SD256 = 25, BFS_NUM_FEATURES = 26,
};

typedef struct bfs_graph_info {
  int64_t n;                 /* vertices */
  int64_t m;                 /* directed CSR entries */
  int64_t deg_summary[5];    /* out-degree min, Q1, median, Q3, max: sorted[floor(k (n-1) / 4)] */
  int64_t deg_sd256;         /* floor(256 * population standard deviation of out-degree) */
  int64_t in_deg_summary[5]; /* the same for in-degree */
  int64_t in_deg_sd256;
  int64_t tot_deg_summary[5]; /* the same for total degree (in + out) */
  int64_t tot_deg_sd256;
  int64_t bytes_resident;    /* device bytes held by the graph (CSR, transpose, stats) */
  int32_t symmetric;         /* 1 if pull reuses the CSR, 0 if a transpose was built */
  int32_t num_workspaces;    /* per-run workspaces currently allocated */
} bfs_graph_info_t;

/* How the level loop is driven (all run the same level code and give the same depths). */
enum bfs_mode {
  BFS_MODE_DEFAULT = 0,    /* persistent when the device supports cooperative launch, else graph */
  BFS_MODE_PERSISTENT = 1, /* one cooperative kernel for the whole traversal; levels separated by a grid barrier */
  BFS_MODE_GRAPH = 2,      /* one CUDA graph per workspace: WHILE node over levels, SWITCH node over
                              the variant kernels; runs on different streams overlap */
  BFS_MODE_HOST_LOOP = 3,  /* the graph's kernels launched level by level from the host (for profilers) */
};

typedef struct bfs_options {
  int32_t forced_variant;    /* BFS_VARIANT_TREE or a fixed bfs_variant (< BFS_NUM_FORCED_VARIANTS) for
                                every level */
  int32_t depth_on_host;     /* 1: depth_out is host memory; the library copies the result there */
  int32_t mode;              /* enum bfs_mode */
  int32_t grid_blocks;       /* persistent driver: blocks of the cooperative grid, 0 for one full
                                occupancy wave (larger values are clamped to it). Fewer blocks let
                                several traversals be resident at once and shorten the grid barrier
                                (latency-bound, high-diameter graphs). Must be 0 for BFS_MODE_GRAPH
                                and BFS_MODE_HOST_LOOP, and >= 0. */
  int32_t count_mode;        /* how the vertex-push variant appends reached vertices to the next queue,
                                the Section 3.1.4 comparison: 0 block-local stage and one global atomic
                                per flush (the default, and the only mode of the other variants), 1 one
                                global atomic per warp, 2 one global atomic per vertex. Nonzero only
                                with BFS_MODE_HOST_LOOP. */
  int32_t host_async;        /* with depth_on_host and no stats: 1 returns once the copy to depth_out is
                                enqueued on `stream` (the caller synchronises `stream` before reading
                                depth_out), so that with pinned host memory one traversal's copy
                                overlaps the next traversal on another stream (a copy to pageable
                                memory completes before the call returns); 0 (the default) returns
                                after the copy has landed */
  int32_t reserved[2];       /* must be zero */
} bfs_options;

typedef struct bfs_run_stats {
  int64_t edges_reached;     /* sum of out-degrees of reached vertices */
  int64_t vertices_reached;  /* vertices with depth >= 0 */
  int32_t levels;            /* nonempty levels (max depth + 1) */
  int32_t status;            /* device-side status word (BFS_OK or BFS_ERR_TIMEOUT) */
  /* Per-level log, optional (set pointers to NULL to skip). Entry L describes
   * the frontier of level L and the variant that expanded it. At most
   * log_capacity entries are written; levels beyond it are counted only. */
  int32_t log_capacity;
  int32_t* log_variant;      /* host, log_capacity entries */
  int64_t* log_frontier;     /* host, vertices in the frontier of level L */
  int64_t* log_frontier_edges; /* host, sum of out-degrees over that frontier */
  int64_t* log_time_ns;      /* host, log_capacity + 1 entries: device %globaltimer (ns) at the start
                                of level L, and entry [levels] at the end (graph and persistent drivers) */
  int64_t start_ns;          /* device %globaltimer (ns) when the run's first kernel started, before the
                                depth initialisation (same clock as log_time_ns) */
} bfs_run_stats;

/* Text of a status code (static storage). */
const char* bfs_status_string(int status);

/* Detail of the calling thread's last failure (thread-local storage; valid until the next call). */
const char* bfs_last_error_detail(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int bfs_version(void);

/*
 * Create a graph from a CSR (Section 4.3: CSR, one int per vertex plus one per
 * edge). row_offsets has n + 1 entries, col_indices m entries; each adjacency
 * list is the out-neighbours of its vertex. The library copies both arrays into
 * device memory it owns (the caller keeps ownership of its buffers), computes
 * the out-degree statistics the decision tree uses (Section 4.1), and, without
 * BFS_SYMMETRIC, builds the transpose that the pull variant reads. Self-loops
 * and duplicate entries are allowed and never change a depth. Synchronous.
 * The CSR is always validated (a malformed one would make kernels read out
 * of bounds). Errors: BFS_ERR_INVALID_ARG (n < 1, n or m >= 2^31, null
 * pointers, unknown flags), BFS_ERR_BAD_GRAPH, BFS_ERR_OOM, BFS_ERR_CUDA.
 */
int bfs_graph_create(const int32_t* row_offsets, const int32_t* col_indices, int64_t n, int64_t m, uint32_t flags,
                     bfs_graph_t* out);

/* Free a graph and its workspaces after waiting for its runs to finish. NULL is a no-op. */
int bfs_graph_destroy(bfs_graph_t g);

/* Sizes and degree statistics of a graph (host struct, filled synchronously). */
int bfs_graph_info(bfs_graph_t g, bfs_graph_info_t* info);

/*
 * Virtual-warp width policy of the push_warp variant, per graph (Section 3.1.3:
 * virtual warps of W lanes per frontier vertex, and the right W depends on the
 * graph and the level). BFS_VW_RULE (the default): the power of two nearest
 * above the level's mean frontier degree floor(e / f), clamped to [4, 32];
 * BFS_VW_RULE_X2 / BFS_VW_RULE_HALF: that width doubled / halved (clamped);
 * BFS_VW_4 .. BFS_VW_32: one width for every level. It applies to every driver
 * and to forced push_warp runs; the tree's choice of variant is unchanged.
 */
enum bfs_warp_width {
  BFS_VW_RULE = 0,
  BFS_VW_RULE_X2 = 1,
  BFS_VW_RULE_HALF = 2,
  BFS_VW_4 = 3,
  BFS_VW_8 = 4,
  BFS_VW_16 = 5,
  BFS_VW_32 = 6,
  BFS_VW_NUM = 7
};

/* Set or read a graph's width policy. Not concurrent with runs on the graph
 * (runs already enqueued keep the policy they were launched with).
 * BFS_ERR_INVALID_ARG for a policy outside [0, BFS_VW_NUM). */
int bfs_set_warp_width(bfs_graph_t g, int32_t policy);
int bfs_get_warp_width(bfs_graph_t g, int32_t* policy);

typedef struct bfs_warp_tune {
  int32_t policy;          /* the fastest policy, now set on the graph */
  int32_t reserved;
  float ms[BFS_VW_NUM];    /* device time of the k traversals under each policy */
} bfs_warp_tune;

/*
 * Autotune the width policy: for each policy, one untimed traversal and then
 * the k traversals from roots (host, 1..4096 int32) timed on `stream` with the
 * default driver and the tree; the fastest policy is set on the graph and
 * returned with every policy's time (host struct). Synchronous; allocates an
 * n-entry depth buffer for its duration. Not concurrent with other runs on the
 * graph.
 */
int bfs_tune_warp_width(bfs_graph_t g, const int32_t* roots, int32_t k, bfs_stream_t stream, bfs_warp_tune* out);

/*
 * Load the process-wide decision tree (Section 2.1, Section 4.3: the trained
 * tree exported as an array plus a lookup function) from a text file, or with
 * NULL restore the built-in tree. File format: optional '#' comment lines, then
 * "bfs-tree 1 <num_nodes>", then one line per node "feature threshold left right
 * value": feature -1 marks a leaf whose value is the predicted variant, or -1
 * for an unknown prediction (Section 4.1); an internal node sends x[feature] <=
 * threshold to `left`, otherwise to `right`. Runs started afterwards use the new
 * tree. Errors: BFS_ERR_NOT_FOUND (file), BFS_ERR_INVALID_ARG (malformed tree).
 */
int bfs_load_tree(const char* path_or_null);

/*
 * Single-source BFS (Section 2.2, Section 3.1). depth_out: device, n int32,
 * caller-owned; on completion depth_out[v] is the hop distance from root, or
 * -1. Asynchronous on `stream`; the result is valid once the stream reaches
 * this point. Errors: BFS_ERR_INVALID_ARG (root not in [0, n), null pointers),
 * BFS_ERR_OOM (no workspace), BFS_ERR_CUDA.
 */
int bfs_run(bfs_graph_t g, int32_t root, int32_t* depth_out, bfs_stream_t stream);

/*
 * bfs_run with options and statistics. With opts->depth_on_host, depth_out is
 * host memory and the call returns after the result has been copied there
 * (with opts->host_async, once the copy is enqueued on `stream`).
 * With stats != NULL the call synchronises `stream` and fills *stats (host);
 * it then also returns the device-side status (BFS_ERR_TIMEOUT if a bounded
 * wait gave up). opts may be NULL (tree switching, device output).
 */
int bfs_run_ex(bfs_graph_t g, int32_t root, int32_t* depth_out, bfs_stream_t stream, const bfs_options* opts,
               bfs_run_stats* stats);

/*
 * Multi-source BFS: k independent traversals of one graph (the result equals k
 * single-source runs, each the level-synchronous BFS of Section 3.1). roots:
 * host, k int32 (repeats allowed). depth_out: device, k * n int32, row-major
 * (row i for roots[i]), caller-owned. Roots are processed in waves of up to 64
 * by one persistent kernel per wave, one bit per root in 64-bit visited /
 * frontier masks per vertex, each level pushing or pulling for all roots at
 * once; the frontier masks of depths 0-14 are kept per depth until the wave
 * ends, when each output row is written once from them (deeper depths are
 * written when found; 164 n bytes of buffers in all, allocated on the first
 * call and kept with the graph).
 * Batches on one graph are ordered after each other on the device.
 * edges_out: optional host array of k int64 reached-edge counts; when given,
 * the call synchronises `stream`. Errors as bfs_run.
 */
int bfs_run_batch(bfs_graph_t g, const int32_t* roots, int32_t k, int32_t* depth_out, bfs_stream_t stream,
                  int64_t* edges_out);

/* Launch shape of the multi-source kernel (chosen by bfs_batch_tune). */
typedef struct bfs_batch_config {
  int32_t push_mode;  /* 0: one thread per frontier vertex, 1: one warp per frontier vertex */
  int32_t alpha;      /* a level pulls when its frontier's edge count x alpha exceeds m */
  float ms;           /* bfs_batch_tune: measured time of one wave with this configuration */
  int32_t grid_blocks; /* blocks of the multi-source kernel (larger values are clamped to one full
                          occupancy wave); 0 for a grid sized to the graph: one block per 4096
                          vertices, at least a quarter of the SMs, at most one full occupancy
                          wave (so that small graphs' waves on several streams run together) */
} bfs_batch_config;

/* Set the graph's multi-source configuration. Errors: BFS_ERR_INVALID_ARG. */
int bfs_batch_set_config(bfs_graph_t g, const bfs_batch_config* cfg);

/*
 * Autotuner: time one wave of the given roots (host, 1..64) with every
 * candidate configuration (push mode x alpha in {2, 4, ..., 64} x grid of a
 * full occupancy wave, a half or a quarter of it; CUDA events on `stream`, one
 * warm-up run each), keep the fastest for the graph and return it in *best.
 * depth_scratch: device, k * n int32, overwritten. Synchronous.
 */
int bfs_batch_tune(bfs_graph_t g, const int32_t* roots, int32_t k, int32_t* depth_scratch, bfs_stream_t stream,
                   bfs_batch_config* best);

/*
 * The autotuner for waves that run together: `concurrency` (1..64) waves of
 * different graphs at once, as with a batch spread over that many streams.
 * The grids tried are those no larger than twice a full occupancy wave
 * divided by `concurrency` (waves of uneven graphs rarely all run at once; at
 * least 1/16 of a full wave), halving, the three largest; the rest as
 * bfs_batch_tune (which is concurrency 1: a full wave, 1/2 and 1/4).
 * Smaller grids let the waves share the device, where one wave alone is
 * fastest on the full grid.
 */
int bfs_batch_tune_ex(bfs_graph_t g, const int32_t* roots, int32_t k, int32_t* depth_scratch, bfs_stream_t stream,
                      int32_t concurrency, bfs_batch_config* best);

/*
 * Single-source BFS that allocates nothing. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while they
 * run (code working inside a memory arena it does not own, a plugin given
 * fixed buffers by its host application, a real-time loop where cudaMalloc may
 * stall or fail). It makes no cudaMalloc, cudaFree or other allocating call,
 * and needs no bfs_graph_t: the caller passes the CSR (row_offsets, n + 1
 * int32; col_indices, m int32) and depth_out (n int32) in device memory it
 * owns, and gets the same depths as bfs_run.
 *
 * Limit: n <= 1,048,576 vertices; larger n returns BFS_ERR_INVALID_ARG. The
 * traversal's scratch (two frontier queues, the visited bitmap, counters) is a
 * fixed device array of about 8.1 MB inside the library, held by every GPU that
 * loads the library until the process exits. Every call looks up that array's
 * device address in the current device's context (cudaGetSymbolAddress, which
 * allocates nothing), so a device reset between calls leaves no stale address;
 * the first call on a device also loads the library's kernels there, so make
 * that first call before any stream capture. `stream` must belong to the
 * current device (BFS_ERR_INVALID_ARG otherwise); NULL is the legacy default
 * stream. A launch that fails returns BFS_ERR_CUDA with the CUDA error text in
 * bfs_last_error_detail(). All calls share
 * the one array, which keeps the previous call's contents (each call clears
 * what it reads first): calls whose work overlaps on the GPU, from any stream
 * or thread, race and corrupt each other, so serialise them. The CSR is
 * validated on every call (BFS_ERR_BAD_GRAPH). Synchronous: the level loop
 * reads each level's frontier size back to the host. Uses a simple one thread
 * per frontier vertex push for every level (no tree switching).
 */
int bfs_run_static(const int32_t* row_offsets, const int32_t* col_indices, int64_t n, int64_t m, int32_t root,
                   int32_t* depth_out, bfs_stream_t stream);

/*
 * Serving: a request loop over graphs resident in HBM (the paper has no
 * serving layer; this wraps the Section 3.1 traversal for many concurrent
 * queries). A dispatcher thread admits submitted single-root queries whenever
 * an in-flight slot and the memory the unit needs fit the budget, first fit
 * over the head of the queue. A unit is one query's traversal (charged its
 * workspace, plus an n-entry depth buffer when the caller passes none) or a
 * multi-source wave merging up to merge_batch queued queries of one graph
 * (charged one wave buffer set, 164 n bytes, plus a depth buffer per query
 * without one): continuous batching. Units run on a pool of streams and overlap
 * on the device; each wave root's depths go straight to its query's buffer.
 * Results are the same as alone: depths are exact. Workspaces, depth buffers
 * and wave sets are allocated when a graph is registered; the dispatcher
 * allocates no device memory (a unit whose pool is empty waits). A serving
 * process should start with CUDA_DEVICE_MAX_CONNECTIONS=32 in its environment
 * (read when the CUDA context is created): with CUDA's default of 8 hardware
 * queues, a unit's completion copy waits in a queue that other streams share,
 * behind long traversals, and short queries wait with it.
 */
typedef struct bfs_server* bfs_server_t;

typedef struct bfs_serve_config {
  int64_t mem_budget_bytes; /* device bytes admitted queries may hold at once; 0 = unlimited */
  int32_t max_inflight;     /* admitted units (queries or merged waves) on the device at once, 1..1024 */
  int32_t num_streams;      /* streams the units are spread over, 1..1024 */
  int32_t queue_capacity;   /* pending submissions before bfs_serve_submit returns BFS_ERR_BUSY */
  int32_t merge_batch;      /* up to this many queued queries to one graph run as one wave (0 or 1: off; <= 64) */
  int32_t merge_policy;     /* 0: merge a graph's queries where the registration probe found a wave
                               cheaper per query than single runs; 1: merge wherever merge_batch allows */
  int32_t reserved;         /* must be zero */
} bfs_serve_config;

typedef struct bfs_serve_stats {
  int64_t submitted, admitted, completed, rejected, failed;
  int64_t peak_bytes_inflight; /* largest admitted memory at once */
  int32_t merged_waves;        /* waves that merged several queries */
  int32_t queued;              /* submissions waiting now */
  double qps;                  /* completed / (last completion - first submission) */
  double p50_ms, p99_ms, max_ms; /* submission-to-completion latency */
  double gteps;                /* sum of edges_reached / 2 over completed queries / the same wall time / 1e9 */
  double wait_p50_ms, wait_p99_ms; /* submission-to-admission part of the latency (time queued) */
} bfs_serve_stats_t;

/* Start a server (and its dispatcher thread) on the current device. */
int bfs_serve_create(const bfs_serve_config* cfg, bfs_server_t* out);
/* Register a graph (same device; up to 256; the caller keeps it alive until
 * bfs_serve_destroy). Synchronous: probe runs on a private stream size the
 * graph's queries. Traversals from vertices 0, n/3, 2n/3 and n-1 pick the one
 * reaching the most edges; it is timed on 8, 16, 32, 64 blocks, one and
 * two per SM and a full occupancy wave, and queries get the count with the least
 * blocks x time among those at most 4x slower than the fastest. One 64-root
 * multi-source wave (roots the probe reached, on the wave grid of at most two
 * blocks per SM that merged queries run on; needs 420 n bytes of temporary
 * memory, skipped if that does not fit) decides whether queued queries are
 * merged (merge_policy 0): when its blocks x time per root is below a single
 * query's. Then the graph's pools are allocated: min(max_inflight, 64, the
 * number the memory budget admits at once) traversal workspaces, and when its
 * queries may merge (merge_batch > 1 and the probe or merge_policy 1 allows
 * it) two wave buffer sets (164 n bytes
 * each, so two waves of the graph can run at once), plus n-entry depth buffers
 * for queries submitted without one (one per workspace and merge_batch per
 * set). Takes a few traversals' time, up to a few seconds on a high-diameter
 * graph of 16M vertices. BFS_ERR_OOM if the pools do not fit. */
int bfs_serve_add_graph(bfs_server_t s, bfs_graph_t g, int32_t* graph_id);
/* The launch shape registration chose for a graph: *query_blocks, the blocks of
 * one query's persistent grid, and *merges, 1 when its queued queries may be
 * merged into waves under merge_policy 0. BFS_ERR_NOT_FOUND for an unknown id. */
int bfs_serve_graph_shape(bfs_server_t s, int32_t graph_id, int32_t* query_blocks, int32_t* merges);
/* Device bytes a single query of the graph is charged against mem_budget_bytes
 * when it is admitted (its traversal workspace, plus an n-entry depth buffer
 * when with_output is 0, i.e. when the caller passes no depth_out).
 * BFS_ERR_NOT_FOUND for an unknown id. */
int bfs_serve_query_bytes(bfs_server_t s, int32_t graph_id, int32_t with_output, int64_t* bytes);
/* Queue a query; non-blocking. depth_out: device, n int32, or NULL (the server
 * supplies a buffer and the depths are not returned). The server's streams do
 * not wait on the caller's streams: depth_out must be ready to be written when
 * submitted, and is valid once the query is done. BFS_ERR_BUSY when the queue
 * is full, BFS_ERR_NOT_FOUND for an unknown graph id. *ticket identifies it. */
int bfs_serve_submit(bfs_server_t s, int32_t graph_id, int32_t root, int32_t* depth_out, uint64_t* ticket);
/* *state: 0 done, 1 queued, 2 running. Returns the query's status once done
 * (BFS_OK before), BFS_ERR_NOT_FOUND for an unknown or long-retired ticket. */
int bfs_serve_poll(bfs_server_t s, uint64_t ticket, int* state);
/* Block until the query is done (timeout_us < 0: no limit). BFS_ERR_TIMEOUT if
 * it is still pending after timeout_us; otherwise the query's status. */
int bfs_serve_wait(bfs_server_t s, uint64_t ticket, int64_t timeout_us);
/* Counters and latency percentiles since creation or the last
 * bfs_serve_reset_stats (host struct). */
int bfs_serve_stats(bfs_server_t s, bfs_serve_stats_t* out);
/* Start a new statistics window: counters, latency records and the wall-time
 * origin are cleared (queries in flight are counted in the new window when they
 * complete). */
int bfs_serve_reset_stats(bfs_server_t s);
/* Load shedding: every query still queued (not yet admitted) finishes with
 * BFS_ERR_CANCELLED; running ones are not touched. *cancelled (optional)
 * receives how many were cancelled. */
int bfs_serve_cancel_queued(bfs_server_t s, int64_t* cancelled);
/* Let running queries finish, cancel queued ones (BFS_ERR_CANCELLED), stop the
 * dispatcher and free the server. A query larger than the whole budget is
 * admitted when nothing else is in flight, so every query eventually runs. */
int bfs_serve_destroy(bfs_server_t s);

/* One level of a profiled traversal. */
typedef struct bfs_level_profile {
  int64_t features[BFS_NUM_FEATURES]; /* the tree's input at this level (enum bfs_feature order) */
  float ms[BFS_NUM_VARIANTS];         /* median device time of each variant expanding this level */
  int32_t tree_variant;               /* the current tree's choice (after the unknown-prediction rule) */
  int32_t pad;
} bfs_level_profile;

/*
 * Per-level timing harness (Section 4.1: the fastest implementation of every
 * level labels the training set). Runs the traversal from `root` level by level
 * with a host round trip per level; at each level every variant expands the
 * level `reps` times from the same state, the state being restored after each
 * run (the level's discoveries undone), the median time is recorded, and the
 * traversal advances with `advance_variant` (or the tree's choice when
 * BFS_VARIANT_TREE). Where the device supports cooperative launch, each run is
 * one level of the persistent driver (the default driver): a cooperative
 * launch of the same level code on the same grid, timed with device
 * timestamps from its start barrier to the end of its level-ending barrier.
 * Otherwise each run is the graph driver's kernels for the level, timed with
 * CUDA events on `stream`. out: host, `capacity` entries; levels beyond it are
 * traversed but not recorded. *num_levels: levels traversed. Synchronous. Uses
 * a private depth buffer (the graph's caller buffers are not touched). Errors:
 * BFS_ERR_INVALID_ARG, BFS_ERR_OOM, BFS_ERR_CUDA, BFS_ERR_TIMEOUT.
 */
int bfs_profile_levels(bfs_graph_t g, int32_t root, int32_t reps, int32_t advance_variant, bfs_stream_t stream,
                       bfs_level_profile* out, int32_t capacity, int32_t* num_levels);

/*
 * Test hook: make the n-th device allocation made by the library from now on
 * fail with BFS_ERR_OOM (n = 0 disables). Lets tests exercise the out-of-memory
 * paths without exhausting a shared GPU.
 */
int bfs_debug_fail_alloc_after(int n);

/*
 * Test hook: make one bounded device-side wait of the next persistent
 * traversal (bfs_run / bfs_run_ex in the persistent driver) or multi-source
 * wave (bfs_run_batch) launched by this process run out, so that tests can
 * check the timeout path without hanging or faulting a GPU. mode 1: the
 * launch's first grid barrier expects one arrival more than the grid has;
 * mode 2: the first level-ending barrier of a traversal, likewise; mode 3: the
 * first adjacency copy staged by the CTA push expects 16 bytes more than it
 * copies (a level the CTA push expands with a list of 512 entries or more).
 * Every wait of the library is bounded (about 2 s), so the kernel gives up,
 * records BFS_ERR_TIMEOUT in its status word (bfs_run_ex with stats, or
 * bfs_run_batch with edges_out, returns it) and exits; the next launch on the
 * same graph resets that state and runs normally. The hook is taken by the
 * first launch that reads it; mode 0 clears it. Errors: BFS_ERR_INVALID_ARG.
 */
int bfs_debug_stall_next_launch(int mode);

#ifdef __cplusplus
}
#endif

#endif /* BFS_GB300_H */
