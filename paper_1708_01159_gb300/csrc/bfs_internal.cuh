// Internal types and device helpers of libbfs (GB300, sm_103a).
//
// Data layout in HBM (one graph):
//   off[n+1], idx[m + pad]      out-edge CSR, int32; idx padded so that
//                               16-byte-aligned bulk copies may overrun by < 16 B
//   in_off/in_idx               transpose for the pull variant (aliases off/idx
//                               when the graph is symmetric)
// Per run (one workspace):
//   q[2][n]                     frontier queues (input / output, swapped per level)
//   vis[2][ceil(n/32)]          visited bitmaps; push updates the current one in
//                               place, pull reads the current and writes the other
//   pe_*                        scratch of the edge-centric variant (degree scan)
//   RunState                    level, counters, variant, status, log pointers
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct bfs_graph;  // the C ABI's graph object (defined in bfs_api.cu)

namespace bfs {

enum Variant : int32_t {
  V_PUSH_THREAD = 0,
  V_PUSH_WARP = 1,
  V_PUSH_CTA = 2,
  V_PUSH_EDGE = 3,
  V_PULL = 4,
  V_NUM = 5,  // the variants the tree predicts
  // Section 3.1.1's two kernels over the whole edge list, selectable as a
  // forced variant (not predicted by the tree)
  V_EDGE_LIST = 5,
  V_REV_EDGE_LIST = 6,
  V_FORCED_NUM = 7,
};

// Virtual-warp width policy of the push_warp variant (Section 3.1.3: the right
// width depends on the graph and the level), chosen per graph by the tuner:
// the rule (the power of two nearest above the frontier's mean degree,
// clamped to [4, 32]), the rule doubled or halved (clamped), or one fixed
// width for every level.
enum WarpWidthPolicy : int32_t {
  VW_RULE = 0,
  VW_RULE_X2 = 1,
  VW_RULE_HALF = 2,
  VW_4 = 3,
  VW_8 = 4,
  VW_16 = 5,
  VW_32 = 6,
  VW_NUM = 7,
};

// How a push level appends the vertices it reaches to the next queue (whose
// tail is the next frontier size). Section 3.1.4 compares a global atomic per
// vertex with warp and block reductions in front of it; the level kernels use
// CM_BLOCK, and the others exist for that comparison (vertex push, host loop).
enum CountMode : int32_t {
  CM_BLOCK = 0,   // block-local shared-memory stage, one global atomic per flush
  CM_WARP = 1,    // one global atomic per group of converged lanes
  CM_ATOMIC = 2,  // one global atomic per vertex
  CM_NUM = 3,
};

// Section 4.1 features, in the order the tree file indexes them: graph size,
// the out-degree 5-number summary and standard deviation, the level's
// frontier and discovered counts, then the in-degree and total-degree
// summaries (Section 4.1 names the degree distribution of in-, out- or total
// degree; for a symmetric graph in-degree equals out-degree).
enum Feature : int32_t {
  F_N = 0, F_M, F_DEG_MIN, F_DEG_Q1, F_DEG_MED, F_DEG_Q3, F_DEG_MAX, F_DEG_SD256,
  F_FRONTIER, F_FRONTIER_PPM, F_DISCOVERED, F_DISCOVERED_PPM, F_FRONTIER_EDGES, F_LEVEL,
  F_IN_DEG_MIN, F_IN_DEG_Q1, F_IN_DEG_MED, F_IN_DEG_Q3, F_IN_DEG_MAX, F_IN_DEG_SD256,
  F_TOT_DEG_MIN, F_TOT_DEG_Q1, F_TOT_DEG_MED, F_TOT_DEG_Q3, F_TOT_DEG_MAX, F_TOT_DEG_SD256,
  F_NUM,
};

// A feature of the graph itself (the same at every level), as opposed to one
// of the level (frontier, discovered, frontier edges, level index).
__host__ __device__ constexpr bool is_graph_feature(int32_t f) { return f < F_FRONTIER || f >= F_IN_DEG_MIN; }

enum Status : int32_t { ST_OK = 0, ST_TIMEOUT = 5 };

// Test hook (bfs_debug_stall_next_launch): which bounded wait of the next
// persistent traversal or multi-source wave is made to run out.
enum Stall : int32_t {
  STALL_NONE = 0,
  STALL_GRID_BARRIER = 1,   // the first grid barrier expects one arrival more than the grid has
  STALL_LEVEL_BARRIER = 2,  // the first level-ending barrier of a traversal, likewise
  STALL_BULK_COPY = 3,      // the first staged adjacency copy of the CTA push expects 16 bytes more than it copies
};

// Section 4.1: an unknown prediction at the first level falls back to the
// edge list implementation (the edge-centric push here).
constexpr int32_t kLevel0Default = V_PUSH_EDGE;

constexpr int kIdxPad = 8;  // int32 entries of slack after idx
constexpr int kHintScan = 64;  // in-list entries examined when a vertex's pull hint is chosen

struct TreeNode {
  long long t;  // threshold: x[f] <= t goes left
  int32_t f;    // feature, -1 for a leaf
  int32_t l, r;
  int32_t v;    // leaf class, -1 = unknown prediction
};
static_assert(sizeof(TreeNode) == 24, "TreeNode layout");

// Bit-parallel form of a small tree (the QuickScorer evaluation of Lucchese et
// al., SIGIR 2015): the leaves are numbered left to right; internal node k,
// when its test x[f] <= t fails, clears the bits of the leaves of its left
// subtree; after every failed test has cleared its bits, the lowest bit left
// is the leaf the walk from the root reaches. All tests are independent, so
// the lanes of a warp evaluate one each and AND the masks, instead of a chain
// of dependent steps. Built on the host for one graph, for trees of at most
// kQsMax internal nodes and kQsMax leaves: the tests on the graph's own
// features (n, m, degree summaries) have the same outcome at every level, so the
// host folds them into `base` and only the tests on level features
// (frontier, discovered, frontier edges, level) remain in node[].
constexpr int kQsMax = 64;
struct QsNode {
  long long t;
  unsigned long long mask;  // all ones except the bits of the left subtree's leaves
  int32_t f;                // a level feature: F_FRONTIER, F_DISCOVERED, F_FRONTIER_EDGES or F_LEVEL
  int32_t pad;
};
struct QsTree {
  int32_t n_int;             // remaining (level-feature) internal nodes
  int32_t n_leaf;            // leaves
  unsigned long long base;   // AND of the masks of the graph-feature tests that fail on this graph
  QsNode node[kQsMax];
  int32_t leaf[kQsMax];  // class of each leaf, left to right (-1: unknown)
  // Box of each leaf: the level-feature values that reach it (its path's
  // tests; empty for a leaf this graph's graph-feature tests rule out).
  // box[b][2k] <= x_k <= box[b][2k + 1] for the level features k = frontier,
  // discovered, frontier edges, level (bounds clamped to int32: every such
  // feature lies in [0, 2^31)). A level whose features stay in the previous
  // level's leaf box reaches the same leaf, so its tree walk can be skipped.
  int32_t box[kQsMax][8];
};

// Origin of every CSR entry (the vertex whose row holds it) and of every
// transpose entry, for the edge-list variants; null until first needed
// (origin_in is origin_out for a symmetric graph).
struct GraphAux {
  const int32_t* origin_out;
  const int32_t* origin_in;
};

struct DevGraph {
  const int32_t* off;
  const int32_t* idx;
  const int32_t* in_off;
  const int32_t* in_idx;
  // visited bitmap a traversal starts from (before the root's bit): bit v set
  // iff v has no edges at all, so no level reaches it and pull never scans it
  const uint32_t* vis_init;
  // device block holding the edge-list variants' origin arrays (filled on
  // their first use; kernels read it at run time, so CUDA graphs built before
  // then see the arrays too)
  const struct GraphAux* aux;
  // per vertex, the in-neighbour with the largest out-degree among the first
  // kHintScan entries of its in-list (-1 without in-edges): the pull variant
  // tests it first, since a high-degree in-neighbour is the likeliest to be
  // in an early frontier
  const int32_t* hint;
  int32_t n;
  int32_t m;
  int32_t words;  // ceil(n / 32)
  int32_t symmetric;
  int32_t n_active;  // vertices with at least one in- or out-edge (the others start visited)
  int32_t vw_policy;  // virtual-warp width policy of the push_warp variant (VW_*)
  long long gfeat[F_NUM];  // the graph features (is_graph_feature); level slots unused
};

struct RunState {
  int32_t* depth;            // caller's output
  const TreeNode* tree;      // device tree
  const QsTree* tree_qs;     // its bit-parallel form, or null
  int32_t tree_nodes;
  int32_t root;
  int32_t forced;            // -1: tree
  int32_t use_handles;       // 1 inside a CUDA graph with conditional nodes
  int32_t level;             // depth of the frontier being expanded
  int32_t variant;           // variant of the current level
  uint32_t qsel;             // q[qsel] = input queue, q[qsel ^ 1] = output queue
  uint32_t vsel;             // vis[vsel] = current visited bitmap
  int32_t frontier;          // f_L
  int32_t status;            // ST_OK / ST_TIMEOUT
  int32_t vw;                // virtual warp width of the push_warp variant at this level
  int32_t levels;            // levels completed (set when the run ends)
  int32_t vw_policy;         // the graph's width policy, copied by k_init (graph and host-loop drivers)
  unsigned long long next_count;  // f_{L+1}: output queue tail
  unsigned long long next_edges;  // e_{L+1}
  long long frontier_edges;  // e_L
  long long discovered;      // sum of f_j, j <= L
  long long edges_reached;   // sum of e_j, j <= L
  unsigned long long h_while;   // cudaGraphConditionalHandle of the level loop
  unsigned long long h_switch;  // cudaGraphConditionalHandle of the variant switch
  long long feat[F_NUM];     // feature vector of the current level (written by decide)
  // persistent driver: level words indexed by level % 3 (level L reads slot
  // L % 3, appends to (L + 1) % 3 and clears (L + 2) % 3). tail3: the output
  // queue tail in the low 32 bits (the next frontier size), the blocks that
  // reached the level-ending barrier in the high 32; edg3: the out-degree sum
  // of the appended vertices in the low 40 bits (e_L <= m < 2^31), arrivals in
  // the high 24. bar64: monotonic arrival count of the other grid barriers.
  unsigned long long tail3[3];
  unsigned long long edg3[3];
  unsigned long long bar64;
  unsigned int run_epoch;       // persistent driver: epoch of the launch whose block 0 reset the barrier state
  int32_t pad3_;
  int32_t log_cap;
  int32_t pad_;
  long long t_entry;  // %globaltimer (ns) when the run's first kernel started (before the depth init)
  long long prof_t0, prof_t1;  // timing harness: %globaltimer at a profiled level's start and end
  unsigned long long prof_e;   // timing harness: the profiled level's next frontier edge count
  unsigned int prof_f;         // timing harness: the profiled level's next frontier size
  int32_t pad4_;
  int32_t* log_variant;
  long long* log_frontier;
  long long* log_edges;
  long long* log_time;  // %globaltimer (ns) at the start of level L; entry `levels` marks the end
};

struct Buffers {
  int32_t* q[2];
  uint32_t* vis[2];
  int32_t* pe_scan;      // exclusive scan of frontier degrees (f + 1 entries)
  int32_t* pe_beg;       // off[u] of each frontier entry
  long long* pe_bsum;    // per-block sums of the scan
  int32_t pe_blocks_cap;
  int32_t pad_;
};

// Records `msg` as the calling thread's bfs_last_error_detail() and returns code.
int set_error_detail(int code, const char* msg);

// Library-internal entry points used by the serving loop (not part of the C ABI).
// run_async: enqueue one traversal on `stream` in the given bfs_mode and, when
// edges_dst (pinned host memory) is not null, an asynchronous copy of its
// reached-edge count there. batch_async: one multi-source wave (k <= 64) on a
// buffer set, root i's depths into rows[i] (device, n int32 each), per-root
// reached-edge counts copied to edges_dst (pinned, 64 entries). grid_blocks > 0 limits a persistent run (or a wave) to that many
// blocks so several can be resident at once. Both return a bfs_status code.
// status_dst (pinned, optional) receives the run's device status word.
int run_async(struct ::bfs_graph* g, int32_t root, int32_t* depth_out, cudaStream_t stream, int32_t mode,
              long long* edges_dst, int32_t grid_blocks, int32_t* status_dst);
int batch_async(struct ::bfs_graph* g, struct MsSet* set, const int32_t* roots, int32_t k, int32_t* const* rows,
                cudaStream_t stream, unsigned long long* edges_dst, int32_t grid_blocks, int32_t* status_dst);
// Create workspaces until the graph holds `count` of them (at most the pool
// limit), so that up to that many concurrent runs allocate nothing.
int reserve_workspaces(struct ::bfs_graph* g, int32_t count);
// Multi-source buffer sets: one wave runs on a set at a time (the caller orders
// waves on one set); a set holds ms_set_bytes(g) device bytes.
struct MsSet;
int ms_set_create(struct ::bfs_graph* g, MsSet** out);
void ms_set_free(MsSet* set);
long long ms_set_bytes(const struct ::bfs_graph* g);
// Device bytes one traversal of the graph holds (workspace), for admission control.
long long workspace_bytes(const struct ::bfs_graph* g);
int32_t graph_vertices(const struct ::bfs_graph* g);
int graph_device(const struct ::bfs_graph* g);
// Blocks of one full occupancy wave of the persistent traversal kernel and of
// the multi-source kernel (0 when cooperative launch is unsupported).
int32_t persistent_grid(const struct ::bfs_graph* g);
int32_t wave_grid(struct ::bfs_graph* g);

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t ld_nc_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Sum `x` over the block and add it to *dst with one atomic. Every thread of
// the block must call it (it synchronises).
__device__ __forceinline__ void block_add_u64(unsigned long long x, unsigned long long* dst) {
  __shared__ unsigned long long part[32];
  x = warp_sum(x);
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) part[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long y = lane_id() < (uint32_t)nw ? part[lane_id()] : 0ull;
    y = warp_sum(y);
    if (lane_id() == 0 && y) atomicAdd(dst, y);
  }
  __syncthreads();
}

// Append v to the output queue with one atomic per group of converged lanes
// (warp-aggregated atomic). The queue tail doubles as the next frontier size;
// a 64-bit tail keeps it in its low 32 bits (the persistent kernel counts
// barrier arrivals in the high half of the same word).
template <typename TailT>
__device__ __forceinline__ void queue_append(int32_t* qout, TailT* tail, int32_t v) {
  const uint32_t mask = __activemask();
  const int leader = __ffs(mask) - 1;
  unsigned int base = 0;
  if ((int)lane_id() == leader) base = (unsigned int)atomicAdd(tail, (TailT)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  qout[base + __popc(mask & lanemask_lt())] = v;
}

// Block-local staging of queue appends. Lanes reserve slots with one
// shared-memory atomic per warp; a block-uniform drain reserves space in the
// output queue with one global atomic per block and copies the slots out with
// coalesced stores. (One global queue tail shared by every warp serialises
// under dense levels; the block stage removes that.) Slots beyond the capacity
// fall back to a warp-aggregated global append.
constexpr int kStageCap = 2048;

struct Stage {
  int32_t* buf;
  unsigned int* cnt;
  unsigned int* base;
};

#define BFS_DECLARE_STAGE(name)                   \
  __shared__ int32_t name##_buf[kStageCap];       \
  __shared__ unsigned int name##_cnt, name##_base; \
  if (threadIdx.x == 0) name##_cnt = 0;           \
  __syncthreads();                                \
  const Stage name { name##_buf, &name##_cnt, &name##_base }

template <typename TailT>
__device__ __forceinline__ void stage_put(const Stage& s, int32_t* out, TailT* tail, int32_t v) {
  const uint32_t mask = __activemask();
  const int leader = __ffs(mask) - 1;
  unsigned int pos = 0;
  if ((int)lane_id() == leader) pos = atomicAdd(s.cnt, (unsigned)__popc(mask));
  pos = __shfl_sync(mask, pos, leader) + (unsigned)__popc(mask & lanemask_lt());
  if (pos < (unsigned)kStageCap)
    s.buf[pos] = v;
  else
    queue_append(out, tail, v);
}

// Copies the staged entries out once at least `threshold` are waiting. Every
// thread of the block must call it (it synchronises).
template <typename TailT>
__device__ __forceinline__ void stage_drain(const Stage& s, int32_t* out, TailT* tail, unsigned int threshold) {
  __syncthreads();
  const unsigned int c = min(*s.cnt, (unsigned)kStageCap);
  if (c == 0 || c < threshold) return;  // uniform: every thread read the same count
  if (threadIdx.x == 0) *s.base = (unsigned int)atomicAdd(tail, (TailT)c);
  __syncthreads();
  const unsigned int b = *s.base;
  for (unsigned int i = threadIdx.x; i < c; i += blockDim.x) out[b + i] = s.buf[i];
  __syncthreads();
  if (threadIdx.x == 0) *s.cnt = 0;
  __syncthreads();
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s bound on any device-side wait

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Sum of x over the block, returned to every thread. Every thread of the block
// must call it (it synchronises).
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x) {
  __shared__ unsigned long long part[33];
  x = warp_sum(x);
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) part[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    unsigned long long y = lane_id() < (uint32_t)nw ? part[lane_id()] : 0ull;
    y = warp_sum(y);
    if (lane_id() == 0) part[32] = y;
  }
  __syncthreads();
  const unsigned long long total = part[32];
  __syncthreads();
  return total;
}

// Grid-wide barrier on a monotonic 64-bit arrival count (cooperative launch:
// every block resident). Thread 0 of each block adds 1 with a release
// reduction (no value comes back, so nothing waits for it) and polls the count
// with acquire loads until every block of this barrier has arrived: `target`,
// a copy each block keeps, advances by the grid size per barrier, so the count
// is never reset within a launch and the last arrival publishes nothing. The
// preceding __syncthreads orders the block's writes before thread 0's release;
// the closing one passes what thread 0 acquired on to the block. `extra`
// (0 normally) makes the barrier wait for that many arrivals more than the
// grid has: the test hook that runs a bounded wait out. The wait ends after
// kWaitLimitNs, or early once *status is not ST_OK; then the status word is
// set and false returned.
__device__ __forceinline__ bool grid_arrive_wait(unsigned long long* count, unsigned long long& target,
                                                 int32_t* status, unsigned int extra = 0u) {
  __syncthreads();
  target += gridDim.x;
  bool ok = true;
  if (threadIdx.x == 0) {
    red_release_add_u64(count, 1ull);
    const unsigned long long want = target + extra;
    if (ld_acquire_u64(count) < want) {
      const unsigned long long t0 = global_ns();
      while (ld_acquire_u64(count) < want) {
        if (*reinterpret_cast<volatile int32_t*>(status) != ST_OK || global_ns() - t0 > kWaitLimitNs) {
          *status = ST_TIMEOUT;
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}

// The barrier that ends a level of the persistent kernel. Two words of the
// next level's slot carry both the arrivals and the next level's inputs:
// *tail holds the output queue tail (f, low 32 bits) and *edges the frontier
// edge sum (e, low 40 bits). Thread 0 adds its block's edge sum e_block
// together with one arrival (bit 40) to *edges, then one arrival (bit 32) to
// *tail, both as release reductions after all of the block's appends; then it
// polls both words until each shows every block's arrival, and reads f and e
// from the same loads. No block waits for an atomic's return, no last block
// publishes anything, and no block reads a counter after the barrier. Bounded
// and hookable like grid_arrive_wait.
__device__ __forceinline__ bool level_arrive_wait(unsigned long long* tail, unsigned long long* edges,
                                                  unsigned long long e_block, int32_t* status, unsigned int* f_out,
                                                  unsigned long long* e_out, unsigned int extra = 0u) {
  __shared__ unsigned long long s_w[2];
  constexpr unsigned long long kLow32 = 0xffffffffull, kLow40 = (1ull << 40) - 1ull;
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) {
    red_release_add_u64(edges, (1ull << 40) + e_block);
    red_release_add_u64(tail, 1ull << 32);
    const unsigned long long want = (unsigned long long)gridDim.x + extra;
    unsigned long long a = ld_acquire_u64(tail), b = ld_acquire_u64(edges);
    if ((a >> 32) < want || (b >> 40) < want) {
      const unsigned long long t0 = global_ns();
      for (;;) {
        a = ld_acquire_u64(tail);
        b = ld_acquire_u64(edges);
        if ((a >> 32) >= want && (b >> 40) >= want) break;
        if (*reinterpret_cast<volatile int32_t*>(status) != ST_OK || global_ns() - t0 > kWaitLimitNs) {
          *status = ST_TIMEOUT;
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    s_w[0] = a;
    s_w[1] = b;
  }
  ok = __syncthreads_and(ok) != 0;
  *f_out = (unsigned int)(s_w[0] & kLow32);
  *e_out = s_w[1] & kLow40;
  return ok;
}

// Try to claim vertex v: set its visited bit. True only for the one thread
// whose atomicOr flipped the bit, so each vertex enters the queue once.
__device__ __forceinline__ bool claim(uint32_t* vis, int32_t v) {
  const uint32_t bit = 1u << (v & 31);
  uint32_t* w = vis + (v >> 5);
  if (*reinterpret_cast<volatile uint32_t*>(w) & bit) return false;  // cheap filter; bits only go 0 -> 1
  return (atomicOr(w, bit) & bit) == 0u;
}

}  // namespace bfs
