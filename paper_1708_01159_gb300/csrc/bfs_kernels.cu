// Level kernels of the per-level switched BFS (sm_103a).
//
// Each variant's level is a device function ("body") written with
// block-uniform loops, so three drivers can share it:
//   - graph path: one thin kernel per body, launched by a CUDA graph whose
//     WHILE node runs the level loop and whose SWITCH node picks the variant
//     set on the device by k_decide;
//   - persistent path: k_bfs_persistent, one cooperative launch per traversal;
//     levels are separated by a grid barrier and every block evaluates the
//     decision tree itself from counters indexed by level % 3;
//   - host loop: the graph path's kernels launched from the host level by
//     level (for profilers and the per-level timing harness).
//
// Newly reached vertices are claimed by an atomicOr on the visited bitmap; the
// single thread that flips a bit writes depth L + 1, stages the vertex in a
// block-local shared-memory buffer that is flushed to the output queue with
// one global atomic per block (the queue tail is the next frontier size:
// Section 3.1.4's first variant, a global atomic counter, with warp and block
// aggregation in front of it), and adds the vertex's out-degree to the next
// level's frontier-edge count.
#include "bfs_kernels.cuh"

namespace bfs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---- mbarrier + bulk async copy (TMA bulk, non-tensor) --------------------

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}

// Wait for the phase with the given parity to complete, giving up after
// kWaitLimitNs. Returns false on timeout.
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}


// ---- output staging and per-edge visit --------------------------------------

// No __restrict__ on the queue or bitmaps: inside the persistent kernel they are
// rewritten every level, so they must not be read through the non-coherent
// read-only cache.
struct Level {
  const int32_t* qin;
  int32_t* qout;
  uint32_t* vis;       // current visited bitmap (push updates it in place; pull reads it)
  uint32_t* vis_next;  // the other bitmap (pull writes it)
  int32_t* depth;
  unsigned long long* tail;  // output queue tail (low 32 bits)
  int32_t next_depth;
  int32_t frontier;
  int32_t latency_bound;  // the level's frontier has fewer than kLatencyEdges edges
  int32_t pull_sparse;    // fewer than 1/16 of the vertices with edges are still unvisited
};

// Below this many frontier edges a level cannot fill the GPU: its time is the
// latency of its chain of dependent memory accesses, not bandwidth. Such a
// level claims targets without reading their bitmap word first (one round trip
// less; the extra atomics cost nothing at this size) and prefetches the first
// adjacency sector of every vertex it reaches into L2, so the next level's
// list reads are L2 hits.
constexpr long long kLatencyEdges = 1ll << 17;

__device__ __forceinline__ Level load_level(const DevGraph& g, const Buffers& b, RunState* st) {
  Level lv;
  // select with ternaries: indexing the by-value parameter arrays would copy them to local memory
  const bool qs = st->qsel != 0u;
  const bool vs = st->vsel != 0u;
  lv.qin = qs ? b.q[1] : b.q[0];
  lv.qout = qs ? b.q[0] : b.q[1];
  lv.vis = vs ? b.vis[1] : b.vis[0];
  lv.vis_next = vs ? b.vis[0] : b.vis[1];
  lv.depth = st->depth;
  lv.tail = &st->next_count;
  lv.next_depth = st->level + 1;
  lv.frontier = st->frontier;
  lv.latency_bound = st->frontier_edges < kLatencyEdges;
  lv.pull_sparse = (long long)g.n_active - st->discovered < (long long)(g.n_active >> 4);
  return lv;
}

// Newly reached vertices go through a block-local stage (see stage_put) into
// the level's output queue.
__device__ __forceinline__ void stage_push(const Stage& s, const Level& lv, int32_t v) {
  stage_put(s, lv.qout, lv.tail, v);
}

__device__ __forceinline__ void stage_flush(const Stage& s, const Level& lv, unsigned int threshold) {
  stage_drain(s, lv.qout, lv.tail, threshold);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Top-down visit of up to K edges u -> v[k] (Section 3.1.2 push). The bitmap
// words of all K targets are read (except on latency-bound levels), then the
// claims (atomicOr) issued, then the winners' row extents read, so the K
// edges' memory round trips overlap instead of forming one dependent chain per
// edge. The one thread whose atomicOr flips a vertex's bit writes its depth,
// counts its out-degree and stages it.
// valid: bit k set when v[k] is an edge to visit.
template <int K, int kCount = CM_BLOCK>
__device__ __forceinline__ void visit_km(const DevGraph& g, const Level& lv, const Stage& s, const int32_t (&v)[K],
                                         uint32_t valid, unsigned long long& edges) {
  const bool filter = !lv.latency_bound;
  uint32_t word[K];
#pragma unroll
  for (int k = 0; k < K; ++k)
    word[k] = (valid >> k) & 1u ? (filter ? ld_volatile_u32(lv.vis + (v[k] >> 5)) : 0u) : 0xffffffffu;
  bool won[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t bit = 1u << (v[k] & 31);
    won[k] = false;
    if (((valid >> k) & 1u) && !(word[k] & bit)) won[k] = (atomicOr(lv.vis + (v[k] >> 5), bit) & bit) == 0u;
  }
  int32_t d[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    d[k] = 0;
    if (won[k]) {
      const int32_t b0 = g.off[v[k]];
      d[k] = g.off[v[k] + 1] - b0;
      if (!filter && d[k] > 0) prefetch_l2(g.idx + b0);
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k)
    if (won[k]) {
      lv.depth[v[k]] = lv.next_depth;
      edges += (unsigned long long)d[k];
      if (kCount == CM_BLOCK)
        stage_push(s, lv, v[k]);
      else if (kCount == CM_WARP)
        queue_append(lv.qout, lv.tail, v[k]);
      else
        lv.qout[(unsigned int)atomicAdd(lv.tail, 1ull)] = v[k];
    }
}

// The first nv entries of v are edges to visit.
template <int K, int kCount = CM_BLOCK>
__device__ __forceinline__ void visit_k(const DevGraph& g, const Level& lv, const Stage& s, const int32_t (&v)[K],
                                        int nv, unsigned long long& edges) {
  visit_km<K, kCount>(g, lv, s, v, nv >= 32 ? 0xffffffffu : (1u << nv) - 1u, edges);
}

template <typename T>
__device__ T block_exclusive_scan(T x, T* total) {
  __shared__ T wsum[32];
  const uint32_t lane = lane_id();
  const int w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  T inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, inc, o);
    if ((int)lane >= o) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    T s = (int)lane < nw ? wsum[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(kFull, s, o);
      if ((int)lane >= o) s += y;
    }
    if ((int)lane < nw) wsum[lane] = s;
  }
  __syncthreads();
  const T base = w > 0 ? wsum[w - 1] : T(0);
  *total = wsum[nw - 1];
  __syncthreads();
  return base + inc - x;
}

// ---------------------------------------------------------------------------
// Init (Section 3.1: all depths infinity, the root 0): depth and bitmap fill
// ---------------------------------------------------------------------------
__device__ __forceinline__ void init_fill(const DevGraph& g, uint32_t* vis0, int32_t* depth, int32_t root) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int32_t n = g.n;
  if ((reinterpret_cast<uintptr_t>(depth) & 15u) == 0) {
    const int64_t n4 = n >> 2;
    int4* d4 = reinterpret_cast<int4*>(depth);
    for (int64_t i = tid; i < n4; i += stride) {
      int4 val = make_int4(-1, -1, -1, -1);
      if ((root >> 2) == i) {
        const int k = root & 3;
        if (k == 0) val.x = 0;
        if (k == 1) val.y = 0;
        if (k == 2) val.z = 0;
        if (k == 3) val.w = 0;
      }
      d4[i] = val;
    }
    for (int64_t i = (n4 << 2) + tid; i < n; i += stride) depth[i] = (i == root) ? 0 : -1;
  } else {
    for (int64_t i = tid; i < n; i += stride) depth[i] = (i == root) ? 0 : -1;
  }
  for (int64_t w = tid; w < g.words; w += stride)
    vis0[w] = g.vis_init[w] | ((w == (root >> 5)) ? (1u << (root & 31)) : 0u);
}

// ---------------------------------------------------------------------------
// Tree evaluation (Section 2.1 walk over the Section 4.1 features, with the
// Section 4.1 unknown-prediction rule). Returns the variant; fills feat[].
// ---------------------------------------------------------------------------
// Value of feature fi at this level, computed on demand: a walk reads at most
// the tree's depth of them, and each ppm share costs a 64-bit division.
__device__ __forceinline__ long long feature_value(const DevGraph& g, int32_t fi, int32_t L, long long f, long long e,
                                                   long long discovered) {
  if (is_graph_feature(fi)) return g.gfeat[fi];
  switch (fi) {
    case F_FRONTIER: return f;
    case F_FRONTIER_PPM: return (1000000ll * f) / g.n;
    case F_DISCOVERED: return discovered;
    case F_DISCOVERED_PPM: return (1000000ll * discovered) / g.n;
    case F_FRONTIER_EDGES: return e;
    default: return L;  // F_LEVEL
  }
}

// The split test x_fi <= t of a tree node, without dividing for the ppm
// shares: floor(1e6 c / n) <= t is 1e6 c < (t + 1) n for 0 <= t < 1e6, always
// true for t >= 1e6 (c <= n) and never for t < 0.
__device__ __forceinline__ bool feature_le(const DevGraph& g, int32_t fi, long long t, int32_t L, long long f,
                                          long long e, long long discovered) {
  if (fi == F_FRONTIER_PPM || fi == F_DISCOVERED_PPM) {
    const long long c = fi == F_FRONTIER_PPM ? f : discovered;
    if (t < 0) return false;
    if (t >= 1000000) return true;
    return 1000000ll * c < (t + 1) * (long long)g.n;
  }
  return feature_value(g, fi, L, f, e, discovered) <= t;
}

// Section 2.1 walk of an integer tree; -1 for an unknown leaf.
__device__ __forceinline__ int32_t walk_tree(const DevGraph& g, const TreeNode* tree, int32_t nodes, int32_t L,
                                             long long f, long long e, long long discovered) {
  int32_t i = 0;
  for (int32_t step = 0; step <= nodes; ++step) {
    const TreeNode nd = tree[i];
    if (nd.f < 0) return nd.v;
    i = feature_le(g, nd.f, nd.t, L, f, e, discovered) ? nd.l : nd.r;
  }
  return -1;
}

// The test x_fi <= t of a level feature without branches, so that the lanes
// of a warp, each on a different feature, do not diverge. The ppm shares do not
// occur here: the host rewrote each as the equivalent test on the count
// (floor(1e6 c / n) <= t is c <= ceil((t + 1) n / 1e6) - 1).
__device__ __forceinline__ bool level_feature_le(int32_t fi, long long t, int32_t L, long long f, long long e,
                                                 long long discovered) {
  long long x = L;
  x = (fi == F_FRONTIER) ? f : x;
  x = (fi == F_DISCOVERED) ? discovered : x;
  x = (fi == F_FRONTIER_EDGES) ? e : x;
  return x <= t;
}

// The leaf the tree's walk reaches, by the bit-parallel form, within one warp:
// lane k tests the level-feature nodes k, k + 32; the graph-feature tests are
// already folded into q.base. Every lane of the warp calls it and gets the
// same result (-1 if none); no block-wide synchronisation.
__device__ __forceinline__ int32_t qs_leaf_warp(const QsTree& q, int32_t L, long long f, long long e,
                                                long long discovered) {
  unsigned long long m = q.base;
  for (int k = lane_id(); k < q.n_int; k += 32) {
    const QsNode nd = q.node[k];
    if (!level_feature_le(nd.f, nd.t, L, f, e, discovered)) m &= nd.mask;
  }
  const uint32_t lo = __reduce_and_sync(kFull, (uint32_t)m);
  const uint32_t hi = __reduce_and_sync(kFull, (uint32_t)(m >> 32));
  const int leaf = __ffsll((long long)(((unsigned long long)hi << 32) | lo)) - 1;
  return (leaf >= 0 && leaf < q.n_leaf) ? leaf : -1;
}

// The tree's prediction (leaf class, -1 for unknown) by the bit-parallel form.
__device__ __forceinline__ int32_t qs_eval_warp(const QsTree& q, int32_t L, long long f, long long e,
                                                long long discovered) {
  const int32_t leaf = qs_leaf_warp(q, L, f, e, discovered);
  return leaf >= 0 ? q.leaf[leaf] : -1;
}

// True (in every lane) when this level's features lie in the box that lanes
// 0-7 of the warp hold in `bound` (lane 2k: lower bound of level feature k,
// lane 2k + 1: upper bound; k = frontier, discovered, frontier edges, level).
__device__ __forceinline__ bool in_leaf_box(int32_t bound, int32_t L, long long f, long long e, long long discovered) {
  const uint32_t lane = lane_id();
  const long long x = lane < 2 ? f : lane < 4 ? discovered : lane < 6 ? e : (long long)L;
  const bool ok = (lane & 1u) ? x <= (long long)bound : x >= (long long)bound;
  return __all_sync(kFull, lane >= 8u || ok);
}

// Section 4.1 unknown-prediction rule on a walk's result (or the forced
// variant), and the virtual-warp width under the graph's policy: the rule is
// the power of two nearest above the frontier's mean degree floor(e / f),
// clamped to [4, 32] (floor(e / f) <= k is e < (k + 1) f).
__device__ __forceinline__ int32_t finish_variant(int32_t v, int32_t L, int32_t prev, long long f, long long e,
                                                  int32_t* vw, bool forced, int32_t policy) {
  if (!forced) {
    if (v < 0 || v >= V_NUM) v = (L == 0) ? kLevel0Default : prev;  // unknown prediction
    if (v < 0 || v >= V_NUM) v = kLevel0Default;
  }
  const int32_t rule = (f <= 0 || e < 5 * f) ? 4 : e < 9 * f ? 8 : e < 17 * f ? 16 : 32;
  *vw = policy == VW_RULE_X2     ? min(32, 2 * rule)
        : policy == VW_RULE_HALF ? max(4, rule / 2)
        : policy == VW_4         ? 4
        : policy == VW_8         ? 8
        : policy == VW_16        ? 16
        : policy == VW_32        ? 32
                                 : rule;
  return v;
}

// ---------------------------------------------------------------------------
// Push, one thread per frontier vertex (Section 3.1.2 vertex push, over an
// explicit queue instead of a scan of all vertices). Each thread walks its
// vertex's adjacency four edges at a time.
// ---------------------------------------------------------------------------
template <int kCount = CM_BLOCK>
__device__ void body_push_thread(const DevGraph& g, const Level& lv, const Stage& stage, unsigned long long& edges) {
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < lv.frontier; base += stride) {
    const int i = base + threadIdx.x;
    if (i < lv.frontier) {
      const int32_t u = lv.qin[i];
      const int32_t end = g.off[u + 1];
      for (int32_t e = g.off[u]; e < end; e += 4) {
        const int nv = min(4, end - e);
        int32_t v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = k < nv ? g.idx[e + k] : 0;
        visit_k<4, kCount>(g, lv, stage, v, nv, edges);
      }
    }
    stage_flush(stage, lv, kStageCap / 2);
  }
}

// ---------------------------------------------------------------------------
// Push, virtual warp of W lanes per frontier vertex (Section 3.1.3, after Hong
// et al. 2011). Lanes stride the adjacency; W = 32 reads long lists with
// 16-byte vector loads.
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void push_vwarp(const DevGraph& g, const Level& lv, const Stage& stage,
                                           unsigned long long& edges) {
  constexpr int G = kThreads / W;  // groups per block
  const int lane = threadIdx.x & (W - 1);
  if (W < 32 && lv.frontier > (int)gridDim.x * G) {
    // More frontier vertices than groups: a group takes kR consecutive
    // frontier vertices per step, and each round every lane visits one edge of
    // each of them (edge lane, lane + W, ...), so kR independent chains of
    // loads are in flight per lane and the level needs a quarter of the steps
    // (a high-diameter graph's levels on a narrow grid). A frontier that fits
    // one step keeps one vertex per group, spread over every block.
    constexpr int kR = 4;
    const int grp = (int)threadIdx.x / W;
    for (int base = blockIdx.x * G * kR; base < lv.frontier; base += gridDim.x * G * kR) {
      int32_t e[kR], end[kR];
#pragma unroll
      for (int j = 0; j < kR; ++j) {
        const int i = base + grp * kR + j;
        e[j] = end[j] = 0;
        if (i < lv.frontier) {
          const int32_t u = lv.qin[i];
          e[j] = g.off[u] + lane;
          end[j] = g.off[u + 1];
        }
      }
      uint32_t valid;
      do {
        int32_t v[kR];
        valid = 0;
#pragma unroll
        for (int j = 0; j < kR; ++j) {
          const bool ok = e[j] < end[j];
          v[j] = ok ? g.idx[e[j]] : 0;
          valid |= (uint32_t)ok << j;
          e[j] += W;
        }
        if (valid) visit_km<kR>(g, lv, stage, v, valid, edges);
      } while (valid);
      stage_flush(stage, lv, kStageCap / 2);
    }
    return;
  }
  for (int base = blockIdx.x * G; base < lv.frontier; base += gridDim.x * G) {
    const int i = base + (int)threadIdx.x / W;
    if (i < lv.frontier) {
      const int32_t u = lv.qin[i];
      const int32_t beg = g.off[u], end = g.off[u + 1];
      if (W == 32 && end - beg >= 256) {
        const int32_t a0 = (beg + 3) & ~3, a1 = end & ~3;
        {
          int32_t v[1] = {beg + lane < a0 ? g.idx[beg + lane] : 0};
          visit_k<1>(g, lv, stage, v, beg + lane < a0 ? 1 : 0, edges);
        }
        for (int32_t e = a0 + 4 * lane; e < a1; e += 128) {
          const int4 q = *reinterpret_cast<const int4*>(g.idx + e);
          int32_t v[4] = {q.x, q.y, q.z, q.w};
          visit_k<4>(g, lv, stage, v, 4, edges);
        }
        {
          int32_t v[1] = {a1 + lane < end ? g.idx[a1 + lane] : 0};
          visit_k<1>(g, lv, stage, v, a1 + lane < end ? 1 : 0, edges);
        }
      } else {
        for (int32_t e = beg + lane; e < end; e += 4 * W) {
          int32_t v[4];
          int nv = 0;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int32_t ek = e + k * W;
            v[k] = ek < end ? g.idx[ek] : 0;
            nv += ek < end ? 1 : 0;
          }
          visit_k<4>(g, lv, stage, v, nv, edges);
        }
      }
    }
    stage_flush(stage, lv, kStageCap / 2);
  }
}

__device__ void body_push_warp(const DevGraph& g, const Level& lv, const Stage& stage, int32_t vw,
                               unsigned long long& edges) {
  switch (vw) {
    case 4: push_vwarp<4>(g, lv, stage, edges); break;
    case 8: push_vwarp<8>(g, lv, stage, edges); break;
    case 16: push_vwarp<16>(g, lv, stage, edges); break;
    default: push_vwarp<32>(g, lv, stage, edges); break;
  }
}

// ---------------------------------------------------------------------------
// Push, one CTA per frontier vertex. Long adjacency lists are streamed into a
// double-buffered shared-memory stage by bulk async copies (cp.async.bulk with
// an mbarrier transaction count); the CTA's threads then test and claim the
// staged neighbours. Copies are 16-byte aligned: the range is widened to
// multiples of 4 entries (idx is padded) and the extra entries are skipped.
// ---------------------------------------------------------------------------
struct CtaPipe {
  int32_t* chunk;  // 2 x kCtaChunk entries of shared memory
  uint64_t* bar;   // 2 mbarriers, initialised once per block
  uint32_t parity0, parity1;
  uint32_t extra_tx;  // test hook: bytes the next copy's barrier expects beyond the copy (0 normally)
};

__device__ __forceinline__ void cta_pipe_init(uint64_t* bar) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
}

// Returns false if a copy never completed (status set; block stopped early).
__device__ bool body_push_cta(const DevGraph& g, const Level& lv, const Stage& stage, CtaPipe& pp, int32_t* status,
                              unsigned long long& edges) {
  const int tid = threadIdx.x;
  constexpr int kPer = kCtaChunk / kThreads;  // staged entries per thread per chunk
  int iter = 0;
  for (int i = blockIdx.x; i < lv.frontier; i += gridDim.x, ++iter) {
    const int32_t u = lv.qin[i];
    const int32_t beg = g.off[u], end = g.off[u + 1];
    if (end - beg < kCtaDirect) {
      // short lists: read directly; check the stage every 4th vertex (4 x 512
      // entries fit it), not after each one, to keep barriers rare
      for (int32_t e = beg + tid; e < end; e += 4 * kThreads) {
        int32_t v[4];
        int nv = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int32_t ek = e + k * kThreads;
          v[k] = ek < end ? g.idx[ek] : 0;
          nv += ek < end ? 1 : 0;
        }
        visit_k<4>(g, lv, stage, v, nv, edges);
      }
      if ((iter & 3) == 3) stage_flush(stage, lv, kStageCap / 2);
      continue;
    }
    stage_flush(stage, lv, 1);  // empty the stage before a long list
    const int32_t abeg = beg & ~3, aend = (end + 3) & ~3;
    const int32_t nch = (aend - abeg + kCtaChunk - 1) / kCtaChunk;
    auto issue = [&](int32_t c) {
      const int32_t cb = abeg + c * kCtaChunk;
      const uint32_t bytes = (uint32_t)min(kCtaChunk, aend - cb) * 4u;
      uint64_t* br = &pp.bar[c & 1];
      mbar_expect_tx(br, bytes + pp.extra_tx);
      pp.extra_tx = 0;
      bulk_g2s(pp.chunk + (c & 1) * kCtaChunk, g.idx + cb, bytes, br);
    };
    if (tid == 0) {
      issue(0);
      if (nch > 1) issue(1);
    }
    for (int32_t c = 0; c < nch; ++c) {
      const int s = c & 1;
      const bool ok = mbar_wait_bounded(&pp.bar[s], s ? pp.parity1 : pp.parity0);
      if (s)
        pp.parity1 ^= 1u;
      else
        pp.parity0 ^= 1u;
      if (ok) {
        const int32_t cb = abeg + c * kCtaChunk;
        const int32_t len = min(kCtaChunk, aend - cb);
        const int32_t* buf = pp.chunk + s * kCtaChunk;
        int32_t v[kPer];
        int nv = 0;
        // entries tid, tid + 256, ... of the chunk, compacted to the valid ones
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          const int32_t kk = tid + k * kThreads;
          const int32_t e = cb + kk;
          if (kk < len && e >= beg && e < end) v[nv++] = buf[kk];
        }
        visit_k<kPer>(g, lv, stage, v, nv, edges);
      }
      stage_flush(stage, lv, kStageCap / 2);
      if (!__syncthreads_and(ok)) {
        // a copy never completed: flag it, let the other in-flight copy land (bounded) and stop
        if (tid == 0) {
          *status = ST_TIMEOUT;
          if (c + 1 < nch) mbar_wait_bounded(&pp.bar[s ^ 1], s ? pp.parity0 : pp.parity1);
        }
        return false;
      }
      if (tid == 0 && c + 2 < nch) issue(c + 2);
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Push, edge-centric (Section 3.1.1 edge list, restricted to the frontier's
// edges): exclusive scan of the frontier degrees, then a load-balanced search
// (merge path of the scan with the edge indices) gives every thread
// kPeItems items (frontier boundaries or edges) regardless of degree skew.
// ---------------------------------------------------------------------------
__device__ void body_pe_reduce(const DevGraph& g, const Level& lv, const Buffers& b) {
  const int f = lv.frontier;
  const int nblk = (f + kPeTile - 1) / kPeTile;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    long long sum = 0;
    const int base = blk * kPeTile;
#pragma unroll
    for (int k = 0; k < kPeItems; ++k) {
      const int i = base + k * kThreads + threadIdx.x;
      if (i < f) {
        const int32_t u = lv.qin[i];
        const int32_t beg = g.off[u];
        const int32_t d = g.off[u + 1] - beg;
        b.pe_beg[i] = beg;
        b.pe_scan[i] = d;
        sum += d;
      }
    }
    long long tot;
    block_exclusive_scan<long long>(sum, &tot);
    if (threadIdx.x == 0) b.pe_bsum[blk] = tot;
  }
}

// One block.
__device__ void body_pe_top(const Buffers& b, int f) {
  const int nblk = (f + kPeTile - 1) / kPeTile;
  long long carry = 0;
  for (int base = 0; base < nblk; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const long long x = i < nblk ? b.pe_bsum[i] : 0;
    long long tot;
    const long long ex = block_exclusive_scan<long long>(x, &tot);
    if (i < nblk) b.pe_bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) b.pe_bsum[nblk] = carry;
}

__device__ void body_pe_scan(const Buffers& b, int f) {
  const int nblk = (f + kPeTile - 1) / kPeTile;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int base = blk * kPeTile + threadIdx.x * kPeItems;
    int32_t d[kPeItems];
#pragma unroll
    for (int k = 0; k < kPeItems; ++k) d[k] = (base + k < f) ? b.pe_scan[base + k] : 0;
    int32_t run = 0;
#pragma unroll
    for (int k = 0; k < kPeItems; ++k) {
      const int32_t t = d[k];
      d[k] = run;
      run += t;
    }
    long long tot;
    const long long ex = block_exclusive_scan<long long>((long long)run, &tot);
    const long long off = b.pe_bsum[blk] + ex;
#pragma unroll
    for (int k = 0; k < kPeItems; ++k)
      if (base + k < f) b.pe_scan[base + k] = (int32_t)(off + d[k]);
    if (blk == nblk - 1 && threadIdx.x == 0) b.pe_scan[f] = (int32_t)b.pe_bsum[nblk];
  }
}

// A frontier of at most kPeSmall vertices fits one scan tile: every block then
// scans the frontier degrees itself, in shared memory, and the level needs no
// grid-wide scan phases (no extra grid barriers in the persistent kernel, no
// work in the reduce/top/scan launches of the other drivers).
constexpr int kPeSmall = kPeTile - 1;

// s_a, s_beg: kPeTile + 1 entries. On return s_a[1 + i] is the exclusive scan
// of the frontier degrees at i (s_a[1 + f] their total) and s_beg[1 + i] the
// row start of frontier entry i; entry 0 of both is 0, the value the expand
// uses before the first frontier entry. f <= kPeSmall.
__device__ void pe_small_scan(const DevGraph& g, const Level& lv, int32_t* s_a, int32_t* s_beg) {
  const int f = lv.frontier;
  const int base = (int)threadIdx.x * kPeItems;
  int32_t d[kPeItems];
  int32_t run = 0;
#pragma unroll
  for (int k = 0; k < kPeItems; ++k) {
    const int i = base + k;
    int32_t deg = 0;
    if (i < f) {
      const int32_t u = lv.qin[i];
      const int32_t b0 = g.off[u];
      deg = g.off[u + 1] - b0;
      s_beg[1 + i] = b0;
    }
    d[k] = run;
    run += deg;
  }
  long long tot;
  const long long ex = block_exclusive_scan<long long>((long long)run, &tot);
#pragma unroll
  for (int k = 0; k < kPeItems; ++k)
    if (base + k < f) s_a[1 + base + k] = (int32_t)(ex + d[k]);
  if (threadIdx.x == 0) {
    s_a[0] = 0;
    s_beg[0] = 0;
    if (f <= kPeSmall) s_a[1 + f] = (int32_t)tot;  // callers guarantee it; the check keeps s_a in bounds
  }
  __syncthreads();
}

// Merge-path split: how many of the first d items of merge(A[0..na), j0+[0..nb))
// are A items, with A first on ties (A[i] <= edge index => boundary first).
__device__ __forceinline__ int merge_split(const int32_t* a, int na, long long j0, int nb, long long d) {
  int lo = (int)max(0ll, d - nb), hi = (int)min(d, (long long)na);
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)a[mid] <= j0 + d - 1 - mid)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// s_a, s_beg: kPeTile + 1 entries of shared memory each; s_split: 2 ints.
// kSmall: the scan is already in s_a / s_beg (pe_small_scan), not in b.
template <bool kSmall>
__device__ void body_pe_expand(const DevGraph& g, const Level& lv, const Buffers& b, const Stage& stage,
                               int32_t* s_a_buf, int32_t* s_beg_buf, int* s_split, unsigned long long& edges) {
  const int f = lv.frontier;
  const int32_t* scan = kSmall ? s_a_buf + 1 : b.pe_scan;
  const int32_t E = scan[f];
  const long long total = (long long)f + E;
  // Tile length: a whole multiple of the block size, as short as spreads the
  // items over every block (one per thread at least), at most kPeTile. A
  // small level (a handful of frontier vertices with some thousands of edges)
  // then runs on many blocks with an item or two per thread instead of a few
  // full tiles, so its latency is one visit chain instead of eight.
  const long long per_block = (total + gridDim.x - 1) / gridDim.x;
  const int tile = (int)min((long long)kPeTile, max((long long)kThreads, (per_block + kThreads - 1) / kThreads * kThreads));
  const int ipt = tile / kThreads;  // items per thread, 1..kPeItems
  const long long ntiles = (total + tile - 1) / tile;
  for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const long long d0 = t * tile;
    const long long d1 = min(d0 + tile, total);
    if (threadIdx.x < 2) s_split[threadIdx.x] = merge_split(scan, f, 0, E, threadIdx.x ? d1 : d0);
    __syncthreads();
    const int i0 = s_split[0], i1 = s_split[1];
    const int na = i1 - i0;
    const int tl = (int)(d1 - d0);
    const int nb = tl - na;
    const long long j0 = d0 - i0;
    // s index k <-> frontier entry i0 - 1 + k (the vertex owning edge j0 may precede the tile)
    const int32_t* s_a = s_a_buf;
    const int32_t* s_beg = s_beg_buf;
    if (kSmall) {
      s_a = s_a_buf + i0;  // s_a_buf[1 + i] holds entry i, s_a_buf[0] the 0 before entry 0
      s_beg = s_beg_buf + i0;
    } else {
      for (int k = threadIdx.x; k <= na; k += blockDim.x) {
        const int gi = i0 - 1 + k;
        s_a_buf[k] = gi >= 0 ? b.pe_scan[gi] : 0;
        s_beg_buf[k] = gi >= 0 ? b.pe_beg[gi] : 0;
      }
      __syncthreads();
    }
    const int td0 = min((int)threadIdx.x * ipt, tl);
    const int td1 = min(td0 + ipt, tl);
    const int ti = merge_split(s_a + 1, na, j0, nb, td0);
    int cur = ti;          // s index of the current vertex
    int anext = ti + 1;    // s index of the next boundary
    long long bj = j0 + (td0 - ti);
    int32_t epos[kPeItems];
    int ne = 0;
    for (int step = td0; step < td1; ++step) {
      if (anext <= na && (long long)s_a[anext] <= bj) {
        cur = anext++;
      } else {
        epos[ne++] = s_beg[cur] + (int32_t)(bj - s_a[cur]);
        ++bj;
      }
    }
    int32_t v[kPeItems];
#pragma unroll
    for (int k = 0; k < kPeItems; ++k) v[k] = k < ne ? g.idx[epos[k]] : 0;
    visit_k<kPeItems>(g, lv, stage, v, ne, edges);
    stage_flush(stage, lv, 1);
  }
}

// ---------------------------------------------------------------------------
// Pull, bottom-up over the visited bitmap (Section 3.1.2 vertex pull). A warp
// owns 32 consecutive vertices (one bitmap word); each unvisited lane scans its
// in-neighbours, four at a time, and stops at the first visited one. At the
// start of level L a visited in-neighbour of an unvisited vertex has depth
// exactly L (a smaller depth would already have reached the vertex), so the
// current bitmap is the frontier test. New bits go to the other bitmap (read
// and write sets stay apart); the found vertices are staged and appended to
// the queue, which is also the bitmap-to-queue conversion a following push
// level needs. kReadOnlyCache: the bitmap is read through the non-coherent
// read-only cache, valid only when no earlier level ran in the same launch
// (graph and host-loop drivers); the persistent kernel passes false.
// ---------------------------------------------------------------------------
template <bool kReadOnlyCache>
__device__ __forceinline__ uint32_t vis_bit(const uint32_t* vis, int32_t u) {
  const uint32_t word = kReadOnlyCache ? ld_nc_u32(vis + (u >> 5)) : vis[u >> 5];
  return (word >> (u & 31)) & 1u;
}

// A warp takes kWords bitmap words (kWords x 32 vertices) per step and each
// lane interleaves the scans of its kWords vertices, four in-neighbours of each
// per round, so kWords times as many independent loads are in flight per
// thread as with one vertex per lane (a scan is a chain of dependent loads:
// row extent, adjacency entries, bitmap words). The bitmap words of the next
// step are loaded at the start of the current one. Found vertices go to a
// warp-private slice of the block stage, flushed by the warp alone (one queue
// atomic per slice), so warps never wait for one another inside the level.
constexpr int kPullWordsLaunch = 2;      // k_pull
constexpr int kPullWordsPersistent = 2;  // pull level of the persistent kernel
constexpr int kWarpStage = kStageCap / (kThreads / 32);
static_assert(kStageCap % (kThreads / 32) == 0, "stage slices");

__device__ __forceinline__ void warp_stage_flush(int32_t* wbuf, unsigned int cnt, const Level& lv) {
  __syncwarp();
  unsigned int base = 0;
  if (lane_id() == 0) base = (unsigned int)atomicAdd(lv.tail, (unsigned long long)cnt);
  base = __shfl_sync(kFull, base, 0);
  for (unsigned int i = lane_id(); i < cnt; i += 32) lv.qout[base + i] = wbuf[i];
  __syncwarp();
}

// A pull level runs in two phases per warp. The hint pass takes kWords bitmap
// words per step (w[j] < 0: none; cw[j] the current word): each lane takes
// vertex w[j] * 32 + lane of every word and, when it is unvisited, tests its
// hint (the in-neighbour of largest out-degree among the first entries of its
// in-list, chosen at graph create); a vertex whose hint is in the frontier is
// found there, without reading its in-list, and the next bitmap's words are
// written. The others (misses) go to the warp's miss list in shared memory;
// whenever it holds 32, the miss pass scans their in-lists, one vertex per
// lane, four in-neighbours per round, stopping at the first visited one, and
// sets the found vertices' bits in the next bitmap. So a step of the hint pass
// costs one round trip to the hint and its bitmap word, and no lane of a miss
// scan waits on vertices that need no scan. Found vertices get their depth and
// a slot of the warp's stage.
template <int kWords>
struct PullMisses {
  static constexpr int kCap = 32 * (kWords + 1);  // up to 31 left over plus one step's misses
  int32_t* v;                                     // kCap entries each, in shared memory
  int32_t* beg;
  int32_t* end;
};

// Shared-memory ints the miss lists of a block's warps take.
template <int kWords>
constexpr int pull_scratch_ints() {
  return (kThreads / 32) * 3 * PullMisses<kWords>::kCap;
}

template <bool kReadOnlyCache, int kWords>
__device__ __forceinline__ void pull_words(const DevGraph& g, const Level& lv, const int32_t (&w)[kWords],
                                           const uint32_t (&cw)[kWords], int32_t* wbuf, unsigned int& wcnt,
                                           const PullMisses<kWords>& ms, int& mcnt, unsigned long long& edges) {
  const uint32_t lane = lane_id();
  int32_t v[kWords], beg[kWords], end[kWords], h[kWords];
  bool active[kWords], found[kWords];
#pragma unroll
  for (int j = 0; j < kWords; ++j) {
    v[j] = w[j] * 32 + (int32_t)lane;
    active[j] = w[j] >= 0 && cw[j] != kFull && v[j] < g.n && !((cw[j] >> lane) & 1u);
    beg[j] = end[j] = 0;
    h[j] = -1;
    if (active[j]) {  // three coalesced loads, issued together
      beg[j] = g.in_off[v[j]];
      end[j] = g.in_off[v[j] + 1];
      h[j] = g.hint[v[j]];
    }
    active[j] = active[j] && beg[j] < end[j];
  }
#pragma unroll
  for (int j = 0; j < kWords; ++j) found[j] = active[j] && h[j] >= 0 && vis_bit<kReadOnlyCache>(lv.vis, h[j]);
#pragma unroll
  for (int j = 0; j < kWords; ++j) {
    const uint32_t fm = __ballot_sync(kFull, found[j]);
    if (found[j]) {
      const int32_t deg = g.symmetric ? end[j] - beg[j] : g.off[v[j] + 1] - g.off[v[j]];
      lv.depth[v[j]] = lv.next_depth;
      edges += (unsigned long long)deg;
      wbuf[wcnt + __popc(fm & lanemask_lt())] = v[j];
    }
    wcnt += (unsigned)__popc(fm);
    if (lane == 0 && w[j] >= 0) lv.vis_next[w[j]] = cw[j] | fm;
    const bool miss = active[j] && !found[j];
    const uint32_t mm = __ballot_sync(kFull, miss);
    if (miss) {
      const int slot = mcnt + __popc(mm & lanemask_lt());
      ms.v[slot] = v[j];
      ms.beg[slot] = beg[j];
      ms.end[slot] = end[j];
    }
    mcnt += __popc(mm);
  }
}

// The miss pass over entries base .. base + cnt - 1 (cnt <= 32) of the warp's
// miss list.
template <bool kReadOnlyCache, int kWords>
__device__ __forceinline__ void pull_misses(const DevGraph& g, const Level& lv, const PullMisses<kWords>& ms,
                                            int base, int cnt, int32_t* wbuf, unsigned int& wcnt,
                                            unsigned long long& edges) {
  // orders the list entries and this warp's next-bitmap word stores before
  // the reads and bit sets below
  __syncwarp();
  const uint32_t lane = lane_id();
  bool active = (int)lane < cnt;
  int32_t v = 0, beg = 0, pos = 0, end = 0;
  if (active) {
    v = ms.v[base + lane];
    beg = ms.beg[base + lane];
    end = ms.end[base + lane];
    pos = beg;
  }
  bool found = false;
  while (__any_sync(kFull, active)) {
    const int nv = active ? min(4, end - pos) : 0;
    int32_t u[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = nv ? g.in_idx[k < nv ? pos + k : pos] : 0;
    if (active) {
      uint32_t hit = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) hit |= vis_bit<kReadOnlyCache>(lv.vis, u[k]);
      pos += 4;
      if (hit) {
        found = true;
        active = false;
      } else if (pos >= end) {
        active = false;
      }
    }
  }
  const uint32_t fm = __ballot_sync(kFull, found);
  if (found) {
    const int32_t deg = g.symmetric ? end - beg : g.off[v + 1] - g.off[v];
    lv.depth[v] = lv.next_depth;
    edges += (unsigned long long)deg;
    wbuf[wcnt + __popc(fm & lanemask_lt())] = v;
    atomicOr(lv.vis_next + (v >> 5), 1u << (v & 31));
  }
  wcnt += (unsigned)__popc(fm);
  __syncwarp();  // the list entries are read before the hint pass overwrites them
}

// After a hint-pass step: scan the misses 32 at a time while the list holds
// that many (all of them when drain), keeping the warp's stage below capacity.
template <bool kReadOnlyCache, int kWords>
__device__ __forceinline__ void pull_settle(const DevGraph& g, const Level& lv, const PullMisses<kWords>& ms,
                                            int& mcnt, bool drain, int32_t* wbuf, unsigned int& wcnt,
                                            unsigned long long& edges) {
  if (wcnt > (unsigned)(kWarpStage - kWords * 32)) {
    warp_stage_flush(wbuf, wcnt, lv);
    wcnt = 0;
  }
  while (mcnt >= 32 || (drain && mcnt > 0)) {  // uniform
    const int take = min(32, mcnt);
    mcnt -= take;
    pull_misses<kReadOnlyCache, kWords>(g, lv, ms, mcnt, take, wbuf, wcnt, edges);
    if (wcnt > (unsigned)(kWarpStage - kWords * 32)) {
      warp_stage_flush(wbuf, wcnt, lv);
      wcnt = 0;
    }
  }
}

// Two walks over the bitmap words share the hint pass. This warp's k-th word
// is (k / kWords) * stride + base0 + (k % kWords) * kWarps (consecutive warps
// take consecutive words; increasing in k), and it takes kWords per step.
//  - dense (most reachable vertices still unvisited): each step's words are
//    loaded one step ahead, and their row extents and hints prefetched into
//    L2, so those round trips overlap the current step;
//  - sparse (few left): a batch of 32 of the warp's words is loaded at once,
//    one per lane; words with no unvisited vertex are settled right there
//    (their next-bitmap word is all ones), the row extents and hints of the
//    others are prefetched into L2, and only those are taken. A late level
//    whose words are nearly all full then costs one round trip per 32 words
//    instead of one per kWords.
// scratch: pull_scratch_ints<kWords>() ints of the block's shared memory.
template <bool kReadOnlyCache>
__device__ __forceinline__ uint32_t pull_load_word(const uint32_t* vis, int32_t w) {
  return kReadOnlyCache ? ld_nc_u32(vis + w) : vis[w];
}

template <bool kReadOnlyCache, int kWords>
__device__ void body_pull(const DevGraph& g, const Level& lv, const Stage& stage, int32_t* scratch,
                          unsigned long long& edges) {
  static_assert(kWords * 32 <= kWarpStage, "a step must fit a stage slice");
  static_assert(32 % kWords == 0, "a batch holds whole steps");
  const uint32_t lane = lane_id();
  constexpr int kWarps = kThreads / 32;
  const int wib = threadIdx.x >> 5;
  int32_t* wbuf = stage.buf + wib * kWarpStage;  // the block stage is empty on entry
  unsigned int wcnt = 0;
  constexpr int kCap = PullMisses<kWords>::kCap;
  int32_t* mine = scratch + wib * 3 * kCap;
  const PullMisses<kWords> ms{mine, mine + kCap, mine + 2 * kCap};
  int mcnt = 0;
  const int stride = gridDim.x * kWarps * kWords;
  const int base0 = blockIdx.x * kWarps * kWords + wib;
  if (!lv.pull_sparse) {
    uint32_t cw_next[kWords];
#pragma unroll
    for (int j = 0; j < kWords; ++j) {
      const int wn = base0 + j * kWarps;
      cw_next[j] = wn < g.words ? pull_load_word<kReadOnlyCache>(lv.vis, wn) : kFull;
    }
    for (int wb = base0; wb < g.words; wb += stride) {
      int32_t w[kWords];
      uint32_t cw[kWords];
#pragma unroll
      for (int j = 0; j < kWords; ++j) {
        w[j] = wb + j * kWarps;
        w[j] = w[j] < g.words ? w[j] : -1;
        cw[j] = cw_next[j];
        const int wn = wb + j * kWarps + stride;
        cw_next[j] = wn < g.words ? pull_load_word<kReadOnlyCache>(lv.vis, wn) : kFull;
        if (wn < g.words) {  // the next step's row extents and hints
          prefetch_l2(g.in_off + (size_t)wn * 32);
          prefetch_l2(g.hint + (size_t)wn * 32);
        }
      }
      pull_words<kReadOnlyCache, kWords>(g, lv, w, cw, wbuf, wcnt, ms, mcnt, edges);
      pull_settle<kReadOnlyCache, kWords>(g, lv, ms, mcnt, false, wbuf, wcnt, edges);
    }
  } else {
    for (int k0 = 0;; k0 += 32) {
      const int kk = k0 + (int)lane;
      const int wl = (kk / kWords) * stride + base0 + (kk % kWords) * kWarps;
      if (__shfl_sync(kFull, wl, 0) >= g.words) break;  // uniform: lane 0 holds the batch's smallest word
      const bool inb = wl < g.words;
      const uint32_t cwl = inb ? pull_load_word<kReadOnlyCache>(lv.vis, wl) : kFull;
      const bool open = inb && cwl != kFull;
      if (inb && !open) lv.vis_next[wl] = kFull;
      if (open) {
        prefetch_l2(g.in_off + (size_t)wl * 32);
        prefetch_l2(g.hint + (size_t)wl * 32);
      }
      uint32_t todo = __ballot_sync(kFull, open);
      while (todo) {  // uniform
        int32_t w[kWords];
        uint32_t cw[kWords];
#pragma unroll
        for (int j = 0; j < kWords; ++j) {
          const int src = todo ? __ffs(todo) - 1 : 0;
          const bool have = todo != 0u;
          todo &= todo - 1u;
          w[j] = have ? __shfl_sync(kFull, wl, src) : -1;
          cw[j] = have ? __shfl_sync(kFull, cwl, src) : kFull;
        }
        pull_words<kReadOnlyCache, kWords>(g, lv, w, cw, wbuf, wcnt, ms, mcnt, edges);
        pull_settle<kReadOnlyCache, kWords>(g, lv, ms, mcnt, false, wbuf, wcnt, edges);
      }
    }
  }
  pull_settle<kReadOnlyCache, kWords>(g, lv, ms, mcnt, true, wbuf, wcnt, edges);
  if (wcnt) warp_stage_flush(wbuf, wcnt, lv);
}

// ---------------------------------------------------------------------------
// Edge list and reverse edge list (Section 3.1.1): one thread per edge of the
// whole graph, every level, four edges per thread per step (coalesced). Edge
// list: CSR entry e is the edge origin_out[e] -> idx[e], whose target is
// reached when its source is in the frontier (depth L). Reverse edge list:
// transpose entry e is in_idx[e] -> origin_in[e]; the destination's bitmap
// bit is read first, so settled destinations cost no depth read. Targets are
// claimed through the visited bitmap like the push variants', so frontier
// counts and queues stay exact.
// ---------------------------------------------------------------------------
template <bool kReverse>
__device__ void body_edge_list(const DevGraph& g, const Level& lv, const Stage& stage, unsigned long long& edges) {
  const int32_t L = lv.next_depth - 1;
  const long long m = g.m;
  const int32_t* origin = kReverse ? g.aux->origin_in : g.aux->origin_out;
  const int32_t* other = kReverse ? g.in_idx : g.idx;
  const long long step = (long long)blockDim.x * 4;
  for (long long base = (long long)blockIdx.x * step; base < m; base += (long long)gridDim.x * step) {
    int32_t v[4] = {0, 0, 0, 0};
    int nv = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const long long e = base + k * (long long)blockDim.x + threadIdx.x;
      if (e < m) {
        if (kReverse) {
          const int32_t dst = origin[e];
          if (!vis_bit<false>(lv.vis, dst) && lv.depth[other[e]] == L) v[nv++] = dst;
        } else {
          if (lv.depth[origin[e]] == L) v[nv++] = other[e];
        }
      }
    }
    visit_k<4>(g, lv, stage, v, nv, edges);
    stage_flush(stage, lv, kStageCap / 2);
  }
}

}  // namespace

// ===========================================================================
// Graph path: init, decide, and one kernel per body
// ===========================================================================
__global__ void __launch_bounds__(kThreads) k_init(DevGraph g, Buffers b, RunState* st, int32_t* depth, int32_t root,
                                                   int32_t forced, const TreeNode* tree, int32_t tree_nodes,
                                                   const QsTree* tree_qs, int32_t use_handles) {
  if (blockIdx.x == 0 && threadIdx.x == 0) st->t_entry = (long long)global_ns();
  init_fill(g, b.vis[0], depth, root);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->depth = depth;
    st->tree = tree;
    st->tree_qs = tree_qs;
    st->tree_nodes = tree_nodes;
    st->root = root;
    st->forced = forced;
    st->use_handles = use_handles;
    st->level = -1;
    st->variant = -1;
    st->qsel = 0;
    st->vsel = 0;
    st->frontier = 0;
    st->status = ST_OK;
    st->vw = 32;
    st->vw_policy = g.vw_policy;
    st->levels = 0;
    st->frontier_edges = 0;
    st->discovered = 0;
    st->edges_reached = 0;
    // the root is the output of "level -1": the first decide turns it into the frontier of level 0
    b.q[1][0] = root;
    st->next_count = 1;
    st->next_edges = (unsigned long long)(g.off[root + 1] - g.off[root]);
  }
}

// First node of the level-loop graph: opens the WHILE loop from the device.
// (The handle has no launch-time default: a value applied by the host when a
// launch is enqueued could reach a still-running earlier launch of the same
// graph on that stream; a kernel inside the launch is ordered with it.)
__global__ void k_loop_start(DevGraph g, Buffers b, RunState* st) {
  (void)g;
  (void)b;
  if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)st->h_while, 1u);
}

// Level end + tree evaluation, between levels on the device. Launched with
// kDecideThreads threads (one warp): lane 0 closes the level and keeps the
// state; the warp evaluates a tree that has a bit-parallel form, else lane 0
// walks it.
__global__ void __launch_bounds__(kDecideThreads) k_decide(DevGraph g, Buffers b, RunState* st) {
  (void)b;
  __shared__ long long s_in[3];  // f, e, discovered
  __shared__ int32_t s_go;       // 1: evaluate the tree this level
  RunState& s = *st;
  int32_t L = 0;
  if (threadIdx.x == 0) {
    // close level L-1: its output queue becomes the frontier of level L
    const unsigned int f = (unsigned int)*reinterpret_cast<volatile unsigned long long*>(&s.next_count);
    const unsigned long long e = *reinterpret_cast<volatile unsigned long long*>(&s.next_edges);
    s.next_count = 0;
    s.next_edges = 0;
    if (s.level >= 0 && s.variant == V_PULL) s.vsel ^= 1u;  // pull wrote the other bitmap
    s.qsel ^= 1u;
    L = s.level + 1;
    s.level = L;
    s.frontier = (int32_t)f;
    s.frontier_edges = (long long)e;
    s.discovered += f;
    s.edges_reached += (long long)e;
    // a traversal has at most n nonempty levels; more means corrupted state, so
    // end the loop with an error instead of iterating on
    if (L > g.n || s.discovered > g.n) s.status = ST_TIMEOUT;
    if (L < s.log_cap) s.log_time[L] = (long long)global_ns();
    s_go = 1;
    if (f == 0 || s.status != ST_OK) {
      s.levels = L;
      if (s.use_handles) {
        cudaGraphSetConditional((cudaGraphConditionalHandle)s.h_while, 0u);
        cudaGraphSetConditional((cudaGraphConditionalHandle)s.h_switch, (unsigned)V_FORCED_NUM);
      }
      s_go = 0;
    }
    s_in[0] = f;
    s_in[1] = (long long)e;
    s_in[2] = s.discovered;
  }
  __syncthreads();
  if (!s_go) return;  // uniform
  const long long f = s_in[0], e = s_in[1], discovered = s_in[2];
  L = st->level;
  int32_t v = s.forced;
  const QsTree* qs = s.tree_qs;
  if (v < 0 && qs != nullptr) v = qs_eval_warp(*qs, L, f, e, discovered);  // the whole warp
  if (threadIdx.x != 0) return;
  if (v < 0 && qs == nullptr && s.tree != nullptr && s.tree_nodes > 0)
    v = walk_tree(g, s.tree, s.tree_nodes, L, f, e, discovered);
  int32_t vw = 32;
  v = finish_variant(v, L, s.variant, f, e, &vw, s.forced >= 0, s.vw_policy);
  for (int i = 0; i < F_NUM; ++i) s.feat[i] = feature_value(g, i, L, f, e, discovered);
  s.variant = v;
  s.vw = vw;
  if (L < s.log_cap) {
    s.log_variant[L] = v;
    s.log_frontier[L] = f;
    s.log_edges[L] = e;
  }
  if (s.use_handles) cudaGraphSetConditional((cudaGraphConditionalHandle)s.h_switch, (unsigned)v);
}

// Vertex push with the other frontier-count modes (Section 3.1.4 comparison).
__global__ void __launch_bounds__(kThreads) k_push_thread_warp_count(DevGraph g, Buffers b, RunState* st) {
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  body_push_thread<CM_WARP>(g, lv, stage, edges);
  block_add_u64(edges, &st->next_edges);
}

__global__ void __launch_bounds__(kThreads) k_push_thread_atomic_count(DevGraph g, Buffers b, RunState* st) {
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  body_push_thread<CM_ATOMIC>(g, lv, stage, edges);
  block_add_u64(edges, &st->next_edges);
}

__global__ void __launch_bounds__(kThreads) k_push_thread(DevGraph g, Buffers b, RunState* st) {
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  body_push_thread(g, lv, stage, edges);
  stage_flush(stage, lv, 1);
  block_add_u64(edges, &st->next_edges);
}

__global__ void __launch_bounds__(kThreads) k_push_warp(DevGraph g, Buffers b, RunState* st) {
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  body_push_warp(g, lv, stage, st->vw, edges);
  stage_flush(stage, lv, 1);
  block_add_u64(edges, &st->next_edges);
}

__global__ void __launch_bounds__(kThreads) k_push_cta(DevGraph g, Buffers b, RunState* st) {
  __shared__ alignas(128) int32_t chunk[2 * kCtaChunk];
  __shared__ alignas(8) uint64_t bar[2];
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  cta_pipe_init(bar);
  CtaPipe pp{chunk, bar, 0u, 0u, 0u};
  unsigned long long edges = 0;
  body_push_cta(g, lv, stage, pp, &st->status, edges);
  stage_flush(stage, lv, 1);
  block_add_u64(edges, &st->next_edges);
}

// (A frontier of at most kPeSmall vertices is scanned by k_pe_expand itself:
// the three scan launches then return at once.)
__global__ void __launch_bounds__(kThreads) k_pe_reduce(DevGraph g, Buffers b, RunState* st) {
  const Level lv = load_level(g, b, st);
  if (lv.frontier <= kPeSmall) return;
  body_pe_reduce(g, lv, b);
}

__global__ void __launch_bounds__(kThreads) k_pe_top(DevGraph g, Buffers b, RunState* st) {
  (void)g;
  const int f = st->frontier;
  if (f <= kPeSmall) return;
  body_pe_top(b, f);
}

__global__ void __launch_bounds__(kThreads) k_pe_scan(DevGraph g, Buffers b, RunState* st) {
  (void)g;
  const int f = st->frontier;
  if (f <= kPeSmall) return;
  body_pe_scan(b, f);
}

__global__ void __launch_bounds__(kThreads) k_pe_expand(DevGraph g, Buffers b, RunState* st) {
  __shared__ int32_t s_a[kPeTile + 1];
  __shared__ int32_t s_beg[kPeTile + 1];
  __shared__ int s_split[2];
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  if (lv.frontier <= kPeSmall) {
    pe_small_scan(g, lv, s_a, s_beg);
    body_pe_expand<true>(g, lv, b, stage, s_a, s_beg, s_split, edges);
  } else {
    body_pe_expand<false>(g, lv, b, stage, s_a, s_beg, s_split, edges);
  }
  block_add_u64(edges, &st->next_edges);
}

__global__ void __launch_bounds__(kThreads) k_edge_list(DevGraph g, Buffers b, RunState* st) {
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  body_edge_list<false>(g, lv, stage, edges);
  stage_flush(stage, lv, 1);
  block_add_u64(edges, &st->next_edges);
}

__global__ void __launch_bounds__(kThreads) k_rev_edge_list(DevGraph g, Buffers b, RunState* st) {
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  body_edge_list<true>(g, lv, stage, edges);
  stage_flush(stage, lv, 1);
  block_add_u64(edges, &st->next_edges);
}

// Origin of every CSR entry: the vertex whose row [off[v], off[v + 1]) holds it.
__global__ void k_build_origin(const int32_t* off, int32_t n, int32_t* origin) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    for (int32_t e = off[v]; e < off[v + 1]; ++e) origin[e] = (int32_t)v;
}

__global__ void __launch_bounds__(kThreads) k_pull(DevGraph g, Buffers b, RunState* st) {
  BFS_DECLARE_STAGE(stage);
  const Level lv = load_level(g, b, st);
  unsigned long long edges = 0;
  __shared__ int32_t s_scratch[pull_scratch_ints<kPullWordsLaunch>()];
  body_pull<true, kPullWordsLaunch>(g, lv, stage, s_scratch, edges);
  stage_flush(stage, lv, 1);
  block_add_u64(edges, &st->next_edges);
}

// ===========================================================================
// Persistent path: the whole traversal in one cooperative launch
// ===========================================================================
// Clears the words the persistent kernel's blocks read before block 0 could
// reset them (a previous run may have stopped with an error).
// Timing harness: undo one level run from the graph path's state. The vertices
// the level discovered are exactly the entries it appended to the output
// queue, so resetting their depth and visited bit restores the state it
// started from, in time proportional to the level's output (pull wrote only
// the other bitmap, which is rewritten whole before it is read again).
__global__ void k_undo_level(Buffers b, RunState* st) {
  const unsigned int count = (unsigned int)st->next_count;
  const int32_t* qout = st->qsel ? b.q[0] : b.q[1];
  uint32_t* vis = st->vsel ? b.vis[1] : b.vis[0];
  int32_t* depth = st->depth;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)count; i += stride) {
    const int32_t v = qout[i];
    depth[v] = -1;
    atomicAnd(&vis[v >> 5], ~(1u << (v & 31)));
  }
}


// One shared-memory buffer serves the CTA variant's copy stage or the
// edge-centric tile of the persistent kernels.
constexpr int kPeSlot = kPeTile + 32;
static_assert(2 * kCtaChunk <= 2 * kPeSlot, "union sizing");
static_assert(pull_scratch_ints<kPullWordsPersistent>() <= 2 * kPeSlot, "union sizing");

// Level L of a persistent traversal (frontier in q[L & 1], appending to
// q[(L + 1) & 1] and to the (L + 1) % 3 level words; current bitmap vis[vsel]).
__device__ __forceinline__ Level persistent_level(const DevGraph& g, const Buffers& b, RunState* st, int32_t* depth,
                                                  int32_t L, unsigned int f, unsigned long long e,
                                                  long long discovered, uint32_t vsel) {
  Level lv;
  lv.qin = (L & 1) ? b.q[1] : b.q[0];
  lv.qout = (L & 1) ? b.q[0] : b.q[1];
  lv.vis = vsel ? b.vis[1] : b.vis[0];
  lv.vis_next = vsel ? b.vis[0] : b.vis[1];
  lv.depth = depth;
  lv.tail = &st->tail3[(L + 1) % 3];
  lv.next_depth = L + 1;
  lv.frontier = (int32_t)f;
  lv.latency_bound = (long long)e < kLatencyEdges;
  lv.pull_sparse = (long long)g.n_active - discovered < (long long)(g.n_active >> 4);
  return lv;
}

// The level's work with variant v inside a persistent kernel (every block of
// the cooperative grid calls it); returns the block's sum of the reached
// vertices' out-degrees, after the block's appends are flushed.
__device__ __forceinline__ unsigned long long persistent_level_work(const DevGraph& g, const Buffers& b, RunState* st,
                                                                    const Level& lv, int32_t v, int32_t vw,
                                                                    const Stage& stage, CtaPipe& pp, int32_t* ubuf,
                                                                    int* s_split, unsigned long long& bar_target) {
  const unsigned int f = (unsigned int)lv.frontier;
  unsigned long long edges = 0;
  switch (v) {
    case V_PUSH_THREAD: body_push_thread(g, lv, stage, edges); break;
    case V_PUSH_WARP: body_push_warp(g, lv, stage, vw, edges); break;
    case V_PUSH_CTA: body_push_cta(g, lv, stage, pp, &st->status, edges); break;
    case V_PUSH_EDGE:
      if ((int)f <= kPeSmall) {
        pe_small_scan(g, lv, ubuf, ubuf + kPeSlot);
        body_pe_expand<true>(g, lv, b, stage, ubuf, ubuf + kPeSlot, s_split, edges);
        break;
      }
      body_pe_reduce(g, lv, b);
      if (!grid_arrive_wait(&st->bar64, bar_target, &st->status)) break;
      if (blockIdx.x == 0) body_pe_top(b, (int)f);
      if (!grid_arrive_wait(&st->bar64, bar_target, &st->status)) break;
      body_pe_scan(b, (int)f);
      if (!grid_arrive_wait(&st->bar64, bar_target, &st->status)) break;
      body_pe_expand<false>(g, lv, b, stage, ubuf, ubuf + kPeSlot, s_split, edges);
      break;
    case V_EDGE_LIST: body_edge_list<false>(g, lv, stage, edges); break;
    case V_REV_EDGE_LIST: body_edge_list<true>(g, lv, stage, edges); break;
    default: body_pull<false, kPullWordsPersistent>(g, lv, stage, ubuf, edges); break;
  }
  stage_flush(stage, lv, 1);
  return block_sum_u64(edges);
}

// epoch: a number the host changes on every launch on this workspace. Block 0
// clears the barrier counter and the status word left by the previous run
// (which a failed run may leave set) and then publishes epoch; every other
// block waits for it before its first barrier, so no separate reset launch is
// needed.
// stall: STALL_NONE, or the test hook's choice of one bounded wait to run out.
__global__ void __launch_bounds__(kThreads, 4) k_bfs_persistent(DevGraph g, Buffers b, RunState* st, int32_t* depth,
                                                             int32_t root, int32_t forced, const TreeNode* tree,
                                                             int32_t tree_nodes, const QsTree* qs, uint32_t epoch,
                                                             int32_t stall) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->t_entry = (long long)global_ns();
    st->bar64 = 0;
    st->status = ST_OK;
    for (int k = 0; k < 3; ++k) {
      st->tail3[k] = 0;
      st->edg3[k] = 0;
    }
    st_release_u32(&st->run_epoch, epoch);
  }
  __shared__ alignas(128) int32_t ubuf[2 * kPeSlot];
  __shared__ alignas(8) uint64_t bar[2];
  __shared__ int s_split[2];
  // the tree is evaluated by every warp every level: its bit-parallel form
  // (trees of up to 64 leaves) is kept in shared memory; larger trees are
  // walked in global memory
  __shared__ QsTree s_qs;
  const bool use_qs = qs != nullptr;
  if (use_qs) {
    static_assert(sizeof(QsTree) % 4 == 0, "QsTree copy");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(qs);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_qs);
    for (int i = threadIdx.x; i < (int)(sizeof(QsTree) / 4); i += blockDim.x) dst[i] = src[i];
  }
  BFS_DECLARE_STAGE(stage);
  init_fill(g, b.vis[0], depth, root);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->depth = depth;
    st->root = root;
    st->forced = forced;
    b.q[0][0] = root;
  }
  cta_pipe_init(bar);
  CtaPipe pp{ubuf, bar, 0u, 0u, stall == STALL_BULK_COPY ? 16u : 0u};
  // the previous run's barrier state is cleared before any block arrives
  if (blockIdx.x != 0 && threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    while (ld_acquire_u32(&st->run_epoch) != epoch)
      if (global_ns() - t0 > kWaitLimitNs) break;  // the first barrier then times out and reports it
  }
  int32_t L = 0;
  long long discovered = 0, reached = 0;
  int32_t prev = -1;
  uint32_t vsel = 0;
  // lanes 0-7 of each warp: the box of the leaf the last evaluated level
  // reached (in_leaf_box); box_leaf < 0 until a level has been evaluated
  int32_t box_bound = 0, box_leaf = -1;
  // level 0's frontier is the root; later levels' f and e arrive with the barrier
  unsigned int f = 1;
  unsigned long long e = (unsigned long long)(g.off[root + 1] - g.off[root]);
  unsigned long long bar_target = 0;  // this block's copy of the grid barriers' arrival target
  bool ok = grid_arrive_wait(&st->bar64, bar_target, &st->status, stall == STALL_GRID_BARRIER ? 1u : 0u);
  for (; ok; ++L) {
    discovered += f;
    reached += (long long)e;
    if (f == 0) break;
    if (L > g.n || discovered > g.n) {  // corrupted state: stop with an error
      if (blockIdx.x == 0 && threadIdx.x == 0) st->status = ST_TIMEOUT;
      break;
    }
    int32_t vw = 32;
    int32_t v = forced;
    if (v < 0 && use_qs) {
      // same leaf box as the previous level: the walk reaches the same leaf, and
      // the level repeats the previous level's choice (for an unknown leaf too)
      if (box_leaf >= 0 && in_leaf_box(box_bound, L, f, (long long)e, discovered)) {
        v = prev;
      } else {
        box_leaf = qs_leaf_warp(s_qs, L, f, (long long)e, discovered);
        v = box_leaf >= 0 ? s_qs.leaf[box_leaf] : -1;
        box_bound = (box_leaf >= 0 && lane_id() < 8u) ? s_qs.box[box_leaf][lane_id()] : 0;
      }
    } else if (v < 0 && tree != nullptr && tree_nodes > 0)
      v = walk_tree(g, tree, tree_nodes, L, f, (long long)e, discovered);
    v = finish_variant(v, L, prev, f, (long long)e, &vw, forced >= 0, g.vw_policy);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->tail3[(L + 2) % 3] = 0;  // the slot of level L - 2's barrier, which every block has left
      st->edg3[(L + 2) % 3] = 0;
      if (L < st->log_cap) {
        st->log_variant[L] = v;
        st->log_frontier[L] = f;
        st->log_edges[L] = (long long)e;
        st->log_time[L] = (long long)global_ns();
      }
    }
    const Level lv = persistent_level(g, b, st, depth, L, f, e, discovered, vsel);
    const unsigned long long e_block = persistent_level_work(g, b, st, lv, v, vw, stage, pp, ubuf, s_split, bar_target);
    if (v == V_PULL) vsel ^= 1u;
    prev = v;
    ok = level_arrive_wait(&st->tail3[(L + 1) % 3], &st->edg3[(L + 1) % 3], e_block, &st->status, &f, &e,
                           (stall == STALL_LEVEL_BARRIER && L == 0) ? 1u : 0u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->levels = L;
    if (L < st->log_cap) st->log_time[L] = (long long)global_ns();
    st->discovered = discovered;
    st->edges_reached = reached;
  }
}

// Per-level timing harness inside the persistent driver: one cooperative
// launch expands level L of a traversal whose state (queues, bitmaps, depths)
// the host has advanced to that level, with variant v, exactly as the
// persistent traversal would (the same level code, grid and barrier), and
// records the device time from the start barrier to the end of the
// level-ending barrier, with the next frontier's size and edge count. The host
// clears the arrival count and the (L + 1) % 3 level words before each launch.
__global__ void __launch_bounds__(kThreads, 4) k_profile_level(DevGraph g, Buffers b, RunState* st, int32_t* depth,
                                                            int32_t L, int32_t v, uint32_t f, unsigned long long e,
                                                            long long discovered, uint32_t vsel) {
  __shared__ alignas(128) int32_t ubuf[2 * kPeSlot];
  __shared__ alignas(8) uint64_t bar[2];
  __shared__ int s_split[2];
  BFS_DECLARE_STAGE(stage);
  cta_pipe_init(bar);
  CtaPipe pp{ubuf, bar, 0u, 0u, 0u};
  int32_t vw = 32;
  v = finish_variant(v, L, -1, f, (long long)e, &vw, true, g.vw_policy);
  unsigned long long bar_target = 0;
  if (!grid_arrive_wait(&st->bar64, bar_target, &st->status)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->prof_t0 = (long long)global_ns();
  const Level lv = persistent_level(g, b, st, depth, L, f, e, discovered, vsel);
  const unsigned long long e_block = persistent_level_work(g, b, st, lv, v, vw, stage, pp, ubuf, s_split, bar_target);
  unsigned int fn = 0;
  unsigned long long en = 0;
  if (!level_arrive_wait(&st->tail3[(L + 1) % 3], &st->edg3[(L + 1) % 3], e_block, &st->status, &fn, &en)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->prof_t1 = (long long)global_ns();
    st->prof_f = fn;
    st->prof_e = en;
  }
}

// Before a profiled level: clear the arrival count, the status and the level
// words the level appends to.
__global__ void k_profile_reset(RunState* st, int32_t slot) {
  st->bar64 = 0;
  st->status = ST_OK;
  st->tail3[slot] = 0;
  st->edg3[slot] = 0;
}

// Undo a profiled level in the persistent layout: the `count` vertices it
// appended to q[qout] lose their depth and their bit in vis[vsel] (pull set no
// bit there; it wrote the other bitmap, which the next pull rewrites whole).
__global__ void k_undo_level_p(Buffers b, int32_t* depth, uint32_t qout, unsigned int count, uint32_t vsel) {
  const int32_t* q = qout ? b.q[1] : b.q[0];
  uint32_t* vis = vsel ? b.vis[1] : b.vis[0];
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (int)count; i += stride) {
    const int32_t v = q[i];
    depth[v] = -1;
    atomicAnd(&vis[v >> 5], ~(1u << (v & 31)));
  }
}

// ---------------------------------------------------------------------------
// Graph creation: validation, out-degree statistics, transpose
// ---------------------------------------------------------------------------
__global__ void k_validate(const int32_t* off, const int32_t* idx, int32_t n, int32_t m, int32_t* bad) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int32_t my = 0;
  if (tid == 0 && (off[0] != 0 || off[n] != m)) my = 1;
  for (int64_t v = tid; v < n; v += stride)
    if (off[v + 1] < off[v]) my = 1;
  for (int64_t e = tid; e < m; e += stride)
    if (idx[e] < 0 || idx[e] >= n) my = 1;
  if (my) atomicOr(bad, 1);
}

// Degree of v for the statistics: the row length in `off`, plus the row
// length in `off2` when given (in-degree + out-degree = total degree).
__device__ __forceinline__ unsigned int stat_degree(const int32_t* off, const int32_t* off2, int64_t v) {
  unsigned int d = (unsigned int)(off[v + 1] - off[v]);
  if (off2) d += (unsigned int)(off2[v + 1] - off2[v]);
  return d;
}

__global__ void k_deg_reduce(const int32_t* off, const int32_t* off2, int32_t n, unsigned long long* s1,
                             unsigned long long* s2, unsigned int* dmin, unsigned int* dmax) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned long long a = 0, q = 0;
  unsigned int lo = 0xffffffffu, hi = 0;
  for (int64_t v = tid; v < n; v += stride) {
    const unsigned int d = stat_degree(off, off2, v);
    a += (unsigned long long)d;
    q += (unsigned long long)d * (unsigned long long)d;
    lo = min(lo, d);
    hi = max(hi, d);
  }
  block_add_u64(a, s1);
  block_add_u64(q, s2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(kFull, lo, o));
    hi = max(hi, __shfl_xor_sync(kFull, hi, o));
  }
  if (lane_id() == 0) {
    atomicMin(dmin, lo);
    atomicMax(dmax, hi);
  }
}

__global__ void k_deg_hist(const int32_t* off, const int32_t* off2, int32_t n, int32_t* hist) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < n; v += stride) atomicAdd(&hist[stat_degree(off, off2, v)], 1);
}

namespace {
__device__ unsigned long long isqrt_u128(unsigned __int128 x) {
  unsigned long long lo = 0, hi = 0xffffffffull << 32 | 0xffffffffull;
  // largest r with r*r <= x (r < 2^64)
  while (lo < hi) {
    const unsigned long long mid = lo + ((hi - lo) >> 1) + 1;
    if ((unsigned __int128)mid * mid <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
}  // namespace

// One block: 5-number summary by nearest rank (q_k = sorted[floor(k (n-1)/4)])
// from the degree histogram, and floor(256 sigma) exactly:
// isqrt(65536 (n S2 - S1^2)) / n.
__global__ void k_deg_finish(const int32_t* hist, int64_t maxdeg, int32_t n, const unsigned long long* s1p,
                             const unsigned long long* s2p, long long* out6) {
  __shared__ long long carry_s;
  long long rank[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) rank[k] = ((long long)k * (n - 1)) / 4;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base <= maxdeg; base += blockDim.x) {
    const int64_t d = base + threadIdx.x;
    const long long c = d <= maxdeg ? hist[d] : 0;
    long long tot;
    const long long ex = block_exclusive_scan<long long>(c, &tot);
    const long long before = carry_s + ex;  // vertices with degree < d
    // d is the k-th quantile when before <= rank_k < before + c
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (c > 0 && before <= rank[k] && rank[k] < before + c) out6[k] = d;
    __syncthreads();
    if (threadIdx.x == 0) carry_s += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned __int128 S1 = *s1p, S2 = *s2p;
    const unsigned __int128 var_n2 = (unsigned __int128)n * S2 - S1 * S1;
    out6[5] = (long long)(isqrt_u128(var_n2 * 65536u) / (unsigned long long)n);
  }
}

__global__ void k_tr_count(const int32_t* idx, int32_t m, int32_t* cnt) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid; e < m; e += stride) atomicAdd(&cnt[idx[e]], 1);
}

// Generic exclusive scan of int32 (three kernels): per-block sums, scan of the
// block sums, apply. Blocks of kThreads threads x kPeItems items.
__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int32_t* in, int32_t len, long long* bsum) {
  const int nblk = (len + kPeTile - 1) / kPeTile;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kPeItems; ++k) {
      const long long i = (long long)blk * kPeTile + k * kThreads + threadIdx.x;
      if (i < len) s += in[i];
    }
    long long tot;
    block_exclusive_scan<long long>(s, &tot);
    if (threadIdx.x == 0) bsum[blk] = tot;
  }
}

__global__ void __launch_bounds__(kThreads) k_scan_top(long long* bsum, int32_t nblk) {
  long long carry = 0;
  for (int base = 0; base < nblk; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const long long x = i < nblk ? bsum[i] : 0;
    long long tot;
    const long long ex = block_exclusive_scan<long long>(x, &tot);
    if (i < nblk) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) bsum[nblk] = carry;
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(const int32_t* in, int32_t len, const long long* bsum,
                                                         int32_t* out) {
  const int nblk = (len + kPeTile - 1) / kPeTile;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const long long base = (long long)blk * kPeTile + threadIdx.x * kPeItems;
    int32_t d[kPeItems];
#pragma unroll
    for (int k = 0; k < kPeItems; ++k) d[k] = (base + k < len) ? in[base + k] : 0;
    long long run = 0;
    long long ex_k[kPeItems];
#pragma unroll
    for (int k = 0; k < kPeItems; ++k) {
      ex_k[k] = run;
      run += d[k];
    }
    long long tot;
    const long long ex = block_exclusive_scan<long long>(run, &tot);
    const long long o = bsum[blk] + ex;
#pragma unroll
    for (int k = 0; k < kPeItems; ++k)
      if (base + k < len) out[base + k] = (int32_t)(o + ex_k[k]);
    if (blk == nblk - 1 && threadIdx.x == 0) out[len] = (int32_t)bsum[nblk];
  }
}

__global__ void k_tr_scatter(const int32_t* off, const int32_t* idx, int32_t n, int32_t* cursor, int32_t* in_idx) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = tid; u < n; u += stride)
    for (int32_t e = off[u]; e < off[u + 1]; ++e) {
      const int32_t v = idx[e];
      in_idx[atomicAdd(&cursor[v], 1)] = (int32_t)u;
    }
}

// Bit v of the starting bitmap: set iff v has neither in- nor out-edges. No
// level can reach such a vertex, and it is nobody's in-neighbour, so marking it
// visited changes no depth; pull then skips it, and skips whole words of them.
// (A vertex with out-edges only must stay clear: pull would take its set bit
// for a frontier in-neighbour.) Bits past n stay clear.
__global__ void k_vis_init(const int32_t* off, const int32_t* in_off, int32_t n, int32_t words, uint32_t* vis_init,
                           unsigned int* isolated_count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < (int64_t)words * 32; v += stride) {
    // 32 consecutive threads share one word; every lane of a warp runs the same trips
    const bool isolated = v < n && off[v + 1] == off[v] && in_off[v + 1] == in_off[v];
    const uint32_t word = __ballot_sync(kFull, isolated);
    if ((v & 31) == 0) {
      vis_init[v >> 5] = word;
      if (word) atomicAdd(isolated_count, (unsigned)__popc(word));
    }
  }
}

// Pull hint of every vertex: among the first kHintScan entries of its in-list,
// the in-neighbour with the largest out-degree (the first such on ties; -1
// without in-edges). Any in-neighbour is a valid first test, so the cap only
// bounds the cost on hubs' long lists.
__global__ void k_pull_hint(const int32_t* off, const int32_t* in_off, const int32_t* in_idx, int32_t n,
                            int32_t* hint) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int32_t b = in_off[v];
    const int32_t e = min(in_off[v + 1], b + kHintScan);
    int32_t best = -1, best_deg = -1;
    for (int32_t k = b; k < e; ++k) {
      const int32_t u = in_idx[k];
      const int32_t d = off[u + 1] - off[u];
      if (d > best_deg) {
        best_deg = d;
        best = u;
      }
    }
    hint[v] = best;
  }
}

}  // namespace bfs
