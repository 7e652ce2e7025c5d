// C ABI of libbfs: graph objects, workspaces, the three level-loop drivers
// (persistent cooperative kernel; k_init followed by one CUDA graph per
// workspace, loop_start -> WHILE(frontier) { decide -> SWITCH(variant) { level
// kernels } }; host loop), the decision-tree store, multi-source batches and
// the per-level timing harness.
#include <algorithm>
#include <array>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <fstream>
#include <functional>
#include <limits>
#include <utility>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "bfs.h"
#include "bfs_kernels.cuh"
#include "bfs_msbfs.cuh"

using namespace bfs;

namespace {

thread_local std::string t_detail;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_detail = buf;
  return code;
}

#define CU(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA, "%s: %s (line %d)", #call, \
                  cudaGetErrorString(e_), __LINE__);                                                  \
    }                                                                                                 \
  } while (0)

#define TRY(expr)              \
  do {                         \
    int r_ = (expr);           \
    if (r_ != BFS_OK) return r_; \
  } while (0)

// Test hook: fail the N-th device allocation from now (0 = off). Lets tests
// exercise the out-of-memory paths without exhausting a shared GPU.
std::atomic<int> g_fail_alloc_countdown{0};

// Test hook: the bounded wait (enum Stall) the next persistent traversal or
// multi-source wave makes run out; taken by the first launch that reads it.
std::atomic<int> g_stall_next{0};
int take_stall() { return g_stall_next.exchange(0); }

int dmalloc(void** p, size_t bytes) {
  int c = g_fail_alloc_countdown.load();
  if (c > 0 && g_fail_alloc_countdown.fetch_sub(1) == 1) {
    *p = nullptr;
    return fail(BFS_ERR_OOM, "injected allocation failure (%zu bytes)", bytes);
  }
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                cudaGetErrorString(e));
  }
  return BFS_OK;
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// ---------------------------------------------------------------------------
// Decision trees
// ---------------------------------------------------------------------------
const TreeNode kBuiltinTree[] = {
#include "default_tree.inc"
};

struct TreeStore {
  std::mutex mu;
  std::vector<TreeNode> nodes;
  uint64_t version = 1;
};

TreeStore& tree_store() {
  static TreeStore* ts = [] {
    auto* t = new TreeStore;
    t->nodes.assign(std::begin(kBuiltinTree), std::end(kBuiltinTree));
    return t;
  }();
  return *ts;
}

// Children must have larger indices than their parent: every walk ends.
int check_tree(const std::vector<TreeNode>& t) {
  if (t.empty()) return fail(BFS_ERR_INVALID_ARG, "tree has no nodes");
  for (size_t i = 0; i < t.size(); ++i) {
    const TreeNode& nd = t[i];
    if (nd.f < -1 || nd.f >= F_NUM) return fail(BFS_ERR_INVALID_ARG, "node %zu: feature %d out of range", i, nd.f);
    if (nd.f >= 0) {
      if (nd.l <= (int)i || nd.r <= (int)i || nd.l >= (int)t.size() || nd.r >= (int)t.size())
        return fail(BFS_ERR_INVALID_ARG, "node %zu: children %d/%d invalid", i, nd.l, nd.r);
    } else if (nd.v < -1 || nd.v >= V_NUM) {
      return fail(BFS_ERR_INVALID_ARG, "node %zu: class %d out of range", i, nd.v);
    }
  }
  return BFS_OK;
}

int parse_tree(const std::string& text, std::vector<TreeNode>* out) {
  std::istringstream in(text);
  std::string line;
  long long count = -1;
  std::vector<TreeNode> nodes;
  while (std::getline(in, line)) {
    size_t p = line.find_first_not_of(" \t\r");
    if (p == std::string::npos || line[p] == '#') continue;
    std::istringstream ls(line);
    if (count < 0) {
      std::string magic;
      int ver = 0;
      if (!(ls >> magic >> ver >> count) || magic != "bfs-tree" || ver != 1 || count <= 0 || count > (1 << 20))
        return fail(BFS_ERR_INVALID_ARG, "bad tree header: %s", line.c_str());
      continue;
    }
    TreeNode nd{};
    long long f, l, r, v;
    if (!(ls >> f >> nd.t >> l >> r >> v)) return fail(BFS_ERR_INVALID_ARG, "bad tree node line: %s", line.c_str());
    // narrowed to int32 below: out-of-range values must not wrap into valid ones
    const auto fits = [](long long x) { return x >= -1 && x <= std::numeric_limits<int32_t>::max(); };
    if (!fits(f) || !fits(l) || !fits(r) || !fits(v))
      return fail(BFS_ERR_INVALID_ARG, "tree node field out of range: %s", line.c_str());
    nd.f = (int32_t)f;
    nd.l = (int32_t)l;
    nd.r = (int32_t)r;
    nd.v = (int32_t)v;
    nodes.push_back(nd);
  }
  if (count < 0 || (long long)nodes.size() != count)
    return fail(BFS_ERR_INVALID_ARG, "tree: expected %lld nodes, read %zu", count, nodes.size());
  TRY(check_tree(nodes));
  *out = std::move(nodes);
  return BFS_OK;
}

// ---------------------------------------------------------------------------
// Workspaces
// ---------------------------------------------------------------------------
struct Workspace {
  Buffers b{};
  RunState* st = nullptr;
  int32_t* log_variant = nullptr;
  long long* log_frontier = nullptr;
  long long* log_edges = nullptr;
  long long* log_time = nullptr;
  int32_t log_cap = 0;
  int32_t* host_depth_stage = nullptr;  // device buffer for runs whose output is host memory
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t start_node = nullptr;
  cudaEvent_t done = nullptr;
  cudaStream_t last_stream = nullptr;
  uint32_t epoch = 0;  // persistent launches so far (the kernel's barrier-state reset handshake)
  bool in_use = false;
  size_t bytes = 0;
  std::vector<void*> allocs;
};

constexpr int kMaxWorkspaces = 64;

struct Shapes {
  int init, push_thread, push_warp, push_cta, pe, pull, edge_list;
  int persist;  // cooperative grid of the persistent kernel (0: not supported)
  int profile;  // cooperative grid of the per-level timing kernel (the persistent grid when it fits)
};

}  // namespace

// One multi-source wave's buffers (bfs::MsSet, declared in bfs_internal.cuh):
// the graph's own set serves bfs_run_batch; the query server holds more so that
// several waves on one graph can run at once.
struct bfs::MsSet {
  MsBuffers mb{};
  MsState* st = nullptr;
  cudaEvent_t done = nullptr;  // recorded after each wave run on the set
  std::vector<void*> allocs;
  size_t bytes = 0;
};

struct bfs_graph {
  int device = 0;
  int sms = 0;
  DevGraph dg{};
  std::vector<void*> allocs;
  size_t bytes = 0;
  bool symmetric = false;
  long long stats6[6] = {0, 0, 0, 0, 0, 0};      // out-degree summary and floor(256 sd)
  long long stats_in6[6] = {0, 0, 0, 0, 0, 0};   // in-degree
  long long stats_tot6[6] = {0, 0, 0, 0, 0, 0};  // total degree
  Shapes shapes{};
  std::mutex mu;
  std::vector<Workspace*> pool;   // every workspace of the graph
  std::deque<Workspace*> idle;    // those not being enqueued, in release order
  // device copies of the process-wide tree, one per version seen (old ones may
  // still be read by runs in flight, so they live until destroy)
  std::vector<TreeNode*> trees;
  TreeNode* tree = nullptr;
  QsTree* tree_qs = nullptr;  // bit-parallel form of the same tree (inside the same allocation), or null
  // edge-list variants: the device GraphAux block and whether it has been filled
  GraphAux* aux = nullptr;
  bool has_origin = false;
  int32_t tree_nodes = 0;
  uint64_t tree_version = 0;
  // the graph's own multi-source buffer set (allocated on the first batch;
  // bfs_run_batch and bfs_batch_tune waves on it are ordered through its event)
  bfs::MsSet* ms_set = nullptr;
  std::mutex ms_mu;
  MsConfig ms_cfg{0, 16};
  int ms_grid = 0;       // one full occupancy wave of the multi-source kernel
  int ms_grid_user = 0;  // configured grid (0: ms_grid)
};

namespace {

int grid_for(const void* func, int sms, int cap_per_sm) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  per_sm = std::max(1, std::min(per_sm, cap_per_sm));
  return sms * per_sm;
}

// Host-to-device copy that has reached the device when it returns. A plain
// cudaMemcpy from pageable memory may return once the source is staged, before
// its DMA lands, and a kernel launched next on a non-blocking stream is not
// ordered after that DMA: it could read the old contents, or have its own
// writes overwritten when the DMA lands.
int upload_now(void* dst, const void* src, size_t bytes) {
  cudaStream_t s;
  CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return fail(BFS_ERR_CUDA, "upload of %zu bytes: %s", bytes, cudaGetErrorString(e));
  return BFS_OK;
}

void free_workspace(Workspace* ws) {
  if (!ws) return;
  if (ws->exec) cudaGraphExecDestroy(ws->exec);
  if (ws->graph) cudaGraphDestroy(ws->graph);
  if (ws->done) cudaEventDestroy(ws->done);
  for (void* p : ws->allocs) cudaFree(p);
  delete ws;
}

int ws_alloc(Workspace* ws, void** p, size_t bytes) {
  TRY(dmalloc(p, bytes));
  ws->allocs.push_back(*p);
  ws->bytes += bytes;
  return BFS_OK;
}

struct KArgs {
  DevGraph g;
  Buffers b;
  RunState* st;
  void* ptrs[3];
};

int add_kernel(cudaGraph_t graph, cudaGraphNode_t* node, const cudaGraphNode_t* dep, const void* func, int grid,
               int block, KArgs& a) {
  a.ptrs[0] = &a.g;
  a.ptrs[1] = &a.b;
  a.ptrs[2] = &a.st;
  cudaKernelNodeParams p{};
  p.func = const_cast<void*>(func);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.sharedMemBytes = 0;
  p.kernelParams = a.ptrs;
  CU(cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &p));
  return BFS_OK;
}

// The workspace's device state before its first run: the log buffers and, once
// the level-loop graph exists, its conditional handles.
int init_run_state(Workspace* ws, unsigned long long h_while, unsigned long long h_switch) {
  RunState init{};
  init.h_while = h_while;
  init.h_switch = h_switch;
  init.use_handles = h_while != 0;
  init.log_cap = ws->log_cap;
  init.log_variant = ws->log_variant;
  init.log_frontier = ws->log_frontier;
  init.log_edges = ws->log_edges;
  init.log_time = ws->log_time;
  return upload_now(ws->st, &init, sizeof init);
}

// Build the level loop of one workspace as a CUDA graph with conditional nodes
// (on the workspace's first run in the graph driver).
// The graph holds the level loop only: k_loop_start opens the WHILE loop on the
// device, and per-run values (root, output, forced variant, tree) reach it
// through RunState, written by a k_init launched on the same stream just
// before. Nothing in the instantiated graph changes between launches, so
// back-to-back launches on one stream cannot see each other's parameters.
int build_graph(bfs_graph* g, Workspace* ws) {
  CU(cudaGraphCreate(&ws->graph, 0));
  KArgs ka{g->dg, ws->b, ws->st, {}};
  TRY(add_kernel(ws->graph, &ws->start_node, nullptr, reinterpret_cast<const void*>(&k_loop_start), 1, 32, ka));

  cudaGraphConditionalHandle hw;
  CU(cudaGraphConditionalHandleCreate(&hw, ws->graph, 0, 0));
  cudaGraphNodeParams wp{};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CU(cudaGraphAddNode(&wnode, ws->graph, &ws->start_node, nullptr, 1, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];

  cudaGraphNode_t decide;
  TRY(add_kernel(body, &decide, nullptr, reinterpret_cast<const void*>(&k_decide), 1, kDecideThreads, ka));

  cudaGraphConditionalHandle hs;
  CU(cudaGraphConditionalHandleCreate(&hs, body, 0, 0));
  cudaGraphNodeParams sp{};
  sp.type = cudaGraphNodeTypeConditional;
  sp.conditional.handle = hs;
  sp.conditional.type = cudaGraphCondTypeSwitch;
  sp.conditional.size = V_FORCED_NUM;
  cudaGraphNode_t snode;
  CU(cudaGraphAddNode(&snode, body, &decide, nullptr, 1, &sp));
  cudaGraph_t* vb = sp.conditional.phGraph_out;
  const Shapes& s = g->shapes;
  cudaGraphNode_t n0, n1, n2, n3;
  TRY(add_kernel(vb[V_PUSH_THREAD], &n0, nullptr, reinterpret_cast<const void*>(&k_push_thread), s.push_thread,
                 kThreads, ka));
  TRY(add_kernel(vb[V_PUSH_WARP], &n0, nullptr, reinterpret_cast<const void*>(&k_push_warp), s.push_warp, kThreads,
                 ka));
  TRY(add_kernel(vb[V_PUSH_CTA], &n0, nullptr, reinterpret_cast<const void*>(&k_push_cta), s.push_cta, kThreads,
                 ka));
  TRY(add_kernel(vb[V_PUSH_EDGE], &n0, nullptr, reinterpret_cast<const void*>(&k_pe_reduce), s.pe, kThreads, ka));
  TRY(add_kernel(vb[V_PUSH_EDGE], &n1, &n0, reinterpret_cast<const void*>(&k_pe_top), 1, kThreads, ka));
  TRY(add_kernel(vb[V_PUSH_EDGE], &n2, &n1, reinterpret_cast<const void*>(&k_pe_scan), s.pe, kThreads, ka));
  TRY(add_kernel(vb[V_PUSH_EDGE], &n3, &n2, reinterpret_cast<const void*>(&k_pe_expand), s.pe, kThreads, ka));
  TRY(add_kernel(vb[V_PULL], &n0, nullptr, reinterpret_cast<const void*>(&k_pull), s.pull, kThreads, ka));
  TRY(add_kernel(vb[V_EDGE_LIST], &n0, nullptr, reinterpret_cast<const void*>(&k_edge_list), s.edge_list, kThreads,
                 ka));
  TRY(add_kernel(vb[V_REV_EDGE_LIST], &n0, nullptr, reinterpret_cast<const void*>(&k_rev_edge_list), s.edge_list,
                 kThreads, ka));
  CU(cudaGraphInstantiate(&ws->exec, ws->graph, 0));
  // the handles live in the device state, where decide sets them each level
  return init_run_state(ws, hw, hs);
}

int create_workspace(bfs_graph* g, Workspace** out) {
  auto* ws = new Workspace;
  const int64_t n = g->dg.n;
  const int64_t words = g->dg.words;
  const int64_t pe_blocks = (n + kPeTile - 1) / kPeTile + 2;
  int r = BFS_OK;
  void* p;
  auto A = [&](size_t bytes) -> void* {
    if (r != BFS_OK) return nullptr;
    r = ws_alloc(ws, &p, bytes);
    return r == BFS_OK ? p : nullptr;
  };
  ws->b.q[0] = static_cast<int32_t*>(A(n * 4));
  ws->b.q[1] = static_cast<int32_t*>(A(n * 4));
  ws->b.vis[0] = static_cast<uint32_t*>(A(words * 4));
  ws->b.vis[1] = static_cast<uint32_t*>(A(words * 4));
  ws->b.pe_scan = static_cast<int32_t*>(A((n + 1) * 4));
  ws->b.pe_beg = static_cast<int32_t*>(A(n * 4));
  ws->b.pe_bsum = static_cast<long long*>(A(pe_blocks * 8));
  ws->b.pe_blocks_cap = (int32_t)pe_blocks;
  ws->st = static_cast<RunState*>(A(sizeof(RunState)));
  ws->log_cap = (int32_t)std::min<int64_t>(n + 1, 1 << 16);
  ws->log_variant = static_cast<int32_t*>(A(ws->log_cap * 4));
  ws->log_frontier = static_cast<long long*>(A(ws->log_cap * 8));
  ws->log_edges = static_cast<long long*>(A(ws->log_cap * 8));
  ws->log_time = static_cast<long long*>(A(ws->log_cap * 8));
  if (r == BFS_OK) {
    cudaError_t e = cudaEventCreateWithFlags(&ws->done, cudaEventDisableTiming);
    if (e != cudaSuccess) r = fail(BFS_ERR_CUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
  }
  if (r == BFS_OK) r = init_run_state(ws, 0, 0);
  if (r != BFS_OK) {
    free_workspace(ws);
    return r;
  }
  *out = ws;
  return BFS_OK;
}

// A workspace free for `stream`: last used on the same stream (stream order
// then protects it), or idle on the device. Released workspaces are kept in
// release order and only the kIdleProbe oldest, the likeliest to have
// finished, are queried, so a busy pool costs a few event queries per acquire,
// not one per workspace. At the pool limit the oldest is reused after
// `stream` waits for its last run.
constexpr int kIdleProbe = 8;
int acquire(bfs_graph* g, cudaStream_t stream, Workspace** out) {
  std::lock_guard<std::mutex> lk(g->mu);
  Workspace* pick = nullptr;
  auto& idle = g->idle;
  for (auto it = idle.begin(); it != idle.end(); ++it)
    if ((*it)->last_stream == stream) {
      pick = *it;
      idle.erase(it);
      break;
    }
  if (!pick) {
    int probed = 0;
    for (auto it = idle.begin(); it != idle.end() && probed < kIdleProbe; ++it, ++probed)
      if (cudaEventQuery((*it)->done) == cudaSuccess) {
        pick = *it;
        idle.erase(it);
        break;
      }
  }
  if (!pick && (int)g->pool.size() < kMaxWorkspaces) {
    Workspace* ws = nullptr;
    TRY(create_workspace(g, &ws));
    g->pool.push_back(ws);
    pick = ws;
  }
  if (!pick) {
    if (idle.empty()) return fail(BFS_ERR_BUSY, "all %d workspaces are being enqueued", kMaxWorkspaces);
    pick = idle.front();
    idle.pop_front();
    CU(cudaStreamWaitEvent(stream, pick->done, 0));
  }
  cudaGetLastError();  // clear a not-ready status from cudaEventQuery
  pick->in_use = true;
  *out = pick;
  return BFS_OK;
}

int release(bfs_graph* g, Workspace* ws, cudaStream_t stream) {
  cudaError_t e = cudaEventRecord(ws->done, stream);
  std::lock_guard<std::mutex> lk(g->mu);
  ws->last_stream = stream;
  ws->in_use = false;
  g->idle.push_back(ws);
  if (e != cudaSuccess) return fail(BFS_ERR_CUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
  return BFS_OK;
}

// A test on a ppm share, floor(1e6 c / n) <= t, as the same test on the count
// c itself: it holds exactly when 1e6 c < (t + 1) n, i.e. when c <= ceil((t +
// 1) n / 1e6) - 1 (never for t < 0, always for t >= 1e6 since c <= n).
long long ppm_to_count_threshold(long long t, long long n) {
  if (t < 0) return -1;
  if (t >= 1000000) return std::numeric_limits<long long>::max();
  const long long a = (t + 1) * n;  // < 2^51 for n < 2^31
  return (a + 999999) / 1000000 - 1;
}

// Bit-parallel form of a tree (QsTree) for one graph: leaves numbered by a
// left-first depth-first walk from node 0, each internal node's mask clearing
// its left subtree's leaves. A test on a graph feature (gfeat: n, m, degree
// summary) is decided here: when it fails its mask goes into base, and either
// way it leaves no node for the device. A test on a ppm share becomes the same
// test on the count. False when the tree is too large for it or node 0 does
// not root a tree (a node reached twice).
// The tree as one graph sees it: every test on a graph feature is decided by
// the graph's own features (the node becomes the child it takes), and a test
// whose two sides end in leaves of one class becomes that leaf, bottom up. The
// prediction is the same for every level of the graph; the level-feature
// tests and leaves left are fewer, so the per-level evaluation is shorter and
// the leaf boxes larger. Children keep larger indices than their parents. An
// input whose shared subtrees would be copied past 4x its size is returned
// unchanged.
std::vector<TreeNode> simplify_tree(const std::vector<TreeNode>& t, const long long* gfeat) {
  std::vector<TreeNode> out;
  const size_t cap = 4 * t.size() + 16;
  bool ok = true;
  std::function<int(int)> rec = [&](int i) -> int {
    while (t[i].f >= 0 && is_graph_feature(t[i].f)) i = gfeat[t[i].f] <= t[i].t ? t[i].l : t[i].r;
    if (!ok || out.size() >= cap) {
      ok = false;
      return 0;
    }
    const int me = (int)out.size();
    out.push_back(t[i]);
    if (t[i].f < 0) return me;
    const int l = rec(t[i].l);
    const int r = rec(t[i].r);
    if (!ok) return 0;
    if (out[l].f < 0 && out[r].f < 0 && out[l].v == out[r].v) {
      out[me] = out[l];  // the two leaves were the last entries appended
      out.resize((size_t)me + 1);
      return me;
    }
    out[me].l = l;
    out[me].r = r;
    return me;
  };
  rec(0);
  return ok ? out : t;
}

bool build_qs(const std::vector<TreeNode>& t, const long long* gfeat, QsTree* q) {
  if (t.empty() || t.size() > 1024) return false;
  std::memset(q, 0, sizeof *q);
  std::vector<int> lo(t.size(), 0), hi(t.size(), 0);
  std::vector<char> seen(t.size(), 0);
  int nleaf = 0, nint = 0;
  bool ok = true;
  std::function<void(int)> dfs = [&](int i) {
    if (!ok || i < 0 || i >= (int)t.size() || seen[i]) {
      ok = false;
      return;
    }
    seen[i] = 1;
    const TreeNode& nd = t[i];
    if (nd.f < 0) {
      if (nleaf >= kQsMax) {
        ok = false;
        return;
      }
      q->leaf[nleaf] = nd.v;
      lo[i] = nleaf;
      hi[i] = ++nleaf;
      return;
    }
    dfs(nd.l);
    dfs(nd.r);
    if (!ok) return;
    lo[i] = lo[nd.l];
    hi[i] = hi[nd.r];
    unsigned long long m = ~0ull;
    for (int b = lo[nd.l]; b < hi[nd.l]; ++b) m &= ~(1ull << b);
    if (is_graph_feature(nd.f)) {
      if (!(gfeat[nd.f] <= nd.t)) q->base &= m;
      return;
    }
    if (nint >= kQsMax) {
      ok = false;
      return;
    }
    QsNode& qn = q->node[nint++];
    qn.t = nd.t;
    qn.f = nd.f;
    if (nd.f == F_FRONTIER_PPM || nd.f == F_DISCOVERED_PPM) {
      qn.f = nd.f == F_FRONTIER_PPM ? F_FRONTIER : F_DISCOVERED;
      qn.t = ppm_to_count_threshold(nd.t, gfeat[F_N]);
    }
    qn.mask = m;
  };
  q->base = ~0ull;
  dfs(0);
  if (!ok) return false;
  q->n_int = nint;
  q->n_leaf = nleaf;
  // leaf boxes: walk again, narrowing the level features' bounds on the way
  // down (x <= t on the left, x >= t + 1 on the right) and deciding the
  // graph-feature tests, leaves numbered in the same left-to-right order
  auto level_slot = [](int32_t f) {
    return f == F_FRONTIER || f == F_FRONTIER_PPM ? 0 : f == F_DISCOVERED || f == F_DISCOVERED_PPM ? 1
           : f == F_FRONTIER_EDGES ? 2 : 3;
  };
  int leaf_no = 0;
  std::function<void(int, std::array<long long, 8>, bool)> boxes = [&](int i, std::array<long long, 8> bx,
                                                                       bool reach) {
    const TreeNode& nd = t[i];
    if (nd.f < 0) {
      const int b = leaf_no++;
      for (int k = 0; k < 8; ++k) {
        const long long v = std::max<long long>(INT32_MIN, std::min<long long>(INT32_MAX, bx[k]));
        q->box[b][k] = (int32_t)v;
      }
      if (!reach) {
        for (int k = 0; k < 4; ++k) {
          q->box[b][2 * k] = INT32_MAX;
          q->box[b][2 * k + 1] = -1;
        }
      }
      return;
    }
    if (is_graph_feature(nd.f)) {
      const bool left = gfeat[nd.f] <= nd.t;
      boxes(nd.l, bx, reach && left);
      boxes(nd.r, bx, reach && !left);
      return;
    }
    long long thr = nd.t;
    if (nd.f == F_FRONTIER_PPM || nd.f == F_DISCOVERED_PPM) thr = ppm_to_count_threshold(nd.t, gfeat[F_N]);
    const int k = level_slot(nd.f);
    std::array<long long, 8> lb = bx, rb = bx;
    lb[2 * k + 1] = std::min(lb[2 * k + 1], thr);
    rb[2 * k] = std::max(rb[2 * k], thr == std::numeric_limits<long long>::max() ? thr : thr + 1);
    boxes(nd.l, lb, reach);
    boxes(nd.r, rb, reach);
  };
  std::array<long long, 8> all{};
  for (int k = 0; k < 4; ++k) {
    all[2 * k] = std::numeric_limits<long long>::min();
    all[2 * k + 1] = std::numeric_limits<long long>::max();
  }
  boxes(0, all, true);
  return true;
}

int sync_tree(bfs_graph* g) {
  TreeStore& ts = tree_store();
  std::lock_guard<std::mutex> lk(ts.mu);
  std::lock_guard<std::mutex> lk2(g->mu);
  if (g->tree_version == ts.version && g->tree) return BFS_OK;
  // one device block: the graph's simplified node array, then its
  // bit-parallel form when it exists
  const std::vector<TreeNode> nodes = simplify_tree(ts.nodes, g->dg.gfeat);
  const size_t tree_bytes = nodes.size() * sizeof(TreeNode);
  const size_t qs_off = (tree_bytes + 15) & ~size_t(15);
  QsTree qs;
  const bool has_qs = build_qs(nodes, g->dg.gfeat, &qs);
  std::vector<char> host(qs_off + sizeof(QsTree), 0);
  std::memcpy(host.data(), nodes.data(), tree_bytes);
  if (has_qs) std::memcpy(host.data() + qs_off, &qs, sizeof qs);
  void* p = nullptr;
  TRY(dmalloc(&p, host.size()));
  const int r = upload_now(p, host.data(), host.size());
  if (r != BFS_OK) {
    cudaFree(p);
    return r;
  }
  g->trees.push_back(static_cast<TreeNode*>(p));
  g->tree = static_cast<TreeNode*>(p);
  g->tree_qs = has_qs ? reinterpret_cast<QsTree*>(static_cast<char*>(p) + qs_off) : nullptr;
  g->tree_nodes = (int32_t)nodes.size();
  g->tree_version = ts.version;
  return BFS_OK;
}

// The edge-list variants' origin arrays, built on their first use (m int32
// each; one array for a symmetric graph) and published through the graph's
// GraphAux block, which the kernels read at run time.
int ensure_origin(bfs_graph* g) {
  std::lock_guard<std::mutex> lk(g->mu);
  if (g->has_origin) return BFS_OK;
  const int64_t m = g->dg.m;
  int32_t* out = nullptr;
  int32_t* in = nullptr;
  TRY(dmalloc(reinterpret_cast<void**>(&out), (size_t)std::max<int64_t>(m, 1) * 4));
  g->allocs.push_back(out);
  g->bytes += (size_t)std::max<int64_t>(m, 1) * 4;
  if (g->symmetric) {
    in = out;
  } else {
    TRY(dmalloc(reinterpret_cast<void**>(&in), (size_t)std::max<int64_t>(m, 1) * 4));
    g->allocs.push_back(in);
    g->bytes += (size_t)std::max<int64_t>(m, 1) * 4;
  }
  cudaStream_t s;
  CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  const int blocks = g->sms * 4;
  k_build_origin<<<blocks, kThreads, 0, s>>>(g->dg.off, g->dg.n, out);
  if (!g->symmetric) k_build_origin<<<blocks, kThreads, 0, s>>>(g->dg.in_off, g->dg.n, in);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return fail(BFS_ERR_CUDA, "origin arrays: %s", cudaGetErrorString(e));
  const GraphAux aux{out, in};
  TRY(upload_now(g->aux, &aux, sizeof aux));
  g->has_origin = true;
  return BFS_OK;
}

int launch_variant(bfs_graph* g, Workspace* ws, int v, cudaStream_t s, int32_t count_mode = CM_BLOCK);

int launch_graph(bfs_graph* g, Workspace* ws, int32_t root, int32_t* depth, int32_t forced, cudaStream_t stream) {
  if (!ws->exec) {
    // first graph-driver run on this workspace: its previous runs (other
    // drivers) finish before the state they use is rewritten
    CU(cudaEventSynchronize(ws->done));
    TRY(build_graph(g, ws));
  }
  k_init<<<g->shapes.init, kThreads, 0, stream>>>(g->dg, ws->b, ws->st, depth, root, forced, g->tree, g->tree_nodes,
                                                  g->tree_qs, 1);
  CU(cudaGetLastError());
  CU(cudaGraphLaunch(ws->exec, stream));
  return BFS_OK;
}

// One cooperative launch runs the whole traversal (k_bfs_persistent).
// grid_blocks > 0 runs the traversal on fewer blocks (every loop strides, the
// barrier counts gridDim), so several traversals can be resident at once.
int launch_persistent(bfs_graph* g, Workspace* ws, int32_t root, int32_t* depth, int32_t forced,
                      cudaStream_t stream, int32_t grid_blocks) {
  DevGraph dg = g->dg;
  Buffers b = ws->b;
  RunState* st = ws->st;
  const TreeNode* tree = g->tree;
  int32_t nodes = g->tree_nodes;
  const QsTree* qs = g->tree_qs;
  uint32_t epoch = ++ws->epoch;  // runs on one workspace are ordered, so consecutive launches differ
  int32_t stall = take_stall();
  void* args[] = {&dg, &b, &st, &depth, &root, &forced, &tree, &nodes, &qs, &epoch, &stall};
  const int grid = grid_blocks > 0 ? std::min(grid_blocks, g->shapes.persist) : g->shapes.persist;
  CU(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_bfs_persistent), dim3(grid), dim3(kThreads), args, 0,
                                 stream));
  return BFS_OK;
}

// The graph's kernels launched level by level from the host, reading each
// level's decision back (synchronous). Profilers can see every kernel here.
int launch_host_loop(bfs_graph* g, Workspace* ws, int32_t root, int32_t* depth, int32_t forced, cudaStream_t s,
                     int32_t count_mode) {
  k_init<<<g->shapes.init, kThreads, 0, s>>>(g->dg, ws->b, ws->st, depth, root, forced, g->tree, g->tree_nodes,
                                             g->tree_qs, 0);
  CU(cudaGetLastError());
  RunState hs{};
  for (;;) {
    k_decide<<<1, kDecideThreads, 0, s>>>(g->dg, ws->b, ws->st);
    CU(cudaMemcpyAsync(&hs, ws->st, sizeof hs, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hs.frontier == 0 || hs.status != ST_OK) break;
    TRY(launch_variant(g, ws, hs.variant, s, count_mode));
  }
  return BFS_OK;
}

int launch_run(bfs_graph* g, Workspace* ws, int32_t root, int32_t* depth, int32_t forced, int32_t mode,
               cudaStream_t stream, int32_t grid_blocks = 0, int32_t count_mode = CM_BLOCK) {
  if (mode == BFS_MODE_DEFAULT) mode = g->shapes.persist > 0 ? BFS_MODE_PERSISTENT : BFS_MODE_GRAPH;
  switch (mode) {
    case BFS_MODE_PERSISTENT:
      if (g->shapes.persist <= 0) return fail(BFS_ERR_INVALID_ARG, "device lacks cooperative launch");
      return launch_persistent(g, ws, root, depth, forced, stream, grid_blocks);
    case BFS_MODE_GRAPH: return launch_graph(g, ws, root, depth, forced, stream);
    case BFS_MODE_HOST_LOOP: return launch_host_loop(g, ws, root, depth, forced, stream, count_mode);
    default: return fail(BFS_ERR_INVALID_ARG, "mode %d", mode);
  }
}

// Launch the kernels of one variant for the current level directly on a
// stream (the host-driven counterpart of one SWITCH body).
int launch_variant(bfs_graph* g, Workspace* ws, int v, cudaStream_t s, int32_t count_mode) {
  const Shapes& sh = g->shapes;
  const DevGraph& dg = g->dg;
  switch (v) {
    case V_PUSH_THREAD:
      if (count_mode == CM_WARP)
        k_push_thread_warp_count<<<sh.push_thread, kThreads, 0, s>>>(dg, ws->b, ws->st);
      else if (count_mode == CM_ATOMIC)
        k_push_thread_atomic_count<<<sh.push_thread, kThreads, 0, s>>>(dg, ws->b, ws->st);
      else
        k_push_thread<<<sh.push_thread, kThreads, 0, s>>>(dg, ws->b, ws->st);
      break;
    case V_PUSH_WARP: k_push_warp<<<sh.push_warp, kThreads, 0, s>>>(dg, ws->b, ws->st); break;
    case V_PUSH_CTA: k_push_cta<<<sh.push_cta, kThreads, 0, s>>>(dg, ws->b, ws->st); break;
    case V_PUSH_EDGE:
      k_pe_reduce<<<sh.pe, kThreads, 0, s>>>(dg, ws->b, ws->st);
      k_pe_top<<<1, kThreads, 0, s>>>(dg, ws->b, ws->st);
      k_pe_scan<<<sh.pe, kThreads, 0, s>>>(dg, ws->b, ws->st);
      k_pe_expand<<<sh.pe, kThreads, 0, s>>>(dg, ws->b, ws->st);
      break;
    case V_PULL: k_pull<<<sh.pull, kThreads, 0, s>>>(dg, ws->b, ws->st); break;
    case V_EDGE_LIST: k_edge_list<<<sh.edge_list, kThreads, 0, s>>>(dg, ws->b, ws->st); break;
    case V_REV_EDGE_LIST: k_rev_edge_list<<<sh.edge_list, kThreads, 0, s>>>(dg, ws->b, ws->st); break;
    default: return fail(BFS_ERR_INVALID_ARG, "variant %d", v);
  }
  CU(cudaGetLastError());
  return BFS_OK;
}

int check_graph(bfs_graph_t g) {
  if (!g) return fail(BFS_ERR_INVALID_ARG, "null graph");
  return BFS_OK;
}

// Blocks of one full occupancy wave of the multi-source kernel (cooperative
// launch required). Called with g->ms_mu held.
int ms_grid_init(bfs_graph* g) {
  if (g->ms_grid > 0) return BFS_OK;
  int coop = 0, per_sm = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(&k_msbfs),
                                                             kMsThreads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return fail(BFS_ERR_CUDA, "multi-source BFS needs cooperative launch");
  }
  g->ms_grid = g->sms * std::min(per_sm, 8);
  return BFS_OK;
}

// The graph's own set. Called with g->ms_mu held.
int ms_prepare(bfs_graph* g) {
  if (g->ms_set) return BFS_OK;
  TRY(ms_grid_init(g));
  return bfs::ms_set_create(g, &g->ms_set);
}

// One wave of up to 64 roots (host array) into the k output rows (host array
// of device pointers) on the given set.
int ms_launch_wave(bfs_graph* g, MsSet* set, const int32_t* roots, int32_t k, int32_t* const* rows_out,
                   cudaStream_t s, MsConfig cfg, int32_t grid_blocks = 0) {
  MsRows rows{};
  for (int32_t i = 0; i < k; ++i) {
    rows.row[i] = rows_out[i];
    rows.root[i] = roots[i];
  }
  k_ms_reset<<<1, 1, 0, s>>>(set->st);
  CU(cudaGetLastError());
  DevGraph dg = g->dg;
  MsBuffers mb = set->mb;
  MsState* st = set->st;
  int32_t stall = take_stall();
  void* args[] = {&dg, &mb, &st, &k, &rows, &cfg, &stall};
  // default: a grid sized to the graph (one block per 4096 vertices, at least
  // a quarter of the SMs, at most one full occupancy wave), so that waves of
  // small graphs on different streams can be resident together
  const long long sized = std::max<long long>(((long long)g->dg.n + 4095) / 4096, std::max(1, g->sms / 4));
  const int grid = grid_blocks > 0 ? std::min(grid_blocks, g->ms_grid) : (int)std::min<long long>(sized, g->ms_grid);
  CU(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_msbfs), dim3(grid), dim3(kMsThreads), args, 0, s));
  return BFS_OK;
}

// Row pointers of a k x n row-major block.
void block_rows(int32_t* base, int64_t n, int32_t k, int32_t** rows) {
  for (int32_t i = 0; i < k; ++i) rows[i] = base + (size_t)i * (size_t)n;
}

}  // namespace

int bfs::set_error_detail(int code, const char* msg) { return fail(code, "%s", msg); }

long long bfs::workspace_bytes(const bfs_graph* g) {
  const long long n = g->dg.n, words = g->dg.words;
  // two queues, two bitmaps, edge-centric scan scratch, logs (a host-output
  // stage of 4 n bytes is added on a workspace's first host-output run)
  return 4 * n * 2 + 4 * words * 2 + 4 * (n + 1) + 4 * n + 8 * ((n + kPeTile - 1) / kPeTile + 2) +
         20 * std::min<long long>(n + 1, 1 << 16) + (long long)sizeof(RunState);
}

int32_t bfs::graph_vertices(const bfs_graph* g) { return g->dg.n; }

int bfs::graph_device(const bfs_graph* g) { return g->device; }

int32_t bfs::persistent_grid(const bfs_graph* g) { return g->shapes.persist; }

int32_t bfs::wave_grid(bfs_graph* g) {
  std::lock_guard<std::mutex> lk(g->ms_mu);
  if (ms_grid_init(g) != BFS_OK) return 0;
  return g->ms_grid;
}

int bfs::reserve_workspaces(bfs_graph* g, int32_t count) {
  DeviceGuard dgd(g->device);
  std::lock_guard<std::mutex> lk(g->mu);
  while ((int32_t)g->pool.size() < std::min<int32_t>(count, kMaxWorkspaces)) {
    Workspace* ws = nullptr;
    TRY(create_workspace(g, &ws));
    g->pool.push_back(ws);
    g->idle.push_back(ws);
  }
  return BFS_OK;
}

int bfs::run_async(bfs_graph* g, int32_t root, int32_t* depth_out, cudaStream_t stream, int32_t mode,
                   long long* edges_dst, int32_t grid_blocks, int32_t* status_dst) {
  if (root < 0 || root >= g->dg.n || !depth_out) return fail(BFS_ERR_INVALID_ARG, "run_async arguments");
  DeviceGuard dgd(g->device);
  TRY(sync_tree(g));
  Workspace* ws = nullptr;
  TRY(acquire(g, stream, &ws));
  int r = launch_run(g, ws, root, depth_out, -1, mode, stream, grid_blocks);
  if (r == BFS_OK && edges_dst) {
    cudaError_t e = cudaMemcpyAsync(edges_dst, &ws->st->edges_reached, sizeof(long long), cudaMemcpyDeviceToHost,
                                    stream);
    if (e != cudaSuccess) r = fail(BFS_ERR_CUDA, "edges copy: %s", cudaGetErrorString(e));
  }
  if (r == BFS_OK && status_dst) {
    cudaError_t e = cudaMemcpyAsync(status_dst, &ws->st->status, sizeof(int32_t), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) r = fail(BFS_ERR_CUDA, "status copy: %s", cudaGetErrorString(e));
  }
  int rr = release(g, ws, stream);
  return r != BFS_OK ? r : rr;
}

long long bfs::ms_set_bytes(const bfs_graph* g) {
  return ms_set_bytes_per_vertex() * (long long)g->dg.n + (long long)sizeof(MsState);
}

int bfs::ms_set_create(bfs_graph* g, MsSet** out) {
  DeviceGuard dgd(g->device);
  auto* set = new MsSet;
  const size_t n = (size_t)g->dg.n;
  int r = BFS_OK;
  auto A = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (r == BFS_OK) r = dmalloc(&p, bytes);
    if (r == BFS_OK) {
      set->allocs.push_back(p);
      set->bytes += bytes;
    }
    return p;
  };
  set->mb.visit = static_cast<unsigned long long*>(A(n * 8));
  set->mb.hist = static_cast<unsigned long long*>(A(n * 8 * (size_t)kMsHistLevels));
  set->mb.front[0] = static_cast<unsigned long long*>(A(n * 8));
  set->mb.front[1] = static_cast<unsigned long long*>(A(n * 8));
  set->mb.next = static_cast<unsigned long long*>(A(n * 8));
  set->mb.flist[0] = static_cast<int32_t*>(A(n * 4));
  set->mb.flist[1] = static_cast<int32_t*>(A(n * 4));
  set->mb.tlist = static_cast<int32_t*>(A(n * 4));
  set->st = static_cast<MsState*>(A(sizeof(MsState)));
  if (r == BFS_OK && cudaEventCreateWithFlags(&set->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    r = fail(BFS_ERR_CUDA, "cudaEventCreate");
  }
  if (r == BFS_OK) {
    // the masks start zero (the kernel keeps them so between waves)
    cudaStream_t zs;
    cudaError_t e = cudaStreamCreateWithFlags(&zs, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      const std::pair<void*, size_t> masks[] = {{set->mb.visit, n * 8},
                                                {set->mb.hist, n * 8 * (size_t)kMsHistLevels},
                                                {set->mb.front[0], n * 8},
                                                {set->mb.front[1], n * 8},
                                                {set->mb.next, n * 8}};
      for (const auto& z : masks)
        if (e == cudaSuccess) e = cudaMemsetAsync(z.first, 0, z.second, zs);
      if (e == cudaSuccess) e = cudaStreamSynchronize(zs);
      cudaStreamDestroy(zs);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      r = fail(BFS_ERR_CUDA, "wave set zeroing: %s", cudaGetErrorString(e));
    }
  }
  if (r == BFS_OK) {
    MsState init{};  // clean_blocks == clean_grid: the masks are zero
    r = upload_now(set->st, &init, sizeof init);
  }
  if (r != BFS_OK) {
    ms_set_free(set);
    return r;
  }
  *out = set;
  return BFS_OK;
}

void bfs::ms_set_free(MsSet* set) {
  if (!set) return;
  if (set->done) {
    cudaEventSynchronize(set->done);
    cudaEventDestroy(set->done);
  }
  for (void* p : set->allocs) cudaFree(p);
  delete set;
}

int bfs::batch_async(bfs_graph* g, MsSet* set, const int32_t* roots, int32_t k, int32_t* const* rows,
                     cudaStream_t stream, unsigned long long* edges_dst, int32_t grid_blocks, int32_t* status_dst) {
  if (!set || k < 1 || k > kMsMaxRoots || !roots || !rows) return fail(BFS_ERR_INVALID_ARG, "batch_async arguments");
  for (int32_t i = 0; i < k; ++i)
    if (!rows[i] || roots[i] < 0 || roots[i] >= g->dg.n) return fail(BFS_ERR_INVALID_ARG, "batch_async row or root");
  DeviceGuard dgd(g->device);
  MsConfig cfg;
  {
    std::lock_guard<std::mutex> lk(g->ms_mu);
    TRY(ms_grid_init(g));
    cfg = g->ms_cfg;
  }
  TRY(ms_launch_wave(g, set, roots, k, rows, stream, cfg, grid_blocks));
  if (edges_dst) CU(cudaMemcpyAsync(edges_dst, set->st->edges, kMsMaxRoots * 8, cudaMemcpyDeviceToHost, stream));
  if (status_dst) CU(cudaMemcpyAsync(status_dst, &set->st->status, 4, cudaMemcpyDeviceToHost, stream));
  CU(cudaEventRecord(set->done, stream));
  return BFS_OK;
}

namespace {

// The 5-number summary (nearest rank) and floor(256 sd) of the degrees of all
// n vertices, on the device: the row lengths of `off`, plus those of `off2`
// when given (in + out = total degree). Synchronous.
int degree_summary(const int32_t* off, const int32_t* off2, int32_t n, int blocks, long long out6[6]) {
  unsigned int* mm = nullptr;  // [0] min, [1] max
  unsigned long long* sums = nullptr;
  int32_t* hist = nullptr;
  long long* st6 = nullptr;
  unsigned int mm_h[2] = {0xffffffffu, 0u};
  cudaError_t e = cudaMalloc(&mm, 8);
  if (e == cudaSuccess) e = cudaMalloc(&sums, 16);
  if (e == cudaSuccess) e = cudaMalloc(&st6, 6 * 8);
  if (e == cudaSuccess) e = cudaMemcpy(mm, mm_h, 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(sums, 0, 16);
  if (e == cudaSuccess) {
    k_deg_reduce<<<blocks, kThreads>>>(off, off2, n, sums, sums + 1, mm, mm + 1);
    e = cudaMemcpy(mm_h, mm, 8, cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess) e = cudaMalloc(&hist, ((size_t)mm_h[1] + 1) * 4);
  if (e == cudaSuccess) e = cudaMemset(hist, 0, ((size_t)mm_h[1] + 1) * 4);
  if (e == cudaSuccess) {
    k_deg_hist<<<blocks, kThreads>>>(off, off2, n, hist);
    k_deg_finish<<<1, kThreads>>>(hist, (int64_t)mm_h[1], n, sums, sums + 1, st6);
    e = cudaMemcpy(out6, st6, 6 * 8, cudaMemcpyDeviceToHost);
  }
  for (void* p : {(void*)mm, (void*)sums, (void*)hist, (void*)st6})
    if (p) cudaFree(p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA, "degree statistics: %s",
                cudaGetErrorString(e));
  }
  return BFS_OK;
}

// The tree's choice for a level on the host (the same walk and unknown-
// prediction rule the device applies): features are exact integers, so every
// test is x[f] <= t.
int32_t host_tree_choice(const std::vector<TreeNode>& t, const long long* x, int32_t L, int32_t prev) {
  int32_t i = 0, v = -1;
  for (size_t step = 0; step <= t.size() && i >= 0 && i < (int32_t)t.size(); ++step) {
    const TreeNode& nd = t[(size_t)i];
    if (nd.f < 0) {
      v = nd.v;
      break;
    }
    i = x[nd.f] <= nd.t ? nd.l : nd.r;
  }
  if (v < 0 || v >= V_NUM) v = L == 0 ? kLevel0Default : prev;
  if (v < 0 || v >= V_NUM) v = kLevel0Default;
  return v;
}

// The timing harness in the persistent driver: every variant expands every
// level from the same state in a cooperative launch of k_profile_level (device
// timestamps around the level, as the traversal kernel runs it), the state is
// restored by k_undo_level_p, and the traversal advances with the chosen
// variant.
int profile_levels_persistent(bfs_graph* g, Workspace* ws, int32_t root, int32_t reps, int32_t advance_variant,
                              cudaStream_t s, int32_t* depth, bfs_level_profile* out, int32_t capacity,
                              int32_t* num_levels) {
  std::vector<TreeNode> tree;
  {
    TreeStore& ts = tree_store();
    std::lock_guard<std::mutex> lk(ts.mu);
    tree = ts.nodes;
  }
  k_init<<<g->shapes.init, kThreads, 0, s>>>(g->dg, ws->b, ws->st, depth, root, -1, g->tree, g->tree_nodes,
                                             g->tree_qs, 0);
  CU(cudaGetLastError());
  int32_t host_root = root;
  int32_t ends[2] = {0, 0};
  CU(cudaMemcpyAsync(ws->b.q[0], &host_root, 4, cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(ends, g->dg.off + root, 8, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  DevGraph dg = g->dg;
  Buffers b = ws->b;
  RunState* st = ws->st;
  const long long n = g->dg.n;
  int32_t L = 0;
  unsigned int f = 1;
  unsigned long long e = (unsigned long long)(ends[1] - ends[0]);
  long long discovered = 1;
  uint32_t vsel = 0;
  int32_t prev = -1;
  std::vector<float> t((size_t)reps);
  struct Rec {
    long long t0, t1;
    unsigned long long pe;
    unsigned int pf;
    int32_t status;
  };
  auto run_level = [&](int32_t v, Rec* rec) -> int {
    k_profile_reset<<<1, 1, 0, s>>>(st, (L + 1) % 3);
    CU(cudaGetLastError());
    int32_t Lv = L, vv = v;
    uint32_t ff = f, vs = vsel;
    unsigned long long ee = e;
    long long dd = discovered;
    void* args[] = {&dg, &b, &st, &depth, &Lv, &vv, &ff, &ee, &dd, &vs};
    CU(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&k_profile_level), dim3(g->shapes.profile),
                                   dim3(kThreads), args, 0, s));
    RunState hs;
    CU(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    rec->t0 = hs.prof_t0;
    rec->t1 = hs.prof_t1;
    rec->pf = hs.prof_f;
    rec->pe = hs.prof_e;
    rec->status = hs.status;
    if (hs.status != ST_OK) return fail(BFS_ERR_TIMEOUT, "a bounded device-side wait gave up");
    return BFS_OK;
  };
  while (f > 0) {
    long long x[F_NUM];
    for (int k = 0; k < F_NUM; ++k) x[k] = g->dg.gfeat[k];
    x[F_FRONTIER] = f;
    x[F_FRONTIER_PPM] = 1000000ll * (long long)f / n;
    x[F_DISCOVERED] = discovered;
    x[F_DISCOVERED_PPM] = 1000000ll * discovered / n;
    x[F_FRONTIER_EDGES] = (long long)e;
    x[F_LEVEL] = L;
    const int32_t tv = host_tree_choice(tree, x, L, prev);
    if (L < capacity) {
      bfs_level_profile& P = out[L];
      for (int k = 0; k < F_NUM; ++k) P.features[k] = x[k];
      P.tree_variant = tv;
      P.pad = 0;
      for (int v = 0; v < V_NUM; ++v) {
        for (int k = 0; k < reps; ++k) {
          Rec rec;
          TRY(run_level(v, &rec));
          t[(size_t)k] = (float)((double)(rec.t1 - rec.t0) * 1e-6);
          k_undo_level_p<<<g->shapes.init, kThreads, 0, s>>>(b, depth, (uint32_t)((L + 1) & 1), rec.pf, vsel);
          CU(cudaGetLastError());
        }
        std::sort(t.begin(), t.end());
        P.ms[v] = t[(size_t)reps / 2];
      }
    }
    // advance to the next level (the resulting state does not depend on the variant)
    const int32_t adv = advance_variant >= 0 ? advance_variant : tv;
    Rec rec;
    TRY(run_level(adv, &rec));
    if (adv == V_PULL) vsel ^= 1u;
    prev = adv;
    f = rec.pf;
    e = rec.pe;
    discovered += f;
    ++L;
    if (L > n) return fail(BFS_ERR_TIMEOUT, "more levels than vertices");
  }
  *num_levels = L;
  return BFS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* bfs_status_string(int status) {
  switch (status) {
    case BFS_OK: return "ok";
    case BFS_ERR_INVALID_ARG: return "invalid argument";
    case BFS_ERR_BAD_GRAPH: return "malformed graph";
    case BFS_ERR_OOM: return "out of memory";
    case BFS_ERR_CUDA: return "CUDA error";
    case BFS_ERR_TIMEOUT: return "timed out";
    case BFS_ERR_BUSY: return "busy";
    case BFS_ERR_CANCELLED: return "cancelled";
    case BFS_ERR_NOT_FOUND: return "not found";
    default: return "unknown status";
  }
}

const char* bfs_last_error_detail(void) { return t_detail.c_str(); }

int bfs_version(void) { return 200; }

// Test hook (not part of the public header's contract): make the n-th device
// allocation from now fail with BFS_ERR_OOM; 0 disables.
int bfs_debug_fail_alloc_after(int n) {
  g_fail_alloc_countdown.store(n < 0 ? 0 : n);
  return BFS_OK;
}

int bfs_debug_stall_next_launch(int mode) {
  if (mode < STALL_NONE || mode > STALL_BULK_COPY) return fail(BFS_ERR_INVALID_ARG, "stall mode %d", mode);
  g_stall_next.store(mode);
  return BFS_OK;
}

int bfs_graph_create(const int32_t* row_offsets, const int32_t* col_indices, int64_t n, int64_t m, uint32_t flags,
                     bfs_graph_t* out) {
  if (!out) return fail(BFS_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  if (!row_offsets || (!col_indices && m > 0)) return fail(BFS_ERR_INVALID_ARG, "null CSR pointer");
  if (n < 1 || n >= INT32_MAX || m < 0 || m > (int64_t)INT32_MAX - 64)
    return fail(BFS_ERR_INVALID_ARG, "sizes out of range (n=%lld, m=%lld)", (long long)n, (long long)m);
  if (flags & ~(uint32_t)(BFS_SYMMETRIC | BFS_INPUT_ON_DEVICE | BFS_VALIDATE))
    return fail(BFS_ERR_INVALID_ARG, "unknown flags 0x%x", flags);
  std::unique_ptr<bfs_graph> g(new bfs_graph);
  CU(cudaGetDevice(&g->device));
  CU(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device));
  g->symmetric = (flags & BFS_SYMMETRIC) != 0;
  auto cleanup = [&]() {
    for (void* p : g->allocs) cudaFree(p);
    g->allocs.clear();
  };
  auto galloc = [&](void** p, size_t bytes) -> int {
    int r = dmalloc(p, bytes);
    if (r == BFS_OK) {
      g->allocs.push_back(*p);
      g->bytes += bytes;
    }
    return r;
  };
  const cudaMemcpyKind kind = (flags & BFS_INPUT_ON_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  int32_t *off = nullptr, *idx = nullptr;
  int r = galloc(reinterpret_cast<void**>(&off), (n + 1) * 4);
  if (r == BFS_OK) r = galloc(reinterpret_cast<void**>(&idx), (m + kIdxPad) * 4);
  if (r != BFS_OK) {
    cleanup();
    return r;
  }
  cudaError_t e = cudaMemcpy(off, row_offsets, (n + 1) * 4, kind);
  if (e == cudaSuccess && m > 0) e = cudaMemcpy(idx, col_indices, m * 4, kind);
  if (e == cudaSuccess) e = cudaMemset(idx + m, 0, kIdxPad * 4);
  // validation is unconditional: a malformed CSR would make kernels read out of bounds
  int32_t* scratch = nullptr;  // [0] bad flag, [1] dmin, [2] dmax
  unsigned long long* sums = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&scratch, 16);
  if (e == cudaSuccess) e = cudaMalloc(&sums, 16);
  if (e != cudaSuccess) {
    if (scratch) cudaFree(scratch);
    cleanup();
    return fail(BFS_ERR_CUDA, "graph upload: %s", cudaGetErrorString(e));
  }
  const int blocks = g->sms * 4;
  int32_t init3[3] = {0, INT32_MAX, 0};
  cudaMemcpy(scratch, init3, 12, cudaMemcpyHostToDevice);
  cudaMemset(sums, 0, 16);
  k_validate<<<blocks, kThreads>>>(off, idx, (int32_t)n, (int32_t)m, scratch);
  int32_t bad = 0;
  e = cudaMemcpy(&bad, scratch, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess || bad) {
    cudaFree(scratch);
    cudaFree(sums);
    cleanup();
    if (e != cudaSuccess) return fail(BFS_ERR_CUDA, "validate: %s", cudaGetErrorString(e));
    return fail(BFS_ERR_BAD_GRAPH, "CSR failed validation (off[0]=0, nondecreasing, off[n]=m, 0<=idx<n)");
  }
  cudaFree(scratch);
  cudaFree(sums);
  // transpose for pull when the graph may be directed
  int32_t *in_off = off, *in_idx = idx;
  if (!g->symmetric) {
    r = galloc(reinterpret_cast<void**>(&in_off), (n + 1) * 4);
    if (r == BFS_OK) r = galloc(reinterpret_cast<void**>(&in_idx), (m + kIdxPad) * 4);
    int32_t* cnt = nullptr;
    long long* bsum = nullptr;
    const int64_t nblk = (n + kPeTile - 1) / kPeTile;
    if (r == BFS_OK) {
      e = cudaMalloc(&cnt, (n + 1) * 4);
      if (e == cudaSuccess) e = cudaMalloc(&bsum, (nblk + 2) * 8);
      if (e == cudaSuccess) e = cudaMemset(cnt, 0, (n + 1) * 4);
      if (e == cudaSuccess) e = cudaMemset(in_idx + m, 0, kIdxPad * 4);
      if (e == cudaSuccess) {
        k_tr_count<<<blocks, kThreads>>>(idx, (int32_t)m, cnt);
        k_scan_reduce<<<blocks, kThreads>>>(cnt, (int32_t)n, bsum);
        k_scan_top<<<1, kThreads>>>(bsum, (int32_t)nblk);
        k_scan_apply<<<blocks, kThreads>>>(cnt, (int32_t)n, bsum, in_off);
        e = cudaMemcpy(cnt, in_off, (n + 1) * 4, cudaMemcpyDeviceToDevice);
      }
      if (e == cudaSuccess) {
        k_tr_scatter<<<blocks, kThreads>>>(off, idx, (int32_t)n, cnt, in_idx);
        e = cudaDeviceSynchronize();
      }
      if (e != cudaSuccess) r = fail(BFS_ERR_CUDA, "transpose: %s", cudaGetErrorString(e));
    }
    if (cnt) cudaFree(cnt);
    if (bsum) cudaFree(bsum);
    if (r != BFS_OK) {
      cleanup();
      return r;
    }
  }
  // starting bitmap: isolated vertices are marked visited up front
  uint32_t* vis_init = nullptr;
  const int64_t words = (n + 31) / 32;
  r = galloc(reinterpret_cast<void**>(&vis_init), words * 4);
  if (r == BFS_OK) r = galloc(reinterpret_cast<void**>(&g->aux), sizeof(GraphAux));
  if (r == BFS_OK) {
    const GraphAux none{nullptr, nullptr};
    r = upload_now(g->aux, &none, sizeof none);
  }
  if (r != BFS_OK) {
    cleanup();
    return r;
  }
  // the pull variant's first test per vertex (k_pull_hint)
  int32_t* hint = nullptr;
  r = galloc(reinterpret_cast<void**>(&hint), (size_t)n * 4);
  if (r != BFS_OK) {
    cleanup();
    return r;
  }
  k_pull_hint<<<blocks, kThreads>>>(off, in_off, in_idx, (int32_t)n, hint);
  unsigned int* iso = nullptr;
  unsigned int iso_h = 0;
  e = cudaMalloc(&iso, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(iso, 0, sizeof(unsigned int));
  if (e == cudaSuccess) {
    k_vis_init<<<blocks, kThreads>>>(off, in_off, (int32_t)n, (int32_t)words, vis_init, iso);
    e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&iso_h, iso, sizeof iso_h, cudaMemcpyDeviceToHost);
  if (iso) cudaFree(iso);
  if (e != cudaSuccess) {
    cleanup();
    return fail(e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA, "graph create: %s",
                cudaGetErrorString(e));
  }
  // degree statistics (Section 4.1 degree distribution): out-degree, in-degree
  // (the transpose's row lengths) and total degree
  r = degree_summary(off, nullptr, (int32_t)n, blocks, g->stats6);
  if (r == BFS_OK) r = degree_summary(in_off, nullptr, (int32_t)n, blocks, g->stats_in6);
  if (r == BFS_OK) r = degree_summary(off, in_off, (int32_t)n, blocks, g->stats_tot6);
  if (r != BFS_OK) {
    cleanup();
    return r;
  }
  DevGraph& dg = g->dg;
  dg.off = off;
  dg.idx = idx;
  dg.in_off = in_off;
  dg.in_idx = in_idx;
  dg.vis_init = vis_init;
  dg.hint = hint;
  dg.aux = g->aux;
  dg.n = (int32_t)n;
  dg.m = (int32_t)m;
  dg.words = (int32_t)((n + 31) / 32);
  dg.symmetric = g->symmetric ? 1 : 0;
  dg.n_active = (int32_t)(n - (int64_t)iso_h);
  dg.gfeat[F_N] = n;
  dg.gfeat[F_M] = m;
  for (int k = 0; k < 6; ++k) {
    dg.gfeat[F_DEG_MIN + k] = g->stats6[k];
    dg.gfeat[F_IN_DEG_MIN + k] = g->stats_in6[k];
    dg.gfeat[F_TOT_DEG_MIN + k] = g->stats_tot6[k];
  }
  Shapes& s = g->shapes;
  s.init = g->sms * 4;
  s.push_thread = grid_for(reinterpret_cast<const void*>(&k_push_thread), g->sms, 8);
  s.push_warp = grid_for(reinterpret_cast<const void*>(&k_push_warp), g->sms, 8);
  s.push_cta = grid_for(reinterpret_cast<const void*>(&k_push_cta), g->sms, 8);
  s.pe = grid_for(reinterpret_cast<const void*>(&k_pe_expand), g->sms, 8);
  s.pull = grid_for(reinterpret_cast<const void*>(&k_pull), g->sms, 8);
  s.edge_list = grid_for(reinterpret_cast<const void*>(&k_edge_list), g->sms, 8);
  // the persistent kernel needs every block resident: one full occupancy wave
  int coop = 0, per_sm = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
  if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(&k_bfs_persistent),
                                                            kThreads, 0) == cudaSuccess && per_sm > 0)
    s.persist = g->sms * std::min(per_sm, 8);
  else
    s.persist = 0;
  per_sm = 0;
  if (s.persist > 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                           &per_sm, reinterpret_cast<const void*>(&k_profile_level), kThreads, 0) == cudaSuccess)
    s.profile = std::min(s.persist, g->sms * std::min(per_sm, 8));
  else
    s.profile = 0;
  cudaGetLastError();
  *out = g.release();
  return BFS_OK;
}

int bfs_graph_destroy(bfs_graph_t g) {
  if (!g) return BFS_OK;
  DeviceGuard dgd(g->device);
  cudaError_t e = cudaDeviceSynchronize();
  for (Workspace* ws : g->pool) free_workspace(ws);
  for (TreeNode* t : g->trees) cudaFree(t);
  bfs::ms_set_free(g->ms_set);
  for (void* p : g->allocs) cudaFree(p);
  delete g;
  if (e != cudaSuccess) return fail(BFS_ERR_CUDA, "destroy: %s", cudaGetErrorString(e));
  return BFS_OK;
}

int bfs_graph_info(bfs_graph_t g, bfs_graph_info_t* info) {
  TRY(check_graph(g));
  if (!info) return fail(BFS_ERR_INVALID_ARG, "info is null");
  std::lock_guard<std::mutex> lk(g->mu);
  info->n = g->dg.n;
  info->m = g->dg.m;
  for (int k = 0; k < 5; ++k) {
    info->deg_summary[k] = g->stats6[k];
    info->in_deg_summary[k] = g->stats_in6[k];
    info->tot_deg_summary[k] = g->stats_tot6[k];
  }
  info->deg_sd256 = g->stats6[5];
  info->in_deg_sd256 = g->stats_in6[5];
  info->tot_deg_sd256 = g->stats_tot6[5];
  size_t b = g->bytes;
  for (Workspace* ws : g->pool) b += ws->bytes;
  info->bytes_resident = (int64_t)b;
  info->symmetric = g->symmetric ? 1 : 0;
  info->num_workspaces = (int32_t)g->pool.size();
  return BFS_OK;
}

static_assert((int)BFS_VW_NUM == (int)VW_NUM && (int)BFS_VW_RULE == (int)VW_RULE && (int)BFS_VW_32 == (int)VW_32,
              "width policy numbering");

int bfs_set_warp_width(bfs_graph_t g, int32_t policy) {
  TRY(check_graph(g));
  if (policy < 0 || policy >= VW_NUM) return fail(BFS_ERR_INVALID_ARG, "width policy %d out of range", policy);
  std::lock_guard<std::mutex> lk(g->mu);
  g->dg.vw_policy = policy;
  return BFS_OK;
}

int bfs_get_warp_width(bfs_graph_t g, int32_t* policy) {
  TRY(check_graph(g));
  if (!policy) return fail(BFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(g->mu);
  *policy = g->dg.vw_policy;
  return BFS_OK;
}

int bfs_tune_warp_width(bfs_graph_t g, const int32_t* roots, int32_t k, bfs_stream_t stream_, bfs_warp_tune* out) {
  TRY(check_graph(g));
  if (!roots || !out || k < 1 || k > 4096) return fail(BFS_ERR_INVALID_ARG, "tune takes 1..4096 roots and an output");
  for (int32_t i = 0; i < k; ++i)
    if (roots[i] < 0 || roots[i] >= g->dg.n) return fail(BFS_ERR_INVALID_ARG, "root %d out of range", roots[i]);
  DeviceGuard dgd(g->device);
  TRY(sync_tree(g));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  void* depth = nullptr;
  TRY(dmalloc(&depth, (size_t)g->dg.n * 4));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int r = BFS_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = fail(BFS_ERR_CUDA, "events");
  // the policy is written between launches of this thread without g->mu
  // (acquire takes it); the call is documented as not concurrent with other
  // runs on the graph
  const int32_t keep = g->dg.vw_policy;
  int32_t best = keep;
  float best_ms = 1e30f;
  for (int32_t p = 0; p < VW_NUM && r == BFS_OK; ++p) {
    g->dg.vw_policy = p;
    float ms = 0.f;
    for (int32_t i = -1; i < k && r == BFS_OK; ++i) {  // i = -1: untimed
      Workspace* ws = nullptr;
      r = acquire(g, s, &ws);
      if (r != BFS_OK) break;
      if (i == 0 && cudaEventRecord(e0, s) != cudaSuccess) r = fail(BFS_ERR_CUDA, "event record");
      if (r == BFS_OK)
        r = launch_run(g, ws, roots[i < 0 ? 0 : i], static_cast<int32_t*>(depth), -1, BFS_MODE_DEFAULT, s);
      const int rr = release(g, ws, s);
      if (r == BFS_OK) r = rr;
    }
    if (r == BFS_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      r = fail(BFS_ERR_CUDA, "tuning run failed");
    if (r != BFS_OK) break;
    out->ms[p] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = p;
    }
  }
  g->dg.vw_policy = r == BFS_OK ? best : keep;
  if (r == BFS_OK) {
    out->policy = best;
    out->reserved = 0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(depth);
  return r;
}

int bfs_load_tree(const char* path_or_null) {
  std::vector<TreeNode> nodes;
  if (!path_or_null) {
    nodes.assign(std::begin(kBuiltinTree), std::end(kBuiltinTree));
  } else {
    std::ifstream f(path_or_null);
    if (!f) return fail(BFS_ERR_NOT_FOUND, "cannot open tree file %s", path_or_null);
    std::stringstream ss;
    ss << f.rdbuf();
    TRY(parse_tree(ss.str(), &nodes));
  }
  TreeStore& ts = tree_store();
  std::lock_guard<std::mutex> lk(ts.mu);
  ts.nodes = std::move(nodes);
  ts.version += 1;
  return BFS_OK;
}

int bfs_run_ex(bfs_graph_t g, int32_t root, int32_t* depth_out, bfs_stream_t stream_, const bfs_options* opts,
               bfs_run_stats* stats) {
  TRY(check_graph(g));
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (!depth_out) return fail(BFS_ERR_INVALID_ARG, "depth_out is null");
  if (root < 0 || root >= g->dg.n) return fail(BFS_ERR_INVALID_ARG, "root %d not in [0, %d)", root, g->dg.n);
  int32_t forced = -1, mode = BFS_MODE_DEFAULT, grid_blocks = 0, count_mode = CM_BLOCK;
  bool host_out = false, host_async = false;
  if (opts) {
    if (opts->forced_variant < -1 || opts->forced_variant >= V_FORCED_NUM)
      return fail(BFS_ERR_INVALID_ARG, "forced_variant %d out of range", opts->forced_variant);
    if (opts->mode < BFS_MODE_DEFAULT || opts->mode > BFS_MODE_HOST_LOOP)
      return fail(BFS_ERR_INVALID_ARG, "mode %d out of range", opts->mode);
    for (int k = 0; k < 2; ++k)
      if (opts->reserved[k]) return fail(BFS_ERR_INVALID_ARG, "reserved option fields must be zero");
    if (opts->count_mode < 0 || opts->count_mode >= CM_NUM)
      return fail(BFS_ERR_INVALID_ARG, "count_mode %d out of range", opts->count_mode);
    if (opts->count_mode != CM_BLOCK && opts->mode != BFS_MODE_HOST_LOOP)
      return fail(BFS_ERR_INVALID_ARG, "count_mode applies to the host-loop driver only");
    count_mode = opts->count_mode;
    if (opts->grid_blocks < 0) return fail(BFS_ERR_INVALID_ARG, "grid_blocks < 0");
    if (opts->grid_blocks > 0 && (opts->mode == BFS_MODE_GRAPH || opts->mode == BFS_MODE_HOST_LOOP))
      return fail(BFS_ERR_INVALID_ARG, "grid_blocks applies to the persistent driver only");
    forced = opts->forced_variant;
    mode = opts->mode;
    host_out = opts->depth_on_host != 0;
    if (opts->host_async != 0 && opts->host_async != 1) return fail(BFS_ERR_INVALID_ARG, "host_async is 0 or 1");
    if (opts->host_async && (!host_out || stats))
      return fail(BFS_ERR_INVALID_ARG, "host_async applies to host output without statistics");
    host_async = opts->host_async != 0;
    grid_blocks = opts->grid_blocks;
  }
  DeviceGuard dgd(g->device);
  TRY(sync_tree(g));
  if (forced == V_EDGE_LIST || forced == V_REV_EDGE_LIST) TRY(ensure_origin(g));
  Workspace* ws = nullptr;
  TRY(acquire(g, stream, &ws));
  int r = BFS_OK;
  if (host_out && !ws->host_depth_stage) {  // allocated on a workspace's first host-output run
    void* p = nullptr;
    r = ws_alloc(ws, &p, (size_t)g->dg.n * 4);
    ws->host_depth_stage = static_cast<int32_t*>(p);
  }
  int32_t* dst = host_out ? ws->host_depth_stage : depth_out;
  if (r == BFS_OK) r = launch_run(g, ws, root, dst, forced, mode, stream, grid_blocks, count_mode);
  RunState hs{};
  if (r == BFS_OK && host_out) {
    cudaError_t e = cudaMemcpyAsync(depth_out, dst, (size_t)g->dg.n * 4, cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) r = fail(BFS_ERR_CUDA, "depth copy: %s", cudaGetErrorString(e));
  }
  if (r == BFS_OK && stats) {
    cudaError_t e = cudaMemcpyAsync(&hs, ws->st, sizeof hs, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && stats->log_capacity > 0) {
      const int32_t cnt = std::min(std::min(hs.levels, ws->log_cap), stats->log_capacity);
      if (cnt > 0) {
        if (stats->log_variant) e = cudaMemcpy(stats->log_variant, ws->log_variant, cnt * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && stats->log_frontier)
          e = cudaMemcpy(stats->log_frontier, ws->log_frontier, cnt * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && stats->log_frontier_edges)
          e = cudaMemcpy(stats->log_frontier_edges, ws->log_edges, cnt * 8, cudaMemcpyDeviceToHost);
        // level start stamps plus the end stamp (entry `levels`) when it fits
        const int32_t tcnt = std::min(std::min(hs.levels + 1, ws->log_cap), stats->log_capacity + 1);
        if (e == cudaSuccess && stats->log_time_ns)
          e = cudaMemcpy(stats->log_time_ns, ws->log_time, tcnt * 8, cudaMemcpyDeviceToHost);
      }
    }
    if (e != cudaSuccess) r = fail(BFS_ERR_CUDA, "stats: %s", cudaGetErrorString(e));
  }
  if (r == BFS_OK && host_out && !stats && !host_async) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) r = fail(BFS_ERR_CUDA, "sync: %s", cudaGetErrorString(e));
  }
  int rr = release(g, ws, stream);
  if (r != BFS_OK) return r;
  if (rr != BFS_OK) return rr;
  if (stats) {
    stats->edges_reached = hs.edges_reached;
    stats->vertices_reached = hs.discovered;
    stats->levels = hs.levels;
    stats->status = hs.status;
    stats->start_ns = hs.t_entry;
    if (hs.status != ST_OK) return fail(BFS_ERR_TIMEOUT, "a bounded device-side wait gave up");
  }
  return BFS_OK;
}

int bfs_run(bfs_graph_t g, int32_t root, int32_t* depth_out, bfs_stream_t stream) {
  return bfs_run_ex(g, root, depth_out, stream, nullptr, nullptr);
}

int bfs_run_batch(bfs_graph_t g, const int32_t* roots, int32_t k, int32_t* depth_out, bfs_stream_t stream,
                  int64_t* edges_out) {
  TRY(check_graph(g));
  if (k < 0) return fail(BFS_ERR_INVALID_ARG, "k < 0");
  if (k == 0) return BFS_OK;
  if (!roots || !depth_out) return fail(BFS_ERR_INVALID_ARG, "null roots or depth_out");
  for (int32_t i = 0; i < k; ++i)
    if (roots[i] < 0 || roots[i] >= g->dg.n)
      return fail(BFS_ERR_INVALID_ARG, "roots[%d] = %d not in [0, %d)", i, roots[i], g->dg.n);
  DeviceGuard dgd(g->device);
  std::lock_guard<std::mutex> lk(g->ms_mu);
  TRY(ms_prepare(g));
  MsSet* set = g->ms_set;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CU(cudaStreamWaitEvent(s, set->done, 0));
  const int64_t n = g->dg.n;
  for (int32_t w0 = 0; w0 < k; w0 += kMsMaxRoots) {
    const int32_t kw = std::min<int32_t>(kMsMaxRoots, k - w0);
    int32_t* rows[kMsMaxRoots];
    block_rows(depth_out + (size_t)w0 * n, n, kw, rows);
    TRY(ms_launch_wave(g, set, roots + w0, kw, rows, s, g->ms_cfg, g->ms_grid_user));
    if (edges_out) {
      unsigned long long e[kMsMaxRoots];
      CU(cudaMemcpyAsync(e, set->st->edges, sizeof e, cudaMemcpyDeviceToHost, s));
      int32_t status = 0;
      CU(cudaMemcpyAsync(&status, &set->st->status, 4, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (status != ST_OK) return fail(BFS_ERR_TIMEOUT, "a bounded device-side wait gave up");
      for (int32_t i = 0; i < kw; ++i) edges_out[w0 + i] = (int64_t)e[i];
    }
  }
  CU(cudaEventRecord(set->done, s));
  return BFS_OK;
}

int bfs_batch_set_config(bfs_graph_t g, const bfs_batch_config* cfg) {
  TRY(check_graph(g));
  if (!cfg || cfg->push_mode < 0 || cfg->push_mode > 1 || cfg->alpha < 1 || cfg->grid_blocks < 0)
    return fail(BFS_ERR_INVALID_ARG, "batch config out of range");
  std::lock_guard<std::mutex> lk(g->ms_mu);
  g->ms_cfg = MsConfig{cfg->push_mode, cfg->alpha};
  g->ms_grid_user = cfg->grid_blocks;
  return BFS_OK;
}

int bfs_batch_tune(bfs_graph_t g, const int32_t* roots, int32_t k, int32_t* depth_scratch, bfs_stream_t stream,
                   bfs_batch_config* best) {
  return bfs_batch_tune_ex(g, roots, k, depth_scratch, stream, 1, best);
}

int bfs_batch_tune_ex(bfs_graph_t g, const int32_t* roots, int32_t k, int32_t* depth_scratch, bfs_stream_t stream,
                      int32_t concurrency, bfs_batch_config* best) {
  TRY(check_graph(g));
  if (k < 1 || k > 64 || !roots || !depth_scratch || !best)
    return fail(BFS_ERR_INVALID_ARG, "tune takes 1..64 roots, a k*n scratch buffer and an output");
  if (concurrency < 1 || concurrency > 64) return fail(BFS_ERR_INVALID_ARG, "concurrency %d not in [1, 64]", concurrency);
  for (int32_t i = 0; i < k; ++i)
    if (roots[i] < 0 || roots[i] >= g->dg.n) return fail(BFS_ERR_INVALID_ARG, "root out of range");
  DeviceGuard dgd(g->device);
  std::lock_guard<std::mutex> lk(g->ms_mu);
  TRY(ms_prepare(g));
  MsSet* set = g->ms_set;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CU(cudaStreamWaitEvent(s, set->done, 0));
  int32_t* rows[kMsMaxRoots];
  block_rows(depth_scratch, g->dg.n, k, rows);
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  const int alphas[] = {2, 4, 8, 16, 32, 64};
  // the grids tried: a full occupancy wave and its halves down to 1/16, those
  // no larger than twice the device's even share of one of `concurrency` waves
  // running together (waves of uneven graphs rarely all run at once), at
  // least the smallest
  const int share = std::max(std::min(g->ms_grid, 2 * g->ms_grid / concurrency), g->ms_grid / 16);
  int grids[5], ng = 0;
  for (int d = 1; d <= 16; d *= 2)
    if (g->ms_grid / d <= share) grids[ng++] = std::max(1, g->ms_grid / d);
  if (ng > 3) ng = 3;  // the three largest that qualify
  float best_ms = 1e30f;
  MsConfig best_cfg = g->ms_cfg;
  int best_grid = g->ms_grid_user;
  int r = BFS_OK;
  for (int gi = 0; gi < ng && r == BFS_OK; ++gi) {
    const int grid = grids[gi];
    for (int pm = 0; pm < 2 && r == BFS_OK; ++pm)
      for (int a : alphas) {
        const MsConfig c{pm, a};
        r = ms_launch_wave(g, set, roots, k, rows, s, c, grid);  // warm-up
        if (r != BFS_OK) break;
        float ms = 0;
        if (cudaEventRecord(e0, s) != cudaSuccess ||
            (r = ms_launch_wave(g, set, roots, k, rows, s, c, grid)) != BFS_OK ||
            cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          if (r == BFS_OK) r = fail(BFS_ERR_CUDA, "tuning run failed");
          break;
        }
        if (ms < best_ms) {
          best_ms = ms;
          best_cfg = c;
          best_grid = grid;
        }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != BFS_OK) return r;
  g->ms_cfg = best_cfg;
  g->ms_grid_user = best_grid;
  best->push_mode = best_cfg.push_mode;
  best->alpha = best_cfg.alpha;
  best->ms = best_ms;
  best->grid_blocks = best_grid;
  CU(cudaEventRecord(set->done, s));
  return BFS_OK;
}

int bfs_profile_levels(bfs_graph_t g, int32_t root, int32_t reps, int32_t advance_variant, bfs_stream_t stream_,
                       bfs_level_profile* out, int32_t capacity, int32_t* num_levels) {
  TRY(check_graph(g));
  if (root < 0 || root >= g->dg.n) return fail(BFS_ERR_INVALID_ARG, "root %d not in [0, %d)", root, g->dg.n);
  if (reps < 1 || reps > 1000) return fail(BFS_ERR_INVALID_ARG, "reps %d not in [1, 1000]", reps);
  if (advance_variant < -1 || advance_variant >= V_NUM) return fail(BFS_ERR_INVALID_ARG, "advance_variant");
  if (capacity < 0 || (capacity > 0 && !out) || !num_levels) return fail(BFS_ERR_INVALID_ARG, "output");
  *num_levels = 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
  DeviceGuard dgd(g->device);
  TRY(sync_tree(g));
  Workspace* ws = nullptr;
  TRY(acquire(g, s, &ws));
  const size_t n = (size_t)g->dg.n;
  int32_t* depth = nullptr;
  RunState* snap_st = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int r = dmalloc(reinterpret_cast<void**>(&depth), n * 4);
  if (r == BFS_OK) r = dmalloc(reinterpret_cast<void**>(&snap_st), sizeof(RunState));
  if (r == BFS_OK && (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess))
    r = fail(BFS_ERR_CUDA, "cudaEventCreate");
  if (r == BFS_OK && g->shapes.profile > 0) {
    // the default driver's own timing: levels inside the persistent kernel
    r = profile_levels_persistent(g, ws, root, reps, advance_variant, s, depth, out, capacity, num_levels);
    cudaStreamSynchronize(s);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    for (void* p : {(void*)depth, (void*)snap_st})
      if (p) cudaFree(p);
    const int rr = release(g, ws, s);
    return r != BFS_OK ? r : rr;
  }
  int32_t L = 0;
  std::vector<float> t(reps);
  auto body = [&]() -> int {
    k_init<<<g->shapes.init, kThreads, 0, s>>>(g->dg, ws->b, ws->st, depth, root, -1, g->tree, g->tree_nodes,
                                               g->tree_qs, 0);
    CU(cudaGetLastError());
    RunState hs{};
    for (;;) {
      k_decide<<<1, kDecideThreads, 0, s>>>(g->dg, ws->b, ws->st);
      CU(cudaMemcpyAsync(&hs, ws->st, sizeof hs, cudaMemcpyDeviceToHost, s));
      CU(cudaStreamSynchronize(s));
      if (hs.frontier == 0 || hs.status != ST_OK) break;
      if (L < capacity) {
        bfs_level_profile& P = out[L];
        for (int k = 0; k < F_NUM; ++k) P.features[k] = hs.feat[k];
        P.tree_variant = hs.variant;
        P.pad = 0;
        CU(cudaMemcpyAsync(snap_st, ws->st, sizeof(RunState), cudaMemcpyDeviceToDevice, s));
        for (int v = 0; v < V_NUM; ++v) {
          for (int k = 0; k < reps; ++k) {
            CU(cudaEventRecord(ev[0], s));
            TRY(launch_variant(g, ws, v, s));
            CU(cudaEventRecord(ev[1], s));
            // undo the level (its discoveries are the output queue) and restore the counters
            k_undo_level<<<g->shapes.init, kThreads, 0, s>>>(ws->b, ws->st);
            CU(cudaMemcpyAsync(ws->st, snap_st, sizeof(RunState), cudaMemcpyDeviceToDevice, s));
            CU(cudaEventSynchronize(ev[1]));
            CU(cudaEventElapsedTime(&t[k], ev[0], ev[1]));
          }
          std::sort(t.begin(), t.end());
          P.ms[v] = t[reps / 2];
        }
      }
      // advance to the next level (the resulting state does not depend on the variant)
      int32_t adv = advance_variant >= 0 ? advance_variant : hs.variant;
      CU(cudaMemcpyAsync(&ws->st->variant, &adv, 4, cudaMemcpyHostToDevice, s));
      TRY(launch_variant(g, ws, adv, s));
      ++L;
    }
    CU(cudaStreamSynchronize(s));
    return BFS_OK;
  };
  if (r == BFS_OK) r = body();
  *num_levels = L;
  cudaStreamSynchronize(s);
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  for (void* p : {(void*)depth, (void*)snap_st})
    if (p) cudaFree(p);
  int rr = release(g, ws, s);
  return r != BFS_OK ? r : rr;
}

}  // extern "C"
