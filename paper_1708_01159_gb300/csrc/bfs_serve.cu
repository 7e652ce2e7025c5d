// bfs_serve: a continuous-batching BFS server over graphs resident in HBM.
//
// A dispatcher thread owns the device side. Submissions enter a FIFO queue;
// whenever an in-flight slot and the memory a unit needs fit the budget, the
// dispatcher admits it, first fit over the head of the queue, so a large query
// waiting for memory does not block smaller ones behind it. A unit is one
// single-root traversal or a multi-source wave: when two or more queries to a
// graph are queued and one of the graph's wave buffer sets is free, up to
// merge_batch of them run as one wave (one bit per query in 64-bit masks), each
// root's depths written straight into its query's buffer. Units run on a pool
// of streams and overlap on the device; each goes to the stream with the fewest
// units in flight. Completion is observed by polling a CUDA event per unit;
// latency runs from submission to that observation.
//
// Everything the dispatcher hands out is allocated when a graph is registered
// (bfs_serve_add_graph): traversal workspaces for single queries, n-entry depth
// buffers for queries submitted without one, and the wave buffer sets. A unit
// that finds its pool empty waits in the queue; the dispatcher itself never
// allocates device memory. Registration also probes the graph's launch shape:
// the block count of its single queries, and whether waves are cheaper per
// query than single runs (merge_policy 0 merges only then).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bfs.h"
#include "bfs_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket;
  int32_t graph_id;
  int32_t root;
  int32_t* depth_out;  // device, or null: the server supplies a buffer
  Clock::time_point t_submit;
};

struct TicketInfo {
  int32_t state;   // 0 done, 1 queued, 2 running
  int32_t status;  // bfs_status once done
};

constexpr int kMaxRoots = 64;
constexpr int kStatusSlot = kMaxRoots;  // pinned slot receiving the unit's device status word

struct Unit {  // one admitted launch: a single query or a merged wave
  std::vector<Request> reqs;
  std::vector<int32_t*> rows;     // output row of each request (caller's buffer or a pooled one)
  std::vector<int32_t*> pooled;   // pooled depth buffers this unit holds
  int32_t graph_id = 0;
  int stream_index = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  long long bytes = 0;
  bool wave = false;
  bfs::MsSet* set = nullptr;
  long long* pinned = nullptr;  // kMaxRoots reached-edge slots, then the status slot
};

// A registered graph, its launch shape and its pools.
struct GraphEntry {
  bfs_graph* g = nullptr;
  int32_t n = 0;
  int32_t single_blocks = 0;  // blocks of a single query's persistent grid
  int32_t wave_blocks = 0;    // blocks of a wave
  bool merge = false;         // the probe found waves cheaper per query
  bool waves = false;         // wave sets allocated: queued queries may merge
  int32_t singles_max = 0;    // workspaces reserved for single queries
  int32_t singles_inflight = 0;
  long long single_bytes = 0;  // one traversal workspace
  long long set_bytes = 0;     // one wave buffer set
  std::vector<int32_t*> depth_all, depth_free;
  std::vector<bfs::MsSet*> sets_all, sets_free;
};

}  // namespace

struct bfs_server {
  bfs_serve_config cfg{};
  int device = 0;
  int32_t sms = 0;
  std::vector<GraphEntry> graphs;  // reserved to kMaxGraphs: entries never move
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_units;  // units in flight per stream (dispatcher thread only)
  std::vector<cudaEvent_t> free_events;
  std::vector<long long*> free_pinned;

  std::mutex mu;
  std::condition_variable work_cv;  // dispatcher wake-up
  std::condition_variable done_cv;  // waiters
  std::list<Request> queue;
  std::unordered_map<uint64_t, TicketInfo> tickets;
  std::deque<uint64_t> done_order;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;

  // statistics (under mu)
  int64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, failed = 0, waves = 0;
  std::vector<double> latency_ms;  // submission to completion
  std::vector<double> wait_ms;     // submission to admission
  double edges_half = 0;
  bool any_submit = false;
  Clock::time_point t_first, t_last;
  long long bytes_inflight = 0, peak_bytes = 0;
};

namespace {

constexpr size_t kTicketCap = 1 << 20;
constexpr size_t kMaxGraphs = 256;
constexpr int kScanDepth = 32;  // queue entries considered per admission pass
// a query's block count may cost up to this factor in latency over the fastest
constexpr float kLatencySlack = 4.0f;
// a merged wave runs on at most this many blocks per SM, leaving room for the
// single queries around it (a full-occupancy wave could only start on an idle
// GPU and would hold all of it)
constexpr int kWaveBlocksPerSm = 2;
constexpr int32_t kSinglesPerGraph = 64;  // most workspaces reserved per graph for single queries
constexpr int32_t kWaveSetsPerGraph = 2;  // waves of one graph that can run at once

void finish_ticket(bfs_server* s, uint64_t t, int status) {
  auto it = s->tickets.find(t);
  if (it != s->tickets.end()) {
    it->second.state = 0;
    it->second.status = status;
  }
  s->done_order.push_back(t);
  while (s->done_order.size() > kTicketCap) {
    s->tickets.erase(s->done_order.front());
    s->done_order.pop_front();
  }
}

// Launch one unit (dispatcher thread, no lock held). Returns a bfs_status.
int launch_unit(bfs_server* s, Unit& u) {
  const GraphEntry& ge = s->graphs[u.graph_id];
  int32_t* status_slot = reinterpret_cast<int32_t*>(&u.pinned[kStatusSlot]);
  *status_slot = BFS_OK;
  if (!u.wave) {
    const int rc = bfs::run_async(ge.g, u.reqs[0].root, u.rows[0], u.stream, BFS_MODE_PERSISTENT, u.pinned,
                                  ge.single_blocks, status_slot);
    if (rc != BFS_OK) return rc;
  } else {
    int32_t roots[kMaxRoots];
    const int k = (int)u.reqs.size();
    for (int i = 0; i < k; ++i) roots[i] = u.reqs[i].root;
    const int rc = bfs::batch_async(ge.g, u.set, roots, k, u.rows.data(), u.stream,
                                    reinterpret_cast<unsigned long long*>(u.pinned), ge.wave_blocks, status_slot);
    if (rc != BFS_OK) return rc;
  }
  if (cudaEventRecord(u.done, u.stream) != cudaSuccess) return BFS_ERR_CUDA;
  return BFS_OK;
}

// Return a unit's resources (with s->mu held).
void release_unit(bfs_server* s, Unit& u) {
  GraphEntry& ge = s->graphs[u.graph_id];
  s->stream_units[u.stream_index] -= 1;
  for (int32_t* p : u.pooled) ge.depth_free.push_back(p);
  if (u.wave)
    ge.sets_free.push_back(u.set);
  else
    ge.singles_inflight -= 1;
  s->free_events.push_back(u.done);
  s->free_pinned.push_back(u.pinned);
  s->bytes_inflight -= u.bytes;
}

// Try to form a unit from the request at `it` (with s->mu held): a wave of up
// to merge_batch queued queries of its graph when a set is free and more than
// one can join, else a single query. False when the pools or the memory budget
// do not allow it now.
bool admit(bfs_server* s, std::list<Request>::iterator& it, bool idle, Unit* u) {
  const int gid = it->graph_id;
  GraphEntry& ge = s->graphs[gid];
  const long long n4 = 4ll * ge.n;
  // candidates for a wave: queued queries of this graph from `it` on; those
  // without an output buffer need a pooled one
  std::vector<std::list<Request>::iterator> pick;
  // a graph whose queries merge waits for a free set rather than starting a
  // single run (the next wave takes every query queued by then); with a set
  // free, a lone query runs single (lower latency than a wave of one)
  if (ge.waves && ge.sets_free.empty()) return false;
  if (ge.waves) {
    size_t bufs = 0;
    const int kmax = std::min(s->cfg.merge_batch, kMaxRoots);
    for (auto jt = it; jt != s->queue.end() && (int)pick.size() < kmax; ++jt) {
      if (jt->graph_id != gid) continue;
      if (!jt->depth_out) {
        if (bufs == ge.depth_free.size()) {
          if (jt == it) break;  // the head query itself cannot join: no wave starts here
          continue;
        }
        ++bufs;
      }
      pick.push_back(jt);
    }
    if (pick.size() < 2) pick.clear();
  }
  long long need = 0;
  if (!pick.empty()) {
    need = ge.set_bytes;
    for (auto& jt : pick)
      if (!jt->depth_out) need += n4;
  } else {
    if (ge.singles_inflight >= ge.singles_max) return false;
    if (!it->depth_out && ge.depth_free.empty()) return false;
    pick.push_back(it);
    need = ge.single_bytes + (it->depth_out ? 0 : n4);
  }
  if (s->cfg.mem_budget_bytes > 0 && s->bytes_inflight + need > s->cfg.mem_budget_bytes && !idle) return false;
  u->graph_id = gid;
  u->wave = pick.size() > 1;
  u->bytes = need;
  if (u->wave) {
    u->set = ge.sets_free.back();
    ge.sets_free.pop_back();
  } else {
    ge.singles_inflight += 1;
  }
  for (auto& jt : pick) {
    int32_t* row = jt->depth_out;
    if (!row) {
      row = ge.depth_free.back();
      ge.depth_free.pop_back();
      u->pooled.push_back(row);
    }
    u->rows.push_back(row);
    u->reqs.push_back(*jt);
  }
  // erase the picked entries (pick[0] is `it`); `it` moves to the first entry
  // after it that was not picked
  for (size_t q = pick.size(); q-- > 1;) s->queue.erase(pick[q]);
  auto next = std::next(it);
  s->queue.erase(it);
  it = next;
  return true;
}

void dispatcher(bfs_server* s) {
  cudaSetDevice(s->device);
  std::vector<Unit> inflight;
  std::vector<Unit> to_launch;
  for (;;) {
    bool progressed = false;
    // 1) completions
    for (size_t i = 0; i < inflight.size();) {
      cudaError_t e = cudaEventQuery(inflight[i].done);
      if (e == cudaErrorNotReady) {
        ++i;
        continue;
      }
      if (e != cudaSuccess) cudaGetLastError();
      const auto now = Clock::now();
      Unit u = std::move(inflight[i]);
      inflight.erase(inflight.begin() + (long)i);
      const int32_t dev_status = *reinterpret_cast<const int32_t*>(&u.pinned[kStatusSlot]);
      const int status = e != cudaSuccess ? BFS_ERR_CUDA : dev_status != BFS_OK ? BFS_ERR_TIMEOUT : BFS_OK;
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t q = 0; q < u.reqs.size(); ++q) {
        const Request& r = u.reqs[q];
        if (status == BFS_OK) {
          s->completed += 1;
          s->latency_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
          s->edges_half += (double)u.pinned[u.wave ? q : 0] / 2.0;
        } else {
          s->failed += 1;
        }
        finish_ticket(s, r.ticket, status);
      }
      s->t_last = now;
      release_unit(s, u);
      progressed = true;
    }
    if (progressed) s->done_cv.notify_all();
    // 2) admissions (first fit over the head of the queue)
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stop) {
        // shutting down: queries never admitted are cancelled; running ones finish
        for (const Request& r : s->queue) finish_ticket(s, r.ticket, BFS_ERR_CANCELLED);
        s->queue.clear();
        s->done_cv.notify_all();
        if (inflight.empty()) break;
      }
      int scanned = 0;
      for (auto it = s->queue.begin(); it != s->queue.end() && scanned < kScanDepth;) {
        if ((int)(inflight.size() + to_launch.size()) >= s->cfg.max_inflight || s->free_events.empty()) break;
        ++scanned;
        Unit u;
        const bool idle = inflight.empty() && to_launch.empty();
        if (!admit(s, it, idle, &u)) {
          ++it;  // does not fit now: try the next one (a query larger than the budget runs alone)
          continue;
        }
        u.done = s->free_events.back();
        s->free_events.pop_back();
        u.pinned = s->free_pinned.back();
        s->free_pinned.pop_back();
        u.stream_index = (int)(std::min_element(s->stream_units.begin(), s->stream_units.end()) -
                               s->stream_units.begin());
        u.stream = s->streams[u.stream_index];
        s->stream_units[u.stream_index] += 1;
        if (u.wave) s->waves += 1;
        const auto t_admit = Clock::now();
        for (const Request& r : u.reqs) {
          auto t = s->tickets.find(r.ticket);
          if (t != s->tickets.end()) t->second.state = 2;
          s->wait_ms.push_back(std::chrono::duration<double, std::milli>(t_admit - r.t_submit).count());
        }
        s->admitted += (int64_t)u.reqs.size();
        s->bytes_inflight += u.bytes;
        s->peak_bytes = std::max(s->peak_bytes, s->bytes_inflight);
        to_launch.push_back(std::move(u));
      }
      if (to_launch.empty() && !progressed) {
        if (inflight.empty())
          s->work_cv.wait_for(lk, std::chrono::milliseconds(2));
        else
          s->work_cv.wait_for(lk, std::chrono::microseconds(20));
        continue;
      }
    }
    for (Unit& u : to_launch) {
      const int rc = launch_unit(s, u);
      if (rc == BFS_OK) {
        inflight.push_back(std::move(u));
      } else {
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Request& r : u.reqs) {
          s->failed += 1;
          finish_ticket(s, r.ticket, rc);
        }
        release_unit(s, u);
        s->done_cv.notify_all();
      }
    }
    to_launch.clear();
  }
}

// Launch shape of a graph's queries, from probe runs at registration
// (synchronous, on a private stream):
//  1. traversals from up to four spread vertices (0, n/3, 2n/3, n-1); the one
//     reaching the most edges is the probe root;
//  2. that traversal timed on 8, 16, 32, 64 blocks, one and two per SM
//     and a full occupancy wave: a query gets the block count that minimises
//     blocks x time (the device share it holds) among those within
//     kLatencySlack of the fastest, so latency-bound graphs run narrow and
//     many of their queries share the GPU;
//  3. one multi-source wave from 64 vertices the probe reached, on the grid
//     waves get (at most kWaveBlocksPerSm blocks per SM): waves are cheaper
//     when their blocks x time per root is below a single query's.
struct Shape {
  int32_t single_blocks = 0;
  int32_t wave_blocks = 0;
  bool merge = false;
};

int probe_shape(bfs_server* s, bfs_graph* g, Shape* out) {
  const int32_t n = bfs::graph_vertices(g);
  const int32_t full = std::max(1, bfs::persistent_grid(g));
  out->single_blocks = std::min(full, s->sms);
  out->merge = false;
  cudaStream_t stream;
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return bfs::set_error_detail(BFS_ERR_CUDA, "probe stream");
  }
  int32_t* depth = nullptr;
  int32_t* wave_out = nullptr;
  bfs::MsSet* set = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = BFS_OK;
  if (cudaMalloc(&depth, (size_t)n * 4) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = bfs::set_error_detail(BFS_ERR_OOM, "probe buffers");
  }
  // 1. probe root
  int32_t root = 0;
  long long best_e = -1;
  const int32_t cand[4] = {0, n / 3, (int32_t)(2LL * n / 3), n - 1};
  for (int c = 0; c < 4 && rc == BFS_OK; ++c) {
    bfs_run_stats st{};
    bfs_options opt{};
    opt.forced_variant = BFS_VARIANT_TREE;
    opt.mode = BFS_MODE_PERSISTENT;
    rc = bfs_run_ex(g, cand[c], depth, stream, &opt, &st);  // with stats: synchronous
    if (rc == BFS_OK && st.edges_reached > best_e) {
      best_e = st.edges_reached;
      root = cand[c];
    }
  }
  // 2. blocks of a single query
  auto timed = [&](auto&& launch, float* ms) -> int {
    if (cudaEventRecord(e0, stream) != cudaSuccess) return BFS_ERR_CUDA;
    const int r = launch();
    if (r != BFS_OK) return r;
    if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return BFS_ERR_CUDA;
    return BFS_OK;
  };
  constexpr int kSizes = 7;
  const int32_t sizes[kSizes] = {8, 16, 32, 64, s->sms, 2 * s->sms, full};
  float t[kSizes] = {0, 0, 0, 0, 0, 0, 0};
  float fastest = 1e30f;
  for (int i = 0; i < kSizes && rc == BFS_OK; ++i) {
    bfs_options opt{};
    opt.forced_variant = BFS_VARIANT_TREE;
    opt.mode = BFS_MODE_PERSISTENT;
    opt.grid_blocks = std::min(sizes[i], full);
    rc = timed([&] { return bfs_run_ex(g, root, depth, stream, &opt, nullptr); }, &t[i]);
    fastest = std::min(fastest, t[i]);
  }
  double single_cost = 0;
  if (rc == BFS_OK) {
    double best_cost = 1e300;
    for (int i = 0; i < kSizes; ++i) {
      const int32_t b = std::min(sizes[i], full);
      const double cost = (double)b * t[i];
      if (t[i] <= kLatencySlack * fastest && cost < best_cost) {
        best_cost = cost;
        out->single_blocks = b;
      }
    }
    single_cost = best_cost;
  }
  // 3. merge or not: a 64-root wave from vertices the probe reached (temporary
  // buffers; a wave that does not fit only disables merging)
  if (rc == BFS_OK) {
    std::vector<int32_t> d((size_t)n);
    if (cudaMemcpy(d.data(), depth, (size_t)n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = BFS_ERR_CUDA;
    std::vector<int32_t> reached;
    for (int32_t v = 0; v < n && rc == BFS_OK; ++v)
      if (d[(size_t)v] >= 0) reached.push_back(v);
    const int32_t wg = std::min(bfs::wave_grid(g), kWaveBlocksPerSm * s->sms);
    out->wave_blocks = std::max(wg, 1);
    if (rc == BFS_OK && wg > 0 && !reached.empty() && cudaMalloc(&wave_out, (size_t)kMaxRoots * n * 4) == cudaSuccess &&
        bfs::ms_set_create(g, &set) == BFS_OK) {
      int32_t roots[kMaxRoots];
      int32_t* rows[kMaxRoots];
      for (int i = 0; i < kMaxRoots; ++i) {
        roots[i] = reached[(size_t)i * reached.size() / kMaxRoots];
        rows[i] = wave_out + (size_t)i * n;
      }
      float wave_ms = 0;
      rc = timed([&] { return bfs::batch_async(g, set, roots, kMaxRoots, rows, stream, nullptr, wg, nullptr); },
                 &wave_ms);
      if (rc == BFS_OK) out->merge = (double)wg * wave_ms / kMaxRoots < single_cost;
    }
    cudaGetLastError();
  }
  bfs::ms_set_free(set);
  if (wave_out) cudaFree(wave_out);
  if (depth) cudaFree(depth);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamDestroy(stream);
  return rc;
}

void free_pools(GraphEntry& ge) {
  for (int32_t* p : ge.depth_all) cudaFree(p);
  for (bfs::MsSet* set : ge.sets_all) bfs::ms_set_free(set);
  ge.depth_all.clear();
  ge.depth_free.clear();
  ge.sets_all.clear();
  ge.sets_free.clear();
}

// The pools a graph's units draw from, allocated once at registration.
int make_pools(bfs_server* s, GraphEntry& ge) {
  // as many single queries as the slots allow, up to the pool limit, and no
  // more than the memory budget could admit at once
  long long cap = std::min<int32_t>(s->cfg.max_inflight, kSinglesPerGraph);
  if (s->cfg.mem_budget_bytes > 0) cap = std::min(cap, s->cfg.mem_budget_bytes / std::max(1ll, ge.single_bytes));
  ge.singles_max = (int32_t)std::max(1ll, cap);
  ge.waves = s->cfg.merge_batch > 1 && (ge.merge || s->cfg.merge_policy == 1);
  int rc = bfs::reserve_workspaces(ge.g, ge.singles_max);
  if (rc != BFS_OK) return rc;
  const int sets = ge.waves ? kWaveSetsPerGraph : 0;
  const int bufs = ge.singles_max + sets * std::min(s->cfg.merge_batch, kMaxRoots);
  for (int i = 0; i < bufs; ++i) {
    int32_t* p = nullptr;
    if (cudaMalloc(&p, (size_t)ge.n * 4) != cudaSuccess) {
      cudaGetLastError();
      free_pools(ge);
      return bfs::set_error_detail(BFS_ERR_OOM, "depth buffer pool");
    }
    ge.depth_all.push_back(p);
  }
  for (int i = 0; i < sets; ++i) {
    bfs::MsSet* set = nullptr;
    rc = bfs::ms_set_create(ge.g, &set);
    if (rc != BFS_OK) {
      free_pools(ge);
      return rc;
    }
    ge.sets_all.push_back(set);
  }
  ge.depth_free = ge.depth_all;
  ge.sets_free = ge.sets_all;
  return BFS_OK;
}

}  // namespace

extern "C" {

int bfs_serve_create(const bfs_serve_config* cfg, bfs_server_t* out) {
  if (!cfg || !out) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  if (cfg->max_inflight < 1 || cfg->max_inflight > 1024 || cfg->num_streams < 1 || cfg->num_streams > 1024 ||
      cfg->queue_capacity < 1 || cfg->merge_batch < 0 || cfg->merge_batch > 64 || cfg->mem_budget_bytes < 0 ||
      cfg->merge_policy < 0 || cfg->merge_policy > 1 || cfg->reserved != 0)
    return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "serve config out of range");
  auto* s = new bfs_server;
  s->cfg = *cfg;
  // graphs are registered while the dispatcher runs: fixed capacity, so the
  // entries never move under it
  s->graphs.reserve(kMaxGraphs);
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
    delete s;
    return bfs::set_error_detail(BFS_ERR_CUDA, "cudaGetDevice failed");
  }
  for (int i = 0; i < cfg->num_streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) break;
    s->streams.push_back(st);
  }
  s->stream_units.assign(s->streams.size(), 0);
  for (int i = 0; i < cfg->max_inflight; ++i) {
    cudaEvent_t e;
    long long* p = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) break;
    if (cudaMallocHost(&p, (kMaxRoots + 1) * sizeof(long long)) != cudaSuccess) {
      cudaEventDestroy(e);
      break;
    }
    s->free_events.push_back(e);
    s->free_pinned.push_back(p);
  }
  if ((int)s->streams.size() != cfg->num_streams || (int)s->free_events.size() != cfg->max_inflight) {
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (long long* p : s->free_pinned) cudaFreeHost(p);
    delete s;
    cudaGetLastError();
    return bfs::set_error_detail(BFS_ERR_OOM, "could not create streams, events or pinned buffers");
  }
  s->worker = std::thread(dispatcher, s);
  *out = s;
  return BFS_OK;
}

int bfs_serve_add_graph(bfs_server_t s, bfs_graph_t g, int32_t* graph_id) {
  if (!s || !g || !graph_id) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  if (bfs::graph_device(g) != s->device)
    return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "graph lives on another device");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->graphs.size() >= kMaxGraphs) return bfs::set_error_detail(BFS_ERR_BUSY, "too many graphs (256)");
  }
  Shape shape;
  int rc = probe_shape(s, g, &shape);
  if (rc != BFS_OK) return rc;
  GraphEntry ge;
  ge.g = g;
  ge.n = bfs::graph_vertices(g);
  ge.single_blocks = shape.single_blocks;
  ge.wave_blocks = shape.wave_blocks;
  ge.merge = shape.merge;
  ge.single_bytes = bfs::workspace_bytes(g);
  ge.set_bytes = bfs::ms_set_bytes(g);
  rc = make_pools(s, ge);
  if (rc != BFS_OK) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->graphs.size() >= kMaxGraphs) {
    free_pools(ge);
    return bfs::set_error_detail(BFS_ERR_BUSY, "too many graphs (256)");
  }
  s->graphs.push_back(std::move(ge));
  *graph_id = (int32_t)s->graphs.size() - 1;
  return BFS_OK;
}

int bfs_serve_graph_shape(bfs_server_t s, int32_t graph_id, int32_t* query_blocks, int32_t* merges) {
  if (!s || !query_blocks || !merges) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size())
    return bfs::set_error_detail(BFS_ERR_NOT_FOUND, "unknown graph id");
  *query_blocks = s->graphs[graph_id].single_blocks;
  *merges = s->graphs[graph_id].merge ? 1 : 0;
  return BFS_OK;
}

int bfs_serve_query_bytes(bfs_server_t s, int32_t graph_id, int32_t with_output, int64_t* bytes) {
  if (!s || !bytes) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size())
    return bfs::set_error_detail(BFS_ERR_NOT_FOUND, "unknown graph id");
  const GraphEntry& ge = s->graphs[graph_id];
  *bytes = ge.single_bytes + (with_output ? 0 : 4ll * ge.n);
  return BFS_OK;
}

int bfs_serve_submit(bfs_server_t s, int32_t graph_id, int32_t root, int32_t* depth_out, uint64_t* ticket) {
  if (!s || !ticket) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size())
    return bfs::set_error_detail(BFS_ERR_NOT_FOUND, "unknown graph id");
  if (root < 0 || root >= s->graphs[graph_id].n)
    return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "root out of range");
  if (s->stop) return bfs::set_error_detail(BFS_ERR_CANCELLED, "server is shutting down");
  if ((int)s->queue.size() >= s->cfg.queue_capacity) {
    s->rejected += 1;
    return bfs::set_error_detail(BFS_ERR_BUSY, "submission queue full");
  }
  const auto now = Clock::now();
  if (!s->any_submit) {
    s->any_submit = true;
    s->t_first = now;
  }
  const uint64_t t = s->next_ticket++;
  s->queue.push_back(Request{t, graph_id, root, depth_out, now});
  s->tickets[t] = TicketInfo{1, BFS_OK};
  s->submitted += 1;
  *ticket = t;
  s->work_cv.notify_one();
  return BFS_OK;
}

int bfs_serve_poll(bfs_server_t s, uint64_t ticket, int* state) {
  if (!s || !state) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return bfs::set_error_detail(BFS_ERR_NOT_FOUND, "unknown ticket");
  *state = it->second.state;
  return it->second.state == 0 ? it->second.status : BFS_OK;
}

int bfs_serve_wait(bfs_server_t s, uint64_t ticket, int64_t timeout_us) {
  if (!s) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto done = [&] {
    auto it = s->tickets.find(ticket);
    return it == s->tickets.end() || it->second.state == 0;
  };
  if (timeout_us < 0)
    s->done_cv.wait(lk, done);
  else if (!s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), done))
    return bfs::set_error_detail(BFS_ERR_TIMEOUT, "query not finished within the timeout");
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end()) return bfs::set_error_detail(BFS_ERR_NOT_FOUND, "unknown ticket");
  return it->second.status;
}

int bfs_serve_stats(bfs_server_t s, bfs_serve_stats_t* out) {
  if (!s || !out) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof *out);
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->failed = s->failed;
  out->merged_waves = (int32_t)s->waves;
  out->peak_bytes_inflight = s->peak_bytes;
  out->queued = (int32_t)s->queue.size();
  auto pct = [](std::vector<double> v, double p) {  // nearest rank
    const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + (long)i, v.end());
    return v[i];
  };
  if (!s->wait_ms.empty()) {
    out->wait_p50_ms = pct(s->wait_ms, 0.50);
    out->wait_p99_ms = pct(s->wait_ms, 0.99);
  }
  if (!s->latency_ms.empty()) {
    out->p50_ms = pct(s->latency_ms, 0.50);
    out->p99_ms = pct(s->latency_ms, 0.99);
    out->max_ms = *std::max_element(s->latency_ms.begin(), s->latency_ms.end());
    const double wall = std::chrono::duration<double>(s->t_last - s->t_first).count();
    if (wall > 0) {
      out->qps = (double)s->completed / wall;
      out->gteps = s->edges_half / wall / 1e9;
    }
  }
  return BFS_OK;
}

int bfs_serve_reset_stats(bfs_server_t s) {
  if (!s) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->submitted = s->admitted = s->completed = s->rejected = s->failed = s->waves = 0;
  s->latency_ms.clear();
  s->wait_ms.clear();
  s->edges_half = 0;
  s->any_submit = false;
  s->peak_bytes = s->bytes_inflight;
  return BFS_OK;
}

int bfs_serve_cancel_queued(bfs_server_t s, int64_t* cancelled) {
  if (!s) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t k = (int64_t)s->queue.size();
  for (const Request& r : s->queue) finish_ticket(s, r.ticket, BFS_ERR_CANCELLED);
  s->queue.clear();
  if (cancelled) *cancelled = k;
  s->done_cv.notify_all();
  return BFS_OK;
}

int bfs_serve_destroy(bfs_server_t s) {
  if (!s) return BFS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->work_cv.notify_all();
  if (s->worker.joinable()) s->worker.join();  // drains the queue and every unit in flight
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
  for (long long* p : s->free_pinned) cudaFreeHost(p);
  for (GraphEntry& ge : s->graphs) free_pools(ge);
  delete s;
  return BFS_OK;
}

}  // extern "C"
