// bfs_serve: a continuous-batching BFS server over graphs resident in HBM.
//
// A dispatcher thread owns the device side. Submissions enter a FIFO queue;
// whenever an in-flight slot and the memory a query needs (its traversal
// workspace, plus a depth buffer when the caller gives none) fit the budget,
// the dispatcher admits it, first fit over the head of the queue, so a large
// query waiting for memory does not block smaller ones behind it. Admitted
// queries run on a pool of streams and overlap on the device; queued queries to
// the same graph are merged into one multi-source wave (up to merge_batch
// roots, one bit each in 64-bit masks). Completion is observed by polling a
// CUDA event per admitted unit; latency runs from submission to that
// observation. Single queries use the persistent driver on one block per SM
// (a quarter of a full cooperative grid), so up to four traversals are
// resident together; a full grid each would serialise them.
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

struct Unit {  // one admitted launch: a single query or a merged wave
  std::vector<Request> reqs;
  int32_t graph_id = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  long long bytes = 0;
  int32_t* scratch = nullptr;  // server-owned depth buffer (single) or wave staging (k x n)
  bool wave = false;
  long long* edges = nullptr;  // pinned: 64 slots
};

}  // namespace

struct bfs_server {
  bfs_serve_config cfg{};
  int device = 0;
  int32_t query_blocks = 0;  // blocks of one single-query persistent traversal (one per SM)
  std::vector<bfs_graph*> graphs;
  std::vector<cudaStream_t> streams;
  size_t next_stream = 0;
  std::vector<cudaEvent_t> free_events;
  std::vector<long long*> free_pinned;
  // per graph: free single-query depth buffers, and one wave staging buffer
  std::vector<std::vector<int32_t*>> free_depth;
  std::vector<int32_t*> wave_staging;
  std::vector<char> wave_busy;

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
  std::vector<double> latency_ms;
  double edges_half = 0;
  bool any_submit = false;
  Clock::time_point t_first, t_last;
  long long bytes_inflight = 0, peak_bytes = 0;
};

namespace {

constexpr size_t kTicketCap = 1 << 20;
constexpr size_t kMaxGraphs = 256;
constexpr int kScanDepth = 32;  // queue entries considered per admission pass

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

long long unit_bytes(bfs_server* s, const Request& r, int k) {
  bfs_graph* g = s->graphs[r.graph_id];
  const long long n = bfs::graph_vertices(g);
  if (k > 1) return 4 * n * k;  // wave staging (the mask buffers stay with the graph)
  return bfs::workspace_bytes(g) + (r.depth_out ? 0 : 4 * n);
}

// Launch one unit (dispatcher thread, no lock held). Returns a bfs_status.
int launch_unit(bfs_server* s, Unit& u) {
  bfs_graph* g = s->graphs[u.graph_id];
  const int64_t n = bfs::graph_vertices(g);
  if (!u.wave) {
    Request& r = u.reqs[0];
    int32_t* out = r.depth_out;
    if (!out) {
      auto& pool = s->free_depth[u.graph_id];
      if (!pool.empty()) {
        out = pool.back();
        pool.pop_back();
      } else if (cudaMalloc(&out, (size_t)n * 4) != cudaSuccess) {
        cudaGetLastError();
        return BFS_ERR_OOM;
      }
      u.scratch = out;
    }
    int rc = bfs::run_async(g, r.root, out, u.stream, BFS_MODE_PERSISTENT, u.edges, s->query_blocks);
    if (rc != BFS_OK) return rc;
  } else {
    int32_t roots[64];
    const int k = (int)u.reqs.size();
    for (int i = 0; i < k; ++i) roots[i] = u.reqs[i].root;
    int32_t* stage = s->wave_staging[u.graph_id];
    if (!stage) {
      if (cudaMalloc(&stage, (size_t)64 * n * 4) != cudaSuccess) {
        cudaGetLastError();
        return BFS_ERR_OOM;
      }
      s->wave_staging[u.graph_id] = stage;
    }
    u.scratch = stage;
    int rc = bfs::batch_async(g, roots, k, stage, u.stream, reinterpret_cast<unsigned long long*>(u.edges));
    if (rc != BFS_OK) return rc;
    for (int i = 0; i < k; ++i)
      if (u.reqs[i].depth_out &&
          cudaMemcpyAsync(u.reqs[i].depth_out, stage + (size_t)i * n, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                          u.stream) != cudaSuccess)
        return BFS_ERR_CUDA;
  }
  if (cudaEventRecord(u.done, u.stream) != cudaSuccess) return BFS_ERR_CUDA;
  return BFS_OK;
}

void release_unit(bfs_server* s, Unit& u) {
  if (!u.wave && u.scratch) s->free_depth[u.graph_id].push_back(u.scratch);
  if (u.wave) s->wave_busy[u.graph_id] = 0;
  s->free_events.push_back(u.done);
  s->free_pinned.push_back(u.edges);
  s->bytes_inflight -= u.bytes;
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
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t q = 0; q < u.reqs.size(); ++q) {
        const Request& r = u.reqs[q];
        if (e == cudaSuccess) {
          s->completed += 1;
          s->latency_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
          s->edges_half += (double)u.edges[u.wave ? q : 0] / 2.0;
          finish_ticket(s, r.ticket, BFS_OK);
        } else {
          s->failed += 1;
          finish_ticket(s, r.ticket, BFS_ERR_CUDA);
        }
      }
      s->t_last = now;
      release_unit(s, u);
      progressed = true;
    }
    if (progressed) s->done_cv.notify_all();
    // 2) admissions (first fit over the head of the queue; same-graph merging)
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
        const int gid = it->graph_id;
        int k = 1;
        if (s->cfg.merge_batch > 1 && !s->wave_busy[gid]) {
          for (auto jt = std::next(it); jt != s->queue.end() && k < s->cfg.merge_batch; ++jt)
            if (jt->graph_id == gid) ++k;
        }
        const long long need = unit_bytes(s, *it, k);
        const bool idle = inflight.empty() && to_launch.empty();
        if (s->cfg.mem_budget_bytes > 0 && s->bytes_inflight + need > s->cfg.mem_budget_bytes && !idle) {
          ++it;  // does not fit now: try the next one (a query larger than the budget runs alone)
          continue;
        }
        Unit u;
        u.graph_id = gid;
        u.wave = k > 1;
        u.bytes = need;
        u.done = s->free_events.back();
        s->free_events.pop_back();
        u.edges = s->free_pinned.back();
        s->free_pinned.pop_back();
        u.stream = s->streams[s->next_stream++ % s->streams.size()];
        u.reqs.push_back(*it);
        it = s->queue.erase(it);  // list: erasing leaves the other iterators valid
        if (u.wave) {
          auto jt = it;
          while (jt != s->queue.end() && (int)u.reqs.size() < k) {
            if (jt->graph_id == gid) {
              u.reqs.push_back(*jt);
              const bool was_it = jt == it;
              jt = s->queue.erase(jt);
              if (was_it) it = jt;
            } else {
              ++jt;
            }
          }
          s->wave_busy[gid] = 1;
          s->waves += 1;
        }
        for (const Request& r : u.reqs) {
          auto t = s->tickets.find(r.ticket);
          if (t != s->tickets.end()) t->second.state = 2;
        }
        s->admitted += (int64_t)u.reqs.size();
        s->bytes_inflight += need;
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

}  // namespace

extern "C" {

int bfs_serve_create(const bfs_serve_config* cfg, bfs_server_t* out) {
  if (!cfg || !out) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  if (cfg->max_inflight < 1 || cfg->max_inflight > 1024 || cfg->num_streams < 1 || cfg->num_streams > 64 ||
      cfg->queue_capacity < 1 || cfg->merge_batch < 0 || cfg->merge_batch > 64 || cfg->mem_budget_bytes < 0)
    return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "serve config out of range");
  auto* s = new bfs_server;
  s->cfg = *cfg;
  // graphs are registered while the dispatcher runs: fixed capacity, so these
  // vectors never reallocate under it
  s->graphs.reserve(kMaxGraphs);
  s->free_depth.reserve(kMaxGraphs);
  s->wave_staging.reserve(kMaxGraphs);
  s->wave_busy.reserve(kMaxGraphs);
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->query_blocks, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
    delete s;
    return bfs::set_error_detail(BFS_ERR_CUDA, "cudaGetDevice failed");
  }
  for (int i = 0; i < cfg->num_streams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) break;
    s->streams.push_back(st);
  }
  for (int i = 0; i < cfg->max_inflight; ++i) {
    cudaEvent_t e;
    long long* p = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) break;
    if (cudaMallocHost(&p, 64 * sizeof(long long)) != cudaSuccess) {
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
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->graphs.size() >= kMaxGraphs) return bfs::set_error_detail(BFS_ERR_BUSY, "too many graphs (256)");
  s->graphs.push_back(g);
  s->free_depth.emplace_back();
  s->wave_staging.push_back(nullptr);
  s->wave_busy.push_back(0);
  *graph_id = (int32_t)s->graphs.size() - 1;
  return BFS_OK;
}

int bfs_serve_submit(bfs_server_t s, int32_t graph_id, int32_t root, int32_t* depth_out, uint64_t* ticket) {
  if (!s || !ticket) return bfs::set_error_detail(BFS_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size())
    return bfs::set_error_detail(BFS_ERR_NOT_FOUND, "unknown graph id");
  if (root < 0 || root >= bfs::graph_vertices(s->graphs[graph_id]))
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
  if (!s->latency_ms.empty()) {
    std::vector<double> v = s->latency_ms;
    auto pct = [&](double p) {
      const size_t i = std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5));
      std::nth_element(v.begin(), v.begin() + (long)i, v.end());
      return v[i];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = *std::max_element(v.begin(), v.end());
    const double wall = std::chrono::duration<double>(s->t_last - s->t_first).count();
    if (wall > 0) {
      out->qps = (double)s->completed / wall;
      out->gteps = s->edges_half / wall / 1e9;
    }
  }
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
  for (auto& pool : s->free_depth)
    for (int32_t* p : pool) cudaFree(p);
  for (int32_t* p : s->wave_staging)
    if (p) cudaFree(p);
  delete s;
  return BFS_OK;
}

}  // extern "C"
