// bfs_run_static: a single-source BFS that allocates no memory.
//
// Some callers cannot allocate device memory while they run: code inside a
// memory-pool arena they do not own, a plugin handed fixed buffers by its host
// application, or a real-time loop where a cudaMalloc (which may synchronise
// the device or fail under fragmentation) is not allowed. For them this file
// keeps the traversal's scratch (two frontier queues, the visited bitmap and
// the level counters) in one file-scope device array of fixed size, and the
// entry point calls no allocating routine at all; the caller passes the graph
// and the output in device memory it already owns.
//
// The level kernel is the one-thread-per-frontier-vertex push of the main
// library, reading its queues and counters from that array. The level loop is
// driven from the host, one small device-to-host read of the next frontier
// size per level.
#include <cstdio>

#include "bfs.h"
#include "bfs_internal.cuh"

namespace {

constexpr int64_t kStaticMaxVertices = 1 << 20;  // 1,048,576 vertices
constexpr int64_t kStaticWords = kStaticMaxVertices / 32;
constexpr int kStaticThreads = 256;

// Layout: queue 0 | queue 1 | visited bitmap | 4 counters (3 used) | error flag
struct StaticScratch {
  int32_t q[2][kStaticMaxVertices];
  uint32_t vis[kStaticWords];
  unsigned int count[4];
  int32_t bad;
  int32_t pad[3];
};

// Held by every GPU that loads the library, until the process exits (about 8.1 MB).
static __device__ __align__(256) StaticScratch g_static_scratch;

// Resets the scratch this call reads before writing (the array keeps the
// previous call's contents) and starts the traversal at `root`.
__global__ void k_static_init(StaticScratch* s, int32_t n, int32_t root, int32_t* depth) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) depth[i] = (i == root) ? 0 : -1;
  const int64_t words = (n + 31) / 32;
  for (int64_t w = tid; w < words; w += stride) s->vis[w] = (w == (root >> 5)) ? (1u << (root & 31)) : 0u;
  if (tid == 0) {
    s->q[0][0] = root;
    s->count[0] = 1;
    s->count[1] = 0;
    s->count[2] = 0;
  }
}

// CSR well-formedness, so a malformed graph is refused instead of read out of bounds.
__global__ void k_static_validate(StaticScratch* s, const int32_t* off, const int32_t* idx, int32_t n, int32_t m) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int32_t my = 0;
  if (tid == 0 && (off[0] != 0 || off[n] != m)) my = 1;
  for (int64_t v = tid; v < n; v += stride)
    if (off[v + 1] < off[v]) my = 1;
  for (int64_t e = tid; e < m; e += stride)
    if (idx[e] < 0 || idx[e] >= n) my = 1;
  if (my) atomicOr(&s->bad, 1);
}

__global__ void k_static_clear_flag(StaticScratch* s) { s->bad = 0; }

// Level L: frontier in q[L & 1] with size count[L % 3]; new vertices go to
// q[(L + 1) & 1] and count[(L + 1) % 3]. count[(L + 2) % 3] was last read by
// level L - 1, which has finished, so it is cleared here for level L + 1.
__global__ void __launch_bounds__(kStaticThreads)
    k_static_level(StaticScratch* s, const int32_t* off, const int32_t* idx, int32_t* depth, int32_t L) {
  const int32_t f = (int32_t)s->count[L % 3];
  const int32_t* qin = s->q[L & 1];
  int32_t* qout = s->q[(L + 1) & 1];
  unsigned int* tail = &s->count[(L + 1) % 3];
  if (blockIdx.x == 0 && threadIdx.x == 0) s->count[(L + 2) % 3] = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < f; i += stride) {
    const int32_t u = qin[i];
    for (int32_t e = off[u]; e < off[u + 1]; ++e) {
      const int32_t v = idx[e];
      if (bfs::claim(s->vis, v)) {
        depth[v] = L + 1;
        bfs::queue_append(qout, tail, v);
      }
    }
  }
}

int static_fail(int code, const char* msg) { return bfs::set_error_detail(code, msg); }

// A launch that could not start (a stream of another device, say) reports its
// CUDA error string instead of surfacing later as a failed copy.
int launch_status(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return BFS_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s launch: %s", what, cudaGetErrorString(e));
  return static_fail(BFS_ERR_CUDA, buf);
}

}  // namespace

#define TRY_LAUNCH(what)                     \
  do {                                       \
    const int r_ = launch_status(what);      \
    if (r_ != BFS_OK) return r_;             \
  } while (0)

extern "C" {

int bfs_run_static(const int32_t* row_offsets, const int32_t* col_indices, int64_t n, int64_t m, int32_t root,
                   int32_t* depth_out, bfs_stream_t stream_) {
  if (!row_offsets || !depth_out || (m > 0 && !col_indices))
    return static_fail(BFS_ERR_INVALID_ARG, "null pointer argument");
  if (n < 1 || n > kStaticMaxVertices)
    return static_fail(BFS_ERR_INVALID_ARG, "n must be in [1, 1048576] for bfs_run_static (fixed scratch size)");
  if (m < 0 || m >= INT32_MAX) return static_fail(BFS_ERR_INVALID_ARG, "m out of range");
  if (root < 0 || root >= n) return static_fail(BFS_ERR_INVALID_ARG, "root not in [0, n)");
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return static_fail(BFS_ERR_CUDA, "cudaGetDevice failed");
  if (stream) {
    int sdev = -1;
    if (cudaStreamGetDevice(stream, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return static_fail(BFS_ERR_INVALID_ARG, "stream is not a valid CUDA stream");
    }
    if (sdev != dev) return static_fail(BFS_ERR_INVALID_ARG, "stream belongs to another device than the current one");
  }
  // The array's device address in the current device's context, looked up on
  // every call (the lookup allocates nothing), so a device reset between calls
  // never leaves a stale address behind; in host code the array's name is only
  // a host-side stand-in and must not be passed to a kernel.
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return static_fail(BFS_ERR_CUDA, "cudaGetSymbolAddress failed");
  }
  StaticScratch* s = static_cast<StaticScratch*>(p);
  const int32_t nn = (int32_t)n, mm = (int32_t)m;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  const int grid = sms * 4;
  k_static_clear_flag<<<1, 1, 0, stream>>>(s);
  TRY_LAUNCH("clear");
  k_static_validate<<<grid, kStaticThreads, 0, stream>>>(s, row_offsets, col_indices, nn, mm);
  TRY_LAUNCH("validate");
  int32_t bad = 0;
  if (cudaMemcpyAsync(&bad, &s->bad, sizeof bad, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return static_fail(BFS_ERR_CUDA, "validation failed to run");
  if (bad) return static_fail(BFS_ERR_BAD_GRAPH, "CSR failed validation");
  k_static_init<<<grid, kStaticThreads, 0, stream>>>(s, nn, root, depth_out);
  TRY_LAUNCH("init");
  for (int32_t L = 0; L <= nn; ++L) {
    k_static_level<<<grid, kStaticThreads, 0, stream>>>(s, row_offsets, col_indices, depth_out, L);
    TRY_LAUNCH("level");
    unsigned int next = 0;
    if (cudaMemcpyAsync(&next, &s->count[(L + 1) % 3], sizeof next, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return static_fail(BFS_ERR_CUDA, "level launch failed");
    if (next == 0) return BFS_OK;
  }
  return static_fail(BFS_ERR_TIMEOUT, "more levels than vertices");
}

}  // extern "C"
