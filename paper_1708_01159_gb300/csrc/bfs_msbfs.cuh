// Multi-source BFS (64 roots per wave, one bit per root in 64-bit masks).
#pragma once

#include "bfs_internal.cuh"

namespace bfs {

constexpr int kMsThreads = 256;
constexpr int kMsMaxRoots = 64;
// Depths up to this value are kept as 4-bit codes (code d + 1) until the wave
// ends; deeper ones (code 15) are written to the output when found.
constexpr int32_t kMsCodeMaxDepth = 13;

// One wave's device buffers (a set): every traversal state the kernel keeps.
struct MsBuffers {
  unsigned long long* visit;     // n masks: bit i = reached by root i
  unsigned long long* front[2];  // n masks each: bit i = in root i's frontier (nonzero only on frontier vertices)
  unsigned long long* next;      // n masks: bits pushed to the vertex during a push level (zero between levels)
  unsigned long long* codes;     // 4 n words: vertex u's 64 nibbles in codes[4u .. 4u + 3], nibble i for root i
  int32_t* flist[2];             // frontier vertex lists (any lane), for level L in flist[L & 1]
  int32_t* tlist;                // vertices whose next mask became nonzero during a push level
};

// Bytes of one set for n vertices (visit, two frontiers, next, codes, three lists).
constexpr long long ms_set_bytes_per_vertex() { return 8 + 16 + 8 + 32 + 12; }

struct MsState {
  unsigned long long bar64;        // monotonic arrival count of the grid barriers (reset before each wave)
  int32_t status;
  int32_t levels;
  unsigned int ftail[4];           // frontier list length (= frontier vertices) of level L in slot L % 4
  unsigned int ttail[2];           // touched list length of a push level L in slot L % 2
  unsigned long long fedges[4];    // out-degree sum of level L's frontier, slot L % 4
  unsigned long long edges[kMsMaxRoots];  // reached-edge count per root
};

struct MsConfig {
  int32_t push_mode;  // 0: thread per frontier vertex, 1: warp per frontier vertex
  int32_t alpha;      // a level pulls when its frontier edges x alpha exceed m
};

// The wave's roots and output rows, passed by value as a kernel parameter
// (no upload): root i's depths go to row[i][0 .. n).
struct MsRows {
  int32_t* row[kMsMaxRoots];
  int32_t root[kMsMaxRoots];
};

// stall: STALL_GRID_BARRIER makes the first grid barrier wait for an arrival
// that never comes (test hook); STALL_NONE otherwise.
__global__ void k_msbfs(DevGraph g, MsBuffers mb, MsState* st, int32_t k, MsRows rows, MsConfig cfg,
                        int32_t stall);
__global__ void k_ms_reset(MsState* st);

}  // namespace bfs
