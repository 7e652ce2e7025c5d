// Multi-source BFS (64 roots per wave, one bit per root in 64-bit masks).
#pragma once

#include "bfs_internal.cuh"

namespace bfs {

constexpr int kMsThreads = 256;
constexpr int kMsMaxRoots = 64;
// Depths below this value are recorded in the per-level history (one mask per
// vertex and depth) until the wave ends; deeper ones are written to the output
// when found.
constexpr int32_t kMsHistLevels = 15;

// One wave's device buffers (a set): every traversal state the kernel keeps.
struct MsBuffers {
  unsigned long long* visit;     // n masks: bit i = reached by root i
  unsigned long long* hist;      // kMsHistLevels x n masks: hist[d n + u] bit i = root i reached u at depth d
                                 // (written once per vertex and depth, read by the final pass; zero between waves)
  unsigned long long* front[2];  // n masks each: bit i = in root i's frontier, level L's in front[L & 1]
  unsigned long long* next;      // n masks: bits pushed to the vertex during a push level (zero between levels)
  int32_t* flist[2];             // frontier vertex lists (any lane), for level L in flist[L & 1]
  int32_t* tlist;                // vertices whose next mask became nonzero during a push level
};

// Bytes of one set for n vertices (visit, history, two frontiers, next, three lists).
constexpr long long ms_set_bytes_per_vertex() { return 8 + 8 * kMsHistLevels + 16 + 8 + 12; }

struct MsState {
  unsigned long long bar64;        // monotonic arrival count of the grid barriers (reset before each wave)
  int32_t status;
  int32_t levels;
  unsigned int ftail[4];           // frontier list length (= frontier vertices) of level L in slot L % 4
  unsigned int ttail[2];           // touched list length of a push level L in slot L % 2
  unsigned long long fedges[4];    // out-degree sum of level L's frontier, slot L % 4
  unsigned long long edges[kMsMaxRoots];  // reached-edge count per root
  // Between waves the history arrays are all zero when clean_blocks ==
  // clean_grid: every block of the last wave cleared what the wave set (the
  // counts are not reset by k_ms_reset; a new set is zeroed when it is
  // allocated).
  unsigned int clean_blocks;
  unsigned int clean_grid;
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
