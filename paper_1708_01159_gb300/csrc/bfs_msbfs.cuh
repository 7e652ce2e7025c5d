// Multi-source BFS (64 roots per wave, one bit per root in 64-bit masks).
#pragma once

#include "bfs_internal.cuh"

namespace bfs {

constexpr int kMsThreads = 256;

struct MsBuffers {
  unsigned long long* visit;     // n masks: bit i = reached by root i
  unsigned long long* front[2];  // n masks each: bit i = in root i's frontier (nonzero only on frontier vertices)
  unsigned long long* next;      // n masks: bits pushed to the vertex during a push level (zero between levels)
  int32_t* flist[2];             // frontier vertex lists (any lane), for level L in flist[L & 1]
  int32_t* tlist;                // vertices whose next mask became nonzero during a push level
  const int32_t* roots;          // device copy of the wave's roots
};

struct MsState {
  unsigned int bar_count;
  unsigned int bar_gen;
  int32_t status;
  int32_t levels;
  unsigned int ftail[4];           // frontier list length (= frontier vertices) of level L in slot L % 4
  unsigned int ttail[2];           // touched list length of a push level L in slot L % 2
  unsigned long long fedges[4];    // out-degree sum of level L's frontier, slot L % 4
  unsigned long long edges[64];    // reached-edge count per root
};

struct MsConfig {
  int32_t push_mode;  // 0: thread per frontier vertex, 1: warp per frontier vertex
  int32_t alpha;      // a level pulls when its frontier edges x alpha exceed m
};

// stall: STALL_GRID_BARRIER makes the first grid barrier wait for an arrival
// that never comes (test hook); STALL_NONE otherwise.
__global__ void k_msbfs(DevGraph g, MsBuffers mb, MsState* st, int32_t k, int32_t* depth, MsConfig cfg,
                        int32_t stall);
__global__ void k_ms_reset(MsState* st);

}  // namespace bfs
