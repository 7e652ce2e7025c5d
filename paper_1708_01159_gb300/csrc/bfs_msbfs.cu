// Multi-source BFS: up to 64 traversals of one graph in one persistent kernel.
//
// Each vertex carries three 64-bit masks: visit (bit i: reached by root i),
// frontier (bit i: at depth L for root i) and next (bits pushed to it during
// the level). Every level runs one direction for all roots at once:
//   push: the vertices of the frontier list OR their frontier mask, minus the
//         target's visited bits, into each neighbour's next mask (atomicOr);
//         a target whose next mask leaves zero joins a touched list, and a
//         commit pass over that list turns next into the new frontier;
//   pull: every vertex still unvisited in some lane ORs its in-neighbours'
//         frontier masks, stopping once every unvisited lane is found.
// Push and commit touch only the frontier and its neighbours (so thousands of
// small levels stay cheap); pull sweeps every vertex, a warp per 32
// consecutive vertices. The result equals k independent single-source
// traversals (each lane is one level-synchronous BFS from its root, Section
// 3.1).
//
// Output. A depth found at a level is not written to the k x n output then:
// each output sector holds 8 vertices of one root, which would be filled piece
// by piece over several levels (and, being far larger than L2, read back and
// merged each time). Instead the frontier masks of depths below kMsHistLevels
// are kept, one n-mask array per depth (the history: hist[d][u] holds the
// roots that reached u at depth d, disjoint over d), and a final pass builds
// every vertex's depths from its history masks and writes every output sector
// once, -1 included. Depths of kMsHistLevels and beyond (high-diameter graphs)
// are written when found; the final pass leaves an entry whose root reached
// the vertex but whose history holds no depth.
//
// The traversal's own frontier masks alternate between front[0] and front[1]
// (zeroed with visit and next when a wave starts, so they stay in L2); the
// history is written beside them, one plain store per vertex and depth it is
// reached at, and read only by the final pass, which zeroes what it read, so
// that the history arrays are zero whenever a wave starts (a wave that did
// not finish leaves the next one to zero them all).
//
// Level L uses frontier slot L % 4 (ftail, fedges), appends to (L + 1) % 4 and
// clears (L + 2) % 4, which every block finished reading two levels ago; the
// previous level's list (slot (L + 3) % 4) names the masks of front[(L+1) & 1]
// to clear before that array receives the new frontier.
#include "bfs_msbfs.cuh"

namespace bfs {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int32_t kMsBlockDegree = 128;  // push_mode 0: degree from which the block expands a vertex together

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(kFullMask, x, o);
  return x;
}

// Bit k of x (k < 16) moved to bit 4k, through a table of the 256 byte
// spreads (lut[x]: bit k of x at bit 4k of a 32-bit word).
__device__ __forceinline__ unsigned long long nibble_spread16(const uint32_t* lut, unsigned long long x) {
  return (unsigned long long)lut[x & 255ull] | ((unsigned long long)lut[(x >> 8) & 255ull] << 32);
}

// Vertex u was reached at depth d by the roots in nb: the history keeps the
// depths below kMsHistLevels; deeper ones are written to their rows now.
__device__ __forceinline__ void ms_record(const MsBuffers& mb, const MsRows& rows, int64_t n, int64_t u,
                                          unsigned long long nb, int32_t d) {
  if (d < kMsHistLevels) {
    mb.hist[(size_t)d * (size_t)n + (size_t)u] = nb;
  } else {
    for (unsigned long long m = nb; m; m &= m - 1) rows.row[__ffsll((long long)m) - 1][u] = d;
  }
}

}  // namespace

__global__ void __launch_bounds__(kMsThreads) k_msbfs(DevGraph g, MsBuffers mb, MsState* st, int32_t k,
                                                       MsRows rows, MsConfig cfg, int32_t stall) {
  __shared__ unsigned long long s_edges[64];
  __shared__ uint32_t s_spread[256];
  __shared__ int32_t s_big[kMsThreads];
  __shared__ int s_nbig;
  BFS_DECLARE_STAGE(stage);
  const int64_t n = g.n;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned long long act = k >= 64 ? ~0ull : ((1ull << k) - 1ull);
  const uint32_t lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  constexpr int kWarps = kMsThreads / 32;
  for (int i = threadIdx.x; i < 64; i += blockDim.x) s_edges[i] = 0;
  for (int x = threadIdx.x; x < 256; x += blockDim.x) {
    uint32_t y = 0;
    for (int b = 0; b < 8; ++b) y |= ((uint32_t)(x >> b) & 1u) << (4 * b);
    s_spread[x] = y;
  }
  // init: visit, frontier and next masks cleared; the history is zero unless
  // the last wave on this set did not finish (then it is zeroed here); the
  // output rows are written once, at the end. Every block reads the counts
  // before the first barrier, block 0 resets them after it.
  const bool hist_dirty = *reinterpret_cast<volatile unsigned int*>(&st->clean_blocks) !=
                          *reinterpret_cast<volatile unsigned int*>(&st->clean_grid);
  for (int64_t v = tid; v < n; v += stride) {
    mb.visit[v] = 0;
    mb.front[0][v] = 0;
    mb.front[1][v] = 0;
    mb.next[v] = 0;
    if (hist_dirty)
      for (int d = 0; d < kMsHistLevels; ++d) mb.hist[(size_t)d * (size_t)n + (size_t)v] = 0;
  }
  unsigned long long bar_target = 0;  // this block's copy of the barriers' arrival target
  if (!grid_arrive_wait(&st->bar64, bar_target, &st->status, stall == STALL_GRID_BARRIER ? 1u : 0u)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->clean_blocks = 0;
    st->clean_grid = gridDim.x;
    // roots: the level 0 frontier; a vertex repeated as several roots carries several bits
    unsigned int fc = 0;
    unsigned long long fe = 0;
    for (int i = 0; i < k; ++i) {
      const int32_t r = rows.root[i];
      if (mb.visit[r] == 0) {
        mb.flist[0][fc++] = r;
        fe += (unsigned long long)(g.off[r + 1] - g.off[r]);
      }
      mb.visit[r] |= 1ull << i;
      mb.front[0][r] |= 1ull << i;
      mb.hist[r] |= 1ull << i;  // depth 0
    }
    for (int i = 0; i < 64; ++i) st->edges[i] = 0;
    for (int s = 0; s < 4; ++s) {
      st->ftail[s] = 0;
      st->fedges[s] = 0;
    }
    st->ftail[0] = fc;
    st->fedges[0] = fe;
    st->ttail[0] = st->ttail[1] = 0;
  }
  bool ok = grid_arrive_wait(&st->bar64, bar_target, &st->status);
  const int64_t words = (n + 31) / 32;
  int32_t L = 0;
  for (; ok; ++L) {
    const unsigned int f = *reinterpret_cast<volatile unsigned int*>(&st->ftail[L % 4]);
    const unsigned int pf = *reinterpret_cast<volatile unsigned int*>(&st->ftail[(L + 3) % 4]);
    const unsigned long long fe = *reinterpret_cast<volatile unsigned long long*>(&st->fedges[L % 4]);
    if (f == 0) break;
    if (L > g.n) {
      if (blockIdx.x == 0 && threadIdx.x == 0) st->status = ST_TIMEOUT;
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->ftail[(L + 2) % 4] = 0;
      st->fedges[(L + 2) % 4] = 0;
      st->ttail[(L + 1) % 2] = 0;
    }
    const unsigned long long* cur = (L & 1) ? mb.front[1] : mb.front[0];
    unsigned long long* nxt = (L & 1) ? mb.front[0] : mb.front[1];
    const int32_t* list = (L & 1) ? mb.flist[1] : mb.flist[0];
    int32_t* out_list = (L & 1) ? mb.flist[0] : mb.flist[1];  // holds level L-1's list until the commit
    unsigned int* out_tail = &st->ftail[(L + 1) % 4];
    unsigned long long my_fe = 0;
    // direction: pull once the frontier's edges exceed m / alpha (Beamer's rule, alpha tuned)
    const bool pull = fe * (unsigned long long)cfg.alpha > (unsigned long long)g.m;
    if (!pull) {
      // nxt still holds level L-1's frontier: clear exactly those masks
      for (int64_t i = tid; i < (int64_t)pf; i += stride) nxt[out_list[i]] = 0;
      unsigned int* ttail = &st->ttail[L % 2];
      if (cfg.push_mode == 0) {
        // a thread per frontier vertex; vertices of degree >= kMsBlockDegree are
        // set aside in shared memory and expanded by the whole block, one after
        // another, so a hub never serialises on one thread
        for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < f; base += stride) {
          if (threadIdx.x == 0) s_nbig = 0;
          __syncthreads();
          const int64_t i = base + threadIdx.x;
          if (i < f) {
            const int32_t v = list[i];
            const int32_t beg = g.off[v], end = g.off[v + 1];
            if (end - beg >= kMsBlockDegree) {
              s_big[atomicAdd(&s_nbig, 1)] = v;
            } else {
              const unsigned long long fv = cur[v];
              // four edges per step: their adjacency entries, then their
              // targets' visit masks, then the pushes, each group issued
              // together rather than one edge's chain after another
              for (int32_t e = beg; e < end; e += 4) {
                const int nv = min(4, end - e);
                int32_t u[4];
                unsigned long long vis[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) u[q] = q < nv ? g.idx[e + q] : 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) vis[q] = q < nv ? mb.visit[u[q]] : ~0ull;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  const unsigned long long nb = fv & ~vis[q];
                  if (nb && atomicOr(&mb.next[u[q]], nb) == 0ull) stage_put(stage, mb.tlist, ttail, u[q]);
                }
              }
            }
          }
          __syncthreads();
          const int nbig = s_nbig;
          for (int b = 0; b < nbig; ++b) {
            const int32_t v = s_big[b];
            const unsigned long long fv = cur[v];
            const int32_t end = g.off[v + 1];
            for (int32_t e = g.off[v] + (int32_t)threadIdx.x; e < end; e += (int32_t)blockDim.x) {
              const int32_t u = g.idx[e];
              const unsigned long long nb = fv & ~mb.visit[u];
              if (nb && atomicOr(&mb.next[u], nb) == 0ull) stage_put(stage, mb.tlist, ttail, u);
            }
            if ((b & 7) == 7) stage_drain(stage, mb.tlist, ttail, kStageCap / 2);
          }
          stage_drain(stage, mb.tlist, ttail, kStageCap / 2);
        }
      } else {
        for (int64_t base = (int64_t)blockIdx.x * kWarps; base < f; base += (int64_t)gridDim.x * kWarps) {
          const int64_t i = base + wib;
          if (i < f) {
            const int32_t v = list[i];
            const unsigned long long fv = cur[v];
            for (int32_t e = g.off[v] + (int32_t)lane; e < g.off[v + 1]; e += 32) {
              const int32_t u = g.idx[e];
              const unsigned long long nb = fv & ~mb.visit[u];
              if (nb && atomicOr(&mb.next[u], nb) == 0ull) stage_put(stage, mb.tlist, ttail, u);
            }
          }
          stage_drain(stage, mb.tlist, ttail, kStageCap / 2);
        }
      }
      stage_drain(stage, mb.tlist, ttail, 1);
      ok = grid_arrive_wait(&st->bar64, bar_target, &st->status);
      if (!ok) break;
      // commit the touched vertices: next -> new frontier, depths, next frontier list
      const unsigned int t = *reinterpret_cast<volatile unsigned int*>(ttail);
      for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < t; base += stride) {
        const int64_t i = base + threadIdx.x;
        if (i < t) {
          const int32_t u = mb.tlist[i];
          const unsigned long long nb = mb.next[u] & ~mb.visit[u];
          mb.next[u] = 0;
          mb.visit[u] |= nb;
          nxt[u] = nb;
          if (nb) {
            my_fe += (unsigned long long)(g.off[u + 1] - g.off[u]);
            stage_put(stage, out_list, out_tail, u);
            ms_record(mb, rows, n, u, nb, L + 1);
          }
        }
        stage_drain(stage, out_list, out_tail, kStageCap / 2);
      }
    } else {
      // pull: OR the in-neighbours' frontier masks until every unvisited lane is found
      for (int64_t wbase = (int64_t)blockIdx.x * kWarps; wbase < words; wbase += (int64_t)gridDim.x * kWarps) {
        const int64_t w = wbase + wib;
        const int64_t u = w * 32 + lane;
        const bool valid = w < words && u < n;
        unsigned long long nb = 0;
        if (valid) {
          const unsigned long long vis = mb.visit[u];
          const unsigned long long unv = ~vis & act;
          if (unv) {
            const int32_t beg = g.in_off[u], end = g.in_off[u + 1];
            unsigned long long acc = 0;
            for (int32_t e = beg; e < end; e += 4) {
              const int nv = min(4, end - e);
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (q < nv) acc |= cur[g.in_idx[e + q]];
              if ((acc & unv) == unv) break;
            }
            nb = acc & unv;
            if (nb) {
              mb.visit[u] = vis | nb;
              my_fe += (unsigned long long)(g.off[u + 1] - g.off[u]);
              stage_put(stage, out_list, out_tail, (int32_t)u);
              ms_record(mb, rows, n, u, nb, L + 1);
            }
          }
          nxt[u] = nb;
        }
        stage_drain(stage, out_list, out_tail, kStageCap - kMsThreads);
      }
    }
    stage_drain(stage, out_list, out_tail, 1);
    block_add_u64(my_fe, &st->fedges[(L + 1) % 4]);
    ok = grid_arrive_wait(&st->bar64, bar_target, &st->status);
  }
  // Final pass, a warp per 32 consecutive vertices: every output sector written
  // once from the history (coalesced 128-byte row segments, one per root),
  // the per-root reached-edge counts (for each root, the sum of out-degrees of
  // the vertices whose visit mask carries its bit), and the history cleared
  // for the next wave. (The loop ended right after a grid barrier, so
  // every block's masks are visible.) Depths 0 .. L - 1 occurred; those below
  // kMsHistLevels are in the history.
  const int32_t dmax = min(L - 1, kMsHistLevels - 1);
  for (int64_t wbase = (int64_t)blockIdx.x * kWarps; wbase < words; wbase += (int64_t)gridDim.x * kWarps) {
    const int64_t w = wbase + wib;
    if (w >= words) continue;  // whole warp
    const int64_t u = w * 32 + lane;
    const bool valid = u < n;
    const unsigned long long vis = valid ? mb.visit[u] : 0ull;
    if (ok && valid) {
      // bit b of the code (d + 1 for depth d) of root i is bit i of plane b
      // (the history masks of u are disjoint); loads five depths at a time
      unsigned long long p0 = 0ull, p1 = 0ull, p2 = 0ull, p3 = 0ull;
      constexpr int kChunk = 5;
      static_assert(kMsHistLevels % kChunk == 0, "whole chunks");
      static_assert(kMsHistLevels <= 15, "codes d + 1 fit four bits");
#pragma unroll 1
      for (int32_t d0 = 0; d0 <= dmax; d0 += kChunk) {
        unsigned long long m[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j)  // an unreached vertex has no history
          m[j] = vis && d0 + j <= dmax ? mb.hist[(size_t)(d0 + j) * (size_t)n + (size_t)u] : 0ull;
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          if (m[j]) {
            mb.hist[(size_t)(d0 + j) * (size_t)n + (size_t)u] = 0ull;
            const int c = d0 + j + 1;
            if (c & 1) p0 |= m[j];
            if (c & 2) p1 |= m[j];
            if (c & 4) p2 |= m[j];
            if (c & 8) p3 |= m[j];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // nibble r: the code of root 16 q + r
        const unsigned long long word = nibble_spread16(s_spread, p0 >> (16 * q)) |
                                        (nibble_spread16(s_spread, p1 >> (16 * q)) << 1) |
                                        (nibble_spread16(s_spread, p2 >> (16 * q)) << 2) |
                                        (nibble_spread16(s_spread, p3 >> (16 * q)) << 3);
        const int rn = min(16, k - 16 * q);
#pragma unroll 1
        for (int r = 0; r < rn; ++r) {
          const int i = 16 * q + r;
          const unsigned int code = (unsigned int)(word >> (4 * r)) & 15u;
          // reached, but not in the history: a deeper depth, written when found
          if (code != 0u || ((vis >> i) & 1ull) == 0ull) rows.row[i][u] = code == 0u ? -1 : (int32_t)code - 1;
        }
      }
    }
    const unsigned deg = valid ? (unsigned)(g.off[u + 1] - g.off[u]) : 0u;
    unsigned long long any = warp_or64(vis);
    while (any) {
      const int i = __ffsll((long long)any) - 1;
      any &= any - 1;
      const unsigned s = __reduce_add_sync(kFullMask, ((vis >> i) & 1ull) ? deg : 0u);
      if (lane == 0 && s) atomicAdd(&s_edges[i], (unsigned long long)s);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (s_edges[i]) atomicAdd(&st->edges[i], s_edges[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->levels = L;
  // this block's share of the history is zero again (a block that stopped
  // early or saw an error does not count, and the next wave zeroes it all)
  if (threadIdx.x == 0 && ok && *reinterpret_cast<volatile int32_t*>(&st->status) == ST_OK)
    atomicAdd(&st->clean_blocks, 1u);
}

__global__ void k_ms_reset(MsState* st) {
  st->status = ST_OK;
  st->bar64 = 0;
}

}  // namespace bfs
