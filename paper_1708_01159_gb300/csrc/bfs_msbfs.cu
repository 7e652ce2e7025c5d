// Multi-source BFS: up to 64 traversals of one graph in one persistent kernel.
//
// Each vertex carries three 64-bit masks: visit (bit i: reached by root i),
// frontier (bit i: at depth L for root i) and next (bits pushed to it during
// the level). Every level runs one direction for all roots at once:
//   push: every vertex with a nonzero frontier mask ORs its mask, minus the
//         target's visited bits, into each neighbour's next mask (atomicOr),
//         then a commit pass turns next into the new frontier;
//   pull: every vertex still unvisited in some lane ORs its in-neighbours'
//         frontier masks, stopping once every unvisited lane is found.
// The result equals k independent single-source traversals (each lane is one
// level-synchronous BFS from its root, Section 3.1). A warp owns 32
// consecutive vertices in the commit and pull passes, so for each root the
// new depths of those vertices are written as one coalesced row segment.
#include "bfs_msbfs.cuh"

namespace bfs {

namespace {

constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x |= __shfl_xor_sync(kFullMask, x, o);
  return x;
}

// Record lane masks `nb` of the warp's 32 vertices (u = w * 32 + lane) as
// newly reached at depth d: depth rows, per-root reached-edge sums (in shared
// memory), and the next level's frontier statistics.
__device__ __forceinline__ void ms_record(int32_t* depth, int64_t n, int32_t u, bool valid, unsigned long long nb,
                                          int32_t deg, int32_t d, unsigned long long* s_edges,
                                          unsigned long long& fcount, unsigned long long& fedges) {
  unsigned long long any = warp_or64(valid ? nb : 0ull);
  if (valid && nb) {
    fcount += 1;
    fedges += (unsigned long long)deg;
  }
  while (any) {
    const int i = __ffsll((long long)any) - 1;
    any &= any - 1;
    const bool has = valid && ((nb >> i) & 1ull);
    const unsigned sum = __reduce_add_sync(kFullMask, has ? (unsigned)deg : 0u);
    if (has) depth[(int64_t)i * n + u] = d;
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&s_edges[i], (unsigned long long)sum);
  }
}

}  // namespace

__global__ void __launch_bounds__(kMsThreads) k_msbfs(DevGraph g, MsBuffers mb, MsState* st, int32_t k,
                                                       int32_t* depth, MsConfig cfg) {
  __shared__ unsigned long long s_edges[64];
  const int64_t n = g.n;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const unsigned long long act = k >= 64 ? ~0ull : ((1ull << k) - 1ull);
  for (int i = threadIdx.x; i < 64; i += blockDim.x) s_edges[i] = 0;
  // init: masks cleared, depth rows -1 (16-byte stores when aligned)
  for (int64_t v = tid; v < n; v += stride) {
    mb.visit[v] = 0;
    mb.front[0][v] = 0;
    mb.front[1][v] = 0;
    mb.next[v] = 0;
  }
  const int64_t total = n * k;
  if ((reinterpret_cast<uintptr_t>(depth) & 15u) == 0) {
    int4* d4 = reinterpret_cast<int4*>(depth);
    const int64_t t4 = total >> 2;
    for (int64_t i = tid; i < t4; i += stride) d4[i] = make_int4(-1, -1, -1, -1);
    for (int64_t i = (t4 << 2) + tid; i < total; i += stride) depth[i] = -1;
  } else {
    for (int64_t i = tid; i < total; i += stride) depth[i] = -1;
  }
  if (!grid_barrier(&st->bar_count, &st->bar_gen, &st->status)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // roots: level 0 frontier; a vertex repeated as several roots carries several bits
    unsigned long long fc = 0, fe = 0;
    for (int i = 0; i < k; ++i) {
      const int32_t r = mb.roots[i];
      const int32_t deg = g.off[r + 1] - g.off[r];
      if (mb.visit[r] == 0) {
        fc += 1;
        fe += (unsigned long long)deg;
      }
      mb.visit[r] |= 1ull << i;
      mb.front[0][r] |= 1ull << i;
      depth[(int64_t)i * n + r] = 0;
      st->edges[i] = (unsigned long long)deg;
    }
    for (int i = k; i < 64; ++i) st->edges[i] = 0;
    st->fcount[0] = fc;
    st->fedges[0] = fe;
    st->fcount[1] = st->fcount[2] = 0;
    st->fedges[1] = st->fedges[2] = 0;
  }
  bool ok = grid_barrier(&st->bar_count, &st->bar_gen, &st->status);
  const uint32_t lane = threadIdx.x & 31;
  const int64_t words = (n + 31) / 32;
  const int64_t warp = tid >> 5;
  const int64_t nwarps = stride >> 5;
  int32_t L = 0;
  for (; ok; ++L) {
    const unsigned long long fc = *reinterpret_cast<volatile unsigned long long*>(&st->fcount[L % 3]);
    const unsigned long long fe = *reinterpret_cast<volatile unsigned long long*>(&st->fedges[L % 3]);
    if (fc == 0) break;
    if (L > g.n) {
      if (blockIdx.x == 0 && threadIdx.x == 0) st->status = ST_TIMEOUT;
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->fcount[(L + 2) % 3] = 0;
      st->fedges[(L + 2) % 3] = 0;
    }
    const unsigned long long* cur = (L & 1) ? mb.front[1] : mb.front[0];
    unsigned long long* nxt = (L & 1) ? mb.front[0] : mb.front[1];
    // direction: pull once the frontier's edges exceed m / alpha (Beamer's rule, alpha tuned)
    const bool pull = fe * (unsigned long long)cfg.alpha > (unsigned long long)g.m;
    unsigned long long my_fc = 0, my_fe = 0;
    if (!pull) {
      if (cfg.push_mode == 0) {
        // thread per frontier vertex
        for (int64_t v = tid; v < n; v += stride) {
          const unsigned long long f = cur[v];
          if (!f) continue;
          for (int32_t e = g.off[v]; e < g.off[v + 1]; ++e) {
            const int32_t u = g.idx[e];
            const unsigned long long nb = f & ~mb.visit[u];
            if (nb) atomicOr(&mb.next[u], nb);
          }
        }
      } else {
        // warp per frontier vertex: the warp's lanes with work take turns, all 32 stride the list
        for (int64_t w = warp; w < words; w += nwarps) {
          const int64_t v0 = w * 32 + lane;
          const unsigned long long f0 = v0 < n ? cur[v0] : 0ull;
          unsigned int todo = __ballot_sync(kFullMask, f0 != 0ull);
          while (todo) {
            const int j = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t v = (int32_t)(w * 32 + j);
            const unsigned long long f = __shfl_sync(kFullMask, f0, j);
            const int32_t beg = g.off[v], end = g.off[v + 1];
            for (int32_t e = beg + (int32_t)lane; e < end; e += 32) {
              const int32_t u = g.idx[e];
              const unsigned long long nb = f & ~mb.visit[u];
              if (nb) atomicOr(&mb.next[u], nb);
            }
          }
        }
      }
      ok = grid_barrier(&st->bar_count, &st->bar_gen, &st->status);
      if (!ok) break;
      // commit: next -> new frontier, depths, statistics
      for (int64_t w = warp; w < words; w += nwarps) {
        const int64_t u = w * 32 + lane;
        const bool valid = u < n;
        unsigned long long nb = 0;
        int32_t deg = 0;
        if (valid) {
          const unsigned long long nx = mb.next[u];
          if (nx) {
            nb = nx & ~mb.visit[u];
            mb.visit[u] |= nb;
            mb.next[u] = 0;
            deg = g.off[u + 1] - g.off[u];
          }
          nxt[u] = nb;
        }
        if (__any_sync(kFullMask, nb != 0ull))
          ms_record(depth, n, (int32_t)u, valid, nb, deg, L + 1, s_edges, my_fc, my_fe);
      }
    } else {
      // pull: OR the in-neighbours' frontier masks until every unvisited lane is found
      for (int64_t w = warp; w < words; w += nwarps) {
        const int64_t u = w * 32 + lane;
        const bool valid = u < n;
        unsigned long long nb = 0;
        int32_t deg = 0;
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
              deg = g.symmetric ? end - beg : g.off[u + 1] - g.off[u];
            }
          }
          nxt[u] = nb;
        }
        if (__any_sync(kFullMask, nb != 0ull))
          ms_record(depth, n, (int32_t)u, valid, nb, deg, L + 1, s_edges, my_fc, my_fe);
      }
    }
    block_add_u64(my_fc, &st->fcount[(L + 1) % 3]);
    block_add_u64(my_fe, &st->fedges[(L + 1) % 3]);
    ok = grid_barrier(&st->bar_count, &st->bar_gen, &st->status);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (s_edges[i]) atomicAdd(&st->edges[i], s_edges[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) st->levels = L;
}

__global__ void k_ms_reset(MsState* st) {
  st->status = ST_OK;
  st->bar_count = 0;
}

}  // namespace bfs
