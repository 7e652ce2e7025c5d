/*
 * graphgen.c -- seeded synthetic graph generators and CSR construction.
 *
 * This module prepares INPUTS only: it holds none of the BFS arithmetic. Both
 * the CPU oracle tests and the GPU path consume the CSR graphs it builds, so it
 * lives apart from both of them.
 *
 * Randomness: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) used in counter mode: draw k of a stream
 * whose state starts at s is mix(s + (k+1) * 0x9E3779B97F4A7C15). Each edge or
 * vertex owns a fixed range of draw indices, so output does not depend on the
 * number of OpenMP threads.
 *
 * Generators:
 *   R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): ef * 2^scale edges, each
 *     built by `scale` quadrant choices with probabilities a, b, c, d.
 *   2D grid: 4-neighbour lattice, each undirected edge dropped with
 *     probability `drop`, vertex ids optionally permuted (Fisher-Yates).
 *   Erdos-Renyi G(n, p): geometric skipping over vertex pairs (Batagelj and
 *     Brandes, "Efficient generation of large random networks", Phys. Rev. E
 *     71, 2005).
 * Every generator symmetrises (R-MAT optionally not), drops self-loops and duplicates, and sorts each
 * adjacency list ascending.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

typedef struct {
  int64_t n;
  int64_t m;
  int32_t* off; /* n + 1 */
  int32_t* idx; /* m */
} gg_csr;

static inline uint64_t gg_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Draw k (0-based) of the SplitMix64 stream whose state starts at `state`. */
uint64_t gg_splitmix64_at(uint64_t state, uint64_t k) {
  return gg_mix(state + (k + 1) * GG_GOLDEN);
}

/* Distinct, well-separated stream start for (seed, purpose tag). */
static uint64_t gg_stream(uint64_t seed, uint64_t tag) {
  return gg_mix(seed * GG_GOLDEN + gg_mix(tag + 0x1234567ULL));
}

/* Uniform double in [0, 1) from the top 53 bits. */
static inline double gg_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

void gg_free(gg_csr* g) {
  if (!g) return;
  free(g->off);
  free(g->idx);
  free(g);
}

static int gg_cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static void gg_sort_row(int32_t* p, int64_t len) {
  if (len <= 24) {
    for (int64_t i = 1; i < len; ++i) {
      int32_t key = p[i];
      int64_t j = i - 1;
      while (j >= 0 && p[j] > key) {
        p[j + 1] = p[j];
        --j;
      }
      p[j + 1] = key;
    }
  } else {
    qsort(p, (size_t)len, sizeof(int32_t), gg_cmp_i32);
  }
}

/*
 * CSR from a list of (src, dst) pairs. Pairs with src == dst are dropped. With
 * `symmetrize`, each pair also contributes (dst, src). Duplicates are removed
 * and rows sorted ascending. Returns NULL on allocation failure or if the
 * result would not fit int32 offsets.
 */
gg_csr* gg_from_pairs(int64_t n, int64_t e, const int32_t* src, const int32_t* dst, int symmetrize) {
  if (n < 0 || n > INT32_MAX || e < 0) return NULL;
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return NULL;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v || u < 0 || v < 0 || u >= n || v >= n) continue;
    __atomic_fetch_add(&cnt[u], 1, __ATOMIC_RELAXED);
    if (symmetrize) __atomic_fetch_add(&cnt[v], 1, __ATOMIC_RELAXED);
  }
  int64_t total = 0;
  for (int64_t u = 0; u < n; ++u) {
    int64_t c = cnt[u];
    cnt[u] = total;
    total += c;
  }
  cnt[n] = total;
  int64_t* cur = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  int32_t* tmp = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!cur || !tmp) {
    free(cnt);
    free(cur);
    free(tmp);
    return NULL;
  }
  memcpy(cur, cnt, ((size_t)n + 1) * sizeof(int64_t));
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    int32_t u = src[i], v = dst[i];
    if (u == v || u < 0 || v < 0 || u >= n || v >= n) continue;
    int64_t p = __atomic_fetch_add(&cur[u], 1, __ATOMIC_RELAXED);
    tmp[p] = v;
    if (symmetrize) {
      int64_t q = __atomic_fetch_add(&cur[v], 1, __ATOMIC_RELAXED);
      tmp[q] = u;
    }
  }
  /* sort + dedupe each row in place; cur[u] becomes the deduplicated degree */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t u = 0; u < n; ++u) {
    int32_t* p = tmp + cnt[u];
    int64_t len = cnt[u + 1] - cnt[u];
    gg_sort_row(p, len);
    int64_t w = 0;
    for (int64_t i = 0; i < len; ++i)
      if (w == 0 || p[i] != p[w - 1]) p[w++] = p[i];
    cur[u] = w;
  }
  int64_t m = 0;
  for (int64_t u = 0; u < n; ++u) m += cur[u];
  if (m > INT32_MAX) {
    free(cnt);
    free(cur);
    free(tmp);
    return NULL;
  }
  gg_csr* g = (gg_csr*)calloc(1, sizeof(gg_csr));
  int32_t* off = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
  int32_t* idx = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  if (!g || !off || !idx) {
    free(g);
    free(off);
    free(idx);
    free(cnt);
    free(cur);
    free(tmp);
    return NULL;
  }
  int64_t acc = 0;
  for (int64_t u = 0; u < n; ++u) {
    off[u] = (int32_t)acc;
    acc += cur[u];
  }
  off[n] = (int32_t)acc;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t u = 0; u < n; ++u) memcpy(idx + off[u], tmp + cnt[u], (size_t)cur[u] * sizeof(int32_t));
  free(cnt);
  free(cur);
  free(tmp);
  g->n = n;
  g->m = m;
  g->off = off;
  g->idx = idx;
  return g;
}

/* Random permutation of 0..n-1 by Fisher-Yates, draws from stream `st`. */
static int32_t* gg_permutation(int64_t n, uint64_t st) {
  int32_t* p = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!p) return NULL;
  for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; --i) {
    uint64_t r = gg_splitmix64_at(st, (uint64_t)i);
    /* multiply-shift range reduction to [0, i] */
    int64_t j = (int64_t)(((unsigned __int128)r * (unsigned __int128)(i + 1)) >> 64);
    int32_t t = p[i];
    p[i] = p[j];
    p[j] = t;
  }
  return p;
}

static void gg_apply_perm(int64_t e, int32_t* src, int32_t* dst, const int32_t* perm) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    src[i] = perm[src[i]];
    dst[i] = perm[dst[i]];
  }
}

/* R-MAT with quadrant probabilities a, b, c and d = 1 - a - b - c. flags: bit 0
 * permutes the vertex ids; bit 1 keeps each generated edge's direction (no
 * symmetrisation: a directed graph, whose in- and out-degree distributions
 * differ when b != c). */
gg_csr* gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed, int flags) {
  const int permute = flags & 1, symmetrize = !(flags & 2);
  if (scale < 1 || scale > 30 || edge_factor < 0) return NULL;
  int64_t n = (int64_t)1 << scale;
  int64_t e = edge_factor * n;
  int32_t* src = (int32_t*)malloc((size_t)(e > 0 ? e : 1) * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)(e > 0 ? e : 1) * sizeof(int32_t));
  if (!src || !dst) {
    free(src);
    free(dst);
    return NULL;
  }
  const double ta = a, tab = a + b, tabc = a + b + c;
  const uint64_t st = gg_stream(seed, 1);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < e; ++i) {
    int64_t u = 0, v = 0;
    for (int j = 0; j < scale; ++j) {
      double r = gg_unit(gg_splitmix64_at(st, (uint64_t)i * (uint64_t)scale + (uint64_t)j));
      int bu, bv;
      if (r < ta) {
        bu = 0;
        bv = 0;
      } else if (r < tab) {
        bu = 0;
        bv = 1;
      } else if (r < tabc) {
        bu = 1;
        bv = 0;
      } else {
        bu = 1;
        bv = 1;
      }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
  if (permute) {
    int32_t* perm = gg_permutation(n, gg_stream(seed, 4));
    if (!perm) {
      free(src);
      free(dst);
      return NULL;
    }
    gg_apply_perm(e, src, dst, perm);
    free(perm);
  }
  gg_csr* g = gg_from_pairs(n, e, src, dst, symmetrize);
  free(src);
  free(dst);
  return g;
}

/* rows x cols 4-neighbour lattice; each undirected edge kept with prob 1-drop. */
gg_csr* gg_grid(int64_t rows, int64_t cols, double drop, uint64_t seed, int permute) {
  if (rows < 1 || cols < 1 || rows * cols > INT32_MAX) return NULL;
  int64_t n = rows * cols;
  int64_t cap = 2 * n; /* right + down edges per vertex at most */
  int32_t* src = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  if (!src || !dst) {
    free(src);
    free(dst);
    return NULL;
  }
  const uint64_t st = gg_stream(seed, 3);
  /* candidate edge 2*v is (v, right), 2*v+1 is (v, down); dropped edges become self-loops (ignored) */
#pragma omp parallel for schedule(static)
  for (int64_t v = 0; v < n; ++v) {
    int64_t r = v / cols, c = v % cols;
    for (int k = 0; k < 2; ++k) {
      int64_t id = 2 * v + k;
      int64_t w = -1;
      if (k == 0 && c + 1 < cols) w = v + 1;
      if (k == 1 && r + 1 < rows) w = v + cols;
      int keep = 0;
      if (w >= 0) keep = gg_unit(gg_splitmix64_at(st, (uint64_t)id)) >= drop;
      src[id] = (int32_t)v;
      dst[id] = keep ? (int32_t)w : (int32_t)v;
    }
  }
  if (permute) {
    int32_t* perm = gg_permutation(n, gg_stream(seed, 4));
    if (!perm) {
      free(src);
      free(dst);
      return NULL;
    }
    gg_apply_perm(cap, src, dst, perm);
    free(perm);
  }
  gg_csr* g = gg_from_pairs(n, cap, src, dst, 1);
  free(src);
  free(dst);
  return g;
}

/* G(n, p) with p = avg_degree / (n - 1), by geometric skipping over pairs w < v. */
gg_csr* gg_er(int64_t n, double avg_degree, uint64_t seed) {
  if (n < 1 || n > INT32_MAX) return NULL;
  double p = n > 1 ? avg_degree / (double)(n - 1) : 0.0;
  if (p < 0) p = 0;
  if (p > 1) p = 1;
  int64_t cap = 1024, e = 0;
  int32_t* src = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  int32_t* dst = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
  if (!src || !dst) {
    free(src);
    free(dst);
    return NULL;
  }
  const uint64_t st = gg_stream(seed, 2);
  if (p > 0) {
    const double lq = log1p(-p); /* log(1 - p); p == 1 handled by the -inf branch */
    int64_t v = 1, w = -1;
    uint64_t k = 0;
    while (v < n) {
      double r = gg_unit(gg_splitmix64_at(st, k++));
      int64_t skip = (p >= 1.0) ? 0 : (int64_t)floor(log1p(-r) / lq);
      w += 1 + skip;
      while (w >= v && v < n) {
        w -= v;
        v += 1;
      }
      if (v < n) {
        if (e == cap) {
          cap *= 2;
          int32_t* s2 = (int32_t*)realloc(src, (size_t)cap * sizeof(int32_t));
          if (!s2) {
            free(src);
            free(dst);
            return NULL;
          }
          src = s2;
          int32_t* d2 = (int32_t*)realloc(dst, (size_t)cap * sizeof(int32_t));
          if (!d2) {
            free(src);
            free(dst);
            return NULL;
          }
          dst = d2;
        }
        src[e] = (int32_t)v;
        dst[e] = (int32_t)w;
        ++e;
      }
    }
  }
  gg_csr* g = gg_from_pairs(n, e, src, dst, 1);
  free(src);
  free(dst);
  return g;
}

static int64_t gg_find(int32_t* parent, int64_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]];
    x = parent[x];
  }
  return x;
}

/*
 * Label of each vertex's connected component (treating every CSR entry as an
 * undirected edge), by union-find. comp[v] = the smallest-index representative
 * chosen by the union rule. Returns the size of the largest component and its
 * label in *giant_label.
 */
int64_t gg_components(int64_t n, const int32_t* off, const int32_t* idx, int32_t* comp, int32_t* giant_label) {
  for (int64_t v = 0; v < n; ++v) comp[v] = (int32_t)v;
  for (int64_t u = 0; u < n; ++u)
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      int64_t a = gg_find(comp, u), b = gg_find(comp, idx[e]);
      if (a == b) continue;
      if (a < b)
        comp[b] = (int32_t)a;
      else
        comp[a] = (int32_t)b;
    }
  for (int64_t v = 0; v < n; ++v) comp[v] = (int32_t)gg_find(comp, v);
  int64_t* sz = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  if (!sz) return -1;
  int64_t best = 0, lab = 0;
  for (int64_t v = 0; v < n; ++v) sz[comp[v]]++;
  for (int64_t v = 0; v < n; ++v)
    if (sz[v] > best) {
      best = sz[v];
      lab = v;
    }
  free(sz);
  if (giant_label) *giant_label = (int32_t)lab;
  return best;
}

/*
 * k distinct roots drawn uniformly (seeded) from the vertices of nonzero
 * out-degree, or, with `giant`, from the largest connected component (among
 * its vertices of nonzero degree). Returns the number written (< k when too
 * few candidates exist), or -1 on allocation failure.
 */
int32_t gg_sample_roots(int64_t n, const int32_t* off, const int32_t* idx, int32_t k, uint64_t seed, int giant,
                        int32_t* roots) {
  int32_t* cand = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!cand) return -1;
  int32_t* comp = NULL;
  int32_t lab = 0;
  if (giant) {
    comp = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!comp || gg_components(n, off, idx, comp, &lab) < 0) {
      free(cand);
      free(comp);
      return -1;
    }
  }
  int64_t nc = 0;
  for (int64_t v = 0; v < n; ++v) {
    if (off[v + 1] == off[v]) continue;
    if (giant && comp[v] != lab) continue;
    cand[nc++] = (int32_t)v;
  }
  free(comp);
  const uint64_t st = gg_stream(seed, 5);
  int32_t got = 0;
  /* partial Fisher-Yates over the candidate list: distinct draws */
  for (int64_t i = 0; i < k && i < nc; ++i) {
    uint64_t r = gg_splitmix64_at(st, (uint64_t)i);
    int64_t j = i + (int64_t)(((unsigned __int128)r * (unsigned __int128)(nc - i)) >> 64);
    int32_t t = cand[i];
    cand[i] = cand[j];
    cand[j] = t;
    roots[got++] = cand[i];
  }
  free(cand);
  return got;
}
