/*
 * bfs_oracle.c -- the CPU oracle for level-synchronous BFS.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this code:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or helper with the GPU library.
 *
 * What it computes is the plain definition of the problem the method solves
 * (Section 2.2: from a root, reach every vertex reachable from it and give its
 * shortest hop distance), with the initialisation and termination of the
 * level-synchronous formulation (Section 3.1: every depth starts at infinity,
 * the root at 0, and the traversal ends when a level discovers nothing). A FIFO
 * queue visits vertices in nondecreasing distance, so the first time a vertex
 * is seen fixes its depth. "Infinity" is written as -1.
 *
 * Besides the depths it reports, per level L, the number of vertices at depth
 * L (the frontier size of Section 3.1 and the "frontier size" feature of
 * Section 4.1) and the sum of their out-degrees, and the reached-edge count:
 * the sum of out-degrees over all reached vertices.
 */
#include <stdint.h>
#include <stdlib.h>

enum {
  ORACLE_OK = 0,
  ORACLE_ERR_INVALID_ARG = 1,
  ORACLE_ERR_BAD_GRAPH = 2,
  ORACLE_ERR_OOM = 3,
};

/* CSR well-formedness: off[0] = 0, off nondecreasing, off[n] = m, 0 <= idx < n. */
int oracle_validate_csr(int64_t n, int64_t m, const int32_t* off, const int32_t* idx) {
  if (n < 0 || m < 0 || n > INT32_MAX || m > INT32_MAX) return ORACLE_ERR_INVALID_ARG;
  if (off[0] != 0) return ORACLE_ERR_BAD_GRAPH;
  for (int64_t v = 0; v < n; ++v)
    if (off[v + 1] < off[v]) return ORACLE_ERR_BAD_GRAPH;
  if (off[n] != m) return ORACLE_ERR_BAD_GRAPH;
  for (int64_t e = 0; e < m; ++e)
    if (idx[e] < 0 || idx[e] >= n) return ORACLE_ERR_BAD_GRAPH;
  return ORACLE_OK;
}

/*
 * Single-source BFS. Writes depth[0..n). If level_count / level_edges are not
 * NULL they receive, for L < cap_levels, the count of vertices at depth L and
 * the sum of their out-degrees; *num_levels gets the number of nonempty levels.
 * Returns the reached-edge count (>= 0) or the negated error code.
 */
int64_t oracle_bfs(int64_t n, const int32_t* off, const int32_t* idx, int32_t root, int32_t* depth,
                   int64_t* level_count, int64_t* level_edges, int64_t cap_levels, int64_t* num_levels) {
  if (n < 1 || root < 0 || root >= n || depth == NULL) return -ORACLE_ERR_INVALID_ARG;
  int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!queue) return -ORACLE_ERR_OOM;

  for (int64_t v = 0; v < n; ++v) depth[v] = -1;
  depth[root] = 0;
  int64_t head = 0, tail = 0;
  queue[tail++] = root;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t e = off[u]; e < off[u + 1]; ++e) {
      int32_t v = idx[e];
      if (depth[v] == -1) {
        depth[v] = depth[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);

  int64_t edges_reached = 0, levels = 0;
  for (int64_t L = 0; L < cap_levels; ++L) {
    if (level_count) level_count[L] = 0;
    if (level_edges) level_edges[L] = 0;
  }
  for (int64_t v = 0; v < n; ++v) {
    int32_t d = depth[v];
    if (d < 0) continue;
    int64_t deg = (int64_t)off[v + 1] - off[v];
    edges_reached += deg;
    if (d + 1 > levels) levels = d + 1;
    if (d < cap_levels) {
      if (level_count) level_count[d] += 1;
      if (level_edges) level_edges[d] += deg;
    }
  }
  if (num_levels) *num_levels = levels;
  return edges_reached;
}

/*
 * k independent single-source runs: the oracle of multi-source (batched) BFS.
 * depth is k rows of n entries, row i for roots[i]. edges[i] gets each run's
 * reached-edge count. Returns 0 or the error code of the first failing run.
 */
int oracle_bfs_batch(int64_t n, const int32_t* off, const int32_t* idx, const int32_t* roots, int64_t k,
                     int32_t* depth, int64_t* edges) {
  for (int64_t i = 0; i < k; ++i) {
    int64_t r = oracle_bfs(n, off, idx, roots[i], depth + i * n, NULL, NULL, 0, NULL);
    if (r < 0) return (int)-r;
    if (edges) edges[i] = r;
  }
  return ORACLE_OK;
}
