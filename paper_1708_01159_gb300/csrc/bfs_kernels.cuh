// Kernel declarations and launch shapes shared by the kernel and host sources.
#pragma once

#include "bfs_internal.cuh"

namespace bfs {

constexpr int kThreads = 256;     // block size of the level kernels
constexpr int kDecideThreads = 32;  // block size of k_decide: one warp evaluates the bit-parallel tree
constexpr int kCtaChunk = 2048;   // int32 per shared-memory stage of the CTA variant (8 KB)
constexpr int kCtaDirect = 512;   // adjacency shorter than this is read directly, not staged
constexpr int kPeItems = 8;       // items per thread in the edge-centric scan / expand
constexpr int kPeTile = kThreads * kPeItems;  // frontier entries per scan block, items per expand tile

__global__ void k_init(DevGraph g, Buffers b, RunState* st, int32_t* depth, int32_t root, int32_t forced,
                       const TreeNode* tree, int32_t tree_nodes, const QsTree* tree_qs, int32_t use_handles);
__global__ void k_decide(DevGraph g, Buffers b, RunState* st);
__global__ void k_loop_start(DevGraph g, Buffers b, RunState* st);
__global__ void k_push_thread(DevGraph g, Buffers b, RunState* st);
__global__ void k_push_warp(DevGraph g, Buffers b, RunState* st);
__global__ void k_push_cta(DevGraph g, Buffers b, RunState* st);
__global__ void k_pe_reduce(DevGraph g, Buffers b, RunState* st);
__global__ void k_pe_top(DevGraph g, Buffers b, RunState* st);
__global__ void k_pe_scan(DevGraph g, Buffers b, RunState* st);
__global__ void k_pe_expand(DevGraph g, Buffers b, RunState* st);
__global__ void k_pull(DevGraph g, Buffers b, RunState* st);
// Vertex push appending by CM_WARP or CM_ATOMIC (count-mode comparison)
__global__ void k_push_thread_warp_count(DevGraph g, Buffers b, RunState* st);
__global__ void k_push_thread_atomic_count(DevGraph g, Buffers b, RunState* st);
__global__ void k_edge_list(DevGraph g, Buffers b, RunState* st);
__global__ void k_rev_edge_list(DevGraph g, Buffers b, RunState* st);
__global__ void k_build_origin(const int32_t* off, int32_t n, int32_t* origin);
__global__ void k_undo_level(Buffers b, RunState* st);
__global__ void k_bfs_persistent(DevGraph g, Buffers b, RunState* st, int32_t* depth, int32_t root, int32_t forced,
                                 const TreeNode* tree, int32_t tree_nodes, const QsTree* qs, uint32_t epoch,
                                 int32_t stall);
__global__ void k_profile_level(DevGraph g, Buffers b, RunState* st, int32_t* depth, int32_t L, int32_t v, uint32_t f,
                                unsigned long long e, long long discovered, uint32_t vsel);
__global__ void k_profile_reset(RunState* st, int32_t slot);
__global__ void k_undo_level_p(Buffers b, int32_t* depth, uint32_t qout, unsigned int count, uint32_t vsel);

// graph creation
__global__ void k_validate(const int32_t* off, const int32_t* idx, int32_t n, int32_t m, int32_t* bad);
// degree statistics: the row lengths of `off`, plus those of `off2` when it is not null
__global__ void k_deg_reduce(const int32_t* off, const int32_t* off2, int32_t n, unsigned long long* s1,
                             unsigned long long* s2, unsigned int* dmin, unsigned int* dmax);
__global__ void k_deg_hist(const int32_t* off, const int32_t* off2, int32_t n, int32_t* hist);
__global__ void k_deg_finish(const int32_t* hist, int64_t maxdeg, int32_t n, const unsigned long long* s1,
                             const unsigned long long* s2, long long* out6);
__global__ void k_tr_count(const int32_t* idx, int32_t m, int32_t* cnt);
__global__ void k_scan_reduce(const int32_t* in, int32_t len, long long* bsum);
__global__ void k_scan_top(long long* bsum, int32_t nblocks);
__global__ void k_scan_apply(const int32_t* in, int32_t len, const long long* bsum, int32_t* out);
__global__ void k_tr_scatter(const int32_t* off, const int32_t* idx, int32_t n, int32_t* cursor, int32_t* in_idx);
__global__ void k_pull_hint(const int32_t* off, const int32_t* in_off, const int32_t* in_idx, int32_t n,
                            int32_t* hint);
__global__ void k_vis_init(const int32_t* off, const int32_t* in_off, int32_t n, int32_t words, uint32_t* vis_init,
                           unsigned int* isolated_count);

}  // namespace bfs
