// Host launcher of the fused edge kernels for one column count K; explicit
// instantiations live in edge_k*.cu so the kernels compile in parallel.
//
// Two kernels compute the same sums: the staged kernel (edge_staged.cuh),
// used whenever a task's entries fit its shared-memory buffers (entries per
// task 32 L / Q <= staged_max_entries(K)), and the direct kernel
// (edge_kernels.cuh) for longer tasks and for batch launches that leave
// graphs out (graph_skip).  The edges-per-lane target L of the handle's task
// set -- set by pspec_tune or PSPEC_EDGES_PER_LANE, 16 Q by default (direct) --
// thus also picks the kernel.
#pragma once

#include <algorithm>
#include <cstdlib>

#include "edge_kernels.cuh"
#include "edge_staged.cuh"
#include "internal.h"

namespace pspec {

inline int env_blocks_per_sm(int occ) {
  if (const char* env = std::getenv("PSPEC_EDGE_BLOCKS_PER_SM")) return std::max(1, std::min(occ, std::atoi(env)));
  return occ;
}

template <int K, int MODE>
pspec_status launch_staged(pspec_graph* g, const EdgeArgs& a, int max_entries, int want, cudaStream_t s) {
  // the largest dynamic shared memory this instantiation is ever given, set
  // once per process (thread-safe initialisation)
  static const cudaError_t attr =
      cudaFuncSetAttribute(edge_staged_kernel<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kWarps * staged_warp_bytes(K, MODE, staged_max_entries(K))));
  PSPEC_CUDA(attr);
  const size_t bytes = kWarps * staged_warp_bytes(K, MODE, max_entries);
  int occ = 0;
  PSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, edge_staged_kernel<K, MODE>, kBlock, bytes));
  occ = env_blocks_per_sm(std::max(occ, 1));
  int blocks = grid_blocks(g, want > 0 ? std::min(want, occ) : occ);
  blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, ((int64_t)a.n_tasks + kWarps - 1) / kWarps));
  edge_staged_kernel<K, MODE><<<blocks, kBlock, bytes, s>>>(a, max_entries);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

// below this many tasks per warp the direct kernel takes contiguous,
// cost-balanced ranges of the (degree-sorted) task list instead of
// round-robin tasks, so the heavy tail is spread evenly; both are fixed
// assignments, so results stay bit-reproducible
constexpr int kSplitTasksPerWarp = 8;

template <int K, int MODE, bool SPLIT, bool GSKIP = false>
int direct_blocks(pspec_graph* g, int64_t n_tasks, int want) {
  // resident blocks at the kernel's register count, once per process
  static const int occ_direct = [] {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, edge_kernel<K, MODE, SPLIT, GSKIP>, kBlock, 0) !=
        cudaSuccess)
      o = 1;
    return std::max(o, 1);
  }();
  const int occ = env_blocks_per_sm(occ_direct);
  const int blocks = grid_blocks(g, want > 0 ? std::min(want, occ) : occ);
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (n_tasks + kWarps - 1) / kWarps));
}

template <int K, int MODE>
pspec_status launch_direct(pspec_graph* g, EdgeArgs a, TaskSet& ts, int want, cudaStream_t s) {
  const int64_t n_tasks = ts.n_tasks;
  a.warp_begin = nullptr;
  if (a.graph_skip) {
    // round-robin tasks: a graph's (contiguous) tasks spread over all warps,
    // so a launch in which few graphs take part is not left to a few warps
    const int blocks = direct_blocks<K, MODE, false, true>(g, n_tasks, want);
    edge_kernel<K, MODE, false, true><<<blocks, kBlock, 0, s>>>(a);
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  const int rr_blocks = direct_blocks<K, MODE, false>(g, n_tasks, want);
  if (n_tasks < (int64_t)kSplitTasksPerWarp * rr_blocks * kWarps) {
    const int blocks = direct_blocks<K, MODE, true>(g, n_tasks, want);
    PSPEC_TRY(ensure_split(ts, blocks * kWarps, s, &a.warp_begin));
    if (a.warp_begin) {
      edge_kernel<K, MODE, true><<<blocks, kBlock, 0, s>>>(a);
      PSPEC_CUDA(cudaGetLastError());
      return PSPEC_OK;
    }
  }
  edge_kernel<K, MODE, false><<<rr_blocks, kBlock, 0, s>>>(a);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

template <int K, bool HVP>
pspec_status launch_edges_k(pspec_graph* g, const EdgeLaunch& L, cudaStream_t s) {
  constexpr int Q = q_of(K);
  PSPEC_TRY(ensure_tasks(g, Q));
  TaskSet& ts = g->tasks[q_index(Q)];
  EdgeArgs a;
  a.cw = g->d_cw_s;
  a.perm = g->d_perm;
  a.U = L.U;
  a.V = L.V;
  a.out_a = L.out_a;
  a.out_b = L.out_b;
  a.tasks = ts.d_tasks;
  a.n_tasks = (int)ts.n_tasks;
  a.hub_part = g->d_hub_part;
  a.hub_first = ts.d_hub_first;
  a.hub_nchunk = ts.d_hub_nchunk;
  a.chunk_hub = ts.d_chunk_hub;
  a.hub_ticket = ts.d_hub_ticket;
  a.p = (float)L.p;
  a.pm2 = (float)L.p - 2.0f;
  a.p64 = L.p;
  a.gr.block_part = g->d_block_part;
  a.gr.group_part = g->d_group_part;
  a.gr.counters = g->d_counters;
  a.scalars = g->d_scalars;
  a.status = g->d_status;
  a.skip = L.skip;
  a.task_part = L.task_part;
  a.alg1 = L.alg1 ? 1 : 0;
  a.keep_nd = L.keep_nd;
  a.warp_begin = nullptr;
  a.graph_skip = L.graph_skip;
  a.task_graph = ts.d_task_graph;
  const int want = g->edge_blocks_per_sm[q_index(Q)];
  TimedScope timer(g, HVP ? "hvp_edges" : "eval_edges", s);
  const int max_entries = ts.chunk_edges;  // 32 L / Q
  if (max_entries <= staged_max_entries(K) && !L.graph_skip) {
    if constexpr (!HVP) return launch_staged<K, kModeEval>(g, a, max_entries, want, s);
    else if (L.keep_nd) return launch_staged<K, kModeHvpKept>(g, a, max_entries, want, s);
    else return launch_staged<K, kModeHvp>(g, a, max_entries, want, s);
  }
  if constexpr (!HVP) return launch_direct<K, kModeEval>(g, a, ts, want, s);
  else if (L.keep_nd) return launch_direct<K, kModeHvpKept>(g, a, ts, want, s);
  else return launch_direct<K, kModeHvp>(g, a, ts, want, s);
}

// resident blocks per SM of the direct kernel of a mode (the HVP one at a
// kept point when `kept`)
template <int K, bool HVP>
pspec_status occupancy_k(int* blocks_per_sm, bool kept) {
  if (HVP && kept)
    PSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, edge_kernel<K, kModeHvpKept, false>,
                                                             kBlock, 0));
  else
    PSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, edge_kernel<K, HVP ? kModeHvp : kModeEval, false>, kBlock, 0));
  return PSPEC_OK;
}

}  // namespace pspec

#define PSPEC_INSTANTIATE_EDGES(K)                                                          \
  template pspec_status pspec::launch_edges_k<K, false>(pspec_graph*, const pspec::EdgeLaunch&, \
                                                        cudaStream_t);                      \
  template pspec_status pspec::launch_edges_k<K, true>(pspec_graph*, const pspec::EdgeLaunch&,  \
                                                       cudaStream_t);                      \
  template pspec_status pspec::occupancy_k<K, false>(int*, bool);                           \
  template pspec_status pspec::occupancy_k<K, true>(int*, bool);
