// Host launcher of the fused edge kernels for one column count K; explicit
// instantiations live in edge_k*.cu so the 32 kernels compile in parallel.
#pragma once

#include <algorithm>
#include <cstdlib>

#include "edge_kernels.cuh"
#include "internal.h"

namespace pspec {

template <int K, bool HVP>
pspec_status launch_edges_k(pspec_graph* g, const EdgeLaunch& L, cudaStream_t s) {
  constexpr int Q = q_of(K);
  PSPEC_TRY(ensure_tasks(g, Q));
  const TaskSet& ts = g->tasks[q_index(Q)];
  static int occ = -1;
  if (occ < 0) {
    PSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, edge_kernel<K, HVP>, kBlock, 0));
    occ = std::max(occ, 1);
    if (const char* env = std::getenv("PSPEC_EDGE_BLOCKS_PER_SM")) occ = std::max(1, std::min(occ, std::atoi(env)));
  }
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
  a.p = L.p;
  a.pm2 = L.p - 2.0f;
  a.gr.block_part = g->d_block_part;
  a.gr.group_part = g->d_group_part;
  a.gr.counters = g->d_counters;
  a.scalars = g->d_scalars;
  a.status = g->d_status;
  a.skip = L.skip;
  a.task_part = L.task_part;
  a.alg1 = L.alg1 ? 1 : 0;
  const int want = g->edge_blocks_per_sm[q_index(Q)];
  int blocks = grid_blocks(g, want > 0 ? std::min(want, occ) : occ);
  blocks = (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (ts.n_tasks + kWarps - 1) / kWarps));
  TimedScope timer(g, HVP ? "hvp_edges" : "eval_edges", s);
  edge_kernel<K, HVP><<<blocks, kBlock, 0, s>>>(a);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

template <int K, bool HVP>
pspec_status occupancy_k(int* blocks_per_sm) {
  PSPEC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, edge_kernel<K, HVP>, kBlock, 0));
  return PSPEC_OK;
}

}  // namespace pspec

#define PSPEC_INSTANTIATE_EDGES(K)                                                          \
  template pspec_status pspec::launch_edges_k<K, false>(pspec_graph*, const pspec::EdgeLaunch&, \
                                                        cudaStream_t);                      \
  template pspec_status pspec::launch_edges_k<K, true>(pspec_graph*, const pspec::EdgeLaunch&,  \
                                                       cudaStream_t);                      \
  template pspec_status pspec::occupancy_k<K, false>(int*);                                 \
  template pspec_status pspec::occupancy_k<K, true>(int*);
