// pspec_solve_batched: the solve of Section 2 (Newton/tCG on the Grassmann
// manifold, p lowered stage by stage toward 1, then k-means and RCut) for every
// graph of a batched handle, each graph its own problem.
//
// Each graph gets a single-graph handle of its own (built on the first call
// and kept on the batched handle: the graph's entries copied out of the
// concatenation with columns rebased to its vertices), and the per-graph
// solves run concurrently: host worker threads take graphs from a shared
// counter, each solve on the private stream of its graph's handle, so the
// device interleaves the kernels of many small graphs.  Every graph's result
// is the same as a pspec_solve on that graph alone.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pspec {

static pspec_status build_subs(pspec_graph* g, cudaStream_t s) {
  if ((int)g->subs.size() == g->n_graphs) return PSPEC_OK;
  const std::vector<int64_t>& off = g->h_node_off;
  const std::vector<int64_t>& rp = g->h_rowptr;
  std::vector<pspec_graph*> subs(g->n_graphs, nullptr);
  pspec_status st = PSPEC_OK;
  for (int q = 0; q < g->n_graphs && st == PSPEC_OK; ++q) {
    const int64_t r0 = off[q], r1 = off[q + 1], n = r1 - r0;
    const int64_t e0 = rp[r0], e1 = rp[r1], nnz = e1 - e0;
    std::vector<int64_t> rowptr(n + 1);
    for (int64_t i = 0; i <= n; ++i) rowptr[i] = rp[r0 + i] - e0;
    std::vector<int32_t> col(std::max<int64_t>(nnz, 1));
    std::vector<float> val(std::max<int64_t>(nnz, 1));
    if (nnz) {
      cudaError_t e = cudaMemcpy(col.data(), g->d_col + e0, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(val.data(), g->d_val32 + e0, sizeof(float) * nnz, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        st = cuda_error(e, "batched solve: graph copy");
        break;
      }
      for (int64_t t = 0; t < nnz; ++t) col[t] -= (int32_t)r0;
    }
    if (n == 0) continue;  // an empty graph has nothing to solve
    st = pspec_graph_create(n, rowptr.data(), col.data(), val.data(), PSPEC_F32, PSPEC_HOST_PTRS, s, &subs[q]);
  }
  if (st != PSPEC_OK) {
    for (pspec_graph* sub : subs) pspec_graph_destroy(sub);
    return st;
  }
  g->subs = std::move(subs);
  return PSPEC_OK;
}

}  // namespace pspec

using namespace pspec;

extern "C" pspec_status pspec_solve_batched(pspec_graph* g, int k, const double* p_schedule, int n_p,
                                            const pspec_solve_opts* opts, float* U_inout,
                                            int32_t* labels_out, double* rcut_out, int32_t* status_out,
                                            int n_threads, void* stream) {
  if (!g) return set_error(PSPEC_ERR_INVALID_ARG, "graph is NULL");
  if (g->h_node_off.empty()) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_solve_batched takes a batched handle");
  if (k < 1 || k > kMaxK) return set_error(PSPEC_ERR_INVALID_ARG, "k must be in [1, 16]");
  if (!U_inout || !labels_out || !rcut_out || !status_out)
    return set_error(PSPEC_ERR_INVALID_ARG, "NULL argument");
  if (n_threads < 1 || n_threads > 256) return set_error(PSPEC_ERR_INVALID_ARG, "n_threads must be in [1, 256]");
  pspec_solve_opts o;
  PSPEC_TRY(check_solve_args(p_schedule, n_p, opts, &o));
  cudaStream_t caller = (cudaStream_t)stream;
  PSPEC_CUDA(cudaStreamSynchronize(caller));  // U_inout and earlier work are ready
  PSPEC_TRY(build_subs(g, caller));
  const int G = g->n_graphs;
  const std::vector<int64_t> off = g->h_node_off;
  int device = 0;
  PSPEC_CUDA(cudaGetDevice(&device));
  std::atomic<int> next{0};
  std::mutex err_mu;
  std::string first_err;
  pspec_status first_st = PSPEC_OK;
  auto worker = [&]() {
    cudaSetDevice(device);
    for (int q = next.fetch_add(1); q < G; q = next.fetch_add(1)) {
      const int64_t r0 = off[q], n = off[q + 1] - r0;
      rcut_out[q] = 0.0;
      pspec_status st;
      if (n < k) {
        st = n == 0 ? PSPEC_OK : set_error(PSPEC_ERR_INVALID_ARG, "a graph has fewer vertices than k");
        rcut_out[q] = n == 0 ? 0.0 : NAN;
      } else {
        st = solve_on_handle(g->subs[q], k, p_schedule, n_p, o, PSPEC_F32, U_inout + r0 * k,
                             labels_out + r0, &rcut_out[q], nullptr, caller);
      }
      status_out[q] = (int32_t)st;
      if (st != PSPEC_OK && st != PSPEC_ERR_NOT_CONVERGED) {
        std::lock_guard<std::mutex> lock(err_mu);
        if (first_st == PSPEC_OK) {
          first_st = st;
          first_err = "graph " + std::to_string(q) + ": " + pspec_last_error();
        }
      }
    }
  };
  const int nt = std::min(n_threads, G);
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int i = 0; i < nt; ++i) pool.emplace_back(worker);
  for (std::thread& th : pool) th.join();
  PSPEC_CUDA(cudaStreamSynchronize(caller));
  if (first_st != PSPEC_OK) return set_error(first_st, first_err);
  for (int q = 0; q < G; ++q)
    if (status_out[q] == PSPEC_ERR_NOT_CONVERGED) return PSPEC_ERR_NOT_CONVERGED;
  return PSPEC_OK;
}
