// pspec_tune: pick the edge kernels' launch shape for one graph and column
// count by timing the candidates on the caller's blocks.
//
// The candidates are the edges-per-lane target L (a row of degree d gets the
// smallest power-of-two number of edge slots E with d <= L*E, and a warp task
// holds 32/(E*Q) rows, so L sets the rows per warp) and the resident blocks
// per SM of the persistent grid.  Each candidate rebuilds the task partition,
// runs one untimed eval + HVP, then `reps` timed ones (CUDA events on the
// caller's stream); the fastest is kept on the handle.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pspec {

// The pair a Newton step repeats: the evaluation at U, keeping Delta_p u, and
// a Hessian product at U reusing it (a batch has no kept form: its plain pair).
static pspec_status run_pair(pspec_graph* g, const float* U, const float* V, int k, double p, float* G,
                             float* H, cudaStream_t s) {
  if (g->n_graphs > 1) {
    PSPEC_TRY(eval_batched(g, U, k, p, nullptr, G, nullptr, s));
    return hvp_batched(g, U, V, k, p, H, s);
  }
  PSPEC_TRY(eval_fast(g, U, k, p, nullptr, G, nullptr, s, /*keep_delta=*/true));
  return hvp_fast(g, U, V, k, p, H, s, nullptr, false, /*delta_kept=*/true);
}

static pspec_status tune_impl(pspec_graph* g, const float* U, const float* V, int k, double p, int reps,
                              pspec_tune_report* rep, cudaStream_t s, float* G, float* H) {
  g->keep_valid = false;  // the timed evaluations overwrite the kept Delta_p u
  const int Q = q_of(k);
  const int qi = q_index(Q);
  // resident blocks per SM of the direct HVP kernel the pair runs (kept
  // form for a single graph): that many (0 = each kernel as many as it
  // fits), one and two fewer
  int occ = 0;
  PSPEC_TRY(edge_occupancy(k, true, &occ, g->n_graphs == 1));
  std::vector<int> bps = {0};
  for (int b = occ - 1; b >= std::max(1, occ - 2); --b) bps.push_back(b);
  const int Ls[] = {Q, 2 * Q, 4 * Q, 8 * Q, 16 * Q};
  cudaEvent_t e0, e1;
  PSPEC_CUDA(cudaEventCreate(&e0));
  PSPEC_CUDA(cudaEventCreate(&e1));
  int n = 0, best = -1, best_b = 0;
  double best_ms = 0.0;
  pspec_status st = PSPEC_OK;
  for (int L : Ls) {
    for (int b : bps) {
      if (n >= PSPEC_TUNE_MAX) break;
      free_tasks(g->tasks[qi]);
      g->edges_per_lane[qi] = L;
      g->edge_blocks_per_sm[qi] = b;
      if ((st = run_pair(g, U, V, k, p, G, H, s)) != PSPEC_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && st == PSPEC_OK; ++r) st = run_pair(g, U, V, k, p, G, H, s);
      cudaEventRecord(e1, s);
      if (st != PSPEC_OK) break;
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) { st = cuda_error(ce, "tune timing"); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      rep->edges_per_lane[n] = L;
      rep->blocks_per_sm[n] = b > 0 ? b : occ;
      rep->ms[n] = (double)ms / reps;
      if (best < 0 || rep->ms[n] < best_ms) {
        best = n;
        best_b = b;
        best_ms = rep->ms[n];
      }
      ++n;
    }
    if (st != PSPEC_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  rep->n_candidates = n;
  rep->chosen = best;
  free_tasks(g->tasks[qi]);
  if (best >= 0) {
    // 0 = as many blocks as each kernel fits (the kernels of a shape differ)
    g->edges_per_lane[qi] = rep->edges_per_lane[best];
    g->edge_blocks_per_sm[qi] = best_b;
  } else {
    g->edges_per_lane[qi] = 0;
    g->edge_blocks_per_sm[qi] = 0;
  }
  if (st != PSPEC_OK) return st;
  return ensure_tasks(g, Q);
}

}  // namespace pspec

using namespace pspec;

extern "C" pspec_status pspec_tune(pspec_graph* g, const float* U, const float* V, int k, double p, int reps,
                                   pspec_tune_report* report, void* stream) {
  if (!g || !U || !V || !report) return set_error(PSPEC_ERR_INVALID_ARG, "NULL argument");
  if (k < 1 || k > kMaxK) return set_error(PSPEC_ERR_INVALID_ARG, "k must be in [1, 16]");
  if (!(p > 1.0 && p <= 2.0)) return set_error(PSPEC_ERR_INVALID_ARG, "p must be in (1, 2]");
  if (reps < 1 || reps > 1000) return set_error(PSPEC_ERR_INVALID_ARG, "reps must be in [1, 1000]");
  PSPEC_TRY(check_block(U, k, PSPEC_F32, "U"));
  PSPEC_TRY(check_block(V, k, PSPEC_F32, "V"));
  *report = pspec_tune_report{};
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = sizeof(float) * (size_t)g->n * k;
  float *G = nullptr, *H = nullptr;
  cudaError_t e = cudaMalloc(&G, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&H, bytes);
  if (e != cudaSuccess) {
    cudaFree(G);
    return cuda_error(e, "cudaMalloc(tune outputs)");
  }
  pspec_status st = tune_impl(g, U, V, k, p, reps, report, s, G, H);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(G);
  cudaFree(H);
  if (st == PSPEC_OK && e2 != cudaSuccess) st = cuda_error(e2, "pspec_tune");
  return st;
}
