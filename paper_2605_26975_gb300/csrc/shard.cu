// Row-partitioned evaluation: the calls one rank of a multi-GPU run makes on
// its shard of W (pspec_graph_create_shard), split at the one exchange step
// the method has.  Every per-column quantity of Section 2 is a sum over rows,
//   N_l = 1/2 sum_i sum_j w_ij |d_ij|^p,  D_l = sum_i |u_i|^p,
//   sigma_N = sum_i (Delta_p u)_i v_i,    sigma_D = sum_i phi_p(u_i) v_i,
// so each rank sums its owned rows (the *_partial calls), the ranks add their
// FP64 sums (an allreduce of 2k or 4k doubles, the caller's), and each rank
// finishes its owned rows from the global sums (the *_finish calls: the
// gradient's and the Hessian product's epilogues).  The rows a rank reads but
// does not own -- the halo, its owned rows' neighbours on other ranks -- are
// the caller's to copy into the block before the partial call.
#include <algorithm>

#include "common.cuh"
#include "edge_kernels.cuh"
#include "internal.h"

namespace pspec {

// FP64 scalars and epilogue coefficients of every column from the global
// sums (N, D[, sigma_N, sigma_D], k each), as the edge kernels' last block
// forms them from its own sums.
__global__ void shard_coef_kernel(const double* sums, int k, double p, int hvp, int alg1, double* sc,
                                  int* status) {
  const int c = threadIdx.x;
  if (c < k) {
    const double sN = hvp ? sums[2 * k + c] : 0.0, sD = hvp ? sums[3 * k + c] : 0.0;
    const int flags = column_scalars(c, sums[c], sums[k + c], sN, sD, hvp != 0, p, alg1, sc);
    if (flags) atomicOr(status, flags);
  }
  __syncthreads();
  if (c == 0) {
    double F = 0.0;
    for (int l = 0; l < k; ++l) F += sc[kScN + l] / sc[kScD + l];
    sc[kScF] = F;
  }
}

static pspec_status check_shard_call(pspec_graph* g, int k, double p, const void* U, const void* out,
                                     const char* what) {
  PSPEC_TRY(check_common(g, k, p));
  if (!g->is_shard) return set_error(PSPEC_ERR_INVALID_ARG, std::string(what) + " takes a shard handle");
  PSPEC_TRY(check_block(U, k, PSPEC_F32, "U"));
  PSPEC_TRY(check_block(out, k, PSPEC_F32, "output block"));
  if (U == out) return set_error(PSPEC_ERR_INVALID_ARG, "the output block aliases U");
  return PSPEC_OK;
}

static pspec_status copy_sums(pspec_graph* g, double* sums_out, int k, bool hvp, cudaStream_t s) {
  if (!sums_out) return set_error(PSPEC_ERR_INVALID_ARG, "sums_out is NULL");
  PSPEC_CUDA(cudaMemcpyAsync(sums_out, g->d_scalars + kScN, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
  PSPEC_CUDA(cudaMemcpyAsync(sums_out + k, g->d_scalars + kScD, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
  if (hvp) {
    PSPEC_CUDA(cudaMemcpyAsync(sums_out + 2 * k, g->d_scalars + kScCN, sizeof(double) * k,
                               cudaMemcpyDeviceToDevice, s));
    PSPEC_CUDA(cudaMemcpyAsync(sums_out + 3 * k, g->d_scalars + kScCD, sizeof(double) * k,
                               cudaMemcpyDeviceToDevice, s));
  }
  return PSPEC_OK;
}

static pspec_status finish_coefs(pspec_graph* g, const double* sums_in, int k, double p, bool hvp, bool alg1,
                                 cudaStream_t s) {
  if (!sums_in) return set_error(PSPEC_ERR_INVALID_ARG, "sums_in is NULL");
  shard_coef_kernel<<<1, 32, 0, s>>>(sums_in, k, p, hvp ? 1 : 0, alg1 ? 1 : 0, g->d_scalars, g->d_status);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

}  // namespace pspec

using namespace pspec;

extern "C" pspec_status pspec_eval_partial(pspec_graph* g, const float* U, int k, double p, float* grad_out,
                                           double* sums_out, void* stream) {
  PSPEC_TRY(check_shard_call(g, k, p, U, grad_out, "pspec_eval_partial"));
  cudaStream_t s = (cudaStream_t)stream;
  EdgeLaunch L{U, nullptr, grad_out, nullptr, p, k};
  PSPEC_TRY(launch_eval_edges(g, L, s));
  return copy_sums(g, sums_out, k, false, s);
}

extern "C" pspec_status pspec_eval_finish(pspec_graph* g, const float* U, int k, double p,
                                          const double* sums_in, double* F_out, float* grad_out,
                                          void* stream) {
  PSPEC_TRY(check_shard_call(g, k, p, U, grad_out, "pspec_eval_finish"));
  cudaStream_t s = (cudaStream_t)stream;
  PSPEC_TRY(finish_coefs(g, sums_in, k, p, false, false, s));
  PSPEC_TRY(run_grad_epilogue(g, U, grad_out, grad_out, k, p, s));
  if (F_out)
    PSPEC_CUDA(cudaMemcpyAsync(F_out, g->d_scalars + kScF, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return PSPEC_OK;
}

extern "C" pspec_status pspec_hvp_partial(pspec_graph* g, const float* U, const float* V, int k, double p,
                                          float* HV_out, double* sums_out, void* stream) {
  PSPEC_TRY(check_shard_call(g, k, p, U, HV_out, "pspec_hvp_partial"));
  PSPEC_TRY(check_block(V, k, PSPEC_F32, "V"));
  if (V == HV_out) return set_error(PSPEC_ERR_INVALID_ARG, "HV_out aliases V");
  cudaStream_t s = (cudaStream_t)stream;
  PSPEC_TRY(ensure_scratch(g, (size_t)g->n * k));
  EdgeLaunch L{U, V, HV_out, g->d_scratch, p, k};
  PSPEC_TRY(launch_hvp_edges(g, L, s));
  return copy_sums(g, sums_out, k, true, s);
}

extern "C" pspec_status pspec_hvp_finish(pspec_graph* g, const float* U, const float* V, int k, double p,
                                         const double* sums_in, float* HV_out, unsigned flags, void* stream) {
  PSPEC_TRY(check_shard_call(g, k, p, U, HV_out, "pspec_hvp_finish"));
  PSPEC_TRY(check_block(V, k, PSPEC_F32, "V"));
  if (!g->d_scratch || g->scratch_elems < (size_t)g->n * k)
    return set_error(PSPEC_ERR_INVALID_ARG, "pspec_hvp_finish without a pspec_hvp_partial before it");
  cudaStream_t s = (cudaStream_t)stream;
  PSPEC_TRY(finish_coefs(g, sums_in, k, p, true, (flags & PSPEC_HVP_ALG1) != 0, s));
  return run_hvp_epilogue(g, U, V, g->d_scratch, HV_out, k, p, s);
}
