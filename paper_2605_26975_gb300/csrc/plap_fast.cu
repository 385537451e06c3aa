// FP32 fast path of pspec_eval / pspec_hvp: dispatch of the fused edge
// kernels by k, the two epilogues that turn row sums into the gradient and
// the Hessian-vector product, and the C entry points (which also route the
// FP64 plain form and host-pointer calls).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace pspec {

template <int K, bool HVP>
pspec_status launch_edges_k(pspec_graph* g, const EdgeLaunch& L, cudaStream_t s);

template <bool HVP>
static pspec_status dispatch_edges(pspec_graph* g, const EdgeLaunch& L, cudaStream_t s) {
  switch (L.k) {
#define CASE(K) \
  case K:       \
    return launch_edges_k<K, HVP>(g, L, s);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
    default:
      return set_error(PSPEC_ERR_INVALID_ARG, "k must be in [1, 16]");
  }
}

pspec_status launch_eval_edges(pspec_graph* g, const EdgeLaunch& L, cudaStream_t s) {
  return dispatch_edges<false>(g, L, s);
}
pspec_status launch_hvp_edges(pspec_graph* g, const EdgeLaunch& L, cudaStream_t s) {
  return dispatch_edges<true>(g, L, s);
}

// grad = (p/D) Delta - (p lambda / D) phi_p(u), in place over Delta.
template <int VW>
__global__ void __launch_bounds__(256) grad_epilogue(const float* __restrict__ U, float* G,
                                                     int64_t n_elems, int K,
                                                     const double* __restrict__ scalars, float pm2) {
  __shared__ float sA[kMaxK], sB[kMaxK];
  if (threadIdx.x < K) {
    sA[threadIdx.x] = (float)scalars[kSlotCoef + threadIdx.x];
    sB[threadIdx.x] = (float)scalars[kSlotCoef + 16 + threadIdx.x];
  }
  __syncthreads();
  const int64_t nv = n_elems / VW;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    float u[VW], d[VW];
    load_vec<VW>(U + v * VW, u);
    if constexpr (VW == 4) {
      float4 t = *reinterpret_cast<const float4*>(G + v * VW);
      d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else if constexpr (VW == 2) {
      float2 t = *reinterpret_cast<const float2*>(G + v * VW);
      d[0] = t.x; d[1] = t.y;
    } else {
      d[0] = G[v];
    }
    const int c = (int)((v * VW) % K);
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      const float phu = abs_pow_pm2_clamped(u[j], pm2) * u[j];
      d[j] = sA[c + j] * d[j] - sB[c + j] * phu;
    }
    store_vec<VW>(G + v * VW, d);
  }
}

// HV = A (S - lambda s_u v) - B (Delta sigma_D + phi_p(u) E), in place over S.
template <int VW>
__global__ void __launch_bounds__(256) hvp_epilogue(const float* __restrict__ U,
                                                    const float* __restrict__ V,
                                                    const float* __restrict__ Dl, float* HV,
                                                    int64_t n_elems, int K,
                                                    const double* __restrict__ scalars, float pm2,
                                                    const int* skip) {
  if (skip && *skip) return;
  __shared__ float sA[kMaxK], sL[kMaxK], sB[kMaxK], sSD[kMaxK], sE[kMaxK];
  if (threadIdx.x < K) {
    const double* c = scalars + kSlotCoef;
    sA[threadIdx.x] = (float)c[threadIdx.x];
    sL[threadIdx.x] = (float)c[16 + threadIdx.x];
    sB[threadIdx.x] = (float)c[32 + threadIdx.x];
    sSD[threadIdx.x] = (float)c[48 + threadIdx.x];
    sE[threadIdx.x] = (float)c[64 + threadIdx.x];
  }
  __syncthreads();
  const bool zero_rule = pm2 != 0.0f;
  const int64_t nv = n_elems / VW;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    float u[VW], x[VW], dl[VW], s[VW];
    load_vec<VW>(U + v * VW, u);
    load_vec<VW>(V + v * VW, x);
    load_vec<VW>(Dl + v * VW, dl);
    if constexpr (VW == 4) {
      float4 t = *reinterpret_cast<const float4*>(HV + v * VW);
      s[0] = t.x; s[1] = t.y; s[2] = t.z; s[3] = t.w;
    } else if constexpr (VW == 2) {
      float2 t = *reinterpret_cast<const float2*>(HV + v * VW);
      s[0] = t.x; s[1] = t.y;
    } else {
      s[0] = HV[v];
    }
    const int c = (int)((v * VW) % K);
#pragma unroll
    for (int j = 0; j < VW; ++j) {
      float su = abs_pow_pm2_clamped(u[j], pm2);
      const float phu = su * u[j];
      if (zero_rule && u[j] == 0.0f) su = 0.0f;
      const int cc = c + j;
      s[j] = sA[cc] * (s[j] - sL[cc] * su * x[j]) - sB[cc] * (dl[j] * sSD[cc] + phu * sE[cc]);
    }
    store_vec<VW>(HV + v * VW, s);
  }
}

static int epi_blocks(pspec_graph* g, int64_t nvec) {
  int64_t want = (nvec + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)g->sm_count * 8));
}

pspec_status eval_fast(pspec_graph* g, const float* U, int k, double p, double* F_out, float* grad,
                       double* parts, cudaStream_t s) {
  EdgeLaunch L{U, nullptr, grad, nullptr, (float)p, k};
  PSPEC_TRY(launch_eval_edges(g, L, s));
  const int64_t ne = g->n * k;
  const float pm2 = (float)p - 2.0f;
  {
    TimedScope timer(g, "grad_epilogue", s);
    if (k % 4 == 0)
      grad_epilogue<4><<<epi_blocks(g, ne / 4), 256, 0, s>>>(U, grad, ne, k, g->d_scalars, pm2);
    else if (k % 2 == 0)
      grad_epilogue<2><<<epi_blocks(g, ne / 2), 256, 0, s>>>(U, grad, ne, k, g->d_scalars, pm2);
    else
      grad_epilogue<1><<<epi_blocks(g, ne), 256, 0, s>>>(U, grad, ne, k, g->d_scalars, pm2);
    PSPEC_CUDA(cudaGetLastError());
  }
  if (F_out)
    PSPEC_CUDA(cudaMemcpyAsync(F_out, g->d_scalars + kSlotF, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (parts) {
    PSPEC_CUDA(cudaMemcpyAsync(parts, g->d_scalars + kSlotN, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
    PSPEC_CUDA(cudaMemcpyAsync(parts + k, g->d_scalars + kSlotD, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
  }
  return PSPEC_OK;
}

static pspec_status ensure_scratch(pspec_graph* g, size_t elems) {
  if (g->scratch_elems >= elems) return PSPEC_OK;
  if (g->d_scratch) cudaFree(g->d_scratch);
  g->d_scratch = nullptr;
  g->scratch_elems = 0;
  PSPEC_CUDA(cudaMalloc(&g->d_scratch, sizeof(float) * elems));
  g->scratch_elems = elems;
  return PSPEC_OK;
}

pspec_status hvp_fast(pspec_graph* g, const float* U, const float* V, int k, double p, float* HV,
                      cudaStream_t s, const int* skip) {
  const int64_t ne = g->n * k;
  PSPEC_TRY(ensure_scratch(g, (size_t)ne));
  EdgeLaunch L{U, V, HV, g->d_scratch, (float)p, k, skip};
  PSPEC_TRY(launch_hvp_edges(g, L, s));
  const float pm2 = (float)p - 2.0f;
  TimedScope timer(g, "hvp_epilogue", s);
  if (k % 4 == 0)
    hvp_epilogue<4><<<epi_blocks(g, ne / 4), 256, 0, s>>>(U, V, g->d_scratch, HV, ne, k, g->d_scalars, pm2, skip);
  else if (k % 2 == 0)
    hvp_epilogue<2><<<epi_blocks(g, ne / 2), 256, 0, s>>>(U, V, g->d_scratch, HV, ne, k, g->d_scalars, pm2, skip);
  else
    hvp_epilogue<1><<<epi_blocks(g, ne), 256, 0, s>>>(U, V, g->d_scratch, HV, ne, k, g->d_scalars, pm2, skip);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

}  // namespace pspec

using namespace pspec;

static size_t elem_size(pspec_dtype t) { return t == PSPEC_F64 ? 8 : 4; }
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" pspec_status pspec_eval(pspec_graph* g, const void* U, int k, double p, pspec_dtype dtype,
                                   double* F_out, void* grad_out, double* parts_out, unsigned flags,
                                   void* stream) {
  PSPEC_TRY(check_common(g, k, p));
  if (dtype != PSPEC_F32 && dtype != PSPEC_F64) return set_error(PSPEC_ERR_INVALID_ARG, "bad dtype");
  if (g->n_graphs != 1) return set_error(PSPEC_ERR_INVALID_ARG, "batched graphs use pspec_eval_batched");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)g->n * k * elem_size(dtype);
  const void* dU = U;
  void* dG = grad_out;
  double* dF = F_out;
  double* dP = parts_out;
  if (flags & PSPEC_HOST_PTRS) {
    if (!U || !grad_out) return set_error(PSPEC_ERR_INVALID_ARG, "U or grad_out is NULL");
    const size_t ab = align_up(bytes);
    PSPEC_TRY(ensure_io(g, 2 * ab + 256 + 8 * 2 * kMaxK));
    char* base = (char*)g->d_io;
    dU = base;
    dG = base + ab;
    dF = (double*)(base + 2 * ab);
    dP = dF + 1;
    PSPEC_CUDA(cudaMemcpyAsync((void*)dU, U, bytes, cudaMemcpyHostToDevice, s));
  } else {
    PSPEC_TRY(check_block(U, k, dtype, "U"));
    PSPEC_TRY(check_block(grad_out, k, dtype, "grad_out"));
    if (U == grad_out) return set_error(PSPEC_ERR_INVALID_ARG, "grad_out aliases U");
  }
  if (dtype == PSPEC_F32)
    PSPEC_TRY(eval_fast(g, (const float*)dU, k, p, dF, (float*)dG, dP, s));
  else
    PSPEC_TRY(eval_plain64(g, (const double*)dU, k, p, dF, (double*)dG, dP, s));
  if (flags & PSPEC_HOST_PTRS) {
    PSPEC_CUDA(cudaMemcpyAsync(grad_out, dG, bytes, cudaMemcpyDeviceToHost, s));
    if (F_out) PSPEC_CUDA(cudaMemcpyAsync(F_out, dF, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (parts_out)
      PSPEC_CUDA(cudaMemcpyAsync(parts_out, dP, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
    return take_status(g, s);
  }
  return PSPEC_OK;
}

extern "C" pspec_status pspec_hvp(pspec_graph* g, const void* U, const void* V, int k, double p,
                                  pspec_dtype dtype, void* HV_out, unsigned flags, void* stream) {
  PSPEC_TRY(check_common(g, k, p));
  if (dtype != PSPEC_F32 && dtype != PSPEC_F64) return set_error(PSPEC_ERR_INVALID_ARG, "bad dtype");
  if (g->n_graphs != 1) return set_error(PSPEC_ERR_INVALID_ARG, "batched graphs use pspec_hvp_batched");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)g->n * k * elem_size(dtype);
  const void* dU = U;
  const void* dV = V;
  void* dH = HV_out;
  if (flags & PSPEC_HOST_PTRS) {
    if (!U || !V || !HV_out) return set_error(PSPEC_ERR_INVALID_ARG, "NULL block");
    const size_t ab = align_up(bytes);
    PSPEC_TRY(ensure_io(g, 3 * ab));
    char* base = (char*)g->d_io;
    dU = base;
    dV = base + ab;
    dH = base + 2 * ab;
    PSPEC_CUDA(cudaMemcpyAsync((void*)dU, U, bytes, cudaMemcpyHostToDevice, s));
    PSPEC_CUDA(cudaMemcpyAsync((void*)dV, V, bytes, cudaMemcpyHostToDevice, s));
  } else {
    PSPEC_TRY(check_block(U, k, dtype, "U"));
    PSPEC_TRY(check_block(V, k, dtype, "V"));
    PSPEC_TRY(check_block(HV_out, k, dtype, "HV_out"));
    if (HV_out == U || HV_out == V) return set_error(PSPEC_ERR_INVALID_ARG, "HV_out aliases an input");
  }
  if (dtype == PSPEC_F32)
    PSPEC_TRY(hvp_fast(g, (const float*)dU, (const float*)dV, k, p, (float*)dH, s));
  else
    PSPEC_TRY(hvp_plain64(g, (const double*)dU, (const double*)dV, k, p, (double*)dH, s));
  if (flags & PSPEC_HOST_PTRS) {
    PSPEC_CUDA(cudaMemcpyAsync(HV_out, dH, bytes, cudaMemcpyDeviceToHost, s));
    return take_status(g, s);
  }
  return PSPEC_OK;
}
