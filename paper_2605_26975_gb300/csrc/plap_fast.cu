// FP32 fast path of pspec_eval / pspec_hvp: dispatch of the fused edge
// kernels by k, the two epilogues that turn row sums into the gradient and
// the Hessian-vector product, and the C entry points (which also route the
// FP64 plain form and host-pointer calls).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "epilogue.cuh"
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

template <int K, bool HVP>
pspec_status occupancy_k(int* blocks_per_sm, bool kept);

pspec_status edge_occupancy(int k, bool hvp, int* blocks_per_sm, bool kept) {
  switch (k) {
#define CASE(K) \
  case K:       \
    return hvp ? occupancy_k<K, true>(blocks_per_sm, kept) : occupancy_k<K, false>(blocks_per_sm, kept);
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

// grad = (p/D) Delta - (p lambda / D) phi_p(u), from the rows Delta into G
// (the same buffer: in place).
template <int VW>
__global__ void __launch_bounds__(256) grad_epilogue(const float* __restrict__ U, const float* Dl,
                                                     float* G, int64_t n_elems, int K,
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
      float4 t = *reinterpret_cast<const float4*>(Dl + v * VW);
      d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
    } else if constexpr (VW == 2) {
      float2 t = *reinterpret_cast<const float2*>(Dl + v * VW);
      d[0] = t.x; d[1] = t.y;
    } else {
      d[0] = Dl[v];
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
      const int cc = c + j;
      const HvpCoef cf{sA[cc], sL[cc], sB[cc], sSD[cc], sE[cc]};
      s[j] = hvp_entry(s[j], u[j], x[j], dl[j], cf, pm2, zero_rule);
    }
    store_vec<VW>(HV + v * VW, s);
  }
}

static int epi_blocks(pspec_graph* g, int64_t nvec) {
  int64_t want = (nvec + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)g->sm_count * 8));
}

static pspec_status ensure_delta_keep(pspec_graph* g, size_t elems) {
  if (g->delta_keep_elems >= elems) return PSPEC_OK;
  if (g->d_delta_keep) cudaFree(g->d_delta_keep);
  g->d_delta_keep = nullptr;
  g->delta_keep_elems = 0;
  g->keep_valid = false;
  if (cudaMalloc(&g->d_delta_keep, sizeof(float) * elems) != cudaSuccess) {
    cudaGetLastError();
    return set_error(PSPEC_ERR_OOM, "device allocation of the kept Delta_p u rows failed");
  }
  g->delta_keep_elems = elems;
  return PSPEC_OK;
}

pspec_status run_grad_epilogue(pspec_graph* g, const float* U, const float* Dl, float* grad, int k, double p,
                               cudaStream_t s) {
  const int64_t ne = g->n_owned * k;
  const float pm2 = (float)p - 2.0f;
  TimedScope timer(g, "grad_epilogue", s);
  if (k % 4 == 0)
    grad_epilogue<4><<<epi_blocks(g, ne / 4), 256, 0, s>>>(U, Dl, grad, ne, k, g->d_scalars, pm2);
  else if (k % 2 == 0)
    grad_epilogue<2><<<epi_blocks(g, ne / 2), 256, 0, s>>>(U, Dl, grad, ne, k, g->d_scalars, pm2);
  else
    grad_epilogue<1><<<epi_blocks(g, ne), 256, 0, s>>>(U, Dl, grad, ne, k, g->d_scalars, pm2);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

pspec_status run_hvp_epilogue(pspec_graph* g, const float* U, const float* V, const float* Dl, float* HV,
                              int k, double p, cudaStream_t s, const int* skip) {
  const int64_t ne = g->n_owned * k;
  const float pm2 = (float)p - 2.0f;
  TimedScope timer(g, "hvp_epilogue", s);
  if (k % 4 == 0)
    hvp_epilogue<4><<<epi_blocks(g, ne / 4), 256, 0, s>>>(U, V, Dl, HV, ne, k, g->d_scalars, pm2, skip);
  else if (k % 2 == 0)
    hvp_epilogue<2><<<epi_blocks(g, ne / 2), 256, 0, s>>>(U, V, Dl, HV, ne, k, g->d_scalars, pm2, skip);
  else
    hvp_epilogue<1><<<epi_blocks(g, ne), 256, 0, s>>>(U, V, Dl, HV, ne, k, g->d_scalars, pm2, skip);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

pspec_status eval_fast(pspec_graph* g, const float* U, int k, double p, double* F_out, float* grad,
                       double* parts, cudaStream_t s, bool keep_delta, float* keep_rows, double* keep_nd) {
  const int64_t ne = g->n_owned * k;
  float* Dl = grad;  // the edge kernel's Delta rows: in place over grad, or kept
  if (keep_delta && !keep_rows) {  // the handle's own kept point (PSPEC_KEEP_DELTA)
    PSPEC_TRY(ensure_delta_keep(g, (size_t)ne));
    keep_rows = g->d_delta_keep;
    keep_nd = g->d_scalars + kSlotKeep;
  }
  if (keep_delta) Dl = keep_rows;
  EdgeLaunch L{U, nullptr, Dl, nullptr, p, k};
  PSPEC_TRY(launch_eval_edges(g, L, s));
  PSPEC_TRY(run_grad_epilogue(g, U, Dl, grad, k, p, s));
  if (keep_delta)  // N[16], D[16] of this point, for the Hessian products that reuse its Delta
    PSPEC_CUDA(cudaMemcpyAsync(keep_nd, g->d_scalars + kSlotN, sizeof(double) * 32, cudaMemcpyDeviceToDevice, s));
  if (F_out)
    PSPEC_CUDA(cudaMemcpyAsync(F_out, g->d_scalars + kSlotF, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (parts) {
    PSPEC_CUDA(cudaMemcpyAsync(parts, g->d_scalars + kSlotN, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
    PSPEC_CUDA(cudaMemcpyAsync(parts + k, g->d_scalars + kSlotD, sizeof(double) * k, cudaMemcpyDeviceToDevice, s));
  }
  return PSPEC_OK;
}

pspec_status ensure_scratch(pspec_graph* g, size_t elems) {
  if (g->scratch_elems >= elems) return PSPEC_OK;
  if (g->d_scratch) cudaFree(g->d_scratch);
  g->d_scratch = nullptr;
  g->scratch_elems = 0;
  PSPEC_CUDA(cudaMalloc(&g->d_scratch, sizeof(float) * elems));
  g->scratch_elems = elems;
  return PSPEC_OK;
}

pspec_status hvp_edges_fast(pspec_graph* g, const float* U, const float* V, int k, double p, float* S,
                            cudaStream_t s, const int* skip, bool alg1) {
  PSPEC_TRY(ensure_scratch(g, (size_t)g->n * k));
  EdgeLaunch L{U, V, S, g->d_scratch, p, k, skip};
  L.alg1 = alg1;
  return launch_hvp_edges(g, L, s);
}

pspec_status hvp_kept_edges(pspec_graph* g, const float* U, const float* V, int k, double p, float* S,
                            const double* keep_nd, cudaStream_t s, const int* skip, bool alg1) {
  EdgeLaunch L{U, V, S, nullptr, p, k, skip};
  L.alg1 = alg1;
  L.keep_nd = keep_nd;
  return launch_hvp_edges(g, L, s);
}

pspec_status hvp_fast(pspec_graph* g, const float* U, const float* V, int k, double p, float* HV,
                      cudaStream_t s, const int* skip, bool alg1, bool delta_kept, const float* keep_rows,
                      const double* keep_nd) {
  const float* Dl;
  if (delta_kept) {  // Delta_p u, N and D of the evaluation at U: the edge kernel skips them
    if (!keep_rows) {  // the handle's own kept point (PSPEC_KEEP_DELTA)
      keep_rows = g->d_delta_keep;
      keep_nd = g->d_scalars + kSlotKeep;
    }
    PSPEC_TRY(hvp_kept_edges(g, U, V, k, p, HV, keep_nd, s, skip, alg1));
    Dl = keep_rows;
  } else {
    PSPEC_TRY(hvp_edges_fast(g, U, V, k, p, HV, s, skip, alg1));
    Dl = g->d_scratch;
  }
  return run_hvp_epilogue(g, U, V, Dl, HV, k, p, s, skip);
}

// ------------------------------------------------------------- batches ---
// One block per graph: the graph's task slots (contiguous) summed in a fixed
// order -- each thread a compensated FP32 sum over every (blockDim/NV)-th
// task, then a float-float tree -- and the graph's FP64 scalars and epilogue
// coefficients written to gs[graph].
__global__ void __launch_bounds__(256) batch_reduce(const float* __restrict__ part,
                                                    const int32_t* __restrict__ graph_task, int K,
                                                    int NQ, double p, bool alg1, double* gs,
                                                    int* status) {
  __shared__ float2 s_part[256];
  __shared__ double s_tot[64];
  const int G = blockIdx.x;
  const int NV = NQ * K;
  const int parts = blockDim.x / NV;
  const int v = threadIdx.x % NV, j = threadIdx.x / NV;
  const int t0 = graph_task[G], t1 = graph_task[G + 1];
  Kahan acc;
  acc.init();
  if (j < parts) {
    // eight slots' loads in flight at a time, added in slot order
    int t = t0 + j;
    for (; t + 7 * parts < t1; t += 8 * parts) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = __ldg(&part[(size_t)(t + u * parts) * NV + v]);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc.add(x[u]);
    }
    for (; t < t1; t += parts) acc.add(part[(size_t)t * NV + v]);
  }
  s_part[threadIdx.x] = kahan_to_ff(acc);
  __syncthreads();
  if (threadIdx.x < NV) {
    float2 tot = make_float2(0.f, 0.f);
    for (int q = 0; q < parts; ++q) tot = ff_add(tot, s_part[q * NV + threadIdx.x]);
    s_tot[threadIdx.x] = ff_to_double(tot);
  }
  __syncthreads();
  double* g = gs + (size_t)G * kGsStride;
  if (threadIdx.x < K) {
    const int c = threadIdx.x;
    const double N = 0.5 * s_tot[c], D = s_tot[K + c];
    const double lam = N / D;
    g[kGsN + c] = N;
    g[kGsD + c] = D;
    int flags = 0;
    if (!isfinite(N) || !isfinite(D)) flags |= kStatusNonFinite;
    else if (!(D > 0.0)) flags |= kStatusZeroColumn;
    if (NQ == 4) {
      const double sN = s_tot[2 * K + c], sD = s_tot[3 * K + c];
      g[kGsC0 + c] = p * (p - 1.0) / D;
      g[kGsC1 + c] = lam;
      g[kGsC2 + c] = alg1 ? 0.0 : p * p / (D * D);
      g[kGsC3 + c] = sD;
      g[kGsC4 + c] = sN - 2.0 * lam * sD;
    } else {
      g[kGsC0 + c] = p / D;
      g[kGsC1 + c] = p * lam / D;
    }
    if (flags) atomicOr(status, flags);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int c = 0; c < K; ++c) F += g[kGsN + c] / g[kGsD + c];
    g[kGsF] = F;
  }
}

// gradient epilogue of a batch: the row's graph picks the coefficients
template <int VW>
__global__ void __launch_bounds__(256) grad_epilogue_b(const float* __restrict__ U, float* G,
                                                       int64_t n_elems, int K,
                                                       const int32_t* __restrict__ row_graph,
                                                       const double* __restrict__ gs, float pm2) {
  const int64_t nv = n_elems / VW;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = v * VW;
    const int64_t row = e0 / K;
    const int c = (int)(e0 - row * K);
    const double* g = gs + (size_t)__ldg(&row_graph[row]) * kGsStride;
    float u[VW], d[VW];
    load_vec<VW>(U + e0, u);
#pragma unroll
    for (int jj = 0; jj < VW; ++jj) d[jj] = G[e0 + jj];
#pragma unroll
    for (int jj = 0; jj < VW; ++jj) {
      const float phu = abs_pow_pm2_clamped(u[jj], pm2) * u[jj];
      d[jj] = (float)g[kGsC0 + c + jj] * d[jj] - (float)g[kGsC1 + c + jj] * phu;
    }
    store_vec<VW>(G + e0, d);
  }
}

template <int VW>
__global__ void __launch_bounds__(256) hvp_epilogue_b(const float* __restrict__ U,
                                                      const float* __restrict__ V,
                                                      const float* __restrict__ Dl, float* HV,
                                                      int64_t n_elems, int K,
                                                      const int32_t* __restrict__ row_graph,
                                                      const double* __restrict__ gs, float pm2) {
  const bool zero_rule = pm2 != 0.0f;
  const int64_t nv = n_elems / VW;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = v * VW;
    const int64_t row = e0 / K;
    const int c = (int)(e0 - row * K);
    const double* g = gs + (size_t)__ldg(&row_graph[row]) * kGsStride;
    float u[VW], x[VW], dl[VW], sv[VW];
    load_vec<VW>(U + e0, u);
    load_vec<VW>(V + e0, x);
    load_vec<VW>(Dl + e0, dl);
#pragma unroll
    for (int jj = 0; jj < VW; ++jj) sv[jj] = HV[e0 + jj];
#pragma unroll
    for (int jj = 0; jj < VW; ++jj) {
      const int cc = c + jj;
      const HvpCoef cf{(float)g[kGsC0 + cc], (float)g[kGsC1 + cc], (float)g[kGsC2 + cc],
                       (float)g[kGsC3 + cc], (float)g[kGsC4 + cc]};
      sv[jj] = hvp_entry(sv[jj], u[jj], x[jj], dl[jj], cf, pm2, zero_rule);
    }
    store_vec<VW>(HV + e0, sv);
  }
}

static pspec_status ensure_task_part(pspec_graph* g, int k) {
  const int64_t nt = task_count(g, k);
  if (nt < 0) return set_error(PSPEC_ERR_CUDA, "task partition");
  const size_t need = (size_t)std::max<int64_t>(1, nt) * 64;
  if (g->task_part_elems >= need) return PSPEC_OK;
  if (g->d_task_part) cudaFree(g->d_task_part);
  g->d_task_part = nullptr;
  g->task_part_elems = 0;
  PSPEC_CUDA(cudaMalloc(&g->d_task_part, sizeof(float) * need));
  g->task_part_elems = need;
  return PSPEC_OK;
}

static const int32_t* graph_task_of(pspec_graph* g, int k) {
  const int Q = q_of(k);
  return g->tasks[Q == 1 ? 0 : Q == 2 ? 1 : 2].d_graph_task;
}

pspec_status eval_batched(pspec_graph* g, const float* U, int k, double p, double* F_out, float* grad,
                          double* parts, cudaStream_t s) {
  PSPEC_TRY(ensure_task_part(g, k));
  EdgeLaunch L{U, nullptr, grad, nullptr, p, k, nullptr, g->d_task_part};
  PSPEC_TRY(launch_eval_edges(g, L, s));
  const int G = g->n_graphs;
  {
    TimedScope timer(g, "batch_reduce", s);
    batch_reduce<<<G, 256, 0, s>>>(g->d_task_part, graph_task_of(g, k), k, 2, p, false,
                                   g->d_graph_scalars, g->d_status);
    PSPEC_CUDA(cudaGetLastError());
  }
  const int64_t ne = g->n * k;
  const float pm2 = (float)p - 2.0f;
  {
    TimedScope timer(g, "grad_epilogue", s);
    if (k % 4 == 0)
      grad_epilogue_b<4><<<epi_blocks(g, ne / 4), 256, 0, s>>>(U, grad, ne, k, g->d_row_graph, g->d_graph_scalars, pm2);
    else if (k % 2 == 0)
      grad_epilogue_b<2><<<epi_blocks(g, ne / 2), 256, 0, s>>>(U, grad, ne, k, g->d_row_graph, g->d_graph_scalars, pm2);
    else
      grad_epilogue_b<1><<<epi_blocks(g, ne), 256, 0, s>>>(U, grad, ne, k, g->d_row_graph, g->d_graph_scalars, pm2);
    PSPEC_CUDA(cudaGetLastError());
  }
  const size_t pitch = sizeof(double) * kGsStride;
  if (F_out)
    PSPEC_CUDA(cudaMemcpy2DAsync(F_out, sizeof(double), g->d_graph_scalars + kGsF, pitch, sizeof(double), G,
                                 cudaMemcpyDeviceToDevice, s));
  if (parts) {
    PSPEC_CUDA(cudaMemcpy2DAsync(parts, sizeof(double) * 2 * k, g->d_graph_scalars + kGsN, pitch,
                                 sizeof(double) * k, G, cudaMemcpyDeviceToDevice, s));
    PSPEC_CUDA(cudaMemcpy2DAsync(parts + k, sizeof(double) * 2 * k, g->d_graph_scalars + kGsD, pitch,
                                 sizeof(double) * k, G, cudaMemcpyDeviceToDevice, s));
  }
  return PSPEC_OK;
}

pspec_status hvp_batched(pspec_graph* g, const float* U, const float* V, int k, double p, float* HV,
                         cudaStream_t s, bool alg1) {
  const int64_t ne = g->n * k;
  PSPEC_TRY(ensure_scratch(g, (size_t)ne));
  PSPEC_TRY(ensure_task_part(g, k));
  EdgeLaunch L{U, V, HV, g->d_scratch, p, k, nullptr, g->d_task_part};
  PSPEC_TRY(launch_hvp_edges(g, L, s));
  {
    TimedScope timer(g, "batch_reduce", s);
    batch_reduce<<<g->n_graphs, 256, 0, s>>>(g->d_task_part, graph_task_of(g, k), k, 4, p, alg1,
                                             g->d_graph_scalars, g->d_status);
    PSPEC_CUDA(cudaGetLastError());
  }
  const float pm2 = (float)p - 2.0f;
  TimedScope timer(g, "hvp_epilogue", s);
  if (k % 4 == 0)
    hvp_epilogue_b<4><<<epi_blocks(g, ne / 4), 256, 0, s>>>(U, V, g->d_scratch, HV, ne, k, g->d_row_graph, g->d_graph_scalars, pm2);
  else if (k % 2 == 0)
    hvp_epilogue_b<2><<<epi_blocks(g, ne / 2), 256, 0, s>>>(U, V, g->d_scratch, HV, ne, k, g->d_row_graph, g->d_graph_scalars, pm2);
  else
    hvp_epilogue_b<1><<<epi_blocks(g, ne), 256, 0, s>>>(U, V, g->d_scratch, HV, ne, k, g->d_row_graph, g->d_graph_scalars, pm2);
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
  if (g->is_shard)
    return set_error(PSPEC_ERR_INVALID_ARG, "a shard handle takes pspec_eval_partial / pspec_eval_finish");
  if (dtype != PSPEC_F32 && dtype != PSPEC_F64) return set_error(PSPEC_ERR_INVALID_ARG, "bad dtype");
  if (g->n_graphs != 1 && dtype != PSPEC_F32)
    return set_error(PSPEC_ERR_INVALID_ARG, "batched graphs run the FP32 path");
  if ((flags & PSPEC_KEEP_DELTA) && (g->n_graphs != 1 || dtype != PSPEC_F32))
    return set_error(PSPEC_ERR_INVALID_ARG, "PSPEC_KEEP_DELTA needs an FP32 call on a single graph");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)g->n * k * elem_size(dtype);
  const void* dU = U;
  void* dG = grad_out;
  double* dF = F_out;
  double* dP = parts_out;
  const int G = g->n_graphs;
  if (flags & PSPEC_HOST_PTRS) {
    if (!U || !grad_out) return set_error(PSPEC_ERR_INVALID_ARG, "U or grad_out is NULL");
    const size_t ab = align_up(bytes);
    // with PSPEC_KEEP_DELTA the staging area is sized for the Hessian
    // products that follow (U, V, HV), so U's device copy stays where they
    // look for it
    size_t need = 2 * ab + 256 + 8 * (size_t)G * (1 + 2 * kMaxK);
    if (flags & PSPEC_KEEP_DELTA) need = std::max(need, 3 * ab);
    PSPEC_TRY(ensure_io(g, need));
    g->io_u_kept = false;
    char* base = (char*)g->d_io;
    dU = base;
    dG = base + ab;
    dF = (double*)(base + 2 * ab);
    dP = dF + G;
    PSPEC_CUDA(cudaMemcpyAsync((void*)dU, U, bytes, cudaMemcpyHostToDevice, s));
  } else {
    PSPEC_TRY(check_block(U, k, dtype, "U"));
    PSPEC_TRY(check_block(grad_out, k, dtype, "grad_out"));
    if (U == grad_out) return set_error(PSPEC_ERR_INVALID_ARG, "grad_out aliases U");
  }
  const bool keep = (flags & PSPEC_KEEP_DELTA) != 0;
  if (keep) g->keep_valid = false;  // until this call's rows are enqueued
  if (G > 1)
    PSPEC_TRY(eval_batched(g, (const float*)dU, k, p, dF, (float*)dG, dP, s));
  else if (dtype == PSPEC_F32)
    PSPEC_TRY(eval_fast(g, (const float*)dU, k, p, dF, (float*)dG, dP, s, keep));
  else
    PSPEC_TRY(eval_plain64(g, (const double*)dU, k, p, dF, (double*)dG, dP, s));
  if (keep) {
    g->keep_valid = true;
    g->io_u_kept = (flags & PSPEC_HOST_PTRS) != 0;  // the staged U is the kept point's
    g->keep_U = U;
    g->keep_host = flags & PSPEC_HOST_PTRS;
    g->keep_k = k;
    g->keep_p = p;
  }
  if (flags & PSPEC_HOST_PTRS) {
    PSPEC_CUDA(cudaMemcpyAsync(grad_out, dG, bytes, cudaMemcpyDeviceToHost, s));
    if (F_out) PSPEC_CUDA(cudaMemcpyAsync(F_out, dF, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
    if (parts_out)
      PSPEC_CUDA(cudaMemcpyAsync(parts_out, dP, sizeof(double) * 2 * k * G, cudaMemcpyDeviceToHost, s));
    return take_status(g, s);
  }
  return PSPEC_OK;
}

extern "C" pspec_status pspec_hvp(pspec_graph* g, const void* U, const void* V, int k, double p,
                                  pspec_dtype dtype, void* HV_out, unsigned flags, void* stream) {
  PSPEC_TRY(check_common(g, k, p));
  if (g->is_shard)
    return set_error(PSPEC_ERR_INVALID_ARG, "a shard handle takes pspec_hvp_partial / pspec_hvp_finish");
  if (dtype != PSPEC_F32 && dtype != PSPEC_F64) return set_error(PSPEC_ERR_INVALID_ARG, "bad dtype");
  if (g->n_graphs != 1 && dtype != PSPEC_F32)
    return set_error(PSPEC_ERR_INVALID_ARG, "batched graphs run the FP32 path");
  const bool kept = (flags & PSPEC_DELTA_KEPT) != 0;
  if (kept) {
    if (g->n_graphs != 1 || dtype != PSPEC_F32)
      return set_error(PSPEC_ERR_INVALID_ARG, "PSPEC_DELTA_KEPT needs an FP32 call on a single graph");
    if (!g->keep_valid || g->keep_U != U || g->keep_k != k || g->keep_p != p ||
        g->keep_host != (flags & PSPEC_HOST_PTRS))
      return set_error(PSPEC_ERR_INVALID_ARG,
                       "PSPEC_DELTA_KEPT: no Delta_p u kept for this U pointer, k and p "
                       "(call pspec_eval with PSPEC_KEEP_DELTA first)");
  }
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
    // at the kept point U's device copy is still staged (and unchanged, as
    // PSPEC_DELTA_KEPT promises), unless another host-pointer call used the area
    if (!(kept && g->io_u_kept))
      PSPEC_CUDA(cudaMemcpyAsync((void*)dU, U, bytes, cudaMemcpyHostToDevice, s));
    g->io_u_kept = kept;
    PSPEC_CUDA(cudaMemcpyAsync((void*)dV, V, bytes, cudaMemcpyHostToDevice, s));
  } else {
    PSPEC_TRY(check_block(U, k, dtype, "U"));
    PSPEC_TRY(check_block(V, k, dtype, "V"));
    PSPEC_TRY(check_block(HV_out, k, dtype, "HV_out"));
    if (HV_out == U || HV_out == V) return set_error(PSPEC_ERR_INVALID_ARG, "HV_out aliases an input");
  }
  const bool alg1 = (flags & PSPEC_HVP_ALG1) != 0;
  if (g->n_graphs > 1)
    PSPEC_TRY(hvp_batched(g, (const float*)dU, (const float*)dV, k, p, (float*)dH, s, alg1));
  else if (dtype == PSPEC_F32)
    PSPEC_TRY(hvp_fast(g, (const float*)dU, (const float*)dV, k, p, (float*)dH, s, nullptr, alg1, kept));
  else
    PSPEC_TRY(hvp_plain64(g, (const double*)dU, (const double*)dV, k, p, (double*)dH, s, alg1));
  if (flags & PSPEC_HOST_PTRS) {
    PSPEC_CUDA(cudaMemcpyAsync(HV_out, dH, bytes, cudaMemcpyDeviceToHost, s));
    return take_status(g, s);
  }
  return PSPEC_OK;
}
