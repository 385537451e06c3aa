// Plain FP64 form of the method on the GPU: one thread per row, one column
// per launch (the loop over columns of Algorithm 1), double precision
// throughout with the CUDA math library's pow().  It is the baseline the
// FP32 fused path is measured against and the precision reference on the
// device.  Reductions are block trees plus the same two-level, ticket-ordered
// grid reduction as the fast path, in double.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace pspec {

constexpr int kPlainBlock = 256;

struct GridReduce64 {
  double* block_part;  // [gridDim][NV]
  double* group_part;  // [groups][NV]
  unsigned* counters;
};

template <int NV>
__device__ bool grid_reduce_f64(const double* mine, double* total, const GridReduce64& gr) {
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  const int nblk = gridDim.x;
  const int ngroups = (nblk + kGroup - 1) / kGroup;
  const int g = blockIdx.x / kGroup;
  if (tid < NV) gr.block_part[(size_t)blockIdx.x * NV + tid] = mine[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    int gsize = min(kGroup, nblk - g * kGroup);
    unsigned t = atomicAdd(&gr.counters[g], 1u);
    s_flag = (t == (unsigned)(gsize - 1));
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  if (tid < NV) {
    double acc = 0.0;
    int b0 = g * kGroup, b1 = min(nblk, b0 + kGroup);
    for (int b = b0; b < b1; ++b) acc += __ldcg(&gr.block_part[(size_t)b * NV + tid]);
    gr.group_part[(size_t)g * NV + tid] = acc;
  }
  if (tid == 0) gr.counters[g] = 0u;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned t = atomicAdd(&gr.counters[ngroups], 1u);
    s_flag = (t == (unsigned)(ngroups - 1));
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  if (tid < NV) {
    double acc = 0.0;
    for (int q = 0; q < ngroups; ++q) acc += __ldcg(&gr.group_part[(size_t)q * NV + tid]);
    total[tid] = acc;
  }
  if (tid == 0) gr.counters[ngroups] = 0u;
  __syncthreads();
  return true;
}

template <int NV>
__device__ void block_sum_f64(double (&v)[NV], double* out) {
  __shared__ double s[NV][kPlainBlock];
#pragma unroll
  for (int q = 0; q < NV; ++q) s[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int h = kPlainBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
#pragma unroll
      for (int q = 0; q < NV; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x < NV) out[threadIdx.x] = s[threadIdx.x][0];
  __syncthreads();
}

__device__ __forceinline__ double phi64(double x, double p) {
  return x == 0.0 ? 0.0 : copysign(pow(fabs(x), p - 1.0), x);
}
// |x|^(p-2), 0 at x == 0 for p < 2 (zero-curvature reading), 1 at p == 2
__device__ __forceinline__ double apm2_64(double x, double p) {
  if (p == 2.0) return 1.0;
  return x == 0.0 ? 0.0 : pow(fabs(x), p - 2.0);
}

struct PlainArgs {
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
  const double* U;
  const double* V;
  double* out_a;  // eval: Delta into grad; hvp: S into HV
  double* out_b;  // hvp: Delta scratch
  int64_t n;
  int k;
  int l;
  double p;
  int alg1;  // HVP in Algorithm 1's form: no rank-two coefficient
  GridReduce64 gr;
  double* scalars;
  int* status;
};

template <bool HVP>
__global__ void __launch_bounds__(kPlainBlock) plain_col_kernel(PlainArgs a) {
  constexpr int NV = HVP ? 4 : 2;
  __shared__ double s_blk[NV], s_tot[NV];
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  const int k = a.k, l = a.l;
  const double p = a.p;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ui = a.U[i * k + l];
    const double vi = HVP ? a.V[i * k + l] : 0.0;
    double delta = 0.0, nn = 0.0, ss = 0.0;
    for (int64_t e = a.rowptr[i]; e < a.rowptr[i + 1]; ++e) {
      const int64_t j = a.col[e];
      const double w = a.val[e];
      const double d = ui - a.U[j * k + l];
      delta += w * phi64(d, p);
      nn += w * pow(fabs(d), p);
      if (HVP) ss += w * apm2_64(d, p) * (vi - a.V[j * k + l]);
    }
    acc[0] += nn;
    acc[1] += pow(fabs(ui), p);
    if (HVP) {
      a.out_a[i * k + l] = ss;
      a.out_b[i * k + l] = delta;
      acc[2] += delta * vi;
      acc[3] += phi64(ui, p) * vi;
    } else {
      a.out_a[i * k + l] = delta;
    }
  }
  block_sum_f64<NV>(acc, s_blk);
  if (!grid_reduce_f64<NV>(s_blk, s_tot, a.gr)) return;
  if (threadIdx.x == 0) {
    const double N = 0.5 * s_tot[0], D = s_tot[1];
    double* sc = a.scalars;
    sc[kSlotN + l] = N;
    sc[kSlotD + l] = D;
    int flags = 0;
    if (!isfinite(N) || !isfinite(D)) flags |= kStatusNonFinite;
    else if (!(D > 0.0)) flags |= kStatusZeroColumn;
    const double lam = N / D;
    double* coef = sc + kSlotCoef;
    if (HVP) {
      sc[kSlotCN + l] = s_tot[2];
      sc[kSlotCD + l] = s_tot[3];
      coef[0 * 16 + l] = p * (p - 1.0) / D;
      coef[1 * 16 + l] = lam;
      coef[2 * 16 + l] = a.alg1 ? 0.0 : p * p / (D * D);
      coef[3 * 16 + l] = s_tot[3];
      coef[4 * 16 + l] = s_tot[2] - 2.0 * lam * s_tot[3];
    } else {
      coef[0 * 16 + l] = p / D;
      coef[1 * 16 + l] = p * lam / D;
    }
    if (l == k - 1) {
      double F = 0.0;
      for (int c = 0; c < k; ++c) F += sc[kSlotN + c] / sc[kSlotD + c];
      sc[kSlotF] = F;
    }
    if (flags) atomicOr(a.status, flags);
  }
}

__global__ void plain_grad_epilogue(const double* U, double* G, int64_t n_elems, int k,
                                    const double* scalars, double p) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % k);
    G[e] = scalars[kSlotCoef + c] * G[e] - scalars[kSlotCoef + 16 + c] * phi64(U[e], p);
  }
}

__global__ void plain_hvp_epilogue(const double* U, const double* V, const double* Dl, double* HV,
                                   int64_t n_elems, int k, const double* scalars, double p) {
  const double* cf = scalars + kSlotCoef;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % k);
    const double u = U[e];
    HV[e] = cf[c] * (HV[e] - cf[16 + c] * apm2_64(u, p) * V[e]) -
            cf[32 + c] * (Dl[e] * cf[48 + c] + phi64(u, p) * cf[64 + c]);
  }
}

static PlainArgs plain_args(pspec_graph* g, const double* U, const double* V, double* a_out,
                            double* b_out, int k, double p) {
  PlainArgs a;
  a.rowptr = g->d_rowptr;
  a.col = g->d_col;
  a.val = g->d_val64;
  a.U = U;
  a.V = V;
  a.out_a = a_out;
  a.out_b = b_out;
  a.n = g->n;
  a.k = k;
  a.l = 0;
  a.p = p;
  a.alg1 = 0;
  a.gr.block_part = g->d_red64;
  a.gr.group_part = g->d_red64 + (size_t)g->max_blocks * 64;
  a.gr.counters = g->d_counters;
  a.scalars = g->d_scalars;
  a.status = g->d_status;
  return a;
}

static int plain_blocks(pspec_graph* g) {
  int64_t want = (g->n + kPlainBlock - 1) / kPlainBlock;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)g->sm_count * 4));
}

pspec_status eval_plain64(pspec_graph* g, const double* U, int k, double p, double* F_out,
                          double* grad, double* parts, cudaStream_t s) {
  PlainArgs a = plain_args(g, U, nullptr, grad, nullptr, k, p);
  const int blocks = plain_blocks(g);
  for (int l = 0; l < k; ++l) {
    a.l = l;
    TimedScope timer(g, "plain64_eval_col", s);
    plain_col_kernel<false><<<blocks, kPlainBlock, 0, s>>>(a);
    PSPEC_CUDA(cudaGetLastError());
  }
  {
    TimedScope timer(g, "plain64_grad_epilogue", s);
    plain_grad_epilogue<<<g->sm_count * 4, 256, 0, s>>>(U, grad, g->n * k, k, g->d_scalars, p);
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

pspec_status hvp_plain64(pspec_graph* g, const double* U, const double* V, int k, double p,
                         double* HV, cudaStream_t s, bool alg1) {
  const size_t need = (size_t)g->n * k * 2;  // doubles stored in the float scratch
  if (g->scratch_elems < need) {
    if (g->d_scratch) cudaFree(g->d_scratch);
    g->d_scratch = nullptr;
    g->scratch_elems = 0;
    PSPEC_CUDA(cudaMalloc(&g->d_scratch, sizeof(float) * need));
    g->scratch_elems = need;
  }
  double* Dl = reinterpret_cast<double*>(g->d_scratch);
  PlainArgs a = plain_args(g, U, V, HV, Dl, k, p);
  a.alg1 = alg1 ? 1 : 0;
  const int blocks = plain_blocks(g);
  for (int l = 0; l < k; ++l) {
    a.l = l;
    TimedScope timer(g, "plain64_hvp_col", s);
    plain_col_kernel<true><<<blocks, kPlainBlock, 0, s>>>(a);
    PSPEC_CUDA(cudaGetLastError());
  }
  TimedScope timer(g, "plain64_hvp_epilogue", s);
  plain_hvp_epilogue<<<g->sm_count * 4, 256, 0, s>>>(U, V, Dl, HV, g->n * k, k, g->d_scalars, p);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

}  // namespace pspec
