// RCut(C_1..C_c) = sum_c cut(C_c, complement C_c) / |C_c| (Section 3.1 of the
// paper), cut(C, C') = sum_{i in C, j in C'} w_ij over both stored triangles,
// so an edge between two clusters counts in both of their cuts.  Empty
// clusters contribute nothing.  FP64, fixed-order reductions.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pspec {

constexpr int kRcBlock = 256;
constexpr int kRcMaxC = 1024;

// per row: w-sum of entries leaving the row's cluster (warp per row)
__global__ void rc_row_cut(const int64_t* rowptr, const int32_t* col, const double* val,
                           const int32_t* labels, int64_t n, double* row_cut) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const int li = labels[i];
    double acc = 0.0;
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32)
      if (labels[col[e]] != li) acc += val[e];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) row_cut[i] = acc;
  }
}

// block (c, s): cut and size of cluster c over row segment s
__global__ void rc_cluster(const double* row_cut, const int32_t* labels, int64_t n, int nseg,
                           double* part) {
  __shared__ double sc[kRcBlock], sn[kRcBlock];
  const int c = blockIdx.x / nseg, sgm = blockIdx.x % nseg;
  const int64_t per = (n + nseg - 1) / nseg;
  const int64_t b0 = sgm * per, b1 = min(n, b0 + per);
  double cut = 0.0, cnt = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x)
    if (labels[i] == c) {
      cut += row_cut[i];
      cnt += 1.0;
    }
  sc[threadIdx.x] = cut;
  sn[threadIdx.x] = cnt;
  __syncthreads();
  for (int h = kRcBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sc[threadIdx.x] += sc[threadIdx.x + h];
      sn[threadIdx.x] += sn[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * (size_t)blockIdx.x] = sc[0];
    part[2 * (size_t)blockIdx.x + 1] = sn[0];
  }
}

__global__ void rc_final(const double* part, int C, int nseg, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r = 0.0;
  for (int c = 0; c < C; ++c) {
    double cut = 0.0, cnt = 0.0;
    for (int s = 0; s < nseg; ++s) {
      cut += part[2 * ((size_t)c * nseg + s)];
      cnt += part[2 * ((size_t)c * nseg + s) + 1];
    }
    if (cnt > 0.0) r += cut / cnt;
  }
  *out = r;
}

__global__ void rc_check_labels(const int32_t* labels, int64_t n, int C, int* bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (labels[i] < 0 || labels[i] >= C) atomicOr(bad, 1);
}

pspec_status rcut_impl(pspec_graph* g, const int32_t* labels, int C, double* out, cudaStream_t s) {
  const int64_t n = g->n;
  const int nseg = (int)std::max<int64_t>(1, std::min<int64_t>(64, (n + 65535) / 65536));
  char* mem = nullptr;
  const size_t bytes = sizeof(double) * ((size_t)n + 2 * (size_t)C * nseg + 2) + 256;
  PSPEC_CUDA(cudaMallocAsync((void**)&mem, bytes, s));
  double* row_cut = (double*)mem;
  double* part = row_cut + n;
  double* res = part + 2 * (size_t)C * nseg;
  int* bad = (int*)(res + 1);
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * 8, (n + 255) / 256));
  rc_check_labels<<<blocks, 256, 0, s>>>(labels, n, C, bad);
  int hbad = 0;
  cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, s);
    return cuda_error(e, "rcut");
  }
  if (hbad) {
    cudaFreeAsync(mem, s);
    cudaStreamSynchronize(s);
    return set_error(PSPEC_ERR_INVALID_ARG, "a label is outside [0, n_clusters)");
  }
  {
    TimedScope timer(g, "rcut_rows", s);
    const int rb = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * 8, (n * 32 + 255) / 256));
    rc_row_cut<<<rb, 256, 0, s>>>(g->d_rowptr, g->d_col, g->d_val64, labels, n, row_cut);
  }
  rc_cluster<<<C * nseg, kRcBlock, 0, s>>>(row_cut, labels, n, nseg, part);
  rc_final<<<1, 1, 0, s>>>(part, C, nseg, res);
  cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(mem, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "rcut");
  return PSPEC_OK;
}

}  // namespace pspec

using namespace pspec;

extern "C" pspec_status pspec_rcut(pspec_graph* g, const int32_t* labels, int n_clusters,
                                   double* rcut_out, void* stream) {
  if (!g || !labels || !rcut_out) return set_error(PSPEC_ERR_INVALID_ARG, "NULL argument");
  if (n_clusters < 1 || n_clusters > kRcMaxC) return set_error(PSPEC_ERR_INVALID_ARG, "n_clusters must be in [1, 1024]");
  if (g->n_graphs != 1) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_rcut takes a single graph");
  if (g->is_shard) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_rcut takes a whole graph, not a shard");
  return rcut_impl(g, labels, n_clusters, rcut_out, (cudaStream_t)stream);
}
