// k-means discretisation of the final U (the paper discretises its
// eigenvector estimates with k-means, Sections 1-2, without further detail).
//
// Reading implemented (same as the CPU oracle's):
//  * k-means++ seeding: first centre = row floor(u n); every further centre is
//    the first row i whose running sum of D^2 exceeds u * sum D^2, D^2 the
//    squared distance to the nearest chosen centre;
//  * uniforms u from SplitMix64(seed): state += 0x9E3779B97F4A7C15, output
//    mix with shifts 30/27/31 and multipliers 0xBF58476D1CE4E5B9 /
//    0x94D049BB133111EB, u = (x >> 11) * 2^-53, one stream per call consumed
//    in order across restarts;
//  * squared distances in FP64, accumulated dimension by dimension, each
//    subtraction, product and sum rounded once (no fused multiply-add), so
//    the nearest-centre decision is taken exactly as the oracle takes it;
//  * Lloyd: assign (ties -> smallest centre), update to means, an empty
//    cluster re-seeded (in cluster order) at the row farthest from its
//    centre, stop when no label changes or after max_iter updates;
//  * restarts: the smallest inertia wins (the first on ties).
// All reductions have a fixed order; only integer counters use atomics.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace pspec {

constexpr int kKmMaxC = 64;
constexpr int kKmMaxDim = 16;
constexpr int kKmBlock = 256;

struct SplitMix64 {
  uint64_t state;
  explicit SplitMix64(uint64_t s) : state(s) {}
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

template <typename T>
__device__ __forceinline__ double sqdist_row(const T* x, const double* mu, int dim) {
  double acc = 0.0;
  for (int j = 0; j < dim; ++j) {
    const double t = __dsub_rn((double)x[j], mu[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

// centre c <- row *idx of X (the index a kernel left in device memory)
template <typename T>
__global__ void km_take_row_at(const T* X, int dim, const int64_t* idx, double* centers, int c) {
  if (threadIdx.x < dim) centers[c * dim + threadIdx.x] = (double)X[(*idx) * dim + threadIdx.x];
}

// centre c <- row idx of X
template <typename T>
__global__ void km_take_row(const T* X, int dim, int64_t idx, double* centers, int c) {
  if (threadIdx.x < dim) centers[c * dim + threadIdx.x] = (double)X[idx * dim + threadIdx.x];
}

// d2[i] = dist(X_i, centre c) (first) or min(d2[i], dist) ; block sums of d2
template <typename T>
__global__ void __launch_bounds__(kKmBlock) km_seed_dist(const T* X, int64_t n, int dim,
                                                         const double* centers, int c, int first,
                                                         double* d2, double* block_sum) {
  __shared__ double mu[kKmMaxDim];
  __shared__ double s[kKmBlock];
  if (threadIdx.x < dim) mu[threadIdx.x] = centers[c * dim + threadIdx.x];
  __syncthreads();
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  double acc = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    double d = sqdist_row(X + i * dim, mu, dim);
    if (!first) d = fmin(d, d2[i]);
    d2[i] = d;
    acc += d;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kKmBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sum[blockIdx.x] = s[0];
}

// first index whose running D^2 sum exceeds u * total (one block of
// kKmBlock threads).  Thread 0 runs over the block sums to the block the
// target falls in; from that block's first row the walk goes on in windows of
// kKmBlock chunks of kPickChunk rows: the threads sum their chunks, thread 0
// adds the chunk sums in order and walks the one chunk the target falls in
// row by row.
constexpr int kPickChunk = 32;

// Lloyd iterations between two host checks of convergence
constexpr int kKmCheckEvery = 8;

__global__ void __launch_bounds__(kKmBlock) km_pick(const double* d2, const double* block_sum,
                                                    int nblocks, int64_t n, double u,
                                                    int64_t* out_idx) {
  __shared__ double csum[kKmBlock];
  __shared__ double s_run, s_target;
  __shared__ int64_t s_i0, s_found;
  const int t = threadIdx.x;
  if (t == 0) {
    double total = 0.0;
    for (int b = 0; b < nblocks; ++b) total += block_sum[b];
    s_found = -1;
    if (total > 0.0) {
      const double target = u * total;
      const int64_t per = (n + nblocks - 1) / nblocks;
      double run = 0.0;
      int b = 0;
      while (b < nblocks - 1 && run + block_sum[b] <= target) run += block_sum[b++];
      s_run = run;
      s_target = target;
      s_i0 = (int64_t)b * per;
    } else {
      s_found = min((int64_t)(u * (double)n), n - 1);
    }
  }
  __syncthreads();
  if (s_found >= 0) {
    if (t == 0) *out_idx = s_found;
    return;
  }
  // the walk may run past the block when the block's tree sum and the
  // running sum round differently
  for (int64_t w0 = s_i0; w0 < n; w0 += (int64_t)kKmBlock * kPickChunk) {
    const int64_t c0 = w0 + (int64_t)t * kPickChunk;
    double cs = 0.0;
    for (int q = 0; q < kPickChunk; ++q)
      if (c0 + q < n) cs += d2[c0 + q];
    csum[t] = cs;
    __syncthreads();
    if (t == 0) {
      double run = s_run;
      for (int c = 0; c < kKmBlock && s_found < 0; ++c) {
        const int64_t r0 = w0 + (int64_t)c * kPickChunk;
        if (r0 >= n) break;
        if (run + csum[c] > s_target) {  // the target is in this chunk: walk it
          // (when rounding says otherwise, the walk goes on in the next chunk)
          for (int q = 0; q < kPickChunk && r0 + q < n; ++q) {
            run += d2[r0 + q];
            if (run > s_target) {
              s_found = r0 + q;
              break;
            }
          }
        } else {
          run += csum[c];
        }
      }
      s_run = run;
    }
    __syncthreads();
    if (s_found >= 0) break;
  }
  if (t == 0) *out_idx = s_found >= 0 ? s_found : n - 1;
}

// labels[i] = argmin_c dist(X_i, mu_c); dmin[i] = that distance; count changes
//
// The decision is the FP64 one (each subtraction, product and sum rounded
// once, ties to the smaller centre).  For FP32 rows it is screened in FP32:
// with u = 2^-24, t_j = fl32(x_j - fl32(mu_j)) differs from a_j = x_j - mu_j by
// at most u'(|a_j| + |mu_j|), u' = u(1+u), and the FP32 sum of the t_j^2 from
// sum a_j^2 by at most
//   (2u' + u + gamma_{dim-1}(1+u) + 2u'^2) d + 2u' |mu| sqrt(d) + 2u'^2 |mu|^2
// (Cauchy-Schwarz on sum |a_j||mu_j|), while the FP64 distance is within
// (dim+2) 2^-53 d of sum a_j^2.  E(c) below is twice the sum of both bounds
// (the factor covers using the computed d32 for d).  When the FP32 winner's
// d32 + E stays below every other centre's d32 - E, the FP64 decision is the
// same centre, and only its FP64 distance is computed; a row that is too
// close to call runs the full FP64 loop.
template <typename T>
__device__ __forceinline__ double km_dist64(const T* xr, const double* mu, int dim) {
  double acc = 0.0;
  for (int j = 0; j < dim; ++j) {
    const double t = __dsub_rn((double)xr[j], mu[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

template <typename T>
__global__ void __launch_bounds__(kKmBlock) km_assign(const T* X, int64_t n, int dim, int C,
                                                      const double* centers, int32_t* labels,
                                                      double* dmin, unsigned* changed,
                                                      const unsigned* done) {
  if (*done) return;
  __shared__ double mu[kKmMaxC * kKmMaxDim];
  __shared__ float mu32[kKmMaxC * kKmMaxDim];
  __shared__ float nmu[kKmMaxC];  // |mu_c|, rounded up
  for (int t = threadIdx.x; t < C * dim; t += blockDim.x) {
    mu[t] = centers[t];
    mu32[t] = (float)centers[t];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double q = 0.0;
    for (int j = 0; j < dim; ++j) q += mu[c * dim + j] * mu[c * dim + j];
    nmu[c] = (float)(sqrt(q) * (1.0 + 1e-6));
  }
  __syncthreads();
  constexpr float u = 5.9604645e-8f;  // 2^-24
  const float k_rel = 2.0f * u * (float)(dim + 3) + 2.0f * (float)(dim + 2) * 1.1102230e-16f;
  unsigned local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T xr[kKmMaxDim];
    for (int j = 0; j < dim; ++j) xr[j] = X[i * dim + j];
    int arg = -1;
    if constexpr (sizeof(T) == 4) {
      float best_hi = 0.f, best_d = 0.f;  // winner's d32 + E and d32
      int c1 = 0;
      float lo1 = 3.4e38f, lo2 = 3.4e38f;  // two smallest d32 - E ...
      int lo1c = -1;                       // ... and the centre of the smallest
      for (int c = 0; c < C; ++c) {
        float d = 0.f;
        for (int j = 0; j < dim; ++j) {
          const float t = xr[j] - mu32[c * dim + j];
          d = fmaf(t, t, d);
        }
        const float e = 2.0f * (k_rel * d + 2.1f * u * nmu[c] * sqrtf(d) + 3.0f * u * u * nmu[c] * nmu[c]);
        if (c == 0 || d < best_d) { best_d = d; best_hi = d + e; c1 = c; }
        const float lo = d - e;
        if (lo < lo1) { lo2 = lo1; lo1 = lo; lo1c = c; }
        else if (lo < lo2) lo2 = lo;
      }
      const float others_lo = (lo1c == c1) ? lo2 : lo1;
      if (best_hi < others_lo) arg = c1;  // separated: the FP64 decision is c1
    }
    double best;
    if (arg >= 0) {
      best = km_dist64(xr, mu + arg * dim, dim);
    } else {
      best = 0.0;
      arg = 0;
      for (int c = 0; c < C; ++c) {
        const double acc = km_dist64(xr, mu + c * dim, dim);
        if (c == 0 || acc < best) { best = acc; arg = c; }
      }
    }
    if (labels[i] != arg) ++local;
    labels[i] = arg;
    dmin[i] = best;
  }
  if (local) atomicAdd(changed, local);
}

// per-block, per-cluster sums of member rows and counts (fixed order):
// warp w owns clusters w, w+8, ...; its lanes stride the block's rows
template <typename T>
__global__ void __launch_bounds__(kKmBlock) km_partial(const T* X, int64_t n, int dim, int C,
                                                       const int32_t* labels, double* part,
                                                       const unsigned* done) {
  if (*done) return;
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* out = part + (size_t)blockIdx.x * C * (dim + 1);
  for (int c = w; c < C; c += kKmBlock / 32) {
    double acc[kKmMaxDim + 1];
    for (int j = 0; j <= dim; ++j) acc[j] = 0.0;
    for (int64_t i = b0 + lane; i < b1; i += 32) {
      if (labels[i] == c) {
        for (int j = 0; j < dim; ++j) acc[j] += (double)X[i * dim + j];
        acc[dim] += 1.0;
      }
    }
    for (int j = 0; j <= dim; ++j) {
      double v = acc[j];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) out[c * (dim + 1) + j] = v;
    }
  }
}

// centres = sums / counts (blocks summed in order); counts to host-visible array
__global__ void km_finish(const double* part, int nblocks, int C, int dim, double* centers,
                          double* counts, const unsigned* done) {
  if (*done) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C * (dim + 1)) return;
  double acc = 0.0;
  for (int b = 0; b < nblocks; ++b) acc += part[(size_t)b * C * (dim + 1) + t];
  const int c = t / (dim + 1), j = t % (dim + 1);
  if (j == dim) {
    counts[c] = acc;
  } else {
    // the count of this cluster, summed in the same order
    double cnt = 0.0;
    for (int b = 0; b < nblocks; ++b) cnt += part[(size_t)b * C * (dim + 1) + c * (dim + 1) + dim];
    if (cnt > 0.0) centers[c * dim + j] = acc / cnt;
  }
}

// Empty clusters, in cluster order: each takes the row farthest from its own
// old centre (dmin, first maximum) as its centre, and that row is excluded
// from the next one (dmin = -1).  One block; returns at once when no cluster
// is empty.
template <typename T>
__global__ void km_reseed(const T* X, int64_t n, int dim, int C, const double* counts, double* dmin,
                          double* centers, const unsigned* done) {
  __shared__ double sv[kKmBlock];
  __shared__ int64_t si[kKmBlock];
  if (*done) return;
  for (int c = 0; c < C; ++c) {
    if (counts[c] != 0.0) continue;  // uniform over the block
    double bv = -1.0;
    int64_t bi = n;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double v = dmin[i];
      if (v > bv) { bv = v; bi = i; }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int h = kKmBlock / 2; h > 0; h >>= 1) {
      if (threadIdx.x < h) {
        const double ov = sv[threadIdx.x + h];
        const int64_t oi = si[threadIdx.x + h];
        if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
          sv[threadIdx.x] = ov;
          si[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    const int64_t far = si[0];
    if (far < n) {
      if (threadIdx.x < dim) centers[c * dim + threadIdx.x] = (double)X[far * dim + threadIdx.x];
      __syncthreads();
      if (threadIdx.x == 0) dmin[far] = -1.0;
    }
    __syncthreads();
  }
}

// end of a Lloyd iteration: an assignment that changed no label is a fixed
// point, and every later iteration leaves the state as it is (done = 1).
__global__ void km_mark(unsigned* changed, unsigned* done) {
  if (*done) return;
  if (*changed == 0) *done = 1;
  *changed = 0;
}

__global__ void km_sum(const double* v, int64_t n, double* out) {
  __shared__ double s[kKmBlock];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += v[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kKmBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

struct KmWork {
  double* d2;
  double* dmin;
  double* part;
  double* centers;
  double* best_centers;
  double* counts;
  int32_t* labels;
  int64_t* idx;
  unsigned* changed;  // [0] labels changed by the last assignment, [1] done
  double* scalar;
  int nblocks;
};

template <typename T>
static pspec_status kmeans_impl(const T* X, int64_t n, int dim, int C, uint64_t seed, int restarts,
                                int max_iter, int32_t* labels_out, double* centers_out,
                                double* inertia_out, cudaStream_t s) {
  KmWork w;
  w.nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (n + 4095) / 4096));
  const size_t part_elems = (size_t)w.nblocks * C * (dim + 1);
  char* mem = nullptr;
  const size_t bytes = sizeof(double) * (2 * (size_t)n + part_elems + 2 * C * dim + C + 4) +
                       sizeof(int32_t) * n + sizeof(int64_t) * 2 + sizeof(unsigned) * 2 + 1024;
  PSPEC_CUDA(cudaMallocAsync((void**)&mem, bytes, s));
  auto carve = [&](size_t b) {
    char* p = mem;
    mem += (b + 127) & ~(size_t)127;
    return p;
  };
  char* base = mem;
  w.d2 = (double*)carve(sizeof(double) * n);
  w.dmin = (double*)carve(sizeof(double) * n);
  w.part = (double*)carve(sizeof(double) * part_elems);
  w.centers = (double*)carve(sizeof(double) * C * dim);
  w.best_centers = (double*)carve(sizeof(double) * C * dim);
  w.counts = (double*)carve(sizeof(double) * C);
  w.scalar = (double*)carve(sizeof(double) * 2);
  w.labels = (int32_t*)carve(sizeof(int32_t) * n);
  w.idx = (int64_t*)carve(sizeof(int64_t) * 2);
  w.changed = (unsigned*)carve(sizeof(unsigned) * 2);
  SplitMix64 rng(seed);
  double best = INFINITY;
  pspec_status st = PSPEC_OK;
  const int ab = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (n + kKmBlock - 1) / kKmBlock));
  for (int r = 0; r < restarts && st == PSPEC_OK; ++r) {
    // ---- k-means++ seeding
    {
      const double u = rng.uniform();
      const int64_t first = std::min<int64_t>((int64_t)(u * (double)n), n - 1);
      km_take_row<T><<<1, 32, 0, s>>>(X, dim, first, w.centers, 0);
      km_seed_dist<T><<<w.nblocks, kKmBlock, 0, s>>>(X, n, dim, w.centers, 0, 1, w.d2, w.part);
      for (int c = 1; c < C; ++c) {
        const double uc = rng.uniform();
        km_pick<<<1, kKmBlock, 0, s>>>(w.d2, w.part, w.nblocks, n, uc, w.idx);
        km_take_row_at<T><<<1, 32, 0, s>>>(X, dim, w.idx, w.centers, c);
        km_seed_dist<T><<<w.nblocks, kKmBlock, 0, s>>>(X, n, dim, w.centers, c, 0, w.d2, w.part);
      }
    }
    if (st != PSPEC_OK) break;
    // ---- Lloyd.  The iterations run in chunks with one host check each: a
    // converged state is marked done on the device and the rest of the chunk
    // skips, so the result is the one of checking after every iteration.
    cudaMemsetAsync(w.labels, 0xff, sizeof(int32_t) * n, s);  // -1: every label "changes"
    cudaMemsetAsync(w.changed, 0, sizeof(unsigned) * 2, s);
    km_assign<T><<<ab, kKmBlock, 0, s>>>(X, n, dim, C, w.centers, w.labels, w.dmin, w.changed, w.changed + 1);
    cudaMemsetAsync(w.changed, 0, sizeof(unsigned), s);
    for (int it = 0; it < max_iter;) {
      const int chunk = std::min(kKmCheckEvery, max_iter - it);
      for (int q = 0; q < chunk; ++q) {
        km_partial<T><<<w.nblocks, kKmBlock, 0, s>>>(X, n, dim, C, w.labels, w.part, w.changed + 1);
        km_finish<<<(C * (dim + 1) + 127) / 128, 128, 0, s>>>(w.part, w.nblocks, C, dim, w.centers, w.counts,
                                                               w.changed + 1);
        // empty clusters re-seed at the farthest rows (dmin = distances to the old centres)
        km_reseed<T><<<1, kKmBlock, 0, s>>>(X, n, dim, C, w.counts, w.dmin, w.centers, w.changed + 1);
        km_assign<T><<<ab, kKmBlock, 0, s>>>(X, n, dim, C, w.centers, w.labels, w.dmin, w.changed,
                                             w.changed + 1);
        km_mark<<<1, 1, 0, s>>>(w.changed, w.changed + 1);
      }
      it += chunk;
      unsigned done = 0;
      cudaMemcpyAsync(&done, w.changed + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { st = cuda_error(e, "kmeans Lloyd"); break; }
      if (done) break;
    }
    if (st != PSPEC_OK) break;
    km_sum<<<1, kKmBlock, 0, s>>>(w.dmin, n, w.scalar);
    double inertia = 0.0;
    cudaMemcpyAsync(&inertia, w.scalar, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (inertia < best) {
      best = inertia;
      cudaMemcpyAsync(labels_out, w.labels, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(w.best_centers, w.centers, sizeof(double) * C * dim, cudaMemcpyDeviceToDevice, s);
    }
  }
  if (st == PSPEC_OK && centers_out)
    cudaMemcpyAsync(centers_out, w.best_centers, sizeof(double) * C * dim, cudaMemcpyDeviceToDevice, s);
  cudaFreeAsync(base, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (st == PSPEC_OK && e != cudaSuccess) st = cuda_error(e, "kmeans");
  if (inertia_out) *inertia_out = best;
  return st;
}

}  // namespace pspec

using namespace pspec;

extern "C" pspec_status pspec_kmeans(const void* X, int64_t n, int dim, pspec_dtype dtype,
                                     int n_clusters, uint64_t seed, int restarts, int max_iter,
                                     int32_t* labels_out, double* centers_out, double* inertia_out,
                                     void* stream) {
  if (!X || !labels_out) return set_error(PSPEC_ERR_INVALID_ARG, "X or labels_out is NULL");
  if (dim < 1 || dim > kKmMaxDim) return set_error(PSPEC_ERR_INVALID_ARG, "dim must be in [1, 16]");
  if (n_clusters < 1 || n_clusters > kKmMaxC) return set_error(PSPEC_ERR_INVALID_ARG, "n_clusters must be in [1, 64]");
  if (n < n_clusters) return set_error(PSPEC_ERR_INVALID_ARG, "n < n_clusters");
  if (restarts < 1 || max_iter < 0) return set_error(PSPEC_ERR_INVALID_ARG, "bad restarts or max_iter");
  cudaStream_t s = (cudaStream_t)stream;
  if (dtype == PSPEC_F32)
    return kmeans_impl((const float*)X, n, dim, n_clusters, seed, restarts, max_iter, labels_out,
                       centers_out, inertia_out, s);
  if (dtype == PSPEC_F64)
    return kmeans_impl((const double*)X, n, dim, n_clusters, seed, restarts, max_iter, labels_out,
                       centers_out, inertia_out, s);
  return set_error(PSPEC_ERR_INVALID_ARG, "bad dtype");
}
