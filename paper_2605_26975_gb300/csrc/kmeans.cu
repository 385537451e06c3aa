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
// The means of FP32 rows are exact fixed-point sums (integer atomics, so
// order-free) scaled back by a power of two; every floating-point reduction
// has a fixed order, so results are reproducible run to run.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
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

// Row loads and distances are built for dim rounded up to DB in {4, 8, 16}
// (register arrays); entries past dim are zero and every loop stops at dim,
// so results are those of the plain dim loop.
__host__ __device__ constexpr int km_bucket(int dim) { return dim <= 4 ? 4 : dim <= 8 ? 8 : 16; }

// row i of X into registers: 16-byte loads when vec (dim == DB and X 16-byte
// aligned, so every row is), else one load per entry
template <typename T> struct KmVec;
template <> struct KmVec<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static void put(const float4& v, float* x) { x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
};
template <> struct KmVec<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static void put(const double2& v, double* x) { x[0] = v.x; x[1] = v.y; }
};

template <typename T, int DB>
__device__ __forceinline__ void km_load_row(const T* __restrict__ X, int64_t i, int dim, bool vec, T (&x)[DB]) {
  if (vec) {
    using KV = KmVec<T>;
    const typename KV::type* p = reinterpret_cast<const typename KV::type*>(X + i * DB);
#pragma unroll
    for (int q = 0; q < DB / KV::W; ++q) KV::put(__ldg(p + q), x + q * KV::W);
  } else {
#pragma unroll
    for (int j = 0; j < DB; ++j) x[j] = j < dim ? X[i * dim + j] : T(0);
  }
}

// the oracle's squared distance: dimension by dimension, each subtraction,
// product and sum rounded once (no fused multiply-add)
template <typename T, int DB>
__device__ __forceinline__ double km_dist64(const T (&x)[DB], const double* mu, int dim) {
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < DB; ++j)
    if (j < dim) {
      const double t = __dsub_rn((double)x[j], mu[j]);
      acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
  return acc;
}

// FP32 squared distance to the FP32-rounded centre, and its error bound E:
// |d32 - d64| <= E / 2 for d64 the FP64 distance above.  With u = 2^-24,
// t_j = fl32(x_j - fl32(mu_j)) differs from a_j = x_j - mu_j by at most
// u'(|a_j| + |mu_j|), u' = u(1+u), and the FP32 sum of the t_j^2 from
// sum a_j^2 by at most
//   (2u' + u + gamma_{dim-1}(1+u) + 2u'^2) d + 2u' |mu| sqrt(d) + 2u'^2 |mu|^2
// (Cauchy-Schwarz on sum |a_j||mu_j|), while the FP64 distance is within
// (dim+2) 2^-53 d of sum a_j^2.  E is twice the sum of both bounds (the
// factor covers using the computed d32 for d), plus 2^-120 for the absolute
// error of products and sums in FP32's subnormal range (at most dim 2^-149),
// so distances that small are always left to the FP64 loop.
template <int DB>
__device__ __forceinline__ float km_dist32(const float (&x)[DB], const float* mu32 /* 16-byte aligned */) {
  float d = 0.f;
#pragma unroll
  for (int q = 0; q < DB / 4; ++q) {  // padded entries add fmaf(0, 0, d) = d
    const float4 m = *reinterpret_cast<const float4*>(mu32 + 4 * q);
    const float mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float t = x[4 * q + j] - mm[j];
      d = fmaf(t, t, d);
    }
  }
  return d;
}
__device__ __forceinline__ float km_err32(float d, float nmu, float k_rel) {
  constexpr float u = 5.9604645e-8f;  // 2^-24
  return 2.0f * (k_rel * d + 2.1f * u * nmu * sqrtf(d) + 3.0f * u * u * nmu * nmu) + 7.5231638e-37f;
}
__device__ __forceinline__ float km_krel(int dim) {
  constexpr float u = 5.9604645e-8f;
  return 2.0f * u * (float)(dim + 3) + 2.0f * (float)(dim + 2) * 1.1102230e-16f;
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

// d2[i] = dist(X_i, centre c) (first) or min(d2[i], dist(X_i, centre c)), and
// the blocks' sums of d2 (contiguous row ranges, fixed-order trees).  For
// FP32 rows the FP64 distance is only computed where the FP32 screen cannot
// show dist >= d2[i] (then the minimum is d2[i] as it stands).  Warps take
// groups of 32 consecutive rows; the rows that need the FP64 distance go to a
// per-warp queue (ballot order) that is worked off 32 rows at a time, so the
// FP64 arithmetic runs with full warps.
template <typename T, int DB>
__global__ void __launch_bounds__(kKmBlock) km_seed_dist(const T* __restrict__ X, int64_t n, int dim,
                                                         bool vec, const double* centers, int c, int first,
                                                         double* d2, double* block_sum) {
  __shared__ double mu[DB];
  __shared__ __align__(16) float mu32[DB];
  __shared__ int queue[kKmBlock / 32][64];
  __shared__ double s[kKmBlock];
  if (threadIdx.x < DB) {
    const double v = threadIdx.x < dim ? centers[c * dim + threadIdx.x] : 0.0;
    mu[threadIdx.x] = v;
    mu32[threadIdx.x] = (float)v;
  }
  __syncthreads();
  double q2 = 0.0;
  for (int j = 0; j < dim; ++j) q2 += mu[j] * mu[j];
  const float nmu = (float)(sqrt(q2) * (1.0 + 1e-6));
  const float k_rel = km_krel(dim);
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int* qw = queue[w];
  int qn = 0;  // warp-uniform queue length
  double acc = 0.0;
  auto drain = [&](int cnt) {  // the first cnt queued rows, one per lane
    if (lane < cnt) {
      const int64_t i = b0 + qw[lane];
      T xr[DB];
      km_load_row<T, DB>(X, i, dim, vec, xr);
      double d = km_dist64<T, DB>(xr, mu, dim);
      if (!first) d = fmin(d, d2[i]);
      d2[i] = d;
      acc += d;
    }
  };
  for (int64_t g0 = b0 + 32 * w; g0 < b1; g0 += kKmBlock) {
    const int64_t i = g0 + lane;
    bool need = false;
    if (i < b1) {
      need = true;
      if constexpr (sizeof(T) == 4) {
        if (!first) {
          T xr[DB];
          km_load_row<T, DB>(X, i, dim, vec, xr);
          const double d = d2[i];
          const float d32 = km_dist32<DB>(xr, mu32);
          if ((double)d32 - (double)km_err32(d32, nmu, k_rel) > d) {
            need = false;
            acc += d;
          }
        }
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (need) qw[qn + __popc(m & ((1u << lane) - 1u))] = (int)(i - b0);
    qn += __popc(m);
    __syncwarp();
    if (qn >= 32) {
      drain(32);
      qn -= 32;
      const int moved = lane < qn ? qw[32 + lane] : 0;
      __syncwarp();
      if (lane < qn) qw[lane] = moved;
      __syncwarp();
    }
  }
  drain(qn);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kKmBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sum[blockIdx.x] = s[0];
}

// first index whose running D^2 sum exceeds u * total (one block of
// kKmBlock threads).  The block sums' prefix sums come from a scan in a fixed
// order (each thread adds its four blocks in order, then a Hillis-Steele scan
// over the threads: a few dependent FP64 adds instead of one per block); the
// first block whose prefix exceeds the target is the one it falls in.  From
// that block's first row the walk goes on in windows of kKmBlock chunks of
// kPickChunk rows: the threads sum their chunks, thread 0 adds the chunk sums
// in order and walks the one chunk the target falls in row by row.
constexpr int kPickChunk = 32;
constexpr int kKmMaxSeedBlocks = 1024;  // row ranges of the seeding

// Lloyd iterations between two host checks of convergence
constexpr int kKmCheckEvery = 8;

__global__ void __launch_bounds__(kKmBlock) km_pick(const double* d2, const double* block_sum,
                                                    int nblocks, int64_t n, double u,
                                                    int64_t* out_idx) {
  constexpr int kPer = kKmMaxSeedBlocks / kKmBlock;  // block sums per thread
  __shared__ double csum[kKmBlock];
  __shared__ double scan[2][kKmBlock];
  __shared__ double s_run, s_target;
  __shared__ int64_t s_i0, s_found;
  __shared__ int s_blk;
  const int t = threadIdx.x;
  double loc[kPer];  // inclusive prefixes of this thread's blocks
  double tsum = 0.0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int b = t * kPer + q;
    if (b < nblocks) tsum += block_sum[b];
    loc[q] = tsum;
  }
  scan[0][t] = tsum;
  if (t == 0) {
    s_blk = nblocks - 1;
    s_found = -1;
  }
  __syncthreads();
  int cur = 0;
  for (int off = 1; off < kKmBlock; off <<= 1) {
    const double v = t >= off ? scan[cur][t] + scan[cur][t - off] : scan[cur][t];
    scan[cur ^ 1][t] = v;
    cur ^= 1;
    __syncthreads();
  }
  const double before = t > 0 ? scan[cur][t - 1] : 0.0;  // the blocks of threads < t
  const double total = scan[cur][kKmBlock - 1];
  const double target = u * total;
  if (total > 0.0) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int b = t * kPer + q;
      if (b < nblocks && before + loc[q] > target) {
        atomicMin(&s_blk, b);
        break;
      }
    }
  }
  __syncthreads();
  if (total > 0.0) {
    if (t == s_blk / kPer) {  // the running sum before the chosen block
      const int q = s_blk % kPer;
      s_run = q > 0 ? before + loc[q - 1] : before;
      s_target = target;
      s_i0 = (int64_t)s_blk * ((n + nblocks - 1) / nblocks);
    }
  } else if (t == 0) {
    s_found = min((int64_t)(u * (double)n), n - 1);
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

// labels[i] = argmin_c dist(X_i, mu_c) and the count of changed labels.
//
// The decision is the FP64 one (reading: ties to the smaller centre).  For
// FP32 rows it is screened in FP32: the FP32 winner is accepted when its
// d32 + E stays below every other centre's d32 - E, which makes it the FP64
// decision too; a row that is too close to call runs the full FP64 loop.
// The distances themselves are not kept: the few steps that need them
// (re-seeding, the inertia) compute them in FP64 from labels and centres.
template <typename T, int DB>
__global__ void __launch_bounds__(kKmBlock) km_assign(const T* __restrict__ X, int64_t n, int dim, bool vec,
                                                      int C, const double* centers, int32_t* labels,
                                                      unsigned* changed, const unsigned* done) {
  if (*done) return;
  __shared__ double mu[kKmMaxC * DB];
  __shared__ __align__(16) float mu32[kKmMaxC * DB];
  __shared__ float nmu[kKmMaxC];  // |mu_c|, rounded up
  for (int t = threadIdx.x; t < C * DB; t += blockDim.x) {
    const int c = t / DB, j = t - (t / DB) * DB;
    const double v = j < dim ? centers[c * dim + j] : 0.0;
    mu[t] = v;
    mu32[t] = (float)v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double q = 0.0;
    for (int j = 0; j < dim; ++j) q += mu[c * DB + j] * mu[c * DB + j];
    nmu[c] = (float)(sqrt(q) * (1.0 + 1e-6));
  }
  __syncthreads();
  const float k_rel = km_krel(dim);
  unsigned local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T xr[DB];
    km_load_row<T, DB>(X, i, dim, vec, xr);
    int arg = -1;
    if constexpr (sizeof(T) == 4) {
      float best_hi = 0.f, best_d = 0.f;  // winner's d32 + E and d32
      int c1 = 0;
      float lo1 = 3.4e38f, lo2 = 3.4e38f;  // two smallest d32 - E ...
      int lo1c = -1;                       // ... and the centre of the smallest
      for (int c = 0; c < C; ++c) {
        const float d = km_dist32<DB>(xr, mu32 + c * DB);
        const float e = km_err32(d, nmu[c], k_rel);
        if (c == 0 || d < best_d) { best_d = d; best_hi = d + e; c1 = c; }
        const float lo = d - e;
        if (lo < lo1) { lo2 = lo1; lo1 = lo; lo1c = c; }
        else if (lo < lo2) lo2 = lo;
      }
      const float others_lo = (lo1c == c1) ? lo2 : lo1;
      if (best_hi < others_lo) arg = c1;  // separated: the FP64 decision is c1
    }
    if (arg < 0) {
      double best = 0.0;
      arg = 0;
      for (int c = 0; c < C; ++c) {
        const double acc = km_dist64<T, DB>(xr, mu + c * DB, dim);
        if (c == 0 || acc < best) { best = acc; arg = c; }
      }
    }
    if (labels[i] != arg) ++local;
    labels[i] = arg;
  }
  if (local) atomicAdd(changed, local);
}

// max |x| over X as float bits (non-negative floats order as their bits)
template <typename T>
__global__ void __launch_bounds__(kKmBlock) km_absmax(const T* __restrict__ X, int64_t m, unsigned* out) {
  __shared__ unsigned s[kKmBlock];
  unsigned b = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    b = max(b, __float_as_uint(fabsf((float)X[e])));
  s[threadIdx.x] = b;
  __syncthreads();
  for (int h = kKmBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] = max(s[threadIdx.x], s[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicMax(out, s[0]);
}

// round(y) as int64 for an FP32 y with |y| < 2^62, in FP32 and integer
// operations only (an integer-valued float above 2^23 is its mantissa shifted)
__device__ __forceinline__ long long km_fixed(float y) {
  if (fabsf(y) < 8388608.0f) return (long long)__float2int_rn(y);
  const unsigned b = __float_as_uint(y);
  const long long v = (long long)((b & 0x7fffffu) | 0x800000u) << (int)(((b >> 23) & 0xffu) - 150u);
  return (b >> 31) ? -v : v;
}

// Per-block, per-cluster sums of member rows and counts.
//
// FP32 rows (fixed = 1): every entry is rounded to a fixed-point integer,
// round(x 2^q) with 2^q chosen on the host from max |x| so that no sum over
// all rows can pass 2^62, and the integers are added exactly with shared-memory
// atomics (so the order does not matter and the result is reproducible); a
// mean is then within 2^-q of the exact mean of the rows, plus one rounding.
// FP64 rows, or FP32 rows too small for a finite scale (fixed = 0): FP64 sums,
// warp w owning clusters w, w+8, ..., its lanes striding the block's rows in
// a fixed order.
template <typename T, int DB>
__global__ void __launch_bounds__(kKmBlock) km_partial(const T* __restrict__ X, int64_t n, int dim, bool vec,
                                                       int C, const int32_t* __restrict__ labels, double* part,
                                                       int fixed, float scale, const unsigned* done) {
  if (*done) return;
  __shared__ unsigned long long acc_fx[kKmMaxC * (kKmMaxDim + 1)];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* out = part + (size_t)blockIdx.x * C * (dim + 1);
  if constexpr (sizeof(T) == 4) {
    if (fixed) {
      const int nv = C * (dim + 1);
      for (int t = threadIdx.x; t < nv; t += blockDim.x) acc_fx[t] = 0ull;
      __syncthreads();
      // warps take 32 consecutive rows at a time; a warp whose rows share one
      // label (clusters of consecutive rows are common) adds its 32 rows with
      // shuffles first, so the shared-memory atomics do not serialise
      for (int64_t base = b0 + 32 * w; base < b1; base += blockDim.x) {
        const int64_t i = base + lane;
        const bool valid = i < b1;
        const int c = valid ? labels[i] : -1;
        float xr[DB];
        if (valid) km_load_row<float, DB>(X, i, dim, vec, xr);
        long long v[DB];
#pragma unroll
        for (int j = 0; j < DB; ++j) v[j] = (valid && j < dim) ? km_fixed(xr[j] * scale) : 0ll;
        const int c0 = __shfl_sync(0xffffffffu, c, 0);
        if (__all_sync(0xffffffffu, c == c0)) {
#pragma unroll
          for (int j = 0; j < DB; ++j)
            if (j < dim)
              for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], off);
          if (lane == 0) {
            unsigned long long* a = acc_fx + c0 * (dim + 1);
#pragma unroll
            for (int j = 0; j < DB; ++j)
              if (j < dim) atomicAdd(a + j, (unsigned long long)v[j]);
            atomicAdd(a + dim, 32ull);
          }
        } else if (valid) {
          unsigned long long* a = acc_fx + c * (dim + 1);
#pragma unroll
          for (int j = 0; j < DB; ++j)
            if (j < dim) atomicAdd(a + j, (unsigned long long)v[j]);
          atomicAdd(a + dim, 1ull);
        }
      }
      __syncthreads();
      long long* o = reinterpret_cast<long long*>(out);
      for (int t = threadIdx.x; t < nv; t += blockDim.x) o[t] = (long long)acc_fx[t];
      return;
    }
  }
  for (int c = w; c < C; c += kKmBlock / 32) {
    double acc[DB];
    double cnt = 0.0;
#pragma unroll
    for (int j = 0; j < DB; ++j) acc[j] = 0.0;
    for (int64_t i = b0 + lane; i < b1; i += 32) {
      if (labels[i] == c) {
        T xr[DB];
        km_load_row<T, DB>(X, i, dim, vec, xr);
#pragma unroll
        for (int j = 0; j < DB; ++j)
          if (j < dim) acc[j] += (double)xr[j];
        cnt += 1.0;
      }
    }
#pragma unroll
    for (int j = 0; j <= DB; ++j) {
      if (j < dim || j == DB) {
        double v = j < DB ? acc[j] : cnt;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) out[c * (dim + 1) + (j < DB ? j : dim)] = v;
      }
    }
  }
}

// One block per cluster: the blocks' partial sums added (fixed point: exact
// int64 sums; FP64: lane-strided, then a shuffle tree, in a fixed order), the
// previous centre kept in prev, the new centre the mean when the cluster has
// members (an empty cluster keeps its centre until it is re-seeded), and the
// count.
__global__ void __launch_bounds__(kKmBlock) km_finish(const double* __restrict__ part, int nblocks, int C,
                                                      int dim, int fixed, double unscale, double* centers,
                                                      double* prev,
                                                      double* counts, const unsigned* done) {
  if (*done) return;
  __shared__ double sums[kKmMaxDim + 1];
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = w; j <= dim; j += kKmBlock / 32) {
    const size_t at = (size_t)c * (dim + 1) + j;
    const size_t stride = (size_t)C * (dim + 1);
    if (fixed) {
      const long long* pl = reinterpret_cast<const long long*>(part);
      long long acc = 0;
      for (int b = lane; b < nblocks; b += 32) acc += pl[b * stride + at];
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane == 0) sums[j] = j == dim ? (double)acc : (double)acc * unscale;  // exact: a power of 2
    } else {
      double acc = 0.0;
      for (int b = lane; b < nblocks; b += 32) acc += part[b * stride + at];
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
      if (lane == 0) sums[j] = acc;
    }
  }
  __syncthreads();
  const double cnt = sums[dim];
  if (threadIdx.x < dim) {
    const int t = c * dim + threadIdx.x;
    prev[t] = centers[t];
    if (cnt > 0.0) centers[t] = sums[threadIdx.x] / cnt;
  }
  if (threadIdx.x == 0) counts[c] = cnt;
}

// dmin[i] = FP64 distance of row i to the centre it was assigned to (prev),
// only when some cluster came out empty (the re-seeding reads it)
template <typename T, int DB>
__global__ void __launch_bounds__(kKmBlock) km_dist_own(const T* __restrict__ X, int64_t n, int dim, bool vec, int C,
                                                        const int32_t* __restrict__ labels,
                                                        const double* prev, const double* counts,
                                                        double* dmin, const unsigned* done) {
  if (*done) return;
  __shared__ double mu[kKmMaxC * DB];
  __shared__ int any_empty;
  if (threadIdx.x == 0) any_empty = 0;
  __syncthreads();
  if (threadIdx.x < C && counts[threadIdx.x] == 0.0) any_empty = 1;
  __syncthreads();
  if (!any_empty) return;
  for (int t = threadIdx.x; t < C * DB; t += blockDim.x) {
    const int c = t / DB, j = t - (t / DB) * DB;
    mu[t] = j < dim ? prev[c * dim + j] : 0.0;
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T xr[DB];
    km_load_row<T, DB>(X, i, dim, vec, xr);
    dmin[i] = km_dist64<T, DB>(xr, mu + labels[i] * DB, dim);
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

// inertia: the blocks' sums (contiguous row ranges, fixed-order trees) of the
// FP64 distance of every row to its centre
template <typename T, int DB>
__global__ void __launch_bounds__(kKmBlock) km_inertia_part(const T* __restrict__ X, int64_t n, int dim,
                                                            bool vec, int C, const int32_t* __restrict__ labels,
                                                            const double* centers, double* block_sum) {
  __shared__ double mu[kKmMaxC * DB];
  __shared__ double s[kKmBlock];
  for (int t = threadIdx.x; t < C * DB; t += blockDim.x) {
    const int c = t / DB, j = t - (t / DB) * DB;
    mu[t] = j < dim ? centers[c * dim + j] : 0.0;
  }
  __syncthreads();
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = blockIdx.x * per, b1 = min(n, b0 + per);
  double acc = 0.0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    T xr[DB];
    km_load_row<T, DB>(X, i, dim, vec, xr);
    acc += km_dist64<T, DB>(xr, mu + labels[i] * DB, dim);
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int h = kKmBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sum[blockIdx.x] = s[0];
}

// the block sums in a fixed order: thread t adds blocks t, t + 256, ...,
// then a tree over the threads (one block of kKmBlock threads)
__global__ void __launch_bounds__(kKmBlock) km_sum_blocks(const double* block_sum, int nblocks, double* out) {
  __shared__ double s[kKmBlock];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc += block_sum[b];
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
  double* part;    // [pblocks][C][dim+1] member sums and counts
  double* bsum;    // [nblocks] block sums of d2 and of the inertia
  double* centers;
  double* prev;    // the centres the current labels were assigned to
  double* best_centers;
  double* counts;
  int32_t* labels;
  int64_t* idx;
  unsigned* changed;  // [0] labels changed by the last assignment, [1] done
  double* scalar;
  int nblocks;  // row ranges of the seeding and the inertia
  int pblocks;  // row ranges of the member sums
};

template <typename T, int DB>
static pspec_status kmeans_impl(const T* X, int64_t n, int dim, int C, uint64_t seed, int restarts,
                                int max_iter, int32_t* labels_out, double* centers_out,
                                double* inertia_out, cudaStream_t s) {
  KmWork w;
  w.nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(kKmMaxSeedBlocks, (n + 1023) / 1024));
  const bool vec = dim == DB && reinterpret_cast<uintptr_t>(X) % 16 == 0;
  w.pblocks = (int)std::max<int64_t>(1, std::min<int64_t>(2048, (n + 1023) / 1024));
  const size_t part_elems = (size_t)w.pblocks * C * (dim + 1);
  char* mem = nullptr;
  const size_t bytes = sizeof(double) * (2 * (size_t)n + part_elems + w.nblocks + 3 * C * dim + C + 4) +
                       sizeof(int32_t) * n + sizeof(int64_t) * 2 + sizeof(unsigned) * 2 + 13 * 128;
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
  w.bsum = (double*)carve(sizeof(double) * w.nblocks);
  w.centers = (double*)carve(sizeof(double) * C * dim);
  w.prev = (double*)carve(sizeof(double) * C * dim);
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
  // fixed-point scale 2^q of the member sums (FP32 rows): max |x| < 2^E and
  // n <= 2^L give |sum| < 2^(62-L) n <= 2^62 for q = 62 - E - L
  int fixed = 0, q = 0;
  if (sizeof(T) == 4) {
    cudaMemsetAsync(w.changed, 0, sizeof(unsigned), s);
    km_absmax<T><<<ab, kKmBlock, 0, s>>>(X, n * dim, w.changed);
    unsigned bits = 0;
    cudaMemcpyAsync(&bits, w.changed, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFreeAsync(base, s);
      return cuda_error(e, "kmeans scale");
    }
    if (bits >= 0x7f800000u) {
      cudaFreeAsync(base, s);
      return set_error(PSPEC_ERR_INVALID_ARG, "X holds a NaN or an infinity");
    }
    float mx;
    std::memcpy(&mx, &bits, sizeof(float));
    const int E = mx > 0.0f ? std::ilogb(mx) + 1 : 0;
    int L = 0;
    while (L < 62 && (int64_t(1) << L) < n) ++L;
    q = 62 - E - L;
    fixed = q >= -120 && q <= 120;  // 2^q a normal float
  }
  const float scale = fixed ? std::ldexp(1.0f, q) : 0.0f;
  const double unscale = fixed ? std::ldexp(1.0, -q) : 1.0;
  for (int r = 0; r < restarts && st == PSPEC_OK; ++r) {
    // ---- k-means++ seeding (the uniforms drawn here, the picks on the device)
    {
      const double u = rng.uniform();
      const int64_t first = std::min<int64_t>((int64_t)(u * (double)n), n - 1);
      km_take_row<T><<<1, 32, 0, s>>>(X, dim, first, w.centers, 0);
      km_seed_dist<T, DB><<<w.nblocks, kKmBlock, 0, s>>>(X, n, dim, vec, w.centers, 0, 1, w.d2, w.bsum);
      for (int c = 1; c < C; ++c) {
        const double uc = rng.uniform();
        km_pick<<<1, kKmBlock, 0, s>>>(w.d2, w.bsum, w.nblocks, n, uc, w.idx);
        km_take_row_at<T><<<1, 32, 0, s>>>(X, dim, w.idx, w.centers, c);
        km_seed_dist<T, DB><<<w.nblocks, kKmBlock, 0, s>>>(X, n, dim, vec, w.centers, c, 0, w.d2, w.bsum);
      }
    }
    // ---- Lloyd.  The iterations run in chunks with one host check each: a
    // converged state is marked done on the device and the rest of the chunk
    // skips, so the result is the one of checking after every iteration.
    cudaMemsetAsync(w.labels, 0xff, sizeof(int32_t) * n, s);  // -1: every label "changes"
    cudaMemsetAsync(w.changed, 0, sizeof(unsigned) * 2, s);
    km_assign<T, DB><<<ab, kKmBlock, 0, s>>>(X, n, dim, vec, C, w.centers, w.labels, w.changed, w.changed + 1);
    cudaMemsetAsync(w.changed, 0, sizeof(unsigned), s);
    for (int it = 0; it < max_iter;) {
      const int chunk = std::min(kKmCheckEvery, max_iter - it);
      for (int q = 0; q < chunk; ++q) {
        km_partial<T, DB><<<w.pblocks, kKmBlock, 0, s>>>(X, n, dim, vec, C, w.labels, w.part, fixed, scale,
                                                         w.changed + 1);
        km_finish<<<C, kKmBlock, 0, s>>>(w.part, w.pblocks, C, dim, fixed, unscale, w.centers, w.prev,
                                         w.counts, w.changed + 1);
        // empty clusters re-seed at the rows farthest from their old centres
        km_dist_own<T, DB><<<ab, kKmBlock, 0, s>>>(X, n, dim, vec, C, w.labels, w.prev, w.counts, w.dmin,
                                                   w.changed + 1);
        km_reseed<T><<<1, kKmBlock, 0, s>>>(X, n, dim, C, w.counts, w.dmin, w.centers, w.changed + 1);
        km_assign<T, DB><<<ab, kKmBlock, 0, s>>>(X, n, dim, vec, C, w.centers, w.labels, w.changed, w.changed + 1);
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
    km_inertia_part<T, DB><<<w.nblocks, kKmBlock, 0, s>>>(X, n, dim, vec, C, w.labels, w.centers, w.bsum);
    km_sum_blocks<<<1, kKmBlock, 0, s>>>(w.bsum, w.nblocks, w.scalar);
    double inertia = 0.0;
    cudaMemcpyAsync(&inertia, w.scalar, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { st = cuda_error(e, "kmeans inertia"); break; }
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

template <typename T>
static pspec_status kmeans_dispatch(const T* X, int64_t n, int dim, int C, uint64_t seed, int restarts,
                                    int max_iter, int32_t* labels_out, double* centers_out,
                                    double* inertia_out, cudaStream_t s) {
  switch (km_bucket(dim)) {
    case 4: return kmeans_impl<T, 4>(X, n, dim, C, seed, restarts, max_iter, labels_out, centers_out, inertia_out, s);
    case 8: return kmeans_impl<T, 8>(X, n, dim, C, seed, restarts, max_iter, labels_out, centers_out, inertia_out, s);
    default: return kmeans_impl<T, 16>(X, n, dim, C, seed, restarts, max_iter, labels_out, centers_out, inertia_out, s);
  }
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
    return kmeans_dispatch((const float*)X, n, dim, n_clusters, seed, restarts, max_iter, labels_out,
                       centers_out, inertia_out, s);
  if (dtype == PSPEC_F64)
    return kmeans_dispatch((const double*)X, n, dim, n_clusters, seed, restarts, max_iter, labels_out,
                       centers_out, inertia_out, s);
  return set_error(PSPEC_ERR_INVALID_ARG, "bad dtype");
}
