// Vector kernels of the Grassmann trust-region Newton / truncated-CG solve:
// Gram products, projections, the CG updates, Cholesky-QR and the scalar
// recurrences of Steihaug-Toint truncated CG, all kept on the device.
//
// Blocks are n x k row-major of type T (float for the fast path, double for
// the plain path).  Cross-thread sums: float-float for T = float (compensated
// per-thread sums, TwoSum trees), double for T = double; both in a fixed
// order.  Every kernel may be handed a `done` flag: once truncated CG has
// stopped, the kernels of the iterations already enqueued return at once.
#pragma once

#include "common.cuh"

namespace pspec {

constexpr int kSolveBlock = 256;

// ------------------------------------------------------------ tCG state ---
struct TcgState {
  double Delta;      // trust-region radius of this subproblem
  double rr;         // <r, r>
  double norm_r0;
  double stop;       // ||r|| threshold
  double e_Pe, e_Pd, d_Pd;  // <eta,eta>, <eta,delta>, <delta,delta>
  double alpha, step, beta;
  double d_Hd;
  int j;             // completed iterations
  int max_inner;
  int done;          // 1 once the subproblem is solved
  int reason;        // 1 negative curvature, 2 radius, 3 converged, 4 max_inner
  int boundary;
  int pad;
};

// accumulation of one partial sum per thread
template <typename T> struct Acc;
template <> struct Acc<float> {
  Kahan k;
  __device__ void init() { k.init(); }
  __device__ void add(float x) { k.add(x); }
  __device__ float2 get() const { return kahan_to_ff(k); }
};
template <> struct Acc<double> {
  double s;
  __device__ void init() { s = 0.0; }
  __device__ void add(double x) { s += x; }
  __device__ double get() const { return s; }
};

template <typename T> struct RedT { using type = float2; };
template <> struct RedT<double> { using type = double; };

__device__ __forceinline__ float2 red_add(float2 a, float2 b) { return ff_add(a, b); }
__device__ __forceinline__ double red_add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 red_zero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double red_zero(double) { return 0.0; }
__device__ __forceinline__ double red_to_double(float2 a) { return ff_to_double(a); }
__device__ __forceinline__ double red_to_double(double a) { return a; }
__device__ __forceinline__ float2 red_shfl(float2 v, int off) { return shfl_xor_ff(v, off); }
__device__ __forceinline__ double red_shfl(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }

struct GridRed {
  void* block_part;
  void* group_part;
  unsigned* counters;
};

// Two-level grid reduction of nv values (nv <= blockDim.x) held in shared
// memory; returns true in the one block that finishes last, with the grid
// totals in `total`.  Order fixed by block and group index.
template <typename R>
__device__ bool grid_reduce_rt(const R* mine, R* total, int nv, const GridRed& gr) {
  __shared__ int s_flag;
  R* bp = (R*)gr.block_part;
  R* gp = (R*)gr.group_part;
  const int tid = threadIdx.x;
  const int nblk = gridDim.x;
  const int ngroups = (nblk + kGroup - 1) / kGroup;
  const int g = blockIdx.x / kGroup;
  if (tid < nv) bp[(size_t)blockIdx.x * nv + tid] = mine[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const int gsize = min(kGroup, nblk - g * kGroup);
    s_flag = atomicAdd(&gr.counters[g], 1u) == (unsigned)(gsize - 1);
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  if (tid < nv) {
    R acc = red_zero(R());
    const int b0 = g * kGroup, b1 = min(nblk, b0 + kGroup);
    for (int b = b0; b < b1; ++b) acc = red_add(acc, __ldcg(&bp[(size_t)b * nv + tid]));
    gp[(size_t)g * nv + tid] = acc;
  }
  if (tid == 0) gr.counters[g] = 0u;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_flag = atomicAdd(&gr.counters[ngroups], 1u) == (unsigned)(ngroups - 1);
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  if (tid < nv) {
    R acc = red_zero(R());
    for (int q = 0; q < ngroups; ++q) acc = red_add(acc, __ldcg(&gp[(size_t)q * nv + tid]));
    total[tid] = acc;
  }
  if (tid == 0) gr.counters[ngroups] = 0u;
  __syncthreads();
  return true;
}

// block sum of ND per-thread values (warp shuffles, then warps in order)
template <typename R, int ND>
__device__ void block_sum(R (&v)[ND], R* out /* shared [ND] */) {
  __shared__ R s[kSolveBlock / 32][ND];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < ND; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] = red_add(v[q], red_shfl(v[q], off));
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < ND; ++q) s[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x < ND) {
    R acc = red_zero(R());
    for (int ww = 0; ww < kSolveBlock / 32; ++ww) acc = red_add(acc, s[ww][threadIdx.x]);
    out[threadIdx.x] = acc;
  }
  __syncthreads();
}

// ----------------------------------------------------------------- gram ---
// G[a][b] = sum_i A_ia B_ib  (k x k, FP64 out).  A warp takes a row at a
// time; lane l owns the pairs (a, b) with a*k + b = l (mod 32).
template <typename T>
__global__ void __launch_bounds__(kSolveBlock) gram_kernel(const T* __restrict__ A,
                                                           const T* __restrict__ B, int64_t n,
                                                           int k, double* G, GridRed gr,
                                                           const int* done) {
  using R = typename RedT<T>::type;
  if (done && *done) return;
  __shared__ R s_w[kSolveBlock / 32][kMaxK * kMaxK];
  __shared__ R s_blk[kMaxK * kMaxK];
  __shared__ R s_tot[kMaxK * kMaxK];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nv = k * k;
  const int npl = (nv + 31) / 32;  // pairs per lane (<= 8)
  Acc<T> acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q].init();
  const int64_t nw = (int64_t)gridDim.x * (kSolveBlock / 32);
  for (int64_t i = (blockIdx.x * (int64_t)kSolveBlock + threadIdx.x) >> 5; i < n; i += nw) {
    const T av = lane < k ? A[i * k + lane] : T(0);
    const T bv = (lane >= 16 && lane - 16 < k) ? B[i * k + lane - 16] : T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q < npl) {
        const int pr = lane + 32 * q;
        const int a = pr / k, b = pr % k;
        const T x = __shfl_sync(0xffffffffu, av, pr < nv ? a : 0);
        const T y = __shfl_sync(0xffffffffu, bv, pr < nv ? 16 + b : 16);
        if (pr < nv) acc[q].add(x * y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int pr = lane + 32 * q;
    if (q < npl && pr < nv) s_w[w][pr] = acc[q].get();
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nv; t += kSolveBlock) {
    R s = red_zero(R());
    for (int ww = 0; ww < kSolveBlock / 32; ++ww) s = red_add(s, s_w[ww][t]);
    s_blk[t] = s;
  }
  __syncthreads();
  if (!grid_reduce_rt<R>(s_blk, s_tot, nv, gr)) return;
  for (int t = threadIdx.x; t < nv; t += kSolveBlock) G[t] = red_to_double(s_tot[t]);
}

// --------------------------------------------------------------- dots ---
// out[q] = <X_q, Y_q> for up to 4 pairs of n x k blocks (flattened length m)
template <typename T>
struct DotPairs {
  const T* x[4];
  const T* y[4];
  int np;
};

template <typename T>
__global__ void __launch_bounds__(kSolveBlock) dots_kernel(DotPairs<T> dp, int64_t m, double* out,
                                                           GridRed gr, const int* done) {
  using R = typename RedT<T>::type;
  if (done && *done) return;
  __shared__ R s_blk[4], s_tot[4];
  Acc<T> acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q].init();
  for (int64_t e = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * kSolveBlock) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < dp.np) acc[q].add(dp.x[q][e] * dp.y[q][e]);
  }
  R v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = acc[q].get();
  block_sum<R, 4>(v, s_blk);
  if (!grid_reduce_rt<R>(s_blk, s_tot, 4, gr)) return;
  if (threadIdx.x < dp.np) out[threadIdx.x] = red_to_double(s_tot[threadIdx.x]);
}

// ---------------------------------------------------------- row combine ---
// out_i = alpha X_i + beta Y_i - (P_i M1) - (Q_i M2)  for rows i, with M1,
// M2 k x k FP64 (either may be NULL) and scalar alpha/beta.
template <typename T>
__global__ void __launch_bounds__(kSolveBlock) combine_kernel(
    T* out, const T* X, double alpha, const T* Y, double beta, const T* P, const double* M1,
    const T* Qm, const double* M2, int64_t n, int k, const int* done) {
  if (done && *done) return;
  __shared__ T m1[kMaxK * kMaxK], m2[kMaxK * kMaxK];
  for (int t = threadIdx.x; t < k * k; t += kSolveBlock) {
    m1[t] = M1 ? (T)M1[t] : T(0);
    m2[t] = M2 ? (T)M2[t] : T(0);
  }
  __syncthreads();
  const int64_t m = n * k;
  for (int64_t e = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * kSolveBlock) {
    const int64_t i = e / k;
    const int b = (int)(e - i * k);
    T v = X ? (T)alpha * X[e] : T(0);
    if (Y) v += (T)beta * Y[e];
    if (M1) {
      const T* pr = P + i * k;
      for (int a = 0; a < k; ++a) v -= pr[a] * m1[a * k + b];
    }
    if (M2) {
      const T* qr = Qm + i * k;
      for (int a = 0; a < k; ++a) v -= qr[a] * m2[a * k + b];
    }
    out[e] = v;
  }
}

// ------------------------------------------------------ Riemannian Hessian ---
// Hd = He - U G - delta M   and the partial sum of <delta, Hd>; the last
// block takes truncated CG's curvature step (alpha, or the boundary tau).
template <typename T>
__global__ void __launch_bounds__(kSolveBlock) hess_kernel(T* Hd, const T* He, const T* U,
                                                           const double* G, const T* delta,
                                                           const double* M, int64_t n, int k,
                                                           TcgState* st, GridRed gr) {
  using R = typename RedT<T>::type;
  if (st->done) return;
  __shared__ T g[kMaxK * kMaxK], mm[kMaxK * kMaxK];
  __shared__ R s_blk[1], s_tot[1];
  for (int t = threadIdx.x; t < k * k; t += kSolveBlock) {
    g[t] = (T)G[t];
    mm[t] = (T)M[t];
  }
  __syncthreads();
  Acc<T> acc;
  acc.init();
  const int64_t m = n * k;
  for (int64_t e = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * kSolveBlock) {
    const int64_t i = e / k;
    const int b = (int)(e - i * k);
    T v = He[e];
    const T* ur = U + i * k;
    const T* dr = delta + i * k;
    for (int a = 0; a < k; ++a) v -= ur[a] * g[a * k + b] + dr[a] * mm[a * k + b];
    Hd[e] = v;
    acc.add(delta[e] * v);
  }
  R v1[1] = {acc.get()};
  block_sum<R, 1>(v1, s_blk);
  if (!grid_reduce_rt<R>(s_blk, s_tot, 1, gr)) return;
  if (threadIdx.x == 0) {
    const double dHd = red_to_double(s_tot[0]);
    st->d_Hd = dHd;
    const double D2 = st->Delta * st->Delta;
    const double alpha = dHd != 0.0 ? st->rr / dHd : INFINITY;
    const double e_Pe_new = st->e_Pe + 2.0 * alpha * st->e_Pd + alpha * alpha * st->d_Pd;
    if (dHd <= 0.0 || e_Pe_new >= D2) {
      const double tau = (-st->e_Pd + sqrt(st->e_Pd * st->e_Pd + st->d_Pd * (D2 - st->e_Pe))) / st->d_Pd;
      st->step = tau;
      st->alpha = 0.0;
      st->boundary = 1;
      st->reason = dHd <= 0.0 ? 1 : 2;
    } else {
      st->step = alpha;
      st->alpha = alpha;
      st->e_Pe = e_Pe_new;
    }
  }
}

// eta += step delta; Heta += step Hd; unless on the boundary r += alpha Hd
// and the partial <r, r>; the last block checks the residual, takes beta.
template <typename T>
__global__ void __launch_bounds__(kSolveBlock) cg_update_kernel(T* eta, T* Heta, T* r,
                                                                const T* delta, const T* Hd,
                                                                int64_t m, TcgState* st,
                                                                GridRed gr) {
  using R = typename RedT<T>::type;
  if (st->done) return;
  __shared__ R s_blk[1], s_tot[1];
  const T step = (T)st->step;
  const T alpha = (T)st->alpha;
  const bool bnd = st->boundary != 0;
  Acc<T> acc;
  acc.init();
  for (int64_t e = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * kSolveBlock) {
    const T h = Hd[e];
    eta[e] += step * delta[e];
    Heta[e] += step * h;
    if (!bnd) {
      const T rn = r[e] + alpha * h;
      r[e] = rn;
      acc.add(rn * rn);
    }
  }
  R v1[1] = {acc.get()};
  block_sum<R, 1>(v1, s_blk);
  if (!grid_reduce_rt<R>(s_blk, s_tot, 1, gr)) return;
  if (threadIdx.x == 0) {
    st->j += 1;
    if (bnd) {
      st->done = 1;
      return;
    }
    const double rr_new = red_to_double(s_tot[0]);
    const double beta = rr_new / st->rr;
    const double alpha_d = st->alpha;
    st->rr = rr_new;
    if (sqrt(rr_new) <= st->stop) {
      st->done = 1;
      st->reason = 3;
      return;
    }
    if (st->j >= st->max_inner) {
      st->done = 1;
      st->reason = 4;
      return;
    }
    st->beta = beta;
    st->e_Pd = beta * (st->e_Pd + alpha_d * st->d_Pd);
    st->d_Pd = rr_new + beta * beta * st->d_Pd;
  }
}

// delta = -r + beta delta
template <typename T>
__global__ void __launch_bounds__(kSolveBlock) direction_kernel(T* delta, const T* r, int64_t m,
                                                                const TcgState* st) {
  if (st->done) return;
  const T beta = (T)st->beta;
  for (int64_t e = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * kSolveBlock)
    delta[e] = -r[e] + beta * delta[e];
}

// --------------------------------------------------------- Cholesky-QR ---
// R^T R = G (k x k, FP64, one thread), then Rinv = R^-1 (upper triangular).
// Sets *bad when G is not numerically positive definite.
__global__ void chol_inv_kernel(const double* G, int k, double* Rinv, int* bad) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double R[kMaxK * kMaxK];
  for (int t = 0; t < k * k; ++t) R[t] = 0.0;
  for (int j = 0; j < k; ++j) {
    double s = G[j * k + j];
    for (int m = 0; m < j; ++m) s -= R[m * k + j] * R[m * k + j];
    if (!(s > 0.0)) {
      *bad = 1;
      s = 1e-300;
    }
    const double d = sqrt(s);
    R[j * k + j] = d;
    for (int c = j + 1; c < k; ++c) {
      double t = G[j * k + c];
      for (int m = 0; m < j; ++m) t -= R[m * k + j] * R[m * k + c];
      R[j * k + c] = t / d;
    }
  }
  // inverse of the upper-triangular R, column by column
  for (int t = 0; t < k * k; ++t) Rinv[t] = 0.0;
  for (int c = 0; c < k; ++c) {
    Rinv[c * k + c] = 1.0 / R[c * k + c];
    for (int rr = c - 1; rr >= 0; --rr) {
      double s = 0.0;
      for (int m = rr + 1; m <= c; ++m) s += R[rr * k + m] * Rinv[m * k + c];
      Rinv[rr * k + c] = -s / R[rr * k + rr];
    }
  }
}

// out_i = A_i Rinv  (rows times an upper-triangular k x k)
template <typename T>
__global__ void __launch_bounds__(kSolveBlock) rmul_kernel(T* out, const T* A, const double* Rinv,
                                                           int64_t n, int k) {
  __shared__ T ri[kMaxK * kMaxK];
  for (int t = threadIdx.x; t < k * k; t += kSolveBlock) ri[t] = (T)Rinv[t];
  __syncthreads();
  const int64_t m = n * k;
  for (int64_t e = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * kSolveBlock) {
    const int64_t i = e / k;
    const int b = (int)(e - i * k);
    const T* ar = A + i * k;
    T v = T(0);
    for (int a = 0; a <= b; ++a) v += ar[a] * ri[a * k + b];
    out[e] = v;
  }
}

}  // namespace pspec
