// pspec_solve_lockstep: the solve of Section 2 -- trust-region Newton with
// truncated-CG subproblems on the Grassmann manifold, p lowered stage by
// stage toward 1, then k-means and RCut -- for every graph of a batched handle
// at once, in lockstep.
//
// One launch serves the whole batch at every step: each evaluation and each
// Hessian product is one launch of the edge kernel over the concatenated CSR
// (per-task sums, then one block per graph), and every n x k operation is one
// launch over the rows of all graphs, split into tiles of kLsTile rows that
// never cross a graph.  Per-graph sums (Gram matrices, dots) are written per
// tile and added per graph in tile order, in FP64.  Every per-graph decision
// -- the truncated-CG recurrences, the trust-region ratio, radius and
// acceptance, the stage's stopping tests -- is taken on the device, one
// thread (or warp) per graph.  The host reads one array of G flags per chunk
// of CG iterations and one per Newton step, for the whole batch, and replays
// the chunk as a CUDA graph.
//
// Each graph runs the algorithm of pspec_solve with the same options: a
// graph whose truncated CG has stopped, whose stage has ended (converged or
// at max_outer) or that is not solved at all (fewer vertices than k) is left
// out of every launch -- its tasks and tiles return at once -- until the
// others catch up, so its iterates are the ones it would have alone.  Only
// the summation order of the reductions differs from pspec_solve.  Stages
// are synchronous: the batch moves to the next p when every graph has
// finished the current one.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "epilogue.cuh"
#include "internal.h"

namespace pspec {

namespace {

constexpr int kLsTile = 256;  // rows per tile = threads per block of the row kernels
constexpr int kLsWarps = kLsTile / 32;
constexpr int kLsMaxStages = 32;

// Per-graph state of the solve (device array, one entry per graph).
struct LsState {
  // truncated CG of the current Newton step (Steihaug-Toint recurrences)
  double cg_Delta;  // radius of the subproblem
  double rr, norm_r0, stop, e_Pe, e_Pd, d_Pd, alpha, step, beta, d_Hd;
  // trust region
  double f, gnorm, gnorm0, Delta;
  double rho;  // the last decision's ratio, and its CG count, stop reason and
  int last_j, last_reason, stepped;  // whether the graph took that step (the verbose trace)
  int j, done, reason, boundary;  // CG iterations, stopped, why (1..4), on the boundary
  int active;                     // still iterating in the current stage
  int converged;                  // the current stage converged
  int outer, inner;               // the current stage's Newton steps and CG iterations
  int accept;                     // the last trial point was accepted
  int status;                     // status bits met since the last decision
  int error_bits;                 // status bits that ended the graph's solve (sticky)
  int chol_bad;                   // Cholesky-QR met a Gram matrix that is not positive definite
  int all_converged;              // every stage so far converged
  int valid;                      // solved at all (n >= k)
};

// Offsets of the per-graph FP64 scalars in sc[G][stride] (kk = k*k).
struct LsOff {
  int M, Mn, Gm, Gram, Rinv;  // U^T egrad (iterate, trial), U^T H delta, Gram, R^-1
  int nd, ndn;                // N[16], D[16] of the iterate and of the trial point
  int F, Fn, gd, gdn, dots;   // F, F trial, <rg,rg>, <rg_new,rg_new>, <rg,eta>, <eta,r>
  int stride;
};

LsOff make_off(int k) {
  const int kk = k * k;
  LsOff o;
  o.M = 0;
  o.Mn = kk;
  o.Gm = 2 * kk;
  o.Gram = 3 * kk;
  o.Rinv = 4 * kk;
  o.nd = 5 * kk;
  o.ndn = o.nd + 32;
  o.F = o.ndn + 32;
  o.Fn = o.F + 1;
  o.gd = o.F + 2;
  o.gdn = o.F + 3;
  o.dots = o.F + 4;
  o.stride = ((o.dots + 2 + 3) / 4) * 4;
  return o;
}

// Options the device decisions need.
struct LsOpts {
  double gtol_rel, gtol_abs, theta, kappa, Delta_bar, Delta0, rho_prime, rho_reg;
  int max_outer, max_inner;
};

// Block sum of ND per-thread float-float values in a fixed order (warp
// trees, then warps in order); out (shared, ND doubles) is valid after the
// call in every thread.
template <int ND>
__device__ __forceinline__ void ls_block_sum(float2 (&v)[ND], double* out) {
  __shared__ float2 s_w[kLsWarps][ND];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < ND; ++q)
    for (int off = 16; off > 0; off >>= 1) v[q] = ff_add(v[q], shfl_xor_ff(v[q], off));
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < ND; ++q) s_w[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x < ND) {
    float2 acc = make_float2(0.f, 0.f);
    for (int ww = 0; ww < kLsWarps; ++ww) acc = ff_add(acc, s_w[ww][threadIdx.x]);
    out[threadIdx.x] = ff_to_double(acc);
  }
  __syncthreads();
}

// The tile's share of A^T B (k x k) from its rows staged in shared memory
// (rows x k, row-major) into part[0..k*k): thread t owns the pair t mod k^2
// and every (256 / k^2)-th row; products in FP32 FMAs, 16 at a time, then a
// compensated sum; the row groups are added in order in float-float.
__device__ __forceinline__ void ls_tile_gram(const float* sa, const float* sb, int rows, int k,
                                             double* part) {
  __shared__ float2 s_p[kLsTile];
  const int nv = k * k;
  const int groups = kLsTile / nv;
  const int t = threadIdx.x;
  const int pr = t % nv, grp = t / nv;
  const bool worker = grp < groups;
  const int x = pr / k, y = pr - (pr / k) * k;
  Kahan acc;
  acc.init();
  if (worker) {
    float part16 = 0.f;
    int cnt = 0;
    for (int r = grp; r < rows; r += groups) {
      part16 = fmaf(sa[r * k + x], sb[r * k + y], part16);
      if (++cnt == 16) {
        acc.add(part16);
        part16 = 0.f;
        cnt = 0;
      }
    }
    acc.add(part16);
  }
  s_p[t] = worker ? kahan_to_ff(acc) : make_float2(0.f, 0.f);
  __syncthreads();
  if (t < nv) {
    float2 s = make_float2(0.f, 0.f);
    for (int q = 0; q < groups; ++q) s = ff_add(s, s_p[q * nv + t]);
    part[t] = ff_to_double(s);
  }
}

// Stage rows [row0, row0 + rows) of an n x k block into shared memory.
__device__ __forceinline__ void ls_stage(float* dst, const float* __restrict__ src, int64_t row0, int rows, int k) {
  const int cnt = rows * k;
  const float* p = src + row0 * k;
  for (int e = threadIdx.x; e < cnt; e += kLsTile) dst[e] = p[e];
}

// A k x k FP64 matrix as floats in shared memory.
__device__ __forceinline__ void ls_stage_matrix(float* dst, const double* M, int k) {
  for (int t = threadIdx.x; t < k * k; t += kLsTile) dst[t] = (float)M[t];
}

// ------------------------------------------------------------ reductions ---
// One block per graph: the graph's per-task sums (two per column) added in
// task order -- each thread a compensated sum over every (256/2K)-th task,
// then the threads in order in float-float -- and the graph's FP64 scalars.
// Evaluation (hvp = 0): N = half the first sums (both triangles stored), D,
// into sc[nd_off]; F = sum N/D into sc[F_off]; the gradient's p/D and
// p lambda/D into gs.  Hessian product at a kept point (hvp = 1): sigma_N,
// sigma_D, with N, D read from sc[nd_off]; the coefficients A = p(p-1)/D,
// lambda, B = p^2/D^2 (0 in Algorithm 1's form), sigma_D and
// E = sigma_N - 2 lambda sigma_D into gs.  Conditions go to the graph's
// status bits.
__global__ void __launch_bounds__(256) ls_reduce_kernel(const float* __restrict__ part,
                                                        const int32_t* __restrict__ graph_task, int K,
                                                        int hvp, double p, int alg1, double* gs, double* sc,
                                                        int stride, int nd_off, int F_off, const int* skip,
                                                        LsState* st) {
  const int b = blockIdx.x;
  if (skip[b]) return;
  __shared__ float2 s_part[256];
  __shared__ double s_tot[2 * kMaxK];
  const int NV = 2 * K;
  const int parts = blockDim.x / NV;
  const int v = threadIdx.x % NV, jj = threadIdx.x / NV;
  const int t0 = graph_task[b], t1 = graph_task[b + 1];
  Kahan acc;
  acc.init();
  if (jj < parts) {
    // eight tasks' loads in flight at a time, added in task order
    int t = t0 + jj;
    for (; t + 7 * parts < t1; t += 8 * parts) {
      float x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = __ldg(&part[(size_t)(t + u * parts) * NV + v]);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc.add(x[u]);
    }
    for (; t < t1; t += parts) acc.add(__ldg(&part[(size_t)t * NV + v]));
  }
  s_part[threadIdx.x] = kahan_to_ff(acc);
  __syncthreads();
  if (threadIdx.x < NV) {
    float2 tot = make_float2(0.f, 0.f);
    for (int q = 0; q < parts; ++q) tot = ff_add(tot, s_part[q * NV + threadIdx.x]);
    s_tot[threadIdx.x] = ff_to_double(tot);
  }
  __syncthreads();
  double* g = gs + (size_t)b * kGsStride;
  double* s = sc + (size_t)b * stride;
  if (threadIdx.x < K) {
    const int c = threadIdx.x;
    int flags = 0;
    if (!hvp) {
      const double N = 0.5 * s_tot[c], D = s_tot[K + c];
      s[nd_off + c] = N;
      s[nd_off + 16 + c] = D;
      if (!isfinite(N) || !isfinite(D)) flags |= kStatusNonFinite;
      else if (!(D > 0.0)) flags |= kStatusZeroColumn;
      g[kGsC0 + c] = p / D;
      g[kGsC1 + c] = p * (N / D) / D;
    } else {
      const double N = s[nd_off + c], D = s[nd_off + 16 + c];
      const double sN = s_tot[c], sD = s_tot[K + c];
      const double lam = N / D;
      if (!isfinite(sN) || !isfinite(sD)) flags |= kStatusNonFinite;
      g[kGsC0 + c] = p * (p - 1.0) / D;
      g[kGsC1 + c] = lam;
      g[kGsC2 + c] = alg1 ? 0.0 : p * p / (D * D);
      g[kGsC3 + c] = sD;
      g[kGsC4 + c] = sN - 2.0 * lam * sD;
    }
    if (flags) atomicOr(&st[b].status, flags);
  }
  if (!hvp) {
    __syncthreads();
    if (threadIdx.x == 0) {
      double F = 0.0;
      for (int c = 0; c < K; ++c) F += s[nd_off + c] / s[nd_off + 16 + c];
      s[F_off] = F;
    }
  }
}

// ------------------------------------------------- per-graph completion ---
// The row kernels walk the tiles grid-stride.  A tile writes its partial
// sums to part[tile]; the block that completes the last tile of a graph
// (per-graph arrival counter, reset by that block) adds the graph's partials
// in tile order and takes the graph's decision in the same launch.  The
// result does not depend on which block finishes last.
struct LsTiles {
  const int4* tiles;          // graph x, first row y, rows z
  const int32_t* graph_tile;  // [G+1] first tile of each graph
  int n;
  unsigned* arrive;           // [G] tiles of the graph done in this launch
  double* part;               // [n][PS] per-tile partial sums
  int PS;
};

__device__ __forceinline__ bool ls_arrive(unsigned* arrive, int b, int ntiles) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&arrive[b], 1u) == (unsigned)(ntiles - 1);
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// nv (<= 256) sums of the graph's tile partials [t0, t1) into out: thread j
// adds entry j mod nv of every (256 / nv)-th tile starting at t0 + j / nv,
// then the groups are added in order
__device__ __forceinline__ void ls_graph_sums(const double* part, int PS, int t0, int t1, int nv, double* out) {
  __shared__ double s_g[kLsTile];
  const int groups = kLsTile / nv;
  const int v = threadIdx.x % nv, grp = threadIdx.x / nv;
  double s = 0.0;
  if (grp < groups)
    for (int t = t0 + grp; t < t1; t += groups) s += __ldcg(&part[(size_t)t * PS + v]);
  s_g[threadIdx.x] = s;
  __syncthreads();
  if ((int)threadIdx.x < nv) {
    double tot = 0.0;
    for (int q = 0; q < groups; ++q) tot += s_g[q * nv + threadIdx.x];
    out[threadIdx.x] = tot;
  }
  __syncthreads();
}

// one sum of the graph's tile partials: thread j takes tiles t0 + j,
// t0 + j + 256, ..., then a fixed tree; every thread returns the total
__device__ __forceinline__ double ls_graph_sum1(const double* part, int PS, int t0, int t1) {
  __shared__ double s_r[kLsTile];
  double s = 0.0;
  for (int t = t0 + threadIdx.x; t < t1; t += kLsTile) s += __ldcg(&part[(size_t)t * PS]);
  s_r[threadIdx.x] = s;
  __syncthreads();
  for (int w = kLsTile / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_r[threadIdx.x] += s_r[threadIdx.x + w];
    __syncthreads();
  }
  const double total = s_r[0];
  __syncthreads();
  return total;
}

// R^T R = Gram (Cholesky) and R^-1, k x k, by one thread; a Gram matrix that
// is not numerically positive definite sets *bad
__device__ void ls_chol_inv(const double* Gm, int k, double* Ri, int* bad) {
  double R[kMaxK * kMaxK];
  for (int t = 0; t < k * k; ++t) R[t] = 0.0;
  for (int j = 0; j < k; ++j) {
    double d2 = Gm[j * k + j];
    for (int m = 0; m < j; ++m) d2 -= R[m * k + j] * R[m * k + j];
    if (!(d2 > 0.0)) {
      *bad = 1;
      d2 = 1e-300;
    }
    const double d = sqrt(d2);
    R[j * k + j] = d;
    for (int c = j + 1; c < k; ++c) {
      double t = Gm[j * k + c];
      for (int m = 0; m < j; ++m) t -= R[m * k + j] * R[m * k + c];
      R[j * k + c] = t / d;
    }
  }
  for (int t = 0; t < k * k; ++t) Ri[t] = 0.0;
  for (int c = 0; c < k; ++c) {
    Ri[c * k + c] = 1.0 / R[c * k + c];
    for (int r = c - 1; r >= 0; --r) {
      double t = 0.0;
      for (int m = r + 1; m <= c; ++m) t += R[r * k + m] * Ri[m * k + c];
      Ri[r * k + c] = -t / R[r * k + r];
    }
  }
}

// ------------------------------------------------------- row kernels ---
// The gradient rows of a tile, egrad = (p/D) Delta - (p lambda/D) phi_p(u)
// with its graph's coefficients (from the kept Delta rows Dl), and the tile's
// share of M = U^T egrad; the graph's last tile writes M.
__global__ void __launch_bounds__(kLsTile) ls_grad_gram_kernel(const float* __restrict__ U,
                                                               const float* __restrict__ Dl, float* egrad,
                                                               int k, const double* __restrict__ gs, float pm2,
                                                               LsTiles T, const int* skip, double* sc, int stride,
                                                               int M_off) {
  __shared__ float sa[kLsTile * kMaxK], sb[kLsTile * kMaxK];
  __shared__ float cA[kMaxK], cB[kMaxK];
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    const int b = td.x;
    if (skip[b]) continue;
    __syncthreads();  // the previous tile's shared data has been used
    if ((int)threadIdx.x < k) {
      const double* g = gs + (size_t)b * kGsStride;
      cA[threadIdx.x] = (float)g[kGsC0 + threadIdx.x];
      cB[threadIdx.x] = (float)g[kGsC1 + threadIdx.x];
    }
    __syncthreads();
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const int c = e % k;
      const float u = U[e0 + e];
      const float phu = abs_pow_pm2_clamped(u, pm2) * u;
      const float gv = cA[c] * Dl[e0 + e] - cB[c] * phu;
      egrad[e0 + e] = gv;
      sa[e] = u;
      sb[e] = gv;
    }
    __syncthreads();
    ls_tile_gram(sa, sb, td.z, k, T.part + (size_t)tile * T.PS);
    const int t0 = T.graph_tile[b], t1 = T.graph_tile[b + 1];
    if (ls_arrive(T.arrive, b, t1 - t0)) {
      ls_graph_sums(T.part, T.PS, t0, t1, k * k, sc + (size_t)b * stride + M_off);
      if (threadIdx.x == 0) T.arrive[b] = 0u;
    }
  }
}

// The Hessian-product rows of a tile from the edge kernel's sparse part S
// (held in HV, overwritten), HV = A (S - lambda |u|^(p-2) v) - B (Delta sigma_D
// + phi_p(u) E) with its graph's coefficients, and the tile's share of
// Gm = U^T HV; the graph's last tile writes Gm.
__global__ void __launch_bounds__(kLsTile) ls_hvp_gram_kernel(const float* __restrict__ U,
                                                              const float* __restrict__ V,
                                                              const float* __restrict__ Dl, float* HV, int k,
                                                              const double* __restrict__ gs, float pm2, LsTiles T,
                                                              const int* skip, double* sc, int stride, int Gm_off) {
  __shared__ float sa[kLsTile * kMaxK], sb[kLsTile * kMaxK];
  __shared__ HvpCoef cf[kMaxK];
  const bool zero_rule = pm2 != 0.0f;
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    const int b = td.x;
    if (skip[b]) continue;
    __syncthreads();
    if ((int)threadIdx.x < k) {
      const double* g = gs + (size_t)b * kGsStride;
      const int c = threadIdx.x;
      cf[c] = HvpCoef{(float)g[kGsC0 + c], (float)g[kGsC1 + c], (float)g[kGsC2 + c], (float)g[kGsC3 + c],
                      (float)g[kGsC4 + c]};
    }
    __syncthreads();
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const int c = e % k;
      const float u = U[e0 + e];
      const float h = hvp_entry(HV[e0 + e], u, V[e0 + e], Dl[e0 + e], cf[c], pm2, zero_rule);
      HV[e0 + e] = h;
      sa[e] = u;
      sb[e] = h;
    }
    __syncthreads();
    ls_tile_gram(sa, sb, td.z, k, T.part + (size_t)tile * T.PS);
    const int t0 = T.graph_tile[b], t1 = T.graph_tile[b + 1];
    if (ls_arrive(T.arrive, b, t1 - t0)) {
      ls_graph_sums(T.part, T.PS, t0, t1, k * k, sc + (size_t)b * stride + Gm_off);
      if (threadIdx.x == 0) T.arrive[b] = 0u;
    }
  }
}

// The tile's share of A^T A; the graph's last tile writes the Gram matrix and
// its Cholesky factor's inverse R^-1 (Cholesky-QR).
__global__ void __launch_bounds__(kLsTile) ls_gram_chol_kernel(const float* __restrict__ A, int k, LsTiles T,
                                                               const int* skip, double* sc, int stride,
                                                               int gram_off, int rinv_off, LsState* st) {
  __shared__ float sa[kLsTile * kMaxK];
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    const int b = td.x;
    if (skip[b]) continue;
    __syncthreads();
    ls_stage(sa, A, td.y, td.z, k);
    __syncthreads();
    ls_tile_gram(sa, sa, td.z, k, T.part + (size_t)tile * T.PS);
    const int t0 = T.graph_tile[b], t1 = T.graph_tile[b + 1];
    if (ls_arrive(T.arrive, b, t1 - t0)) {
      double* x = sc + (size_t)b * stride;
      ls_graph_sums(T.part, T.PS, t0, t1, k * k, x + gram_off);
      if (threadIdx.x == 0) {
        ls_chol_inv(x + gram_off, k, x + rinv_off, &st[b].chol_bad);
        T.arrive[b] = 0u;
      }
    }
  }
}

// rg = egrad - U M (M = U^T egrad of the graph) and the tile's <rg, rg>; the
// graph's last tile writes <rg, rg>.
__global__ void __launch_bounds__(kLsTile) ls_proj_dot_kernel(float* rg, const float* __restrict__ egrad,
                                                              const float* __restrict__ U, double* sc, int stride,
                                                              int M_off, int gd_off, int k, LsTiles T,
                                                              const int* skip) {
  __shared__ float su[kLsTile * kMaxK];
  __shared__ float sm[kMaxK * kMaxK];
  __shared__ double s_out[1];
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    const int b = td.x;
    if (skip[b]) continue;
    __syncthreads();
    ls_stage(su, U, td.y, td.z, k);
    ls_stage_matrix(sm, sc + (size_t)b * stride + M_off, k);
    __syncthreads();
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    Kahan acc;
    acc.init();
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const int r = e / k, c = e - (e / k) * k;
      float v = egrad[e0 + e];
      for (int a = 0; a < k; ++a) v -= su[r * k + a] * sm[a * k + c];
      rg[e0 + e] = v;
      acc.add(v * v);
    }
    float2 v1[1] = {kahan_to_ff(acc)};
    ls_block_sum<1>(v1, s_out);
    if (threadIdx.x == 0) T.part[(size_t)tile * T.PS] = s_out[0];
    const int t0 = T.graph_tile[b], t1 = T.graph_tile[b + 1];
    if (ls_arrive(T.arrive, b, t1 - t0)) {
      const double tot = ls_graph_sum1(T.part, T.PS, t0, t1);
      if (threadIdx.x == 0) {
        sc[(size_t)b * stride + gd_off] = tot;
        T.arrive[b] = 0u;
      }
    }
  }
}

// The Riemannian Hessian's rows Hd = He - U Gm - delta M (Gm = U^T He, M =
// U^T egrad of the graph) and the tile's <delta, Hd>.  The graph's last tile
// takes truncated CG's curvature step: alpha = <r,r> / <delta, H delta>, or,
// on negative curvature or when the step would leave the trust region, the
// step tau to the boundary.
__global__ void __launch_bounds__(kLsTile) ls_hess_kernel(float* Hd, const float* __restrict__ He,
                                                          const float* __restrict__ U,
                                                          const float* __restrict__ delta, const double* sc,
                                                          int stride, int Gm_off, int M_off, int k, LsTiles T,
                                                          const int* skip, LsState* st) {
  __shared__ float su[kLsTile * kMaxK], sd[kLsTile * kMaxK];
  __shared__ float sg[kMaxK * kMaxK], sm[kMaxK * kMaxK];
  __shared__ double s_out[1];
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    const int b = td.x;
    if (skip[b]) continue;
    __syncthreads();
    ls_stage(su, U, td.y, td.z, k);
    ls_stage(sd, delta, td.y, td.z, k);
    const double* x = sc + (size_t)b * stride;
    ls_stage_matrix(sg, x + Gm_off, k);
    ls_stage_matrix(sm, x + M_off, k);
    __syncthreads();
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    Kahan acc;
    acc.init();
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const int r = e / k, c = e - (e / k) * k;
      float v = He[e0 + e];
      for (int a = 0; a < k; ++a) v -= su[r * k + a] * sg[a * k + c] + sd[r * k + a] * sm[a * k + c];
      Hd[e0 + e] = v;
      acc.add(sd[e] * v);
    }
    float2 v1[1] = {kahan_to_ff(acc)};
    ls_block_sum<1>(v1, s_out);
    if (threadIdx.x == 0) T.part[(size_t)tile * T.PS] = s_out[0];
    const int t0 = T.graph_tile[b], t1 = T.graph_tile[b + 1];
    if (ls_arrive(T.arrive, b, t1 - t0)) {
      const double dHd = ls_graph_sum1(T.part, T.PS, t0, t1);
      if (threadIdx.x == 0) {
        LsState& q = st[b];
        q.d_Hd = dHd;
        const double D2 = q.cg_Delta * q.cg_Delta;
        const double alpha = dHd != 0.0 ? q.rr / dHd : INFINITY;
        const double e_Pe_new = q.e_Pe + 2.0 * alpha * q.e_Pd + alpha * alpha * q.d_Pd;
        if (dHd <= 0.0 || e_Pe_new >= D2) {
          q.step = (-q.e_Pd + sqrt(q.e_Pd * q.e_Pd + q.d_Pd * (D2 - q.e_Pe))) / q.d_Pd;
          q.alpha = 0.0;
          q.boundary = 1;
          q.reason = dHd <= 0.0 ? 1 : 2;
        } else {
          q.step = alpha;
          q.alpha = alpha;
          q.e_Pe = e_Pe_new;
        }
        T.arrive[b] = 0u;
      }
    }
  }
}

// eta += step delta and r += step Hd, with the tile's <r, r> unless the step
// ended on the boundary (H eta is not kept: r starts at rg and takes every
// step's Hd, so H eta = r - rg when CG stops).  The graph's last tile ends
// the CG iteration: stop on the boundary, at the residual threshold or at
// max_inner (the graph is then flagged in skip); otherwise beta and the
// recurrences for <eta, delta> and <delta, delta>.
__global__ void __launch_bounds__(kLsTile) ls_cg_update_kernel(float* eta, float* r,
                                                               const float* __restrict__ delta,
                                                               const float* __restrict__ Hd, int k, LsTiles T,
                                                               int* skip, LsState* st, int max_inner) {
  __shared__ double s_out[1];
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    const int b = td.x;
    if (skip[b]) continue;
    const float step = (float)st[b].step;
    const bool bnd = st[b].boundary != 0;
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    Kahan acc;
    acc.init();
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const int64_t i = e0 + e;
      eta[i] += step * delta[i];
      const float rn = r[i] + step * Hd[i];
      r[i] = rn;
      if (!bnd) acc.add(rn * rn);
    }
    float2 v1[1] = {kahan_to_ff(acc)};
    ls_block_sum<1>(v1, s_out);
    if (threadIdx.x == 0) T.part[(size_t)tile * T.PS] = s_out[0];
    const int t0 = T.graph_tile[b], t1 = T.graph_tile[b + 1];
    if (ls_arrive(T.arrive, b, t1 - t0)) {
      const double rr_new = ls_graph_sum1(T.part, T.PS, t0, t1);
      if (threadIdx.x == 0) {
        LsState& q = st[b];
        q.j += 1;
        if (q.boundary) {
          q.done = 1;
        } else {
          const double beta = rr_new / q.rr;
          const double alpha_d = q.alpha;
          q.rr = rr_new;
          if (sqrt(rr_new) <= q.stop) {
            q.done = 1;
            q.reason = 3;
          } else if (q.j >= max_inner) {
            q.done = 1;
            q.reason = 4;
          } else {
            q.beta = beta;
            q.e_Pd = beta * (q.e_Pd + alpha_d * q.d_Pd);
            q.d_Pd = rr_new + beta * beta * q.d_Pd;
          }
        }
        if (q.done) skip[b] = 1;
        T.arrive[b] = 0u;
      }
    }
  }
}

// delta = -r + beta delta
__global__ void __launch_bounds__(kLsTile) ls_direction_kernel(float* delta, const float* __restrict__ r, int k,
                                                               LsTiles T, const int* skip, const LsState* st) {
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    if (skip[td.x]) continue;
    const float beta = (float)st[td.x].beta;
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    for (int e = threadIdx.x; e < cnt; e += kLsTile) delta[e0 + e] = -r[e0 + e] + beta * delta[e0 + e];
  }
}

// truncated CG's start: eta = 0, r = rg, delta = -rg
__global__ void __launch_bounds__(kLsTile) ls_tcg_init_kernel(float* eta, float* r, float* delta,
                                                              const float* __restrict__ rg, int k, LsTiles T,
                                                              const int* skip) {
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    if (skip[td.x]) continue;
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const float g = rg[e0 + e];
      eta[e0 + e] = 0.f;
      r[e0 + e] = g;
      delta[e0 + e] = -g;
    }
  }
}

// out = X + Y
__global__ void __launch_bounds__(kLsTile) ls_add_kernel(float* out, const float* __restrict__ X,
                                                         const float* __restrict__ Y, int k, LsTiles T,
                                                         const int* skip) {
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    if (skip[td.x]) continue;
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    for (int e = threadIdx.x; e < cnt; e += kLsTile) out[e0 + e] = X[e0 + e] + Y[e0 + e];
  }
}

// the tile's <rg, eta> and <eta, r> (the model's decrease, <eta, H eta> =
// <eta, r> - <eta, rg>); the graph's
// last tile writes both
__global__ void __launch_bounds__(kLsTile) ls_dots2_kernel(const float* __restrict__ rg,
                                                           const float* __restrict__ eta,
                                                           const float* __restrict__ r, int k, LsTiles T,
                                                           const int* skip, double* sc, int stride, int dots_off) {
  __shared__ double s_out[2];
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    const int b = td.x;
    if (skip[b]) continue;
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    Kahan a0, a1;
    a0.init();
    a1.init();
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const float x = eta[e0 + e];
      a0.add(rg[e0 + e] * x);
      a1.add(x * r[e0 + e]);
    }
    float2 v2[2] = {kahan_to_ff(a0), kahan_to_ff(a1)};
    ls_block_sum<2>(v2, s_out);
    if (threadIdx.x < 2) T.part[(size_t)tile * T.PS + threadIdx.x] = s_out[threadIdx.x];
    const int t0 = T.graph_tile[b], t1 = T.graph_tile[b + 1];
    if (ls_arrive(T.arrive, b, t1 - t0)) {
      ls_graph_sums(T.part, T.PS, t0, t1, 2, sc + (size_t)b * stride + dots_off);
      if (threadIdx.x == 0) T.arrive[b] = 0u;
    }
  }
}

// out = A R^-1 (R^-1 upper triangular, the graph's); in place when out == A
// (the tile is staged first)
__global__ void __launch_bounds__(kLsTile) ls_rmul_kernel(float* out, const float* A, const double* sc,
                                                          int stride, int R_off, int k, LsTiles T,
                                                          const int* skip) {
  __shared__ float sa[kLsTile * kMaxK];
  __shared__ float sr[kMaxK * kMaxK];
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    if (skip[td.x]) continue;
    __syncthreads();
    ls_stage(sa, A, td.y, td.z, k);
    ls_stage_matrix(sr, sc + (size_t)td.x * stride + R_off, k);
    __syncthreads();
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const int r = e / k, c = e - (e / k) * k;
      float v = 0.f;
      for (int a = 0; a <= c; ++a) v += sa[r * k + a] * sr[a * k + c];
      out[e0 + e] = v;
    }
  }
}

// the rows of every graph whose trial point was accepted move to the iterate
__global__ void __launch_bounds__(kLsTile) ls_accept_rows_kernel(float* U, const float* __restrict__ Un,
                                                                 float* eg, const float* __restrict__ egn,
                                                                 float* dk, const float* __restrict__ dkn,
                                                                 float* rg, const float* __restrict__ rgn, int k,
                                                                 LsTiles T, const LsState* st) {
  for (int tile = blockIdx.x; tile < T.n; tile += gridDim.x) {
    const int4 td = __ldg(&T.tiles[tile]);
    if (!st[td.x].accept) continue;
    const int64_t e0 = (int64_t)td.y * k;
    const int cnt = td.z * k;
    for (int e = threadIdx.x; e < cnt; e += kLsTile) {
      const int64_t i = e0 + e;
      U[i] = Un[i];
      eg[i] = egn[i];
      dk[i] = dkn[i];
      rg[i] = rgn[i];
    }
  }
}

// ------------------------------------------------- per-graph decisions ---
// Opens the graph's next Newton step, or ends its stage: converged when
// ||rg|| <= max(gtol_abs, gtol_rel ||rg_0||), ended at max_outer.  An open
// step starts truncated CG at eta = 0 with the stopping threshold
// ||rg|| min(||rg||^theta, kappa).
__device__ void ls_next_step(LsState& s, const LsOpts& o, int* skip_newton, int* skip_cg) {
  if (s.active) {
    if (s.gnorm <= fmax(o.gtol_abs, o.gtol_rel * s.gnorm0)) {
      s.converged = 1;
      s.active = 0;
    } else if (s.outer >= o.max_outer) {
      s.active = 0;
    }
  }
  if (!s.active) {
    s.done = 1;
    *skip_newton = 1;
    *skip_cg = 1;
    return;
  }
  s.outer += 1;
  s.cg_Delta = s.Delta;
  s.rr = s.gnorm * s.gnorm;
  s.norm_r0 = s.gnorm;
  s.stop = s.gnorm * fmin(pow(s.gnorm, o.theta), o.kappa);
  s.e_Pe = 0.0;
  s.e_Pd = 0.0;
  s.d_Pd = s.rr;
  s.alpha = s.step = s.beta = s.d_Hd = 0.0;
  s.j = 0;
  s.done = 0;
  s.reason = 0;
  s.boundary = 0;
  *skip_newton = 0;
  *skip_cg = 0;
}

__global__ void ls_init_kernel(LsState* st, const int* valid, int G) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < G; b += gridDim.x * blockDim.x) {
    LsState s{};
    s.valid = valid[b];
    s.all_converged = 1;
    s.done = 1;
    st[b] = s;
  }
}

// A stage opens: every graph that is solved and has met no error iterates.
__global__ void ls_stage_open_kernel(LsState* st, int* skip_newton, int* skip_cg, int G) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < G; b += gridDim.x * blockDim.x) {
    LsState& s = st[b];
    s.active = s.valid && s.error_bits == 0;
    s.converged = 0;
    s.outer = 0;
    s.inner = 0;
    s.status = 0;
    s.accept = 0;
    s.done = 1;
    skip_newton[b] = s.active ? 0 : 1;
    skip_cg[b] = 1;
  }
}

// After the stage's first evaluation: a graph whose evaluation met a
// non-finite value or a zero column stops with that error; the others take
// f, ||rg||, the radius Delta_0 and open their first Newton step.
__global__ void ls_stage_begin_kernel(LsState* st, const double* sc, LsOff off, LsOpts o, int* skip_newton,
                                      int* skip_cg, int G) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < G; b += gridDim.x * blockDim.x) {
    LsState& s = st[b];
    if (s.active) {
      const double* x = sc + (size_t)b * off.stride;
      if (s.status != 0) {
        s.error_bits = s.status;
        s.active = 0;
      } else {
        s.f = x[off.F];
        s.gnorm = sqrt(fmax(x[off.gd], 0.0));
        s.gnorm0 = s.gnorm;
        s.Delta = o.Delta0;
      }
      s.status = 0;
    }
    ls_next_step(s, o, &skip_newton[b], &skip_cg[b]);
  }
}

// The trust-region decision of every graph that took a Newton step: the
// ratio of actual to model decrease (regularised by rho_reg max(1, |f|)),
// the 1/4 and 3/4 radius rules, acceptance when the model decreased and
// rho > rho_prime (a trial point whose evaluation or Hessian products met a
// non-finite value or a zero column is rejected); an accepted point's F,
// ||rg||, U^T egrad and N, D become the iterate's.  Then the graph's next
// Newton step opens (or its stage ends).
__global__ void ls_decide_kernel(LsState* st, double* sc, LsOff off, LsOpts o, int kk, int* skip_newton,
                                 int* skip_cg, int G) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < G; b += gridDim.x * blockDim.x) {
    LsState& s = st[b];
    s.accept = 0;
    s.stepped = 0;
    if (skip_newton[b]) continue;  // took no step
    double* x = sc + (size_t)b * off.stride;
    s.inner += s.j;
    s.stepped = 1;
    s.last_j = s.j;
    s.last_reason = s.reason;
    const bool on_boundary = s.boundary != 0;
    const double f_new = x[off.Fn];
    const bool trial_bad = s.status != 0 || !isfinite(f_new);
    s.status = 0;
    const double reg = o.rho_reg * fmax(1.0, fabs(s.f));
    const double num = s.f - f_new + reg;
    const double den = -(x[off.dots] + 0.5 * (x[off.dots + 1] - x[off.dots])) + reg;  // <rg,eta> + <eta,H eta>/2
    const bool model_decreased = den >= 0.0 && !trial_bad;
    const double rho = trial_bad ? NAN : (den != 0.0 ? num / den : -INFINITY);
    s.rho = rho;
    if (!model_decreased || rho < 0.25 || isnan(rho))
      s.Delta *= 0.25;
    else if (rho > 0.75 && on_boundary)
      s.Delta = fmin(2.0 * s.Delta, o.Delta_bar);
    if (model_decreased && rho > o.rho_prime) {
      s.accept = 1;
      s.f = f_new;
      s.gnorm = sqrt(fmax(x[off.gdn], 0.0));
      for (int t = 0; t < kk; ++t) x[off.M + t] = x[off.Mn + t];
      for (int t = 0; t < 32; ++t) x[off.nd + t] = x[off.ndn + t];
    }
    ls_next_step(s, o, &skip_newton[b], &skip_cg[b]);
  }
}

// A stage ends: its counters, F and ||rg|| per graph into the statistics.
__global__ void ls_stage_close_kernel(LsState* st, int ip, int* s_outer, int* s_inner, double* s_f,
                                      double* s_gnorm, int G) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < G; b += gridDim.x * blockDim.x) {
    LsState& s = st[b];
    if (ip < kLsMaxStages) {
      const size_t q = (size_t)b * kLsMaxStages + ip;
      s_outer[q] = s.outer;
      s_inner[q] = s.inner;
      s_f[q] = s.f;
      s_gnorm[q] = s.gnorm;
    }
    if (s.valid && s.error_bits == 0 && !s.converged) s.all_converged = 0;
  }
}

// ------------------------------------------------------------------ RCut ---
// RCut of every graph (Section 3.1): per row the weight of its entries
// leaving its cluster (a warp per row, FP64), then per graph and cluster the
// cut and the size in a fixed order, RCut = sum of cut / size over non-empty
// clusters.  Entries never leave their graph, so labels compare within it.
__global__ void __launch_bounds__(256) ls_row_cut_kernel(const int64_t* __restrict__ rowptr,
                                                         const int32_t* __restrict__ col,
                                                         const double* __restrict__ val,
                                                         const int32_t* __restrict__ labels, int64_t n,
                                                         double* row_cut) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    const int li = labels[i];
    double acc = 0.0;
    for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32)
      if (labels[col[e]] != li) acc += val[e];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) row_cut[i] = acc;
  }
}

__global__ void __launch_bounds__(256) ls_rcut_kernel(const double* __restrict__ row_cut,
                                                      const int32_t* __restrict__ labels,
                                                      const int64_t* __restrict__ node_off, int k,
                                                      const int* solved, double* rcut) {
  const int b = blockIdx.x;
  if (!solved[b]) return;
  __shared__ double s_cut[256], s_cnt[256];
  const int64_t r0 = node_off[b], r1 = node_off[b + 1];
  double total = 0.0;
  for (int c = 0; c < k; ++c) {
    double cut = 0.0, cnt = 0.0;
    for (int64_t i = r0 + threadIdx.x; i < r1; i += 256)
      if (labels[i] == c) {
        cut += row_cut[i];
        cnt += 1.0;
      }
    s_cut[threadIdx.x] = cut;
    s_cnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) {
        s_cut[threadIdx.x] += s_cut[threadIdx.x + w];
        s_cnt[threadIdx.x] += s_cnt[threadIdx.x + w];
      }
      __syncthreads();
    }
    if (s_cnt[0] > 0.0) total += s_cut[0] / s_cnt[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) rcut[b] = total;
}

// ------------------------------------------------------------------ host ---
struct LsWork {
  std::vector<void*> allocs;
  float *U = nullptr, *Un, *eg, *egn, *rg, *rgn, *dk, *dkn, *eta, *r, *delta, *He, *Hd, *tmp;
  int4* tiles = nullptr;
  int32_t* graph_tile = nullptr;
  int n_tiles = 0;
  double* part = nullptr;
  int PS = 4;
  double* sc = nullptr;
  LsOff off;
  LsState* st = nullptr;
  int *skip_newton = nullptr, *skip_cg = nullptr, *valid = nullptr;
  int *s_outer = nullptr, *s_inner = nullptr;
  double *s_f = nullptr, *s_gnorm = nullptr;
  float* task_part = nullptr;
  double* row_cut = nullptr;
  double* rcut = nullptr;
  unsigned* arrive = nullptr;  // [G] per-graph tile arrival counters (zero between launches)
  int* h_flags = nullptr;      // pinned [2G]
  ~LsWork() {
    for (void* q : allocs) cudaFree(q);
    if (h_flags) cudaFreeHost(h_flags);
  }
  template <typename T>
  pspec_status alloc(T** out, size_t count) {
    void* q = nullptr;
    PSPEC_CUDA(cudaMalloc(&q, sizeof(T) * std::max<size_t>(1, count)));
    allocs.push_back(q);
    *out = (T*)q;
    return PSPEC_OK;
  }
};

struct Lockstep {
  pspec_graph* g = nullptr;
  int k = 0, kk = 0, G = 0;
  cudaStream_t s = nullptr;
  LsWork w;
  LsOpts o;
  int alg1 = 0;
  const int32_t* graph_task = nullptr;
  LsTiles T;
  int rows_blocks = 1;  // grid of the row kernels (they walk the tiles grid-stride)

  // F, N, D, Delta_p u (kept in dk), the Euclidean gradient, M = U^T egrad
  // and the Riemannian gradient rg with <rg, rg>, for every graph not in
  // skip_newton
  pspec_status eval(const float* U, double p, float* dk, float* eg, float* rg, int nd_off, int F_off, int M_off,
                    int gd_off) {
    const int* skip = w.skip_newton;
    EdgeLaunch L{U, nullptr, dk, nullptr, p, k, nullptr, w.task_part};
    L.graph_skip = skip;
    PSPEC_TRY(launch_eval_edges(g, L, s));
    TimedScope timer(g, "lockstep_eval_rows", s);
    ls_reduce_kernel<<<G, 256, 0, s>>>(w.task_part, graph_task, k, 0, p, 0, g->d_graph_scalars, w.sc,
                                       w.off.stride, nd_off, F_off, skip, w.st);
    ls_grad_gram_kernel<<<rows_blocks, kLsTile, 0, s>>>(U, dk, eg, k, g->d_graph_scalars, (float)p - 2.0f, T,
                                                        skip, w.sc, w.off.stride, M_off);
    ls_proj_dot_kernel<<<rows_blocks, kLsTile, 0, s>>>(rg, eg, U, w.sc, w.off.stride, M_off, gd_off, k, T, skip);
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  // one truncated-CG iteration of every graph not in skip_cg: the Hessian
  // product at the iterate (its kept Delta_p u, N and D) with U^T (H delta),
  // the Riemannian Hessian and the curvature step, the updates of eta, H eta
  // and r with the stopping tests, and the new direction
  pspec_status cg_iter(double p) {
    const int* skip = w.skip_cg;
    EdgeLaunch L{w.U, w.delta, w.He, nullptr, p, k, nullptr, w.task_part};
    L.keep_nd = w.sc;  // selects the kept-point kernel; a batch launch reads no N, D
    L.graph_skip = skip;
    L.alg1 = alg1 != 0;
    PSPEC_TRY(launch_hvp_edges(g, L, s));
    {
      TimedScope timer(g, "ls_reduce", s);
      ls_reduce_kernel<<<G, 256, 0, s>>>(w.task_part, graph_task, k, 1, p, alg1, g->d_graph_scalars, w.sc,
                                         w.off.stride, w.off.nd, 0, skip, w.st);
    }
    {
      TimedScope timer(g, "ls_hvp_gram", s);
      ls_hvp_gram_kernel<<<rows_blocks, kLsTile, 0, s>>>(w.U, w.delta, w.dk, w.He, k, g->d_graph_scalars,
                                                         (float)p - 2.0f, T, skip, w.sc, w.off.stride, w.off.Gm);
    }
    {
      TimedScope timer(g, "ls_hess", s);
      ls_hess_kernel<<<rows_blocks, kLsTile, 0, s>>>(w.Hd, w.He, w.U, w.delta, w.sc, w.off.stride, w.off.Gm,
                                                     w.off.M, k, T, skip, w.st);
    }
    {
      TimedScope timer(g, "ls_cg_update", s);
      ls_cg_update_kernel<<<rows_blocks, kLsTile, 0, s>>>(w.eta, w.r, w.delta, w.Hd, k, T, w.skip_cg,
                                                          w.st, o.max_inner);
    }
    {
      TimedScope timer(g, "ls_direction", s);
      ls_direction_kernel<<<rows_blocks, kLsTile, 0, s>>>(w.delta, w.r, k, T, skip, w.st);
    }
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  // Un = qf(U + eta) by Cholesky-QR twice
  pspec_status trial_point() {
    const int* skip = w.skip_newton;
    TimedScope timer(g, "lockstep_retraction", s);
    ls_add_kernel<<<rows_blocks, kLsTile, 0, s>>>(w.tmp, w.U, w.eta, k, T, skip);
    const float* src = w.tmp;
    for (int pass = 0; pass < 2; ++pass) {
      ls_gram_chol_kernel<<<rows_blocks, kLsTile, 0, s>>>(src, k, T, skip, w.sc, w.off.stride, w.off.Gram,
                                                          w.off.Rinv, w.st);
      ls_rmul_kernel<<<rows_blocks, kLsTile, 0, s>>>(w.Un, src, w.sc, w.off.stride, w.off.Rinv, k, T, skip);
      src = w.Un;
    }
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  // the pinned copy of a flag array; returns how many graphs are not flagged
  pspec_status count_open(const int* flags, int* open) {
    PSPEC_CUDA(cudaMemcpyAsync(w.h_flags, flags, sizeof(int) * G, cudaMemcpyDeviceToHost, s));
    PSPEC_CUDA(cudaStreamSynchronize(s));
    int c = 0;
    for (int b = 0; b < G; ++b) c += w.h_flags[b] == 0;
    *open = c;
    return PSPEC_OK;
  }
};

struct ChunkGraphs {
  bool enabled = true;
  std::vector<std::pair<double, cudaGraphExec_t>> entries;
  ~ChunkGraphs() {
    for (auto& e : entries) cudaGraphExecDestroy(e.second);
  }
};

pspec_status setup(Lockstep& S, const std::vector<int64_t>& off, int k) {
  pspec_graph* g = S.g;
  const int G = S.G;
  LsWork& w = S.w;
  const size_t m = (size_t)g->n * k;
  float** vecs[14] = {&w.U, &w.Un, &w.eg, &w.egn, &w.rg, &w.rgn, &w.dk, &w.dkn,
                      &w.eta, &w.r, &w.delta, &w.He, &w.Hd, &w.tmp};
  for (float** v : vecs) PSPEC_TRY(w.alloc(v, m));
  std::vector<int4> tiles;
  std::vector<int32_t> graph_tile(G + 1, 0);
  std::vector<int> valid(G, 0);
  for (int b = 0; b < G; ++b) {
    graph_tile[b] = (int32_t)tiles.size();
    const int64_t n_b = off[b + 1] - off[b];
    valid[b] = n_b >= k && n_b > 0;
    if (!valid[b]) continue;
    for (int64_t r0 = off[b]; r0 < off[b + 1]; r0 += kLsTile)
      tiles.push_back(make_int4(b, (int)r0, (int)std::min<int64_t>(kLsTile, off[b + 1] - r0), 0));
  }
  graph_tile[G] = (int32_t)tiles.size();
  w.n_tiles = (int)tiles.size();
  PSPEC_TRY(w.alloc(&w.tiles, tiles.size()));
  PSPEC_TRY(w.alloc(&w.graph_tile, G + 1));
  PSPEC_TRY(w.alloc(&w.valid, G));
  if (!tiles.empty())
    PSPEC_CUDA(cudaMemcpyAsync(w.tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, S.s));
  PSPEC_CUDA(cudaMemcpyAsync(w.graph_tile, graph_tile.data(), sizeof(int32_t) * (G + 1), cudaMemcpyHostToDevice, S.s));
  PSPEC_CUDA(cudaMemcpyAsync(w.valid, valid.data(), sizeof(int) * G, cudaMemcpyHostToDevice, S.s));
  w.PS = std::max(k * k, 4);
  PSPEC_TRY(w.alloc(&w.part, (size_t)std::max(1, w.n_tiles) * w.PS));
  w.off = make_off(k);
  PSPEC_TRY(w.alloc(&w.sc, (size_t)G * w.off.stride));
  PSPEC_CUDA(cudaMemsetAsync(w.sc, 0, sizeof(double) * G * w.off.stride, S.s));
  PSPEC_TRY(w.alloc(&w.st, G));
  PSPEC_TRY(w.alloc(&w.skip_newton, G));
  PSPEC_TRY(w.alloc(&w.skip_cg, G));
  PSPEC_TRY(w.alloc(&w.s_outer, (size_t)G * kLsMaxStages));
  PSPEC_TRY(w.alloc(&w.s_inner, (size_t)G * kLsMaxStages));
  PSPEC_TRY(w.alloc(&w.s_f, (size_t)G * kLsMaxStages));
  PSPEC_TRY(w.alloc(&w.s_gnorm, (size_t)G * kLsMaxStages));
  PSPEC_CUDA(cudaMemsetAsync(w.s_outer, 0, sizeof(int) * G * kLsMaxStages, S.s));
  PSPEC_CUDA(cudaMemsetAsync(w.s_inner, 0, sizeof(int) * G * kLsMaxStages, S.s));
  PSPEC_CUDA(cudaMemsetAsync(w.s_f, 0, sizeof(double) * G * kLsMaxStages, S.s));
  PSPEC_CUDA(cudaMemsetAsync(w.s_gnorm, 0, sizeof(double) * G * kLsMaxStages, S.s));
  const int64_t nt = task_count(g, k);
  if (nt < 0) return set_error(PSPEC_ERR_CUDA, "task partition");
  PSPEC_TRY(w.alloc(&w.task_part, (size_t)std::max<int64_t>(1, nt) * 2 * k));
  S.graph_task = g->tasks[q_index(q_of(k))].d_graph_task;
  if (!S.graph_task || !g->tasks[q_index(q_of(k))].d_task_graph || !g->d_graph_scalars || !g->d_node_off)
    return set_error(PSPEC_ERR_INVALID_ARG, "pspec_solve_lockstep: the handle has no per-graph task map");
  PSPEC_TRY(w.alloc(&w.row_cut, g->n));
  PSPEC_TRY(w.alloc(&w.rcut, G));
  PSPEC_CUDA(cudaMallocHost(&w.h_flags, sizeof(int) * 2 * std::max(1, G)));
  PSPEC_TRY(w.alloc(&w.arrive, G));
  PSPEC_CUDA(cudaMemsetAsync(w.arrive, 0, sizeof(unsigned) * G, S.s));
  S.T = LsTiles{w.tiles, w.graph_tile, w.n_tiles, w.arrive, w.part, w.PS};
  // the row kernels' grid: one block per tile, or with
  // PSPEC_LOCKSTEP_BLOCKS_PER_SM = b > 0 that many blocks per SM walking the
  // tiles
  int64_t rb = w.n_tiles;
  if (const char* env = std::getenv("PSPEC_LOCKSTEP_BLOCKS_PER_SM"))
    if (std::atoi(env) > 0) rb = std::min<int64_t>(rb, (int64_t)g->sm_count * std::atoi(env));
  S.rows_blocks = (int)std::max<int64_t>(1, rb);
  ls_init_kernel<<<(G + 255) / 256, 256, 0, S.s>>>(w.st, w.valid, G);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

pspec_status run_stages(Lockstep& S, const double* sched, int n_p, int verbose) {
  LsWork& w = S.w;
  const int G = S.G;
  const int chunk = 6;  // CG iterations per host check
  ChunkGraphs graphs;
  graphs.enabled = !S.g->timing.enabled && !(std::getenv("PSPEC_SOLVE_EAGER") &&
                                             std::getenv("PSPEC_SOLVE_EAGER")[0] == '1');
  for (int ip = 0; ip < n_p; ++ip) {
    const double p = sched[ip];
    ls_stage_open_kernel<<<(G + 255) / 256, 256, 0, S.s>>>(w.st, w.skip_newton, w.skip_cg, G);
    PSPEC_TRY(S.eval(w.U, p, w.dk, w.eg, w.rg, w.off.nd, w.off.F, w.off.M, w.off.gd));
    ls_stage_begin_kernel<<<1, 256, 0, S.s>>>(w.st, w.sc, w.off, S.o, w.skip_newton, w.skip_cg, G);
    PSPEC_CUDA(cudaGetLastError());
    int active = 0;
    PSPEC_TRY(S.count_open(w.skip_newton, &active));
    int step = 0;
    while (active > 0) {
      ++step;
      ls_tcg_init_kernel<<<S.rows_blocks, kLsTile, 0, S.s>>>(w.eta, w.r, w.delta, w.rg, S.k, S.T,
                                                              w.skip_cg);
      PSPEC_CUDA(cudaGetLastError());
      int chunks = 0;
      for (int it = 0; it < S.o.max_inner; it += chunk, ++chunks) {
        if (graphs.enabled && (step > 1 || it > 0)) {
          cudaGraphExec_t exec = nullptr;
          for (auto& e : graphs.entries)
            if (e.first == p) exec = e.second;
          if (!exec) {  // captured once per p: the buffers never move
            PSPEC_CUDA(cudaStreamBeginCapture(S.s, cudaStreamCaptureModeThreadLocal));
            pspec_status st = PSPEC_OK;
            for (int c = 0; c < chunk && st == PSPEC_OK; ++c) st = S.cg_iter(p);
            cudaGraph_t cg = nullptr;
            const cudaError_t e = cudaStreamEndCapture(S.s, &cg);
            if (st != PSPEC_OK) {
              if (cg) cudaGraphDestroy(cg);
              return st;
            }
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture(lockstep tCG chunk)");
            const cudaError_t ei = cudaGraphInstantiate(&exec, cg, 0);
            cudaGraphDestroy(cg);
            if (ei != cudaSuccess) return cuda_error(ei, "cudaGraphInstantiate(lockstep tCG chunk)");
            graphs.entries.push_back({p, exec});
          }
          PSPEC_CUDA(cudaGraphLaunch(exec, S.s));
        } else {
          for (int c = 0; c < std::min(chunk, S.o.max_inner - it); ++c) PSPEC_TRY(S.cg_iter(p));
        }
        int running = 0;
        PSPEC_TRY(S.count_open(w.skip_cg, &running));
        if (running == 0) break;
      }
      PSPEC_TRY(S.trial_point());
      PSPEC_TRY(S.eval(w.Un, p, w.dkn, w.egn, w.rgn, w.off.ndn, w.off.Fn, w.off.Mn, w.off.gdn));
      ls_dots2_kernel<<<S.rows_blocks, kLsTile, 0, S.s>>>(w.rg, w.eta, w.r, S.k, S.T, w.skip_newton, w.sc,
                                                           w.off.stride, w.off.dots);
      ls_decide_kernel<<<1, 256, 0, S.s>>>(w.st, w.sc, w.off, S.o, S.kk, w.skip_newton, w.skip_cg, G);
      ls_accept_rows_kernel<<<S.rows_blocks, kLsTile, 0, S.s>>>(w.U, w.Un, w.eg, w.egn, w.dk, w.dkn, w.rg, w.rgn,
                                                                S.k, S.T, w.st);
      PSPEC_CUDA(cudaGetLastError());
      const int before = active;
      if (verbose >= 2) {  // each graph that took this step: its decision, before the next step opens
        std::vector<LsState> hs(G);
        PSPEC_CUDA(cudaMemcpyAsync(hs.data(), w.st, sizeof(LsState) * G, cudaMemcpyDeviceToHost, S.s));
        PSPEC_CUDA(cudaStreamSynchronize(S.s));
        for (int b = 0; b < G; ++b)
          if (hs[b].stepped)
            std::fprintf(stderr, "pspec lockstep graph=%d p=%.3f step=%d f=%.10e |g|=%.3e tcg=%d(%d) rho=%.3f Delta=%.3e %s\n",
                         b, p, step, hs[b].f, hs[b].gnorm, hs[b].last_j, hs[b].last_reason, hs[b].rho, hs[b].Delta,
                         hs[b].accept ? "acc" : "rej");
      }
      PSPEC_TRY(S.count_open(w.skip_newton, &active));
      if (verbose)
        std::fprintf(stderr, "pspec lockstep p=%.3f step=%d graphs=%d tcg_chunks=%d still=%d\n", p, step, before,
                     chunks + 1, active);
    }
    ls_stage_close_kernel<<<(G + 255) / 256, 256, 0, S.s>>>(w.st, ip, w.s_outer, w.s_inner, w.s_f, w.s_gnorm, G);
    PSPEC_CUDA(cudaGetLastError());
  }
  return PSPEC_OK;
}

// The whole call on the handle's private stream (validated arguments).
pspec_status lockstep_impl(pspec_graph* g, int k, const double* p_schedule, int n_p, const pspec_solve_opts& o,
                           float* U_inout, int32_t* labels_out, double* rcut_out, int32_t* status_out,
                           pspec_solve_stats* stats_out, int n_threads, cudaStream_t s,
                           std::chrono::steady_clock::time_point t0) {
  const int G = g->n_graphs;
  const std::vector<int64_t>& off = g->h_node_off;
  Lockstep S;
  S.g = g;
  S.k = k;
  S.kk = k * k;
  S.G = G;
  S.s = s;
  S.alg1 = o.hessian_form == PSPEC_HESSIAN_ALG1 ? 1 : 0;
  const double Delta_bar = o.delta_bar_scale * std::sqrt((double)k);
  S.o = LsOpts{o.gtol_rel, o.gtol_abs, o.theta, o.kappa, Delta_bar, o.delta0_scale * Delta_bar, o.rho_prime,
               o.rho_reg, o.max_outer, o.max_inner};
  PSPEC_TRY(setup(S, off, k));
  LsWork& w = S.w;
  const size_t m = (size_t)g->n * k;
  PSPEC_CUDA(cudaMemcpyAsync(w.U, U_inout, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
  if (w.n_tiles > 0) PSPEC_TRY(run_stages(S, p_schedule, n_p, o.verbose));
  PSPEC_CUDA(cudaMemcpyAsync(U_inout, w.U, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
  std::vector<LsState> hs(G);
  std::vector<int> h_outer((size_t)G * kLsMaxStages), h_inner((size_t)G * kLsMaxStages);
  std::vector<double> h_f((size_t)G * kLsMaxStages), h_gn((size_t)G * kLsMaxStages);
  PSPEC_CUDA(cudaMemcpyAsync(hs.data(), w.st, sizeof(LsState) * G, cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaMemcpyAsync(h_outer.data(), w.s_outer, sizeof(int) * h_outer.size(), cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaMemcpyAsync(h_inner.data(), w.s_inner, sizeof(int) * h_inner.size(), cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaMemcpyAsync(h_f.data(), w.s_f, sizeof(double) * h_f.size(), cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaMemcpyAsync(h_gn.data(), w.s_gnorm, sizeof(double) * h_gn.size(), cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaStreamSynchronize(s));
  // per-graph status; the graphs whose solve ended without an error are
  // discretised and scored
  std::vector<int> solved(G, 0);
  for (int b = 0; b < G; ++b) {
    const LsState& x = hs[b];
    const int64_t n_b = off[b + 1] - off[b];
    rcut_out[b] = n_b == 0 ? 0.0 : NAN;
    pspec_status st = PSPEC_OK;
    if (n_b == 0) st = PSPEC_OK;
    else if (!x.valid) st = set_error(PSPEC_ERR_INVALID_ARG, "a graph has fewer vertices than k");
    else if (x.error_bits) st = status_error(x.error_bits);
    else if (x.chol_bad) st = set_error(PSPEC_ERR_NONFINITE, "Cholesky-QR met a Gram matrix that is not positive definite");
    else {
      st = x.all_converged ? PSPEC_OK : PSPEC_ERR_NOT_CONVERGED;
      solved[b] = 1;
    }
    status_out[b] = (int32_t)st;
  }
  std::vector<double> inertia(G, 0.0);
  {  // k-means of each solved graph's rows, host threads on streams of their own
    int device = 0;
    PSPEC_CUDA(cudaGetDevice(&device));
    std::atomic<int> next{0};
    auto worker = [&]() {
      cudaSetDevice(device);
      cudaStream_t ws = nullptr;
      const bool own = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) == cudaSuccess;
      for (int b = next.fetch_add(1); b < G; b = next.fetch_add(1)) {
        if (!solved[b]) continue;
        const int64_t r0 = off[b], n_b = off[b + 1] - r0;
        const pspec_status st =
            own ? pspec_kmeans(U_inout + r0 * k, n_b, k, PSPEC_F32, k, o.seed, o.kmeans_restarts, o.kmeans_max_iter,
                               labels_out + r0, nullptr, &inertia[b], ws)
                : PSPEC_ERR_CUDA;
        if (st != PSPEC_OK) {
          status_out[b] = (int32_t)st;
          solved[b] = 0;
        }
      }
      if (own) cudaStreamDestroy(ws);
    };
    std::vector<std::thread> pool;
    const int nt = std::max(1, std::min(n_threads, G));
    for (int i = 0; i < nt; ++i) pool.emplace_back(worker);
    for (std::thread& th : pool) th.join();
  }
  PSPEC_CUDA(cudaMemcpyAsync(w.valid, solved.data(), sizeof(int) * G, cudaMemcpyHostToDevice, s));
  const int rc_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((g->n + 7) / 8, (int64_t)g->sm_count * 16));
  ls_row_cut_kernel<<<rc_blocks, 256, 0, s>>>(g->d_rowptr, g->d_col, g->d_val64, labels_out, g->n, w.row_cut);
  ls_rcut_kernel<<<G, 256, 0, s>>>(w.row_cut, labels_out, g->d_node_off, k, w.valid, w.rcut);
  PSPEC_CUDA(cudaGetLastError());
  std::vector<double> h_rcut(G, 0.0);
  PSPEC_CUDA(cudaMemcpyAsync(h_rcut.data(), w.rcut, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaStreamSynchronize(s));
  const double seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int b = 0; b < G; ++b) {
    if (solved[b]) rcut_out[b] = h_rcut[b];
    if (!stats_out) continue;
    pspec_solve_stats& x = stats_out[b];
    std::memset(&x, 0, sizeof(x));
    x.n_stages = n_p;
    int64_t outer = 0, inner = 0;
    for (int ip = 0; ip < std::min(n_p, kLsMaxStages); ++ip) {
      const size_t q = (size_t)b * kLsMaxStages + ip;
      x.outer[ip] = h_outer[q];
      x.inner[ip] = h_inner[q];
      x.f[ip] = h_f[q];
      x.gnorm[ip] = h_gn[q];
      outer += h_outer[q];
      inner += h_inner[q];
    }
    x.hvp_calls = inner;
    x.eval_calls = hs[b].valid ? n_p + outer : 0;
    x.seconds = seconds;
    x.kmeans_inertia = inertia[b];
  }
  bool any_nc = false;
  for (int b = 0; b < G; ++b) {
    if (status_out[b] == PSPEC_ERR_NOT_CONVERGED) any_nc = true;
    else if (status_out[b] != PSPEC_OK)
      return set_error((pspec_status)status_out[b], "graph " + std::to_string(b) + ": the solve did not complete");
  }
  return any_nc ? PSPEC_ERR_NOT_CONVERGED : PSPEC_OK;
}

}  // namespace

}  // namespace pspec

using namespace pspec;

extern "C" pspec_status pspec_solve_lockstep(pspec_graph* g, int k, const double* p_schedule, int n_p,
                                             const pspec_solve_opts* opts, float* U_inout, int32_t* labels_out,
                                             double* rcut_out, int32_t* status_out, pspec_solve_stats* stats_out,
                                             int n_threads, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!g) return set_error(PSPEC_ERR_INVALID_ARG, "graph is NULL");
  if (g->h_node_off.empty()) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_solve_lockstep takes a batched handle");
  if (k < 1 || k > kMaxK) return set_error(PSPEC_ERR_INVALID_ARG, "k must be in [1, 16]");
  if (!U_inout || !labels_out || !rcut_out || !status_out)
    return set_error(PSPEC_ERR_INVALID_ARG, "NULL argument");
  if (n_threads < 1 || n_threads > 256) return set_error(PSPEC_ERR_INVALID_ARG, "n_threads must be in [1, 256]");
  if (g->n >= (int64_t)INT32_MAX - kLsTile)
    return set_error(PSPEC_ERR_INVALID_ARG, "pspec_solve_lockstep takes fewer than 2^31 - 256 vertices");
  pspec_solve_opts o;
  PSPEC_TRY(check_solve_args(p_schedule, n_p, opts, &o));
  PSPEC_TRY(check_block(U_inout, k, PSPEC_F32, "U_inout"));
  // the solve runs on the handle's private stream (CUDA graphs are captured
  // on it), after the caller's earlier work and before its later work
  cudaStream_t caller = (cudaStream_t)stream;
  if (!g->solve_stream) {
    PSPEC_CUDA(cudaStreamCreateWithFlags(&g->solve_stream, cudaStreamNonBlocking));
    PSPEC_CUDA(cudaEventCreateWithFlags(&g->solve_event, cudaEventDisableTiming));
  }
  PSPEC_CUDA(cudaEventRecord(g->solve_event, caller));
  PSPEC_CUDA(cudaStreamWaitEvent(g->solve_stream, g->solve_event, 0));
  const pspec_status st = lockstep_impl(g, k, p_schedule, n_p, o, U_inout, labels_out, rcut_out, status_out,
                                        stats_out, n_threads, g->solve_stream, t0);
  cudaEventRecord(g->solve_event, g->solve_stream);
  cudaStreamWaitEvent(caller, g->solve_event, 0);
  return st;
}
