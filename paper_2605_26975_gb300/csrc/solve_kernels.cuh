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
#include "epilogue.cuh"

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

// 16-byte vectors of T for the elementwise loops (all blocks are carved at
// 256-byte boundaries, so element 0 of every block is 16-byte aligned)
template <typename T> struct Vec16;
template <> struct Vec16<float> {
  static constexpr int W = 4;
  using type = float4;
  __device__ static float get(const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }
  __device__ static void set(float4& v, int i, float x) {
    if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
  }
};
template <> struct Vec16<double> {
  static constexpr int W = 2;
  using type = double2;
  __device__ static double get(const double2& v, int i) { return i == 0 ? v.x : v.y; }
  __device__ static void set(double2& v, int i, double x) {
    if (i == 0) v.x = x; else v.y = x;
  }
};

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
// G[a][b] = sum_i A_ia B_ib  (k x k, FP64 out).  A block stages tiles of
// kGramTile consecutive rows of A and B in shared memory (one coalesced copy
// of tile*k contiguous values each); thread t owns the pair p = t mod k^2 and
// the rows r = t div k^2 (mod 256 div k^2) of every tile, so all 256 threads
// work for any k.  A thread's share of a tile (at most 128 products) is
// summed with FMAs and added to its compensated running sum; then the row
// groups in order, then the grid.
constexpr int kGramTile = 128;

template <typename T>
__global__ void __launch_bounds__(kSolveBlock) gram_kernel(const T* __restrict__ A,
                                                           const T* __restrict__ B, int64_t n,
                                                           int k, double* G, GridRed gr,
                                                           const int* done) {
  using R = typename RedT<T>::type;
  if (done && *done) return;
  __shared__ __align__(16) T sa[kGramTile * kMaxK];
  __shared__ __align__(16) T sb[kGramTile * kMaxK];
  __shared__ R s_part[kSolveBlock];
  __shared__ R s_blk[kMaxK * kMaxK];
  __shared__ R s_tot[kMaxK * kMaxK];
  const int nv = k * k;
  const int groups = kSolveBlock / nv;  // row groups (>= 1 since k <= 16)
  const int t = threadIdx.x;
  const int pr = t % nv, grp = t / nv;
  const bool worker = grp < groups;
  const int a = pr / k, b = pr - (pr / k) * k;
  Acc<T> acc;
  acc.init();
  const int64_t ntiles = (n + kGramTile - 1) / kGramTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t r0 = tile * kGramTile;
    const int rows = (int)min((int64_t)kGramTile, n - r0);
    const int cnt = rows * k;
    __syncthreads();  // the previous tile has been consumed
    {  // tiles start at multiples of kGramTile rows: 16-byte aligned
      using V = Vec16<T>;
      using VT = typename V::type;
      const int cv = cnt / V::W;
      const VT* ga = reinterpret_cast<const VT*>(A + r0 * k);
      const VT* gb = reinterpret_cast<const VT*>(B + r0 * k);
      for (int e = t; e < cv; e += kSolveBlock) {
        reinterpret_cast<VT*>(sa)[e] = ga[e];
        reinterpret_cast<VT*>(sb)[e] = gb[e];
      }
      for (int e = cv * V::W + t; e < cnt; e += kSolveBlock) {
        sa[e] = A[r0 * k + e];
        sb[e] = B[r0 * k + e];
      }
    }
    __syncthreads();
    if (worker) {  // the tile's share in plain FMAs, then one compensated add
      T part = T(0);
      for (int r = grp; r < rows; r += groups) part = fma(sa[r * k + a], sb[r * k + b], part);
      acc.add(part);
    }
  }
  s_part[t] = worker ? acc.get() : red_zero(R());
  __syncthreads();
  if (t < nv) {
    R sum = red_zero(R());
    for (int q = 0; q < groups; ++q) sum = red_add(sum, s_part[q * nv + t]);
    s_blk[t] = sum;
  }
  __syncthreads();
  if (!grid_reduce_rt<R>(s_blk, s_tot, nv, gr)) return;
  for (int q = threadIdx.x; q < nv; q += kSolveBlock) G[q] = red_to_double(s_tot[q]);
}

// The FP32 Gram product for k a multiple of 4, with the tiles streamed by the
// TMA unit: a ring of kGramStages stages per block, each holding one full
// tile of A and of B, filled by two 1-D bulk copies (one elected thread) that
// complete on the stage's mbarrier; a stage is refilled with the block's tile
// kGramStages ahead as soon as all threads have read it.  Full tiles are 128
// rows of k floats (512k bytes, 16-byte aligned in the 256-byte aligned
// solver buffers); a ragged last tile is read with plain loads.  A thread
// owns a 4 x 4 block of the k x k output and a share of every tile's rows: a
// row costs it two 16-byte shared loads and 16 FMAs (each staged value is
// read k/4 times, not k).  Per-thread sums are FP32 within four tiles, then
// compensated.  Every wait is bounded: a block that gives up records a
// timeout in *status, waits (bounded) for its copies still in flight and
// leaves the sums undone.
constexpr int kGramStages = 3;
constexpr uint32_t kGramWaitTries = 2000;  // x up to 1 ms each
constexpr size_t kGramTileFloats = (size_t)kGramTile * kMaxK;
constexpr size_t gram_tma_smem_bytes() {
  return sizeof(float) * 2 * kGramTileFloats * kGramStages + sizeof(uint64_t) * kGramStages;
}

__global__ void __launch_bounds__(kSolveBlock) gram_tma_kernel(const float* __restrict__ A,
                                                               const float* __restrict__ B,
                                                               int64_t n, int k, double* G,
                                                               GridRed gr, const int* done,
                                                               int* status) {
  using R = float2;
  if (done && *done) return;
  extern __shared__ __align__(128) unsigned char gsm[];
  float* tiles = reinterpret_cast<float*>(gsm);  // [stage][A|B][kGramTileFloats]
  uint64_t* bars = reinterpret_cast<uint64_t*>(gsm + sizeof(float) * 2 * kGramTileFloats * kGramStages);
  __shared__ R s_blk[kMaxK * kMaxK];
  __shared__ R s_tot[kMaxK * kMaxK];
  const int nv = k * k;
  const int nb = k / 4;                  // 4 x 4 output blocks per side
  const int nblk = nb * nb;
  const int groups = kSolveBlock / nblk;  // row groups
  const int t = threadIdx.x;
  const int pb = t % nblk, grp = t / nblk;
  const bool worker = grp < groups;
  const int a0 = 4 * (pb / nb), b0 = 4 * (pb % nb);
  const int64_t nfull = n / kGramTile;
  const uint32_t tbytes = (uint32_t)(kGramTile * k * sizeof(float));
  auto issue = [&](int stage, int64_t tile) {
    float* dst = tiles + (size_t)stage * 2 * kGramTileFloats;
    mbar_arrive_expect_tx(&bars[stage], 2u * tbytes);
    tma_load_1d(dst, A + tile * kGramTile * k, tbytes, &bars[stage]);
    tma_load_1d(dst + kGramTileFloats, B + tile * kGramTile * k, tbytes, &bars[stage]);
  };
  if (t == 0) {
    for (int st = 0; st < kGramStages; ++st) mbar_init(&bars[st], 1);
    mbar_init_fence();
    for (int st = 0; st < kGramStages; ++st) {
      const int64_t tile = blockIdx.x + (int64_t)st * gridDim.x;
      if (tile < nfull) issue(st, tile);
    }
  }
  __syncthreads();
  Kahan acc[16];
  float part[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    acc[q].init();
    part[q] = 0.f;
  }
  // rows [r_lo, r_hi) of a staged tile into the 4 x 4 block
  auto accumulate = [&](const float* sa, const float* sb, int rows) {
    for (int r = grp; r < rows; r += groups) {
      const float4 av = *reinterpret_cast<const float4*>(sa + r * k + a0);
      const float4 bv = *reinterpret_cast<const float4*>(sb + r * k + b0);
      const float aa[4] = {av.x, av.y, av.z, av.w};
      const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i * 4 + j] = fmaf(aa[i], bb[j], part[i * 4 + j]);
    }
  };
  auto flush = [&]() {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      acc[q].add(part[q]);
      part[q] = 0.f;
    }
  };
  uint32_t phase = 0;
  int it = 0;
  bool timed_out = false;
  for (int64_t tile = blockIdx.x; tile < nfull; tile += gridDim.x, ++it) {
    const int st = it % kGramStages;
    const bool got = mbar_wait_bounded(&bars[st], (phase >> st) & 1u, kGramWaitTries);
    if (!__syncthreads_and(got)) {
      timed_out = true;
      break;
    }
    phase ^= 1u << st;
    const float* sa = tiles + (size_t)st * 2 * kGramTileFloats;
    const float* sb = sa + kGramTileFloats;
    if (worker) {
      accumulate(sa, sb, kGramTile);
      if ((it & 3) == 3) flush();
    }
    __syncthreads();  // every thread has read the stage: refill it
    if (t == 0) {
      const int64_t next = tile + (int64_t)kGramStages * gridDim.x;
      if (next < nfull) {
        fence_proxy_async_smem();
        issue(st, next);
      }
    }
  }
  if (timed_out) {
    if (t == 0) {
      atomicOr(status, kStatusTimeout);
      // wait (bounded) for this block's copies still in flight
      int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
      for (int q = 0; q < kGramStages && tile < nfull; ++q, ++it, tile += gridDim.x) {
        const int st = it % kGramStages;
        mbar_wait_bounded(&bars[st], (phase >> st) & 1u, kGramWaitTries);
        phase ^= 1u << st;
      }
    }
    __syncthreads();
    return;
  }
  // the ragged last tile, read with plain loads by the block whose turn it is
  const int rows = (int)(n - nfull * kGramTile);
  if (rows > 0 && blockIdx.x == (int)(nfull % gridDim.x)) {
    float* sa = tiles;  // every copy of this block has landed and been read
    float* sb = tiles + kGramTileFloats;
    const int64_t r0 = nfull * kGramTile;
    for (int e = t; e < rows * k; e += kSolveBlock) {
      sa[e] = A[r0 * k + e];
      sb[e] = B[r0 * k + e];
    }
    __syncthreads();
    if (worker) accumulate(sa, sb, rows);
  }
  if (worker) flush();
  // the row groups of each output entry in order (the stages are free now:
  // every copy of this block has landed and been read)
  __syncthreads();
  float2* s_part = reinterpret_cast<float2*>(tiles);  // [16][kSolveBlock]
#pragma unroll
  for (int q = 0; q < 16; ++q) s_part[q * kSolveBlock + t] = worker ? kahan_to_ff(acc[q]) : make_float2(0.f, 0.f);
  __syncthreads();
  if (t < nv) {
    const int a = t / k, b = t - (t / k) * k;
    const int blk = (a / 4) * nb + (b / 4), q = (a % 4) * 4 + (b % 4);
    R sum = make_float2(0.f, 0.f);
    for (int g2 = 0; g2 < groups; ++g2) sum = red_add(sum, s_part[q * kSolveBlock + g2 * nblk + blk]);
    s_blk[t] = sum;
  }
  __syncthreads();
  if (!grid_reduce_rt<R>(s_blk, s_tot, nv, gr)) return;
  for (int q = threadIdx.x; q < nv; q += kSolveBlock) G[q] = red_to_double(s_tot[q]);
}

// The fast path's HVP epilogue fused with G = U^T HV (k a multiple of 4), the
// two products truncated CG needs back to back.  The grid, the order of the
// tiles and the 4 x 4 output blocks of the threads are those of
// gram_tma_kernel, and every HV entry is hvp_entry's, so HV and G equal the
// two-kernel result bit for bit; the U and HV rows of a tile come into shared
// memory from the epilogue's own loads instead of being read again.  A block
// stages kEpiTiles tiles per step (more loads in flight per thread).  S (the
// edge kernel's sparse part) is read from HV and overwritten.
constexpr int kEpiTiles = 2;

__global__ void __launch_bounds__(kSolveBlock, 3) hvp_epi_gram_kernel(
    const float* __restrict__ U, const float* __restrict__ V, const float* __restrict__ Dl, float* HV,
    int64_t n, int k, const double* __restrict__ scalars, float pm2, double* G, GridRed gr,
    const int* done) {
  using R = float2;
  if (done && *done) return;
  __shared__ __align__(16) float tiles[kEpiTiles * 2 * kGramTileFloats];  // [tile][U | HV]
  __shared__ HvpCoef coef[kMaxK];
  __shared__ R s_blk[kMaxK * kMaxK];
  __shared__ R s_tot[kMaxK * kMaxK];
  const int t = threadIdx.x;
  if (t < k) {
    const double* c = scalars + kSlotCoef;
    coef[t] = HvpCoef{(float)c[t], (float)c[16 + t], (float)c[32 + t], (float)c[48 + t], (float)c[64 + t]};
  }
  const bool zero_rule = pm2 != 0.0f;
  const int nv = k * k;
  const int nb = k / 4;
  const int nblk = nb * nb;
  const int groups = kSolveBlock / nblk;
  const int pb = t % nblk, grp = t / nblk;
  const bool worker = grp < groups;
  const int a0 = 4 * (pb / nb), b0 = 4 * (pb % nb);
  const int64_t nfull = n / kGramTile;
  const int rows_last = (int)(n - nfull * kGramTile);
  const int64_t ntiles = nfull + (rows_last > 0 ? 1 : 0);
  Kahan acc[16];
  float part[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    acc[q].init();
    part[q] = 0.f;
  }
  int it = 0;  // full tiles of this block accumulated so far
  for (int64_t base = blockIdx.x; base < ntiles; base += (int64_t)kEpiTiles * gridDim.x) {
    __syncthreads();  // coefficients staged; the previous step's tiles consumed
    for (int q = 0; q < kEpiTiles; ++q) {
      const int64_t tile = base + (int64_t)q * gridDim.x;
      if (tile >= ntiles) break;
      const int rows = tile < nfull ? kGramTile : rows_last;
      const int cv = rows * k / 4;
      float4* su = reinterpret_cast<float4*>(tiles + (size_t)q * 2 * kGramTileFloats);
      float4* sh = su + kGramTileFloats / 4;
      const int64_t e0 = tile * kGramTile * k / 4;  // first float4 of the tile
      for (int e = t; e < cv; e += kSolveBlock) {
        const float4 u = __ldg(reinterpret_cast<const float4*>(U) + e0 + e);
        const float4 x = __ldg(reinterpret_cast<const float4*>(V) + e0 + e);
        const float4 dl = __ldg(reinterpret_cast<const float4*>(Dl) + e0 + e);
        const float4 sv = reinterpret_cast<const float4*>(HV)[e0 + e];
        const int c = (e * 4) % k;
        float4 h;
        h.x = hvp_entry(sv.x, u.x, x.x, dl.x, coef[c], pm2, zero_rule);
        h.y = hvp_entry(sv.y, u.y, x.y, dl.y, coef[c + 1], pm2, zero_rule);
        h.z = hvp_entry(sv.z, u.z, x.z, dl.z, coef[c + 2], pm2, zero_rule);
        h.w = hvp_entry(sv.w, u.w, x.w, dl.w, coef[c + 3], pm2, zero_rule);
        reinterpret_cast<float4*>(HV)[e0 + e] = h;
        su[e] = u;
        sh[e] = h;
      }
    }
    __syncthreads();
    for (int q = 0; q < kEpiTiles; ++q) {
      const int64_t tile = base + (int64_t)q * gridDim.x;
      if (tile >= ntiles) break;
      const int rows = tile < nfull ? kGramTile : rows_last;
      const float* sa = tiles + (size_t)q * 2 * kGramTileFloats;
      const float* sb = sa + kGramTileFloats;
      if (worker) {
        for (int r = grp; r < rows; r += groups) {
          const float4 av = *reinterpret_cast<const float4*>(sa + r * k + a0);
          const float4 bv = *reinterpret_cast<const float4*>(sb + r * k + b0);
          const float aa[4] = {av.x, av.y, av.z, av.w};
          const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[i * 4 + j] = fmaf(aa[i], bb[j], part[i * 4 + j]);
        }
        if (tile < nfull && (it & 3) == 3) {
#pragma unroll
          for (int w = 0; w < 16; ++w) {
            acc[w].add(part[w]);
            part[w] = 0.f;
          }
        }
      }
      if (tile < nfull) ++it;
    }
  }
  if (worker) {
#pragma unroll
    for (int w = 0; w < 16; ++w) acc[w].add(part[w]);
  }
  // the row groups of each output entry in order, as gram_tma_kernel
  __syncthreads();
  float2* s_part = reinterpret_cast<float2*>(tiles);  // [16][kSolveBlock]
#pragma unroll
  for (int q = 0; q < 16; ++q) s_part[q * kSolveBlock + t] = worker ? kahan_to_ff(acc[q]) : make_float2(0.f, 0.f);
  __syncthreads();
  if (t < nv) {
    const int a = t / k, b = t - (t / k) * k;
    const int blk = (a / 4) * nb + (b / 4), q = (a % 4) * 4 + (b % 4);
    R sum = make_float2(0.f, 0.f);
    for (int g2 = 0; g2 < groups; ++g2) sum = red_add(sum, s_part[q * kSolveBlock + g2 * nblk + blk]);
    s_blk[t] = sum;
  }
  __syncthreads();
  if (!grid_reduce_rt<R>(s_blk, s_tot, nv, gr)) return;
  for (int q = threadIdx.x; q < nv; q += kSolveBlock) G[q] = red_to_double(s_tot[q]);
}
static_assert(sizeof(float) * kEpiTiles * 2 * kGramTileFloats >= sizeof(float2) * 16 * kSolveBlock,
              "the staged tiles hold the per-thread partial sums at the end");

// k rounded up to the register-array width the row kernels are built for
__host__ __device__ constexpr int k_bucket(int k) { return k <= 4 ? 4 : k <= 8 ? 8 : 16; }

// a k x k FP64 matrix as T in shared memory with row stride KM, zero padded
template <typename T, int KM>
__device__ __forceinline__ void stage_matrix(T* dst, const double* M, int k) {
  for (int t = threadIdx.x; t < KM * KM; t += blockDim.x) {
    const int a = t / KM, b = t - (t / KM) * KM;
    dst[t] = (M && a < k && b < k) ? (T)M[a * k + b] : T(0);
  }
}

// row i of an n x k block into registers (zero padded to KM); 16-byte loads
// when k fills the bucket (rows are then 16-byte aligned)
template <typename T, int KM>
__device__ __forceinline__ void load_krow(const T* __restrict__ src, int64_t i, int k, T (&v)[KM]) {
  using V = Vec16<T>;
  using VT = typename V::type;
  if (k == KM) {
    const VT* p = reinterpret_cast<const VT*>(src + i * KM);
#pragma unroll
    for (int c = 0; c < KM / V::W; ++c) {
      const VT x = p[c];
#pragma unroll
      for (int w = 0; w < V::W; ++w) v[c * V::W + w] = V::get(x, w);
    }
  } else {
#pragma unroll
    for (int a = 0; a < KM; ++a) v[a] = a < k ? src[i * k + a] : T(0);
  }
}

template <typename T, int KM>
__device__ __forceinline__ void store_krow(T* dst, int64_t i, int k, const T (&v)[KM]) {
  using V = Vec16<T>;
  using VT = typename V::type;
  if (k == KM) {
    VT* p = reinterpret_cast<VT*>(dst + i * KM);
#pragma unroll
    for (int c = 0; c < KM / V::W; ++c) {
      VT x;
#pragma unroll
      for (int w = 0; w < V::W; ++w) V::set(x, w, v[c * V::W + w]);
      p[c] = x;
    }
  } else {
#pragma unroll
    for (int a = 0; a < KM; ++a)
      if (a < k) dst[i * k + a] = v[a];
  }
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
  using V = Vec16<T>;
  using VT = typename V::type;
  constexpr int W = V::W;
  Acc<T> acc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q].init();
  const int64_t mv = m / W;
  const int64_t tid = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * kSolveBlock;
  for (int64_t e = tid; e < mv; e += nth) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < dp.np) {
        const VT x = reinterpret_cast<const VT*>(dp.x[q])[e];
        const VT y = reinterpret_cast<const VT*>(dp.y[q])[e];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[q].add(V::get(x, w) * V::get(y, w));
      }
  }
  for (int64_t e = mv * W + tid; e < m; e += nth) {
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
// M2 k x k FP64 (either may be NULL) and scalar alpha/beta.  A thread per row.
template <typename T, int KM>
__global__ void __launch_bounds__(kSolveBlock) combine_kernel(
    T* out, const T* X, double alpha, const T* Y, double beta, const T* P, const double* M1,
    const T* Qm, const double* M2, int64_t n, int k, const int* done) {
  if (done && *done) return;
  __shared__ T m1[KM * KM], m2[KM * KM];
  stage_matrix<T, KM>(m1, M1, k);
  stage_matrix<T, KM>(m2, M2, k);
  __syncthreads();
  // read through volatile views: one shared-memory load per use, so the
  // k x k matrices are not hoisted into registers across rows
  const volatile T* v1 = m1;
  const volatile T* v2 = m2;
  for (int64_t i = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kSolveBlock) {
    T v[KM], xr[KM], pr[KM];
    if (X) {
      load_krow<T, KM>(X, i, k, xr);
#pragma unroll
      for (int b = 0; b < KM; ++b) v[b] = (T)alpha * xr[b];
    } else {
#pragma unroll
      for (int b = 0; b < KM; ++b) v[b] = T(0);
    }
    if (Y) {
      load_krow<T, KM>(Y, i, k, xr);
#pragma unroll
      for (int b = 0; b < KM; ++b) v[b] += (T)beta * xr[b];
    }
    if (M1) {  // padded rows/columns of the staged matrix are zero
      load_krow<T, KM>(P, i, k, pr);
#pragma unroll
      for (int a = 0; a < KM; ++a)
#pragma unroll
        for (int b = 0; b < KM; ++b) v[b] -= pr[a] * v1[a * KM + b];
    }
    if (M2) {
      load_krow<T, KM>(Qm, i, k, pr);
#pragma unroll
      for (int a = 0; a < KM; ++a)
#pragma unroll
        for (int b = 0; b < KM; ++b) v[b] -= pr[a] * v2[a * KM + b];
    }
    store_krow<T, KM>(out, i, k, v);
  }
}

// ------------------------------------------------------ Riemannian Hessian ---
// Hd = He - U G - delta M   and the partial sum of <delta, Hd>; the last
// block takes truncated CG's curvature step (alpha, or the boundary tau).
// A thread per row.
template <typename T, int KM>
__global__ void __launch_bounds__(kSolveBlock) hess_kernel(T* Hd, const T* He, const T* U,
                                                           const double* G, const T* delta,
                                                           const double* M, int64_t n, int k,
                                                           TcgState* st, GridRed gr) {
  using R = typename RedT<T>::type;
  if (st->done) return;
  __shared__ T g[KM * KM], mm[KM * KM];
  __shared__ R s_blk[1], s_tot[1];
  stage_matrix<T, KM>(g, G, k);
  stage_matrix<T, KM>(mm, M, k);
  __syncthreads();
  const volatile T* gv = g;  // one shared-memory load per use (see combine_kernel)
  const volatile T* mv = mm;
  Acc<T> acc;
  acc.init();
  for (int64_t i = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kSolveBlock) {
    T v[KM], ur[KM], dr[KM];
    load_krow<T, KM>(He, i, k, v);
    load_krow<T, KM>(U, i, k, ur);
    load_krow<T, KM>(delta, i, k, dr);
#pragma unroll
    for (int a = 0; a < KM; ++a)
#pragma unroll
      for (int b = 0; b < KM; ++b) v[b] -= ur[a] * gv[a * KM + b] + dr[a] * mv[a * KM + b];
    store_krow<T, KM>(Hd, i, k, v);
#pragma unroll
    for (int b = 0; b < KM; ++b)
      if (b < k) acc.add(dr[b] * v[b]);
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

// eta += step delta and r += step Hd, with the partial <r, r> unless the step
// ended on the boundary; the last block checks the residual, takes beta.
// H eta is not kept: r starts at the Riemannian gradient rg and takes every
// step's Hd (the boundary step's too), so H eta = r - rg when CG stops.
template <typename T>
__global__ void __launch_bounds__(kSolveBlock) cg_update_kernel(T* eta, T* r, const T* delta, const T* Hd,
                                                                int64_t m, TcgState* st, GridRed gr) {
  using R = typename RedT<T>::type;
  if (st->done) return;
  __shared__ R s_blk[1], s_tot[1];
  const T step = (T)st->step;
  const bool bnd = st->boundary != 0;
  using V = Vec16<T>;
  using VT = typename V::type;
  constexpr int W = V::W;
  Acc<T> acc;
  acc.init();
  const int64_t mv = m / W;
  const int64_t tid = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * kSolveBlock;
  for (int64_t e = tid; e < mv; e += nth) {
    const VT h = reinterpret_cast<const VT*>(Hd)[e];
    const VT d = reinterpret_cast<const VT*>(delta)[e];
    VT et = reinterpret_cast<VT*>(eta)[e];
    VT rr = reinterpret_cast<VT*>(r)[e];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      V::set(et, w, V::get(et, w) + step * V::get(d, w));
      const T rn = V::get(rr, w) + step * V::get(h, w);
      V::set(rr, w, rn);
      if (!bnd) acc.add(rn * rn);
    }
    reinterpret_cast<VT*>(eta)[e] = et;
    reinterpret_cast<VT*>(r)[e] = rr;
  }
  for (int64_t e = mv * W + tid; e < m; e += nth) {
    eta[e] += step * delta[e];
    const T rn = r[e] + step * Hd[e];
    r[e] = rn;
    if (!bnd) acc.add(rn * rn);
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
  using V = Vec16<T>;
  using VT = typename V::type;
  constexpr int W = V::W;
  const int64_t mv = m / W;
  const int64_t tid = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * kSolveBlock;
  for (int64_t e = tid; e < mv; e += nth) {
    const VT rr = reinterpret_cast<const VT*>(r)[e];
    VT d = reinterpret_cast<VT*>(delta)[e];
#pragma unroll
    for (int w = 0; w < W; ++w) V::set(d, w, -V::get(rr, w) + beta * V::get(d, w));
    reinterpret_cast<VT*>(delta)[e] = d;
  }
  for (int64_t e = mv * W + tid; e < m; e += nth) delta[e] = -r[e] + beta * delta[e];
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

// out_i = A_i Rinv  (rows times an upper-triangular k x k); a thread per row
template <typename T, int KM>
__global__ void __launch_bounds__(kSolveBlock) rmul_kernel(T* out, const T* A, const double* Rinv,
                                                           int64_t n, int k) {
  __shared__ T ri[KM * KM];
  stage_matrix<T, KM>(ri, Rinv, k);
  __syncthreads();
  const volatile T* rv = ri;  // one shared-memory load per use (see combine_kernel)
  for (int64_t i = blockIdx.x * (int64_t)kSolveBlock + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kSolveBlock) {
    T v[KM], ar[KM];
    load_krow<T, KM>(A, i, k, ar);
#pragma unroll
    for (int b = 0; b < KM; ++b) v[b] = T(0);
#pragma unroll
    for (int a = 0; a < KM; ++a)
#pragma unroll
      for (int b = a; b < KM; ++b) v[b] += ar[a] * rv[a * KM + b];  // Rinv upper triangular
    store_krow<T, KM>(out, i, k, v);
  }
}

}  // namespace pspec
