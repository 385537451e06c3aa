// Fused FP32 edge kernels of the p-Laplacian (Section 2 of the paper):
//
//  eval:  per row i and column l
//           Delta_i = sum_j w_ij phi_p(u_i - u_j)              -> out_a
//         and per column the sums
//           N = 1/2 sum_ij w_ij |u_i - u_j|^p,  D = sum_i |u_i|^p
//  hvp:   additionally, for a direction V,
//           S_i = sum_j w_ij |u_i - u_j|^(p-2) (v_i - v_j)      -> out_a
//           Delta_i                             -> out_b (skipped if NULL)
//         and sigma_N = sum_i Delta_i v_i, sigma_D = sum_i phi_p(u_i) v_i.
//
// Arithmetic.  Every stored entry (i, j) costs one lg2 and one ex2 per column,
// with log2 w_ij stored in the graph's sorted copy (computed once, in double,
// at upload): the objective forms w_ij phi_p(d) = sign(d) 2^((p-1) log2|d| +
// log2 w_ij) and |d|^p w_ij = that * d; the Hessian product forms
// w_ij |d|^(p-2) = 2^((p-2) log2|d| + log2 w_ij) and phi from it.  A zero
// difference (a subnormal one flushed to zero) gives phi = 0 for any weight
// and, for p < 2, no curvature term.
//
// Data movement.  The kernels read a copy of W whose rows are stably sorted
// by degree (perm maps a sorted row back to its vertex), with each entry's
// column and log2 weight interleaved in one 8-byte word.  A warp task is a run
// of consecutive sorted rows of one degree, so its entries are contiguous and
// every lane knows its exact entry count: the lanes stream their entries
// with plain 8-byte loads (the warp's loads of one step cover a contiguous
// window, so they coalesce in L1), the next group's entries are loaded while
// the current group's neighbour rows are in flight, and the loop has no
// padding or per-entry bounds test.
//
// Work split.  A row is handled by a team of E edge slots x Q column lanes; a
// lane owns CPL = K/Q consecutive columns (16/8/4-byte vectors).  Typical rows
// get E = 1 (a lane walks its row, UNR entries per step, no shuffles); longer
// rows are shared by E slots and reduced by warp shuffles; rows above the hub
// threshold are split into chunks whose partial sums the warp finishing the
// row's last chunk adds in chunk order (atomic ticket, no spinning).
// Per-column sums live per lane in registers (compensated for the objective),
// then are reduced across the warp, block and grid in float-float in a fixed
// order, so every result is bit-reproducible run to run.
#pragma once

#include "common.cuh"

namespace pspec {

struct EdgeArgs {
  const int2* cw;         // degree-sorted entries: x = column, y = bits of log2 w
  const int32_t* perm;    // sorted row -> vertex
  const float* U;
  const float* V;
  float* out_a;
  float* out_b;
  const int4* tasks;
  int n_tasks;
  float* hub_part;
  const int32_t* hub_first;
  const int32_t* hub_nchunk;
  const int32_t* chunk_hub;
  unsigned* hub_ticket;
  float p;
  float pm2;
  double p64;  // p exactly, for the FP64 scalars and coefficients
  GridReduce gr;
  double* scalars;
  int* status;
  const int* skip;
  // batches: per-task column sums go to task_part[task][NV] instead of the
  // grid reduction (NULL for a single graph)
  float* task_part;
  // HVP in Algorithm 1's form: the epilogue's rank-two coefficient is zero
  int alg1;
  // HVP with Delta_p u kept from the evaluation at the same U: that
  // evaluation's N[16], D[16] (the staged kernel then sums only sigma_N and
  // sigma_D); NULL otherwise
  const double* keep_nd;
  // contiguous task ranges, warp w taking [warp_begin[w], warp_begin[w+1]);
  // NULL: round-robin
  const int32_t* warp_begin;
  // batches: the tasks of graph q are left out while graph_skip[q] is
  // nonzero (task_graph: the graph of each task); read only by the direct
  // kernel's GSKIP instantiation
  const int* graph_skip;
  const int32_t* task_graph;
};

// What an edge kernel sums: the objective (N, D, Delta_p u), the Hessian
// product (N, D, sigma_N, sigma_D, S, and Delta_p u unless out_b is NULL), or
// the Hessian product at a point whose Delta_p u and N, D were kept by its
// evaluation (sigma_N, sigma_D and S only).
constexpr int kModeEval = 0, kModeHvp = 1, kModeHvpKept = 2;

// Scalar slots of the per-call FP64 array (d_scalars)
constexpr int kScN = 0, kScD = 16, kScCN = 32, kScCD = 48, kScF = 64, kScCoef = 80, kScKeep = 256;

template <int K, int CPL, int VW>
__device__ __forceinline__ void load_row(const float* base, int64_t row, int c0, float* dst) {
#pragma unroll
  for (int j = 0; j < CPL; j += VW) load_vec<VW>(base + row * K + c0 + j, dst + j);
}

template <int K, int CPL, int VW>
__device__ __forceinline__ void store_row(float* base, int64_t row, int c0, const float* src) {
#pragma unroll
  for (int j = 0; j < CPL; j += VW) store_vec<VW>(base + row * K + c0 + j, src + j);
}

// Per-lane running sums of the per-column quantities (N, D and, for the
// Hessian product, sigma_N and sigma_D): compensated for the objective's
// sums, plain for the Hessian product's (whose rank-two coefficients need
// ~1e-6 only).  For a lane of at most 8 columns they live in shared memory,
// one slot per thread laid out [slot][thread] (a warp's accesses hit 32
// banks), which frees the registers they would take for occupancy; wider
// lanes keep them in registers.
template <int CPL, int NQ, bool COMP, bool SMEM> struct AccBank;

template <int CPL, int NQ, bool COMP>
struct AccBank<CPL, NQ, COMP, true> {
  static constexpr int kSlots = NQ * CPL * (COMP ? 2 : 1);
  float* base;  // this thread's first slot; slot i at base[i * kBlock]
  __device__ __forceinline__ void init(float* smem) {
    base = smem + threadIdx.x;
#pragma unroll
    for (int i = 0; i < kSlots; ++i) base[i * kBlock] = 0.f;
  }
  __device__ __forceinline__ void add(int q, int c, float x) {
    const int i = q * CPL + c;
    if constexpr (COMP) {
      Kahan k{base[(2 * i) * kBlock], base[(2 * i + 1) * kBlock]};
      k.add(x);
      base[(2 * i) * kBlock] = k.s;
      base[(2 * i + 1) * kBlock] = k.c;
    } else {
      base[i * kBlock] += x;
    }
  }
  __device__ __forceinline__ float2 ff(int q, int c) const {
    const int i = q * CPL + c;
    if constexpr (COMP) return kahan_to_ff(Kahan{base[(2 * i) * kBlock], base[(2 * i + 1) * kBlock]});
    return make_float2(base[i * kBlock], 0.f);
  }
};

template <int CPL, int NQ, bool COMP>
struct AccBank<CPL, NQ, COMP, false> {
  static constexpr int kSlots = 1;
  Kahan k[NQ][CPL];
  __device__ __forceinline__ void init(float*) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int c = 0; c < CPL; ++c) k[q][c].init();
  }
  __device__ __forceinline__ void add(int q, int c, float x) {
    if constexpr (COMP) k[q][c].add(x);
    else k[q][c].s += x;
  }
  __device__ __forceinline__ float2 ff(int q, int c) const {
    if constexpr (COMP) return kahan_to_ff(k[q][c]);
    return make_float2(k[q][c].s, 0.f);
  }
};

// Resident blocks per SM the kernel is compiled for: with lanes of at most
// four columns the kernels fit four blocks of 256 threads (64 registers)
// without spilling, and the Hessian product at a kept point (no |d|^p sum,
// two column sums instead of four) fits five (48 registers) for k = 8 (at
// k = 16 that register budget made it slower than four blocks at 64); the
// gathers' latency is hidden by that many warps.
template <int K, int MODE, bool SPLIT>
__host__ __device__ constexpr int edge_min_blocks() {
  return K / q_of(K) <= 4 ? ((MODE == kModeHvpKept && K >= 8 && K < 16 && !SPLIT) ? 5 : 4) : 1;
}

// task descriptor fields (see ensure_tasks)
__device__ __forceinline__ bool task_is_hub(int4 t) { return ((t.z >> 8) & 1) != 0; }

// G entries of a lane's row: gather the neighbour rows, then accumulate
//   dsum += w phi_p(d),  nsum += w |d|^p,  ssum += w |d|^(p-2) (v_i - v_j)
// `ex` is the exponent of the power formed per entry: p - 1 for the
// objective, p - 2 for the Hessian product.
//  * objective: w phi_p(d) = sign(d) 2^((p-1) log2|d| + log2 w) directly; a tie
//    (d == 0) has log2|d| = -inf and gives 0 for every weight.
//  * Hessian product: w |d|^(p-2) = 2^((p-2) max(log2|d|, -126) + log2 w), then
//    phi = that * d.  A tie is selected away before the product (p < 2: no
//    curvature term; p = 2: the term is w), so a large weight never meets
//    inf * 0.
template <int K, int CPL, int VW, bool HVP, bool KEPT, int G>
__device__ __forceinline__ void edge_group(const EdgeArgs& a, const int2 (&e)[G], int c0,
                                           const float (&ui)[CPL], const float (&vi)[CPL], float ex,
                                           bool zero_rule, float (&dsum)[CPL], float (&nsum)[CPL],
                                           float (&ssum)[CPL]) {
  float uj[G][CPL], vj[G][CPL];
#pragma unroll
  for (int u = 0; u < G; ++u) {
    load_row<K, CPL, VW>(a.U, (int64_t)(uint32_t)e[u].x, c0, uj[u]);
    if constexpr (HVP) load_row<K, CPL, VW>(a.V, (int64_t)(uint32_t)e[u].x, c0, vj[u]);
  }
#pragma unroll
  for (int u = 0; u < G; ++u) {
    const float lw = __int_as_float(e[u].y);
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const float d = sub_ftz(ui[c], uj[u][c]);
      if constexpr (HVP) {
        const float sw = ex2_approx(fmaf(ex, fmaxf(lg2_approx(fabsf(d)), -126.0f), lw));
        const float sz = (zero_rule && d == 0.0f) ? 0.0f : sw;  // w |d|^(p-2)
        const float ph = sz * d;                                 // w phi_p(d)
        dsum[c] += ph;
        if constexpr (!KEPT) nsum[c] = fmaf(ph, d, nsum[c]);
        ssum[c] = fmaf(sz, vi[c] - vj[u][c], ssum[c]);
      } else {
        const float ph = copysignf(ex2_approx(fmaf(ex, lg2_approx(fabsf(d)), lw)), d);  // w phi_p(d)
        dsum[c] += ph;
        nsum[c] = fmaf(ph, d, nsum[c]);  // w |d|^p
      }
    }
  }
}

// Column c's FP64 scalars and epilogue coefficients from its sums N, D (and,
// for the Hessian product, sigma_N, sigma_D) into the scalar array sc (slots
// kSc*): the gradient's p/D and p lambda/D, or the Hessian product's
// A = p(p-1)/D, lambda, B = p^2/D^2 (0 in Algorithm 1's form), sigma_D and
// E = sigma_N - 2 lambda sigma_D.  Returns the status bits it found.
__device__ __forceinline__ int column_scalars(int c, double N, double D, double sN, double sD, bool hvp,
                                              double p, int alg1, double* sc) {
  sc[kScN + c] = N;
  sc[kScD + c] = D;
  int flags = 0;
  if (!isfinite(N) || !isfinite(D)) flags |= kStatusNonFinite;
  else if (!(D > 0.0)) flags |= kStatusZeroColumn;
  const double lam = N / D;
  double* coef = sc + kScCoef;  // 6 x 16
  if (hvp) {
    sc[kScCN + c] = sN;
    sc[kScCD + c] = sD;
    if (!isfinite(sN) || !isfinite(sD)) flags |= kStatusNonFinite;
    coef[0 * 16 + c] = p * (p - 1.0) / D;              // A
    coef[1 * 16 + c] = lam;                            // lambda
    coef[2 * 16 + c] = alg1 ? 0.0 : p * p / (D * D);  // B
    coef[3 * 16 + c] = sD;                             // sigma_D
    coef[4 * 16 + c] = sN - 2.0 * lam * sD;            // E
  } else {
    coef[0 * 16 + c] = p / D;
    coef[1 * 16 + c] = p * lam / D;
  }
  return flags;
}

// The per-column sums of a launch, from each lane's float-float values v
// (quantity qq of column c0 + c): lanes of equal q are added over the warp,
// warps over the block and blocks over the grid, all in float-float and in a
// fixed order; the last block then writes the FP64 scalars and the epilogue
// coefficients.  Quantities: N, D (objective); N, D, sigma_N, sigma_D
// (Hessian product); sigma_N, sigma_D with N, D from a.keep_nd (Hessian
// product at a point whose Delta_p u was kept).
template <int K, int NQ, bool HVP, bool KEPT, int CPL>
__device__ __forceinline__ void finish_edges(float2 (&v)[NQ][CPL], const EdgeArgs& a) {
  constexpr int Q = q_of(K);
  constexpr int NV = NQ * K;
  __shared__ float2 s_warp[kWarps][NV];
  __shared__ float2 s_blk[NV];
  __shared__ float2 s_tot[NV];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int c0 = (lane % Q) * CPL;
#pragma unroll
  for (int off = Q; off < 32; off <<= 1)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
      for (int c = 0; c < CPL; ++c) v[qq][c] = ff_add(v[qq][c], shfl_xor_ff(v[qq][c], off));
  if (lane < Q)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
      for (int c = 0; c < CPL; ++c) s_warp[wib][qq * K + c0 + c] = v[qq][c];
  __syncthreads();
  if (threadIdx.x < NV) {
    float2 acc = make_float2(0.f, 0.f);
    for (int w = 0; w < kWarps; ++w) acc = ff_add(acc, s_warp[w][threadIdx.x]);
    s_blk[threadIdx.x] = acc;
  }
  __syncthreads();
  if (!grid_reduce_ff<NV>(s_blk, s_tot, a.gr)) return;

  // last block: FP64 scalars and epilogue coefficients
  if (threadIdx.x < K) {
    const int c = threadIdx.x;
    double N, D;
    if constexpr (KEPT) {
      N = a.keep_nd[c];
      D = a.keep_nd[16 + c];
    } else {
      N = 0.5 * ff_to_double(s_tot[c]);  // both triangles stored
      D = ff_to_double(s_tot[K + c]);
    }
    double sN = 0.0, sD = 0.0;
    if constexpr (HVP) {
      constexpr int o = KEPT ? 0 : 2;  // sigma_N, sigma_D after N, D unless N, D are kept
      sN = ff_to_double(s_tot[o * K + c]);
      sD = ff_to_double(s_tot[(o + 1) * K + c]);
    }
    const int flags = column_scalars(c, N, D, sN, sD, HVP, a.p64, a.alg1, a.scalars);
    if (flags) atomicOr(a.status, flags);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int c = 0; c < K; ++c) F += a.scalars[kScN + c] / a.scalars[kScD + c];
    a.scalars[kScF] = F;
  }
}

template <int G>
__device__ __forceinline__ void load_entries(const int2* __restrict__ cw, int E, int2 (&e)[G]) {
#pragma unroll
  for (int u = 0; u < G; ++u) e[u] = __ldg(cw + u * E);
}

// A lane's part of a warp task (see ensure_tasks): its team (row) and edge
// slot, its entries cw[start + slot + j E] for j < n_my, the sorted row whose
// vertex perm[prow] it works on.
struct LaneTask {
  bool hub, active;
  int elog, E, T, team, slot, cnt, start, n_my, prow;
};

template <int Q>
__device__ __forceinline__ LaneTask lane_task(int4 task, int lane) {
  LaneTask v;
  v.hub = task_is_hub(task);
  v.elog = task.z & 0xff;
  v.E = 1 << v.elog;
  v.T = v.E * Q;
  v.team = lane / v.T;
  v.slot = (lane % v.T) / Q;
  if (!v.hub) {
    const int deg = task.y >> 8;
    v.active = v.team < (task.y & 0xff);
    v.cnt = deg;
    v.start = task.w + v.team * deg;
  } else {
    v.active = true;
    v.cnt = task.z >> 10;
    v.start = task.w;
  }
  v.n_my = (v.active && v.slot < v.cnt) ? ((v.cnt - v.slot + v.E - 1) >> v.elog) : 0;
  v.prow = task.x + (v.hub ? 0 : v.team);
  return v;
}

// SPLIT: the warps take contiguous, cost-balanced task ranges (a.warp_begin)
// instead of round-robin tasks.  GSKIP: batch launches that leave out the
// tasks of graphs flagged in a.graph_skip (a separate instantiation, so the
// other launches carry no per-task test).
template <int K, int MODE, bool SPLIT, bool GSKIP = false>
__global__ void __launch_bounds__(kBlock, edge_min_blocks<K, MODE, SPLIT>()) edge_kernel(EdgeArgs a) {
  constexpr bool HVP = MODE != kModeEval;
  constexpr bool KEPT = MODE == kModeHvpKept;
  constexpr int Q = q_of(K);
  constexpr int CPL = K / Q;
  constexpr int VW = vw_of(K);
  constexpr int NQ = MODE == kModeHvp ? 4 : 2;  // N, D (, sigma_N, sigma_D) | sigma_N, sigma_D
  constexpr int NV = NQ * K;
  constexpr int UNR = HVP ? (CPL > 8 ? 1 : 2) : (CPL > 8 ? 2 : 4);  // entries per lane per step
  constexpr bool COMP = !HVP;

  constexpr bool SMEM_ACC = CPL <= 8;
  using Acc = AccBank<CPL, NQ, COMP, SMEM_ACC>;

  if (a.skip && *a.skip) return;  // uniform over the grid
  __shared__ float s_acc[SMEM_ACC ? Acc::kSlots * kBlock : 1];

  const int lane = threadIdx.x & 31;
  const int q = lane % Q;
  const int c0 = q * CPL;
  const int gwarp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const float pm2 = a.pm2;
  const float ex = HVP ? pm2 : a.p - 1.0f;  // exponent of the per-entry power
  const bool zero_rule = pm2 != 0.0f;  // p < 2: a zero difference has no curvature

  Acc acc;
  acc.init(s_acc);

  const int t_first = SPLIT ? __ldg(&a.warp_begin[gwarp]) : gwarp;
  const int t_end = SPLIT ? __ldg(&a.warp_begin[gwarp + 1]) : a.n_tasks;
  for (int t = t_first; t < t_end; t += SPLIT ? 1 : nwarps) {
    if constexpr (GSKIP) {
      if (a.graph_skip[__ldg(&a.task_graph[t])]) continue;  // uniform over the warp
    }
    const int4 task = __ldg(&a.tasks[t]);
    const LaneTask lt = lane_task<Q>(task, lane);
    const bool hub = lt.hub;
    const int elog = lt.elog, E = lt.E, T = lt.T, slot = lt.slot, n_my = lt.n_my;
    const bool active = lt.active;
    const int2* cw = a.cw + lt.start + slot;  // this lane's entries: cw[j * E], j < n_my
    int2 nx[UNR];
    if (n_my >= UNR) load_entries<UNR>(cw, E, nx);
    const int64_t row = active ? (int64_t)__ldg(&a.perm[lt.prow]) : 0;

    float ui[CPL], vi[CPL], dsum[CPL], nsum[CPL], ssum[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) { ui[c] = 0.f; vi[c] = 0.f; dsum[c] = 0.f; nsum[c] = 0.f; ssum[c] = 0.f; }
    if (active) {
      load_row<K, CPL, VW>(a.U, row, c0, ui);
      if constexpr (HVP) load_row<K, CPL, VW>(a.V, row, c0, vi);
    }
    int j = 0;
    for (; j + UNR <= n_my; j += UNR) {
      int2 e[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) e[u] = nx[u];
      if (j + 2 * UNR <= n_my) load_entries<UNR>(cw + (j + UNR) * E, E, nx);  // next step's entries
      edge_group<K, CPL, VW, HVP, KEPT, UNR>(a, e, c0, ui, vi, ex, zero_rule, dsum, nsum, ssum);
    }
    if constexpr (UNR >= 4) {
      if (n_my - j >= 2) {
        int2 e[2];
        load_entries<2>(cw + j * E, E, e);
        edge_group<K, CPL, VW, HVP, KEPT, 2>(a, e, c0, ui, vi, ex, zero_rule, dsum, nsum, ssum);
        j += 2;
      }
    }
    if constexpr (UNR >= 2) {
      if (j < n_my) {  // at most one entry left
        int2 e[1];
        load_entries<1>(cw + j * E, E, e);
        edge_group<K, CPL, VW, HVP, KEPT, 1>(a, e, c0, ui, vi, ex, zero_rule, dsum, nsum, ssum);
      }
    }
    // row sums across the E edge slots of each team (lanes of equal q)
    for (int off = Q; off < T; off <<= 1) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        dsum[c] += __shfl_xor_sync(0xffffffffu, dsum[c], off);
        if constexpr (!KEPT) nsum[c] += __shfl_xor_sync(0xffffffffu, nsum[c], off);
        if constexpr (HVP) ssum[c] += __shfl_xor_sync(0xffffffffu, ssum[c], off);
      }
    }
    const bool lead = active && slot == 0;
    const bool first_chunk = !hub || ((task.z >> 9) & 1);
    // this task's contributions of this lane to the per-column sums
    float tq[NQ][CPL];
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
      for (int c = 0; c < CPL; ++c) tq[qq][c] = 0.f;
    if (lead) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        float phu = 0.f;
        if (first_chunk) phu = abs_pow_pm2_clamped(ui[c], pm2) * ui[c];  // phi_p(u_i), once per row
        if constexpr (MODE == kModeEval) {
          tq[0][c] = nsum[c];
          tq[1][c] = phu * ui[c];  // |u_i|^p
        } else if constexpr (MODE == kModeHvp) {
          tq[0][c] = nsum[c];
          tq[1][c] = phu * ui[c];
          tq[2][c] = dsum[c] * vi[c];  // sigma_N: a row's Delta_i v_i, or a chunk's share
          tq[3][c] = phu * vi[c];      // sigma_D
        } else {
          tq[0][c] = dsum[c] * vi[c];
          tq[1][c] = phu * vi[c];
        }
      }
      if (!hub) {
        if constexpr (HVP) {
          store_row<K, CPL, VW>(a.out_a, row, c0, ssum);
          if (a.out_b) store_row<K, CPL, VW>(a.out_b, row, c0, dsum);
        } else {
          store_row<K, CPL, VW>(a.out_a, row, c0, dsum);
        }
      }
    }
    if (!a.task_part) {
      if (lead) {
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
          for (int c = 0; c < CPL; ++c) acc.add(qq, c, tq[qq][c]);
      }
    } else {
      // one graph of a batch: fold the task's sums over the warp (lanes of
      // equal q) and publish them in the task's slot
      for (int off = Q; off < 32; off <<= 1)
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
          for (int c = 0; c < CPL; ++c) tq[qq][c] += __shfl_xor_sync(0xffffffffu, tq[qq][c], off);
      if (lane < Q) {
        float* tp = a.task_part + (size_t)t * NV;
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
          for (int c = 0; c < CPL; ++c) tp[qq * K + c0 + c] = tq[qq][c];
      }
    }
    if (hub) {
      // publish this chunk's partial row sums; the last chunk adds them up.
      // (sigma_N's share of the row was taken chunk by chunk above, by the
      // chunk's own warp -- a static assignment, not by whichever finishes last.)
      const int slot_id = task.y;
      if (lead) {
        float* hp = a.hub_part + (size_t)slot_id * 2 * K;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          hp[c0 + c] = dsum[c];
          if constexpr (HVP) hp[K + c0 + c] = ssum[c];
        }
      }
      __threadfence();
      __syncwarp();
      const int h = __ldg(&a.chunk_hub[slot_id]);
      const int first = __ldg(&a.hub_first[h]);
      const int nch = __ldg(&a.hub_nchunk[h]);
      unsigned tk = 0;
      if (lane == 0) tk = atomicAdd(&a.hub_ticket[h], 1u);
      tk = __shfl_sync(0xffffffffu, tk, 0);
      if (tk == (unsigned)(nch - 1)) {
        __threadfence();
        if (lead) {
          Kahan td[CPL], ts[CPL];
#pragma unroll
          for (int c = 0; c < CPL; ++c) { td[c].init(); ts[c].init(); }
          for (int ch = 0; ch < nch; ++ch) {
            const float* hp = a.hub_part + (size_t)(first + ch) * 2 * K;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              td[c].add(__ldcg(hp + c0 + c));
              if constexpr (HVP) ts[c].add(__ldcg(hp + K + c0 + c));
            }
          }
          float rd[CPL], rs[CPL];
#pragma unroll
          for (int c = 0; c < CPL; ++c) { rd[c] = td[c].s - td[c].c; rs[c] = ts[c].s - ts[c].c; }
          if constexpr (HVP) {
            store_row<K, CPL, VW>(a.out_a, row, c0, rs);
            if (a.out_b) store_row<K, CPL, VW>(a.out_b, row, c0, rd);
          } else {
            store_row<K, CPL, VW>(a.out_a, row, c0, rd);
          }
        }
        if (lane == 0) a.hub_ticket[h] = 0u;
      }
    }
  }
  if (a.task_part) return;  // batches: per-graph sums are reduced by batch_reduce
  float2 v[NQ][CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) v[qq][c] = acc.ff(qq, c);
  finish_edges<K, NQ, HVP, KEPT>(v, a);
}

}  // namespace pspec
