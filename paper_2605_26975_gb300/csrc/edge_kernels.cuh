// Fused FP32 edge kernels of the p-Laplacian (Section 2 of the paper):
//
//  eval:  per row i and column l
//           Delta_i = sum_j w_ij phi_p(u_i - u_j)              -> out_a
//         and per column the sums
//           N = 1/2 sum_ij w_ij |u_i - u_j|^p,  D = sum_i |u_i|^p
//  hvp:   additionally, for a direction V,
//           S_i = sum_j w_ij |u_i - u_j|^(p-2) (v_i - v_j)      -> out_a
//           Delta_i                                              -> out_b
//         and sigma_N = sum_i Delta_i v_i, sigma_D = sum_i phi_p(u_i) v_i.
//
// One pass over the CSR: every stored entry (i, j) costs one lg2 and one ex2
// per column, w_ij |d|^(p-2) = 2^((p-2) log2|d| + log2 w_ij) with log2 w
// computed once per entry, then phi = that * d and |d|^p = phi * d.  An exact
// zero difference gives phi = 0 (the log is clamped, see common.cuh) and, for
// p < 2, no curvature term in S.
//
// Work decomposition: each warp walks warp tasks (TaskSet) in a fixed
// grid-stride order.  A task's rows are handled by teams of E edge slots x Q
// column lanes; a lane owns CPL = K/Q columns loaded as 16/8/4-byte vectors,
// so the gather of a neighbour row is one or a few vector loads.  Row sums are
// reduced across the E slots by warp shuffles; per-column objective sums are
// folded across teams and kept per warp in compensated (Kahan) FP32 in shared
// memory, then reduced across warps and blocks in float-float.  Long rows are
// split into chunks whose partial row sums the warp finishing the row's last
// chunk adds in chunk order.  Nothing depends on scheduling order, so every
// result is bit-reproducible run to run.
#pragma once

#include "common.cuh"

namespace pspec {

struct EdgeArgs {
  const int64_t* rowptr;
  const int32_t* col;
  const float* val;
  const float* U;
  const float* V;
  float* out_a;
  float* out_b;
  const int4* tasks;
  int n_tasks;
  int chunk_edges;
  float* hub_part;
  const int32_t* hub_first;
  const int32_t* hub_nchunk;
  const int32_t* chunk_hub;
  unsigned* hub_ticket;
  float p;
  float pm2;
  GridReduce gr;
  double* scalars;
  int* status;
  const int* skip;
};

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

template <int K, bool HVP>
__global__ void __launch_bounds__(kBlock) edge_kernel(EdgeArgs a) {
  constexpr int Q = q_of(K);
  constexpr int CPL = K / Q;
  constexpr int VW = vw_of(K);
  constexpr int NQ = HVP ? 4 : 2;  // N, D (, sigma_N, sigma_D)
  constexpr int NV = NQ * K;

  if (a.skip && *a.skip) return;  // uniform over the grid
  __shared__ float s_acc[kWarps][NV][2];  // per-warp Kahan (sum, compensation)
  __shared__ float2 s_blk[NV];
  __shared__ float2 s_tot[NV];

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int q = lane % Q;
  const int c0 = q * CPL;
  const int gwarp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const float pm2 = a.pm2;
  const bool zero_rule = pm2 != 0.0f;  // p < 2: a zero difference has no curvature

  for (int i = lane; i < NV; i += 32) {
    s_acc[wib][i][0] = 0.f;
    s_acc[wib][i][1] = 0.f;
  }
  __syncwarp();

  for (int t = gwarp; t < a.n_tasks; t += nwarps) {
    const int4 task = __ldg(&a.tasks[t]);
    const int elog = task.z & 0xff;
    const bool hub = (task.z >> 8) != 0;
    const int E = 1 << elog;
    const int T = E * Q;
    const int team = lane / T;
    const int slot = (lane % T) / Q;
    int64_t row, e_beg = 0, e_end = 0;
    bool active;
    if (!hub) {
      row = (int64_t)task.x + team;
      active = team < task.y;
      if (active) {
        e_beg = __ldg(&a.rowptr[row]);
        e_end = __ldg(&a.rowptr[row + 1]);
      }
    } else {
      row = task.x;
      active = true;
      const int64_t rb = __ldg(&a.rowptr[row]);
      const int64_t re = __ldg(&a.rowptr[row + 1]);
      e_beg = rb + (int64_t)task.y * a.chunk_edges;
      e_end = min(re, e_beg + (int64_t)a.chunk_edges);
    }

    float ui[CPL], vi[CPL], dsum[CPL], nsum[CPL], ssum[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) { ui[c] = 0.f; vi[c] = 0.f; dsum[c] = 0.f; nsum[c] = 0.f; ssum[c] = 0.f; }
    if (active) {
      load_row<K, CPL, VW>(a.U, row, c0, ui);
      if constexpr (HVP) load_row<K, CPL, VW>(a.V, row, c0, vi);
      for (int64_t e = e_beg + slot; e < e_end; e += 2 * E) {
        const int64_t e2 = e + E;
        const bool has2 = e2 < e_end;
        const int j1 = __ldg(&a.col[e]);
        const float w1 = __ldg(&a.val[e]);
        const int j2 = has2 ? __ldg(&a.col[e2]) : j1;
        const float w2 = has2 ? __ldg(&a.val[e2]) : 0.0f;  // weight 0: contributes nothing
        float uj1[CPL], uj2[CPL], vj1[CPL], vj2[CPL];
        load_row<K, CPL, VW>(a.U, j1, c0, uj1);
        load_row<K, CPL, VW>(a.U, j2, c0, uj2);
        if constexpr (HVP) {
          load_row<K, CPL, VW>(a.V, j1, c0, vj1);
          load_row<K, CPL, VW>(a.V, j2, c0, vj2);
        }
        const float lw1 = lg2_approx(w1);
        const float lw2 = lg2_approx(w2);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const float d1 = ui[c] - uj1[c];
          const float d2 = ui[c] - uj2[c];
          const float sw1 = ex2_approx(fmaf(pm2, fmaxf(lg2_approx(fabsf(d1)), -126.0f), lw1));
          const float sw2 = ex2_approx(fmaf(pm2, fmaxf(lg2_approx(fabsf(d2)), -126.0f), lw2));
          const float ph1 = sw1 * d1;  // w phi_p(d)
          const float ph2 = sw2 * d2;
          dsum[c] += ph1;
          dsum[c] += ph2;
          nsum[c] = fmaf(ph1, d1, nsum[c]);  // w |d|^p
          nsum[c] = fmaf(ph2, d2, nsum[c]);
          if constexpr (HVP) {
            const float s1 = (zero_rule && d1 == 0.0f) ? 0.0f : sw1;
            const float s2 = (zero_rule && d2 == 0.0f) ? 0.0f : sw2;
            ssum[c] = fmaf(s1, vi[c] - vj1[c], ssum[c]);
            ssum[c] = fmaf(s2, vi[c] - vj2[c], ssum[c]);
          }
        }
      }
    }
    // row sums across the E edge slots of each team (lanes of equal q)
    for (int off = Q; off < T; off <<= 1) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        dsum[c] += __shfl_xor_sync(0xffffffffu, dsum[c], off);
        nsum[c] += __shfl_xor_sync(0xffffffffu, nsum[c], off);
        if constexpr (HVP) ssum[c] += __shfl_xor_sync(0xffffffffu, ssum[c], off);
      }
    }
    const bool lead = active && slot == 0;
    // per-row vertex terms on the lead lanes; everything else contributes 0
    float dpart[CPL], cnpart[CPL], cdpart[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      dpart[c] = 0.f; cnpart[c] = 0.f; cdpart[c] = 0.f;
      if (!lead) nsum[c] = 0.f;
    }
    const bool vertex = lead && (!hub || task.y == 0);
    if (vertex) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const float phu = abs_pow_pm2_clamped(ui[c], pm2) * ui[c];  // phi_p(u_i)
        dpart[c] = phu * ui[c];                                     // |u_i|^p
        if constexpr (HVP) cdpart[c] = phu * vi[c];
      }
    }
    if (lead && !hub) {
      if constexpr (HVP) {
        store_row<K, CPL, VW>(a.out_a, row, c0, ssum);
        store_row<K, CPL, VW>(a.out_b, row, c0, dsum);
#pragma unroll
        for (int c = 0; c < CPL; ++c) cnpart[c] = dsum[c] * vi[c];
      } else {
        store_row<K, CPL, VW>(a.out_a, row, c0, dsum);
      }
    }
    if (hub) {
      // publish this chunk's partial row sums; the last chunk adds them up
      const int slot_id = task.w;
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
            store_row<K, CPL, VW>(a.out_b, row, c0, rd);
#pragma unroll
            for (int c = 0; c < CPL; ++c) cnpart[c] = rd[c] * vi[c];
          } else {
            store_row<K, CPL, VW>(a.out_a, row, c0, rd);
          }
        }
        if (lane == 0) a.hub_ticket[h] = 0u;
      }
    }
    // fold the task's per-column sums across teams, then into the warp's
    // compensated accumulators (lanes 0..Q-1 own distinct columns)
    for (int off = T; off < 32; off <<= 1) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        nsum[c] += __shfl_xor_sync(0xffffffffu, nsum[c], off);
        dpart[c] += __shfl_xor_sync(0xffffffffu, dpart[c], off);
        if constexpr (HVP) {
          cnpart[c] += __shfl_xor_sync(0xffffffffu, cnpart[c], off);
          cdpart[c] += __shfl_xor_sync(0xffffffffu, cdpart[c], off);
        }
      }
    }
    if (lane < Q) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const float vals[4] = {nsum[c], dpart[c], cnpart[c], cdpart[c]};
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
          float* acc = s_acc[wib][qq * K + c0 + c];
          const float y = vals[qq] - acc[1];
          const float tt = acc[0] + y;
          acc[1] = (tt - acc[0]) - y;
          acc[0] = tt;
        }
      }
    }
    __syncwarp();
  }

  // block: warps in order, float-float
  __syncthreads();
  if (threadIdx.x < NV) {
    float2 acc = make_float2(0.f, 0.f);
    for (int w = 0; w < kWarps; ++w)
      acc = ff_add(acc, two_sum(s_acc[w][threadIdx.x][0], -s_acc[w][threadIdx.x][1]));
    s_blk[threadIdx.x] = acc;
  }
  __syncthreads();
  if (!grid_reduce_ff<NV>(s_blk, s_tot, a.gr)) return;

  // last block: FP64 scalars and epilogue coefficients
  if (threadIdx.x < K) {
    const int c = threadIdx.x;
    const double N = 0.5 * ff_to_double(s_tot[c]);  // both triangles stored
    const double D = ff_to_double(s_tot[K + c]);
    double* sc = a.scalars;
    sc[0 + c] = N;   // kSlotN
    sc[16 + c] = D;  // kSlotD
    int flags = 0;
    if (!isfinite(N) || !isfinite(D)) flags |= kStatusNonFinite;
    else if (!(D > 0.0)) flags |= kStatusZeroColumn;
    const double p = (double)a.p;
    const double lam = N / D;
    double* coef = sc + 80;  // kSlotCoef: 6 x 16
    if constexpr (HVP) {
      const double sN = ff_to_double(s_tot[2 * K + c]);
      const double sD = ff_to_double(s_tot[3 * K + c]);
      sc[32 + c] = sN;
      sc[48 + c] = sD;
      if (!isfinite(sN) || !isfinite(sD)) flags |= kStatusNonFinite;
      coef[0 * 16 + c] = p * (p - 1.0) / D;  // A
      coef[1 * 16 + c] = lam;                // lambda
      coef[2 * 16 + c] = p * p / (D * D);    // B
      coef[3 * 16 + c] = sD;                 // sigma_D
      coef[4 * 16 + c] = sN - 2.0 * lam * sD;
    } else {
      coef[0 * 16 + c] = p / D;
      coef[1 * 16 + c] = p * lam / D;
    }
    if (flags) atomicOr(a.status, flags);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double F = 0.0;
    for (int c = 0; c < K; ++c) F += a.scalars[c] / a.scalars[16 + c];
    a.scalars[64] = F;  // kSlotF
  }
}

}  // namespace pspec
