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
// Arithmetic.  Every stored entry (i, j) costs one lg2 and one ex2 per column:
// w_ij |d|^(p-2) = 2^((p-2) log2|d| + log2 w_ij) with log2 w computed once per
// entry, then phi = that * d and |d|^p = phi * d.  An exact zero difference
// gives phi = 0 (the log is clamped, see common.cuh) and, for p < 2, no
// curvature term in S.
//
// Data movement.  The kernels read a copy of W whose rows are stably sorted
// by degree (perm maps a sorted row back to its vertex).  A warp task is a run
// of consecutive sorted rows of one degree, so its entries are contiguous.
// Each warp owns a ring of kStages shared-memory stages; lane 0 fills a stage
// with the task's column indices, weights and perm slice by three TMA bulk
// copies completing on the stage's mbarrier, kStages tasks ahead of use, so
// the CSR stream never stalls the lanes: they wait only on the 16-byte
// gathers of neighbour rows of U (and V).  All barrier waits are bounded; a
// wait that gives up records a timeout in the status word and the warp stops.
//
// Work split.  A row is handled by a team of E edge slots x Q column lanes; a
// lane owns CPL = K/Q consecutive columns (16/8/4-byte vectors).  Typical rows
// get E = 1 (a lane walks its row UNR entries at a time, no shuffles); longer
// rows are shared by E slots and reduced by warp shuffles; rows above the hub
// threshold are split into chunks whose partial sums the warp finishing the
// row's last chunk adds in chunk order (atomic ticket, no spinning).
// Per-column sums live per lane in registers (compensated for the objective),
// then are reduced across the warp, block and grid in float-float in a fixed
// order, so every result is bit-reproducible run to run.
#pragma once

#include "common.cuh"

namespace pspec {

// Entries per lane per row before a row gets more edge slots: 8*Q, so the
// largest task (32/Q lanes x that) is 256 entries for every column split.
__host__ __device__ constexpr int edges_per_lane(int Q) { return 8 * Q; }
__host__ __device__ constexpr int task_max_entries(int Q) { return 32 * edges_per_lane(Q) / Q; }
constexpr int kStages = 3;
constexpr uint32_t kWaitTries = 2000;  // x up to 1 ms each: about 2 s before a timeout

template <int Q>
struct StageBuf {
  static constexpr int SEG = task_max_entries(Q) + 8;  // + alignment slack
  int4 desc;
  int32_t col[SEG];
  float val[SEG];
  int32_t perm[40];
};

template <int Q>
__host__ __device__ constexpr size_t edge_smem_bytes() {
  return sizeof(StageBuf<Q>) * kStages * kWarps + sizeof(uint64_t) * kStages * kWarps;
}

struct EdgeArgs {
  const int64_t* rowptr;  // degree-sorted rows
  const int32_t* col;
  const float* val;
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
  GridReduce gr;
  double* scalars;
  int* status;
  const int* skip;
  // batches: per-task column sums go to task_part[task][NV] instead of the
  // grid reduction (NULL for a single graph)
  float* task_part;
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

// per-lane accumulator: compensated for the objective's sums, plain for the
// Hessian product's (whose rank-two coefficients need ~1e-6 only)
template <bool COMP> struct LaneAcc;
template <> struct LaneAcc<true> {
  Kahan k;
  __device__ __forceinline__ void init() { k.init(); }
  __device__ __forceinline__ void add(float x) { k.add(x); }
  __device__ __forceinline__ float2 ff() const { return kahan_to_ff(k); }
};
template <> struct LaneAcc<false> {
  float s;
  __device__ __forceinline__ void init() { s = 0.f; }
  __device__ __forceinline__ void add(float x) { s += x; }
  __device__ __forceinline__ float2 ff() const { return make_float2(s, 0.f); }
};

// task descriptor fields (see ensure_tasks)
__device__ __forceinline__ bool task_is_hub(int4 t) { return ((t.z >> 8) & 1) != 0; }
__device__ __forceinline__ int task_entries(int4 t) {
  return task_is_hub(t) ? (t.z >> 10) : (t.y & 0xff) * (t.y >> 8);
}
__device__ __forceinline__ int task_rows(int4 t) { return task_is_hub(t) ? 1 : (t.y & 0xff); }

// lane 0: start the three bulk copies of task t into stage st.  Windows are
// widened to 16-byte granules (the arrays are padded past their ends).
template <int Q>
__device__ __forceinline__ void issue_stage(const EdgeArgs& a, int4 t, StageBuf<Q>* st, uint64_t* bar) {
  st->desc = t;
  const int cnt = task_entries(t);
  const int nr = task_rows(t);
  const int oc = t.w & 3;  // entries before the task in its first granule
  const int op = t.x & 3;
  const uint32_t bc = (uint32_t)((oc + cnt + 3) & ~3) * 4u;
  const uint32_t bp = (uint32_t)((op + nr + 3) & ~3) * 4u;
  mbar_arrive_expect_tx(bar, (cnt > 0 ? 2u * bc : 0u) + bp);
  if (cnt > 0) {
    tma_load_1d(st->col, a.col + (t.w - oc), bc, bar);
    tma_load_1d(st->val, a.val + (t.w - oc), bc, bar);
  }
  tma_load_1d(st->perm, a.perm + (t.x - op), bp, bar);
}

template <int K, bool HVP>
__global__ void __launch_bounds__(kBlock) edge_kernel(EdgeArgs a) {
  constexpr int Q = q_of(K);
  constexpr int CPL = K / Q;
  constexpr int VW = vw_of(K);
  constexpr int NQ = HVP ? 4 : 2;  // N, D (, sigma_N, sigma_D)
  constexpr int NV = NQ * K;
  constexpr int UNR = HVP ? (CPL > 8 ? 1 : 2) : (CPL > 8 ? 2 : 4);  // entries per lane per trip
  constexpr bool COMP = !HVP;

  if (a.skip && *a.skip) return;  // uniform over the grid
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float2 s_warp[kWarps][NV];
  __shared__ float2 s_blk[NV];
  __shared__ float2 s_tot[NV];

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  StageBuf<Q>* stages = reinterpret_cast<StageBuf<Q>*>(smem_raw) + wib * kStages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + sizeof(StageBuf<Q>) * kStages * kWarps) +
                   wib * kStages;
  const int q = lane % Q;
  const int c0 = q * CPL;
  const int gwarp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const float pm2 = a.pm2;
  const bool zero_rule = pm2 != 0.0f;  // p < 2: a zero difference has no curvature

  LaneAcc<COMP> accN[CPL], accD[CPL];
  LaneAcc<false> accCN[HVP ? CPL : 1], accCD[HVP ? CPL : 1];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    accN[c].init();
    accD[c].init();
    if constexpr (HVP) {
      accCN[c].init();
      accCD[c].init();
    }
  }

  // ---- prologue: barriers, then the first kStages tasks of this warp in flight
  if (lane == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
    mbar_init_fence();
    for (int s = 0; s < kStages; ++s) {
      const int t = gwarp + s * nwarps;
      if (t < a.n_tasks) issue_stage<Q>(a, __ldg(&a.tasks[t]), &stages[s], &bars[s]);
    }
  }
  __syncwarp();

  uint32_t phase = 0;  // bit s: parity of the next completion of stage s
  bool timed_out = false;
  int it = 0;
  for (int t = gwarp; t < a.n_tasks; t += nwarps, ++it) {
    const int s = it % kStages;
    // every lane observes the completion itself (acquire); the decision to go
    // on is taken by the whole warp
    const bool got = mbar_wait_bounded(&bars[s], (phase >> s) & 1u, kWaitTries);
    if (!__all_sync(0xffffffffu, got)) {
      timed_out = true;
      break;
    }
    phase ^= 1u << s;
    StageBuf<Q>& st = stages[s];
    const int4 task = st.desc;
    const bool hub = task_is_hub(task);
    const int elog = task.z & 0xff;
    const int E = 1 << elog;
    const int T = E * Q;
    const int team = lane / T;
    const int slot = (lane % T) / Q;
    const int oc = task.w & 3;
    const int op = task.x & 3;
    int l_beg, l_end;  // entries of this lane's row within the stage
    bool active;
    if (!hub) {
      const int deg = task.y >> 8;
      active = team < (task.y & 0xff);
      l_beg = oc + team * deg;
      l_end = l_beg + deg;
    } else {
      active = true;
      l_beg = oc;
      l_end = oc + (task.z >> 10);
    }
    const int64_t row = active ? (int64_t)st.perm[op + (hub ? 0 : team)] : 0;

    float ui[CPL], vi[CPL], dsum[CPL], nsum[CPL], ssum[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) { ui[c] = 0.f; vi[c] = 0.f; dsum[c] = 0.f; nsum[c] = 0.f; ssum[c] = 0.f; }
    if (active) {
      load_row<K, CPL, VW>(a.U, row, c0, ui);
      if constexpr (HVP) load_row<K, CPL, VW>(a.V, row, c0, vi);
      for (int e = l_beg + slot; e < l_end; e += UNR * E) {
        int jj[UNR];
        float lw[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int eu = e + u * E;
          const bool ok = eu < l_end;
          jj[u] = ok ? st.col[eu] : (int)row;  // off the end: own row, weight 0
          lw[u] = ok ? st.val[eu] : 0.0f;
        }
        float uj[UNR][CPL], vj[UNR][CPL];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          load_row<K, CPL, VW>(a.U, jj[u], c0, uj[u]);
          if constexpr (HVP) load_row<K, CPL, VW>(a.V, jj[u], c0, vj[u]);
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) lw[u] = lg2_approx(lw[u]);  // log2 0 = -inf: no contribution
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const float d = ui[c] - uj[u][c];
            const float sw = ex2_approx(fmaf(pm2, fmaxf(lg2_approx(fabsf(d)), -126.0f), lw[u]));
            const float ph = sw * d;  // w phi_p(d)
            dsum[c] += ph;
            nsum[c] = fmaf(ph, d, nsum[c]);  // w |d|^p
            if constexpr (HVP) {
              const float sz = (zero_rule && d == 0.0f) ? 0.0f : sw;
              ssum[c] = fmaf(sz, vi[c] - vj[u][c], ssum[c]);
            }
          }
        }
      }
    }
    // every lane has read the stage: refill it with this warp's task kStages ahead
    __syncwarp();
    if (lane == 0) {
      const int tn = t + kStages * nwarps;
      if (tn < a.n_tasks) {
        fence_proxy_async_smem();
        issue_stage<Q>(a, __ldg(&a.tasks[tn]), &st, &bars[s]);
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
    const bool first_chunk = !hub || ((task.z >> 9) & 1);
    // this task's contributions of this lane to the per-column sums
    float tN[CPL], tD[CPL], tCN[CPL], tCD[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) { tN[c] = 0.f; tD[c] = 0.f; tCN[c] = 0.f; tCD[c] = 0.f; }
    if (lead) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) tN[c] = nsum[c];
      if (first_chunk) {  // vertex terms once per row
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const float phu = abs_pow_pm2_clamped(ui[c], pm2) * ui[c];  // phi_p(u_i)
          tD[c] = phu * ui[c];                                        // |u_i|^p
          if constexpr (HVP) tCD[c] = phu * vi[c];
        }
      }
      // sigma_N: a whole row's Delta_i v_i, or a chunk's share of it
#pragma unroll
      for (int c = 0; c < CPL; ++c)
        if constexpr (HVP) tCN[c] = dsum[c] * vi[c];
      if (!hub) {
        if constexpr (HVP) {
          store_row<K, CPL, VW>(a.out_a, row, c0, ssum);
          store_row<K, CPL, VW>(a.out_b, row, c0, dsum);
        } else {
          store_row<K, CPL, VW>(a.out_a, row, c0, dsum);
        }
      }
    }
    if (!a.task_part) {
      if (lead) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          accN[c].add(tN[c]);
          accD[c].add(tD[c]);
          if constexpr (HVP) {
            accCN[c].add(tCN[c]);
            accCD[c].add(tCD[c]);
          }
        }
      }
    } else {
      // one graph of a batch: fold the task's sums over the warp (lanes of
      // equal q) and publish them in the task's slot
      for (int off = Q; off < 32; off <<= 1)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          tN[c] += __shfl_xor_sync(0xffffffffu, tN[c], off);
          tD[c] += __shfl_xor_sync(0xffffffffu, tD[c], off);
          if constexpr (HVP) {
            tCN[c] += __shfl_xor_sync(0xffffffffu, tCN[c], off);
            tCD[c] += __shfl_xor_sync(0xffffffffu, tCD[c], off);
          }
        }
      if (lane < Q) {
        float* tp = a.task_part + (size_t)t * NV;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          tp[c0 + c] = tN[c];
          tp[K + c0 + c] = tD[c];
          if constexpr (HVP) {
            tp[2 * K + c0 + c] = tCN[c];
            tp[3 * K + c0 + c] = tCD[c];
          }
        }
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
            store_row<K, CPL, VW>(a.out_b, row, c0, rd);
          } else {
            store_row<K, CPL, VW>(a.out_a, row, c0, rd);
          }
        }
        if (lane == 0) a.hub_ticket[h] = 0u;
      }
    }
  }
  if (timed_out) {
    // drain this warp's copies still in flight (bounded), then report
    if (lane == 0) {
      atomicOr(a.status, kStatusTimeout);
      int t = gwarp + it * nwarps;
      for (int k2 = 0; k2 < kStages && t < a.n_tasks; ++k2, ++it, t += nwarps) {
        const int s = it % kStages;
        mbar_wait_bounded(&bars[s], (phase >> s) & 1u, kWaitTries);
        phase ^= 1u << s;
      }
    }
    __syncwarp();
  }

  if (a.task_part) return;  // batches: per-graph sums are reduced by batch_reduce

  // warp: lanes of equal q in float-float; lanes 0..Q-1 hold the warp sums
  {
    float2 v[NQ][CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      v[0][c] = accN[c].ff();
      v[1][c] = accD[c].ff();
      if constexpr (HVP) {
        v[2][c] = accCN[c].ff();
        v[3][c] = accCD[c].ff();
      }
    }
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
  }
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
