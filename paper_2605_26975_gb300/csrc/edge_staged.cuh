// Staged edge kernels: the computation of edge_kernel (edge_kernels.cuh) --
// the objective's Delta_p u, N, D and the Hessian product's sparse part,
// sigma_N, sigma_D (Section 2, Algorithm 1) -- with the memory traffic of a
// warp task reorganised to shorten its chain of dependent loads.
//
// The direct kernel walks a task as: descriptor -> (perm, entries) ->
// neighbour rows, the last in steps of a few entries, each step a memory
// round trip.  Here, per warp:
//  * the entries and perm of the NEXT task are copied into shared memory with
//    cp.async while the current task is worked on (its descriptor was loaded
//    one task earlier still), so a task starts with its entries on chip;
//  * all neighbour rows of the task (U, and V for the Hessian product) are
//    requested at once with cp.async into shared memory -- no registers held
//    for loads in flight, one round trip per task -- together with the own
//    rows, then the arithmetic runs from shared memory.
// The arithmetic per entry is the direct kernel's (edge_group), so results
// agree with it to rounding of the summation order only.
//
// Shared memory per warp (dynamic, sized by the task set's entries per task
// M = 32 L / Q): entries 2 x M x 8 bytes, perm 2 x 32 x 4, neighbour rows
// M x K x 4 (x 2 for the Hessian product).  The task set's L must keep
// M <= staged_max_entries(K) (the launcher checks it).
//
// Modes: objective (N, D, Delta_p u), Hessian product (N, D, sigma_N,
// sigma_D, S, optionally Delta_p u), Hessian product at a point whose Delta_p u
// and N, D were kept by the evaluation (sigma_N, sigma_D and S only).
#pragma once

#include "edge_kernels.cuh"

namespace pspec {

// Most entries a task may hold for the staged kernel of column count K: the
// neighbour rows of U and V for that many entries take at most 8 KB per warp.
__host__ __device__ constexpr int staged_max_entries(int K) {
  return (8192 / (8 * K)) > 256 ? 256 : (8192 / (8 * K));
}

__host__ __device__ constexpr size_t staged_warp_bytes(int K, int mode, int max_entries) {
  return (size_t)max_entries * 8 * 2 + 32 * 4 * 2 +
         (size_t)max_entries * K * 4 * (mode == kModeEval ? 1 : 2);
}

__device__ __forceinline__ void cp_async_4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_16(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int VW>
__device__ __forceinline__ void cp_async_vec(uint32_t dst, const float* src) {
  if constexpr (VW == 4) cp_async_16(dst, src);
  else if constexpr (VW == 2) cp_async_8(dst, src);
  else cp_async_4(dst, src);
}

// CPL columns of row `row` of a row-major n x K block into shared memory at dst
template <int K, int CPL, int VW>
__device__ __forceinline__ void stage_row(uint32_t dst, const float* base, int64_t row, int c0) {
#pragma unroll
  for (int j = 0; j < CPL; j += VW) cp_async_vec<VW>(dst + 4 * j, base + row * K + c0 + j);
}

template <int CPL, int VW>
__device__ __forceinline__ void lds_row(const float* src, float* dst) {
#pragma unroll
  for (int j = 0; j < CPL; j += VW) {
    if constexpr (VW == 4) {
      const float4 t = *reinterpret_cast<const float4*>(src + j);
      dst[j] = t.x; dst[j + 1] = t.y; dst[j + 2] = t.z; dst[j + 3] = t.w;
    } else if constexpr (VW == 2) {
      const float2 t = *reinterpret_cast<const float2*>(src + j);
      dst[j] = t.x; dst[j + 1] = t.y;
    } else {
      dst[j] = src[j];
    }
  }
}

// entries count of a task and its number of rows (1 for a hub chunk)
__device__ __forceinline__ int task_entries(int4 t) {
  return task_is_hub(t) ? (t.z >> 10) : (t.y & 0xff) * (t.y >> 8);
}
__device__ __forceinline__ int task_rows(int4 t) { return task_is_hub(t) ? 1 : (t.y & 0xff); }

// copy a task's entries and perm into this warp's shared buffers (all lanes)
__device__ __forceinline__ void stage_task(const EdgeArgs& a, int4 t, uint32_t ent, uint32_t prm, int lane) {
  const int ne = task_entries(t);
  const int2* src = a.cw + t.w;
  for (int i = lane; i < ne; i += 32) cp_async_8(ent + 8 * i, src + i);
  if (lane < task_rows(t)) cp_async_4(prm + 4 * lane, a.perm + t.x + lane);
}

// One entry of a lane's row from the staged buffers: the arithmetic of
// edge_group (edge_kernels.cuh), with the neighbour row read from shared
// memory.  With KEPT the objective's sum |d|^p is not formed (N is kept).
template <int K, int CPL, int VW, bool HVP, bool KEPT>
__device__ __forceinline__ void staged_entry(const int2* ent, const float* gu, const float* gv, int idx,
                                             int c0, const float (&ui)[CPL], const float (&vi)[CPL],
                                             float ex, bool zero_rule, float (&dsum)[CPL],
                                             float (&nsum)[CPL], float (&ssum)[CPL]) {
  const float lw = __int_as_float(ent[idx].y);
  float uj[CPL], vj[CPL];
  lds_row<CPL, VW>(gu + idx * K + c0, uj);
  if constexpr (HVP) lds_row<CPL, VW>(gv + idx * K + c0, vj);
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const float d = sub_ftz(ui[c], uj[c]);
    if constexpr (HVP) {
      const float sw = ex2_approx(fmaf(ex, fmaxf(lg2_approx(fabsf(d)), -126.0f), lw));
      const float sz = (zero_rule && d == 0.0f) ? 0.0f : sw;  // w |d|^(p-2)
      const float ph = sz * d;                                 // w phi_p(d)
      dsum[c] += ph;
      if constexpr (!KEPT) nsum[c] = fmaf(ph, d, nsum[c]);
      ssum[c] = fmaf(sz, vi[c] - vj[c], ssum[c]);
    } else {
      const float ph = copysignf(ex2_approx(fmaf(ex, lg2_approx(fabsf(d)), lw)), d);  // w phi_p(d)
      dsum[c] += ph;
      nsum[c] = fmaf(ph, d, nsum[c]);  // w |d|^p
    }
  }
}

template <int K, int MODE>
__global__ void __launch_bounds__(kBlock, 2) edge_staged_kernel(EdgeArgs a, int max_entries) {
  constexpr bool HVP = MODE != kModeEval;
  constexpr bool KEPT = MODE == kModeHvpKept;
  constexpr int Q = q_of(K);
  constexpr int CPL = K / Q;
  constexpr int VW = vw_of(K);
  constexpr int NQ = (MODE == kModeHvp) ? 4 : 2;  // N, D (, sigma_N, sigma_D) | sigma_N, sigma_D
  constexpr bool COMP = !HVP;
  using Acc = AccBank<CPL, NQ, COMP, false>;

  if (a.skip && *a.skip) return;  // uniform over the grid
  extern __shared__ __align__(16) unsigned char s_dyn[];

  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int q = lane % Q;
  const int c0 = q * CPL;
  const int gwarp = (blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * kBlock) >> 5;
  const float pm2 = a.pm2;
  const float ex = HVP ? pm2 : a.p - 1.0f;
  const bool zero_rule = pm2 != 0.0f;

  // this warp's buffers
  unsigned char* wbase = s_dyn + (size_t)wib * staged_warp_bytes(K, MODE, max_entries);
  int2* ent_s = reinterpret_cast<int2*>(wbase);                          // [2][max_entries]
  int* prm_s = reinterpret_cast<int*>(wbase + (size_t)max_entries * 16);  // [2][32]
  float* gu = reinterpret_cast<float*>(wbase + (size_t)max_entries * 16 + 256);  // [max_entries][K]
  float* gv = gu + (size_t)max_entries * K;                                        // HVP: [max_entries][K]
  const uint32_t ent_a = smem_u32(ent_s), prm_a = smem_u32(prm_s);
  const uint32_t gu_a = smem_u32(gu), gv_a = smem_u32(gv);

  Acc acc;
  acc.init(nullptr);

  int t = gwarp;
  int4 cur = make_int4(0, 0, 0, 0), nxt = make_int4(0, 0, 0, 0);
  if (t < a.n_tasks) {
    cur = __ldg(&a.tasks[t]);
    stage_task(a, cur, ent_a, prm_a, lane);
  }
  cp_async_commit();
  if (t + nwarps < a.n_tasks) nxt = __ldg(&a.tasks[t + nwarps]);
  int buf = 0;

  for (; t < a.n_tasks; t += nwarps) {
    const int4 task = cur;
    cp_async_wait<0>();  // this task's entries and perm
    __syncwarp();
    const int2* ent = ent_s + buf * max_entries;
    const int* prm = prm_s + buf * 32;

    const bool hub = task_is_hub(task);
    const int elog = task.z & 0xff;
    const int E = 1 << elog;
    const int T = E * Q;
    const int team = lane / T;
    const int slot = (lane % T) / Q;
    int cnt, off;  // entries of this lane's row (or hub chunk), offset of the row in the task
    bool active;
    if (!hub) {
      const int deg = task.y >> 8;
      active = team < (task.y & 0xff);
      cnt = deg;
      off = team * deg;
    } else {
      active = true;
      cnt = task.z >> 10;
      off = 0;
    }
    const int n_my = (active && slot < cnt) ? ((cnt - slot + E - 1) >> elog) : 0;
    const int64_t row = active ? (int64_t)prm[hub ? 0 : team] : 0;

    // own row into registers, every neighbour row into shared memory
    float ui[CPL], vi[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) { ui[c] = 0.f; vi[c] = 0.f; }
    if (active) {
      load_row<K, CPL, VW>(a.U, row, c0, ui);
      if constexpr (HVP) load_row<K, CPL, VW>(a.V, row, c0, vi);
    }
    for (int j = 0; j < n_my; ++j) {
      const int idx = off + slot + (j << elog);
      const int64_t col = (int64_t)(uint32_t)ent[idx].x;
      const uint32_t o = 4u * (uint32_t)(idx * K + c0);
      stage_row<K, CPL, VW>(gu_a + o, a.U, col, c0);
      if constexpr (HVP) stage_row<K, CPL, VW>(gv_a + o, a.V, col, c0);
    }
    cp_async_commit();
    // the next task's entries and perm into the other buffer, and the
    // descriptor of the task after it
    const int tn = t + nwarps;
    if (tn < a.n_tasks) stage_task(a, nxt, ent_a + 8u * (uint32_t)((buf ^ 1) * max_entries),
                                   prm_a + 4u * (uint32_t)((buf ^ 1) * 32), lane);
    cp_async_commit();
    cur = nxt;
    if (tn + nwarps < a.n_tasks) nxt = __ldg(&a.tasks[tn + nwarps]);
    cp_async_wait<1>();  // the neighbour rows (the entries of the next task may still fly)

    float dsum[CPL], nsum[CPL], ssum[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) { dsum[c] = 0.f; nsum[c] = 0.f; ssum[c] = 0.f; }
    int j = 0;
    for (; j + 2 <= n_my; j += 2) {
#pragma unroll
      for (int u = 0; u < 2; ++u)
        staged_entry<K, CPL, VW, HVP, KEPT>(ent, gu, gv, off + slot + ((j + u) << elog), c0, ui, vi, ex,
                                            zero_rule, dsum, nsum, ssum);
    }
    if (j < n_my)
      staged_entry<K, CPL, VW, HVP, KEPT>(ent, gu, gv, off + slot + (j << elog), c0, ui, vi, ex, zero_rule,
                                          dsum, nsum, ssum);
    // row sums across the E edge slots of each team (lanes of equal q)
    for (int o = Q; o < T; o <<= 1) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        dsum[c] += __shfl_xor_sync(0xffffffffu, dsum[c], o);
        if constexpr (!KEPT) nsum[c] += __shfl_xor_sync(0xffffffffu, nsum[c], o);
        if constexpr (HVP) ssum[c] += __shfl_xor_sync(0xffffffffu, ssum[c], o);
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
      for (int o = Q; o < 32; o <<= 1)
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
          for (int c = 0; c < CPL; ++c) tq[qq][c] += __shfl_xor_sync(0xffffffffu, tq[qq][c], o);
      if (lane < Q) {
        float* tp = a.task_part + (size_t)t * (NQ * K);
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
#pragma unroll
          for (int c = 0; c < CPL; ++c) tp[qq * K + c0 + c] = tq[qq][c];
      }
    }
    if (hub) {
      // publish this chunk's partial row sums; the warp that finishes the
      // row's last chunk adds them up in chunk order (as the direct kernel)
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
    buf ^= 1;
  }
  cp_async_wait<0>();  // nothing left in flight before the warp leaves its buffers
  if (a.task_part) return;  // batches: per-graph sums are reduced by batch_reduce

  float2 v[NQ][CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) v[qq][c] = acc.ff(qq, c);
  finish_edges<K, NQ, HVP, KEPT>(v, a);
}

}  // namespace pspec
