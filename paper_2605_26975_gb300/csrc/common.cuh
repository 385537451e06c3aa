// Device helpers shared by the kernels of the p-spectral clustering library.
//
//  * fast transcendental wrappers (PTX lg2.approx / ex2.approx, flush to zero)
//  * compensated FP32 accumulation (Kahan) and float-float (double-single)
//    addition built on Knuth's TwoSum, used for every cross-thread reduction
//    so that no reduction depends on the GPU's slow FP64 pipe
//  * the deterministic two-level grid reduction: each block writes its
//    partials, the last block of every group of 32 blocks sums its group in
//    block order, and the last group finisher sums the groups in group order.
//    Finishing order is decided by atomic tickets, never by spinning, so
//    nothing here can wait forever.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pspec {

constexpr int kMaxK = 16;
constexpr int kBlock = 256;          // threads per block of the edge kernels
constexpr int kWarps = kBlock / 32;
constexpr int kGroup = 32;           // blocks per first-level reduction group

// status bits recorded by kernels (mapped to pspec_status on the host)
constexpr int kStatusZeroColumn = 1;
constexpr int kStatusNonFinite = 2;
constexpr int kStatusTimeout = 4;

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// a - b with a subnormal result flushed to zero, the same flush lg2.approx.ftz
// applies to its argument: a difference is either zero (a tie) or has a
// finite base-2 logarithm.
__device__ __forceinline__ float sub_ftz(float a, float b) {
  float y;
  asm("sub.ftz.f32 %0, %1, %2;" : "=f"(y) : "f"(a), "f"(b));
  return y;
}

// |x|^(p-2) for x != 0; for x == 0 the log is clamped so that the result is
// finite (2^(126 (2-p))) and x * result == 0, which gives phi_p(0) = 0.
// Only for terms without a weight: with a weight w the clamped value
// w 2^(126 (2-p)) can overflow, and the edge kernels select on x == 0 instead.
__device__ __forceinline__ float abs_pow_pm2_clamped(float x, float pm2) {
  float t = fmaxf(lg2_approx(fabsf(x)), -126.0f);
  return ex2_approx(pm2 * t);
}

// ------------------------------------------------- TMA bulk copy + mbarrier ---
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this thread's earlier shared-memory accesses before later async-proxy writes
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// One potentially blocking test: the thread is suspended in hardware until
// the phase with this parity completes or about kMbarSuspendNs pass, so a
// waiting warp issues a handful of instructions, not a spin loop.
constexpr uint32_t kMbarSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kMbarSuspendNs)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity: gives up after
// `max_tries` tests and returns false (the caller records a timeout).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_tries) {
  for (uint32_t i = 0; i < max_tries; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size multiple of
// 16) completing on `bar` with a transaction count of `bytes`.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ---------------------------------------------------------------- Kahan ---
struct Kahan {
  float s, c;  // running sum and compensation (true sum ~= s - c)
  __device__ __forceinline__ void init() { s = 0.0f; c = 0.0f; }
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// ---------------------------------------------------------- float-float ---
// value = hi + lo with |lo| <= ulp(hi)/2
__device__ __forceinline__ float2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float v = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  float2 t = two_sum(a.y, b.y);
  float e = __fadd_rn(s.y, t.x);
  float2 u = two_sum(s.x, e);
  e = __fadd_rn(u.y, t.y);
  return two_sum(u.x, e);
}
__device__ __forceinline__ float2 kahan_to_ff(const Kahan& k) { return two_sum(k.s, -k.c); }
__device__ __forceinline__ double ff_to_double(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float2 shfl_xor_ff(float2 v, int off) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, off);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, off);
  return v;
}

// ------------------------------------------------------------ grid reduce ---
// Scratch for the two-level reduction of NV float-float values per block.
struct GridReduce {
  float2* block_part;   // [gridDim.x][NV]
  float2* group_part;   // [ceil(gridDim.x / kGroup)][NV]
  unsigned* counters;   // [ceil(gridDim.x / kGroup) + 1], zero between launches
};

// Called by every thread of every block after the block's NV partials are in
// shared memory `mine`.  Returns true in exactly one block (the last to
// finish), in which `total[0..NV)` (shared memory) then holds the grid sums.
// Summation order is fixed (block index, then group index), so the result
// does not depend on which block finishes last.
template <int NV>
__device__ bool grid_reduce_ff(const float2* mine, float2* total, const GridReduce& gr) {
  __shared__ int s_flag;
  const int tid = threadIdx.x;
  const int nblk = gridDim.x;
  const int ngroups = (nblk + kGroup - 1) / kGroup;
  const int g = blockIdx.x / kGroup;
  if (tid < NV) gr.block_part[(size_t)blockIdx.x * NV + tid] = mine[tid];
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    int gsize = min(kGroup, nblk - g * kGroup);
    unsigned t = atomicAdd(&gr.counters[g], 1u);
    s_flag = (t == (unsigned)(gsize - 1));
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  if (tid < NV) {
    float2 acc = make_float2(0.f, 0.f);
    int b0 = g * kGroup, b1 = min(nblk, b0 + kGroup);
    for (int b = b0; b < b1; ++b) acc = ff_add(acc, __ldcg(&gr.block_part[(size_t)b * NV + tid]));
    gr.group_part[(size_t)g * NV + tid] = acc;
  }
  if (tid == 0) gr.counters[g] = 0u;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    unsigned t = atomicAdd(&gr.counters[ngroups], 1u);
    s_flag = (t == (unsigned)(ngroups - 1));
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  if (tid < NV) {
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < ngroups; ++q) acc = ff_add(acc, __ldcg(&gr.group_part[(size_t)q * NV + tid]));
    total[tid] = acc;
  }
  if (tid == 0) gr.counters[ngroups] = 0u;
  __syncthreads();
  return true;
}

// ------------------------------------------------------ vector load/store ---
template <int VW> struct VecT;
template <> struct VecT<1> { using T = float; };
template <> struct VecT<2> { using T = float2; };
template <> struct VecT<4> { using T = float4; };

template <int VW>
__device__ __forceinline__ void load_vec(const float* p, float* dst) {
  if constexpr (VW == 4) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
  } else if constexpr (VW == 2) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    dst[0] = v.x; dst[1] = v.y;
  } else {
    dst[0] = __ldg(p);
  }
}
template <int VW>
__device__ __forceinline__ void store_vec(float* p, const float* src) {
  if constexpr (VW == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(src[0], src[1], src[2], src[3]);
  } else if constexpr (VW == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(src[0], src[1]);
  } else {
    p[0] = src[0];
  }
}

// Column split of a k-column row: Q lanes share one edge, each lane owning
// CPL = K/Q consecutive columns loaded as vectors of VW floats.
__host__ __device__ constexpr int q_of(int K) {
  return (K % 4 == 0 && K / 4 >= 4) ? 4 : (K % 2 == 0 && K / 2 >= 4) ? 2 : 1;
}
__host__ __device__ constexpr int vw_of(int K) {
  return ((K / q_of(K)) % 4 == 0) ? 4 : ((K / q_of(K)) % 2 == 0) ? 2 : 1;
}

}  // namespace pspec
