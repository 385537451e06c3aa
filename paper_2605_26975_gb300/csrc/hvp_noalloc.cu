// pspec_hvp_noalloc: the Hessian-vector product of pspec_hvp for callers that
// cannot allocate device memory -- code whose device memory is owned by
// another runtime's allocator (a framework's caching pool, an embedding
// application that hands out fixed buffers), or a latency-critical path that
// must not enter cudaMalloc, which can synchronise the device.  It takes the
// CSR arrays and blocks directly (no graph handle: creating one allocates)
// and keeps its working memory -- the rows of Delta_p u and the partial sums
// of the grid reduction -- in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.  The
// call enqueues kernels and a memset, so like any CUDA call it must not be
// made from a host function running on a stream (cudaLaunchHostFunc).
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress (host code cannot use the
// array's name as a device pointer) and keeps it for the life of the process;
// that first call should come before any stream capture, and the function
// must not be used across a cudaDeviceReset of that device in the same
// process (the kept address would be stale).  Calls share the array: two
// calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race and corrupt each other's results; serialise
// them.  There is no status word: a non-finite intermediate shows up as a NaN
// or an infinity in HV_out.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace pspec {
namespace {

constexpr int64_t kNaMaxElems = 1 << 19;  // n * k limit: 2 MB of Delta rows
constexpr int kNaMaxBlocks = 1024;
constexpr int kNaMaxNV = 4 * kMaxK;
constexpr int kNaGroups = kNaMaxBlocks / kGroup + 1;
constexpr int kNaEdgeSlots = 4;  // edge slots per row

// byte layout of the scratch array
constexpr size_t kOffDelta = 0;
constexpr size_t kOffBlock = kOffDelta + sizeof(float) * kNaMaxElems;
constexpr size_t kOffGroup = kOffBlock + sizeof(float2) * kNaMaxBlocks * kNaMaxNV;
constexpr size_t kOffCount = kOffGroup + sizeof(float2) * kNaGroups * kNaMaxNV;
constexpr size_t kOffScal = kOffCount + 256;  // counters: kNaGroups + 1 unsigned
constexpr size_t kNaBytes = kOffScal + sizeof(double) * 128;

static __device__ __align__(256) unsigned char g_na_scratch[kNaBytes];

struct NaArgs {
  const int64_t* rowptr;
  const int32_t* col;
  const float* val;
  const float* U;
  const float* V;
  float* S;      // sparse part, into the caller's output
  float* delta;  // scratch
  int64_t n;
  float pm2;
  double p;  // exactly as passed (the FP64 coefficients use it)
  GridReduce gr;
  double* coef;  // scratch: A, lambda, B, sigma_D, E per column (5 x 16)
};

// One pass over the rows: a team of kNaEdgeSlots x Q lanes per row, rows in
// grid-stride order; the same arithmetic and reductions as the edge kernel of
// pspec_hvp, without its degree-sorted layout or prefetch ring.
template <int K>
__global__ void __launch_bounds__(kBlock) na_hvp_edges(NaArgs a) {
  constexpr int Q = q_of(K);
  constexpr int CPL = K / Q;
  constexpr int VW = vw_of(K);
  constexpr int T = kNaEdgeSlots * Q;
  constexpr int RPW = 32 / T;  // rows per warp step
  constexpr int NV = 4 * K;
  __shared__ float2 s_warp[kWarps][NV];
  __shared__ float2 s_blk[NV];
  __shared__ float2 s_tot[NV];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = lane % Q, c0 = q * CPL;
  const int team = lane / T, slot = (lane % T) / Q;
  const int64_t gwarp = (blockIdx.x * (int64_t)kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
  const bool zero_rule = a.pm2 != 0.0f;
  float accN[CPL], accD[CPL], accCN[CPL], accCD[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) accN[c] = accD[c] = accCN[c] = accCD[c] = 0.f;

  for (int64_t base = gwarp * RPW; base < a.n; base += nwarps * RPW) {
    const int64_t row = base + team;
    const bool active = row < a.n;
    float ui[CPL], vi[CPL], ds[CPL], ns[CPL], ss[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) ui[c] = vi[c] = ds[c] = ns[c] = ss[c] = 0.f;
    if (active) {
#pragma unroll
      for (int j = 0; j < CPL; j += VW) {
        load_vec<VW>(a.U + row * K + c0 + j, ui + j);
        load_vec<VW>(a.V + row * K + c0 + j, vi + j);
      }
      const int64_t e1 = a.rowptr[row + 1];
      for (int64_t e = a.rowptr[row] + slot; e < e1; e += kNaEdgeSlots) {
        const int64_t jr = a.col[e];
        const float lw = lg2_approx(a.val[e]);
        float uj[CPL], vj[CPL];
#pragma unroll
        for (int j = 0; j < CPL; j += VW) {
          load_vec<VW>(a.U + jr * K + c0 + j, uj + j);
          load_vec<VW>(a.V + jr * K + c0 + j, vj + j);
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          // w |d|^(p-2); a tie (d == 0, subnormal differences flushed) has no
          // curvature term for p < 2 and is selected away before phi = that * d,
          // so a large weight never meets inf * 0
          const float d = sub_ftz(ui[c], uj[c]);
          const float sw = ex2_approx(fmaf(a.pm2, fmaxf(lg2_approx(fabsf(d)), -126.0f), lw));
          const float sz = (zero_rule && d == 0.0f) ? 0.0f : sw;
          const float ph = sz * d;
          ds[c] += ph;
          ns[c] = fmaf(ph, d, ns[c]);
          ss[c] = fmaf(sz, vi[c] - vj[c], ss[c]);
        }
      }
    }
#pragma unroll
    for (int off = Q; off < T; off <<= 1)
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        ds[c] += __shfl_xor_sync(0xffffffffu, ds[c], off);
        ns[c] += __shfl_xor_sync(0xffffffffu, ns[c], off);
        ss[c] += __shfl_xor_sync(0xffffffffu, ss[c], off);
      }
    if (active && slot == 0) {
#pragma unroll
      for (int j = 0; j < CPL; j += VW) {
        store_vec<VW>(a.S + row * K + c0 + j, ss + j);
        store_vec<VW>(a.delta + row * K + c0 + j, ds + j);
      }
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const float phu = abs_pow_pm2_clamped(ui[c], a.pm2) * ui[c];
        accN[c] += ns[c];
        accD[c] += phu * ui[c];
        accCN[c] += ds[c] * vi[c];
        accCD[c] += phu * vi[c];
      }
    }
  }
  // warp, block and grid sums in float-float, fixed order
  float2 v[4][CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    v[0][c] = make_float2(accN[c], 0.f);
    v[1][c] = make_float2(accD[c], 0.f);
    v[2][c] = make_float2(accCN[c], 0.f);
    v[3][c] = make_float2(accCD[c], 0.f);
  }
#pragma unroll
  for (int off = Q; off < 32; off <<= 1)
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)
#pragma unroll
      for (int c = 0; c < CPL; ++c) v[qq][c] = ff_add(v[qq][c], shfl_xor_ff(v[qq][c], off));
  if (lane < Q)
#pragma unroll
    for (int qq = 0; qq < 4; ++qq)
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
  if (threadIdx.x < K) {
    const int c = threadIdx.x;
    const double N = 0.5 * ff_to_double(s_tot[c]);
    const double D = ff_to_double(s_tot[K + c]);
    const double sN = ff_to_double(s_tot[2 * K + c]);
    const double sD = ff_to_double(s_tot[3 * K + c]);
    const double p = a.p, lam = N / D;
    a.coef[0 * 16 + c] = p * (p - 1.0) / D;
    a.coef[1 * 16 + c] = lam;
    a.coef[2 * 16 + c] = p * p / (D * D);
    a.coef[3 * 16 + c] = sD;
    a.coef[4 * 16 + c] = sN - 2.0 * lam * sD;
  }
}

// HV = A (S - lambda s_u v) - B (Delta sigma_D + phi_p(u) E), in place over S
__global__ void __launch_bounds__(256) na_hvp_epilogue(const float* U, const float* V,
                                                       const float* delta, float* HV, int64_t m,
                                                       int K, const double* coef, float pm2) {
  __shared__ float c5[5][kMaxK];
  if (threadIdx.x < 5 * kMaxK) c5[threadIdx.x / kMaxK][threadIdx.x % kMaxK] =
      (float)coef[(threadIdx.x / kMaxK) * 16 + threadIdx.x % kMaxK];
  __syncthreads();
  const bool zero_rule = pm2 != 0.0f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % K);
    const float u = U[e];
    float su = abs_pow_pm2_clamped(u, pm2);
    const float phu = su * u;
    if (zero_rule && u == 0.0f) su = 0.0f;
    HV[e] = c5[0][c] * (HV[e] - c5[1][c] * su * V[e]) - c5[2][c] * (delta[e] * c5[3][c] + phu * c5[4][c]);
  }
}

std::mutex g_na_mutex;
void* g_na_ptr[64] = {};

pspec_status na_scratch(void** out) {
  int dev = 0;
  PSPEC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_error(PSPEC_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    PSPEC_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return PSPEC_OK;
}

template <int K>
pspec_status na_launch(const NaArgs& a, int sm_count, cudaStream_t s) {
  static const int occ = [] {  // once per instantiation, thread-safe
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, na_hvp_edges<K>, kBlock, 0) != cudaSuccess) o = 1;
    return std::max(o, 1);
  }();
  constexpr int RPW = 32 / (kNaEdgeSlots * q_of(K));
  const int64_t want = (a.n + (int64_t)RPW * kWarps - 1) / ((int64_t)RPW * kWarps);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)sm_count * occ, kNaMaxBlocks}));
  na_hvp_edges<K><<<blocks, kBlock, 0, s>>>(a);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}

}  // namespace
}  // namespace pspec

using namespace pspec;

extern "C" pspec_status pspec_hvp_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                                          const float* val, const float* U, const float* V, int k,
                                          double p, float* HV_out, void* stream) {
  if (n < 1 || !rowptr || !col || !val || !U || !V || !HV_out)
    return set_error(PSPEC_ERR_INVALID_ARG, "pspec_hvp_noalloc: NULL pointer or n < 1");
  if (k < 1 || k > kMaxK) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_hvp_noalloc: k must be in [1, 16]");
  if (!(p > 1.0 && p <= 2.0)) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_hvp_noalloc: p must be in (1, 2]");
  if (n * (int64_t)k > kNaMaxElems)
    return set_error(PSPEC_ERR_INVALID_ARG,
                     "pspec_hvp_noalloc: n * k exceeds the 524288-element limit of its static scratch");
  PSPEC_TRY(check_block(U, k, PSPEC_F32, "U"));
  PSPEC_TRY(check_block(V, k, PSPEC_F32, "V"));
  PSPEC_TRY(check_block(HV_out, k, PSPEC_F32, "HV_out"));
  void* base = nullptr;
  PSPEC_TRY(na_scratch(&base));
  unsigned char* sb = static_cast<unsigned char*>(base);
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  PSPEC_CUDA(cudaGetDevice(&dev));
  PSPEC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  NaArgs a;
  a.rowptr = rowptr;
  a.col = col;
  a.val = val;
  a.U = U;
  a.V = V;
  a.S = HV_out;
  a.delta = reinterpret_cast<float*>(sb + kOffDelta);
  a.n = n;
  a.p = p;
  a.pm2 = (float)p - 2.0f;
  a.gr.block_part = reinterpret_cast<float2*>(sb + kOffBlock);
  a.gr.group_part = reinterpret_cast<float2*>(sb + kOffGroup);
  a.gr.counters = reinterpret_cast<unsigned*>(sb + kOffCount);
  a.coef = reinterpret_cast<double*>(sb + kOffScal);
  // the grid reduction's tickets must start at zero
  PSPEC_CUDA(cudaMemsetAsync(sb + kOffCount, 0, 256, s));
  pspec_status st;
  switch (k) {
#define CASE(K) \
  case K:       \
    st = na_launch<K>(a, sms, s); \
    break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
    default:
      st = PSPEC_ERR_INVALID_ARG;
  }
  if (st != PSPEC_OK) return st;
  const int64_t m = n * k;
  const int eb = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)sms * 8));
  na_hvp_epilogue<<<eb, 256, 0, s>>>(U, V, a.delta, HV_out, m, k, a.coef, a.pm2);
  PSPEC_CUDA(cudaGetLastError());
  return PSPEC_OK;
}
