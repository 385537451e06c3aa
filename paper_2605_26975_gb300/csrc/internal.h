// Host-side internals of the p-spectral clustering library: the graph handle,
// its device workspace, error plumbing and per-kernel timing.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "pspec.h"

namespace pspec {

// ------------------------------------------------------------ row tasks ---
// The edge kernels walk a list of warp tasks over the degree-sorted rows.  A
// plain task covers `nrows` consecutive sorted rows starting at `row`, each
// processed by a team of E = 2^elog edge slots x Q column lanes
// (E*Q*nrows <= 32); sorting makes the rows of a task (nearly) equally long.  A hub chunk task
// covers edges [rowptr[row] + chunk*chunk_edges, ...) of one long row with the
// whole warp; its partial row sums go to hub slot `slot`, and the warp that
// finishes the row's last chunk adds the chunks up in chunk order.
struct TaskSet {
  bool built = false;
  int Q = 0;
  int L = 0;            // edges-per-lane target the set was built with
  int chunk_edges = 0;  // = most entries of one task, 32 L / Q
  int64_t n_tasks = 0;
  int n_hubs = 0;
  int n_chunks = 0;
  int4* d_tasks = nullptr;          // x=row, y=nrows|chunk, z=elog|(hub<<8), w=slot
  int32_t* d_hub_row = nullptr;     // [n_hubs]
  int32_t* d_hub_first = nullptr;   // [n_hubs] first slot of the hub's chunks
  int32_t* d_hub_nchunk = nullptr;  // [n_hubs]
  unsigned* d_hub_ticket = nullptr; // [n_hubs] chunk completion counters
  int32_t* d_chunk_hub = nullptr;   // [n_chunks] hub index of each chunk
  int32_t* d_task_graph = nullptr;  // [n_tasks] graph of each task (batches)
  int32_t* d_graph_task = nullptr;  // [G+1] first task of each graph (batches)
  // splits of the task list into contiguous, equally costly warp ranges
  // (launches with few tasks per warp): prefix sums of each task's
  // estimated cost, and per warp count the uploaded first task of each warp
  std::vector<int64_t> h_cost;                      // [n_tasks + 1]
  std::vector<std::pair<int, int32_t*>> splits;     // (warps, device [warps + 1])
};

struct Timing {
  bool enabled = false;
  struct Pending {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, std::pair<long long, double>> totals;
};

}  // namespace pspec

struct pspec_graph {
  int64_t n = 0, nnz = 0;
  // rows the edge kernels and epilogues cover: n, or for a shard of a
  // row-partitioned graph its owned rows (the first n_owned local vertices;
  // the rest are halo vertices, read only as neighbours)
  int64_t n_owned = 0;
  bool is_shard = false;
  int32_t n_graphs = 1;
  int device = 0;
  int sm_count = 0;
  // device CSR in the caller's row order
  int64_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  float* d_val32 = nullptr;
  double* d_val64 = nullptr;
  std::vector<int64_t> h_rowptr;     // host copy (task building, batching)
  // the same matrix with its rows stably sorted by degree (fast edge kernels):
  // sorted row r is row d_perm[r] of W; column indices are unchanged; each
  // entry is one 8-byte word {column, bits of (float)log2(w)}
  int2* d_cw_s = nullptr;
  int32_t* d_perm = nullptr;
  std::vector<int64_t> h_rowptr_s;
  std::vector<int32_t> h_perm;
  // batched graphs
  std::vector<int64_t> h_node_off;
  int64_t* d_node_off = nullptr;
  int32_t* d_row_graph = nullptr;     // [n] graph of each vertex
  double* d_graph_scalars = nullptr;  // [G][128]: N, D, sigma_N, sigma_D, coefficients, F
  float* d_task_part = nullptr;       // [n_tasks][64] per-task column sums
  size_t task_part_elems = 0;
  // edge-kernel partitions, one per column split Q in {1, 2, 4}
  pspec::TaskSet tasks[3];
  // launch shape per column split (index q_index(Q)); 0 = built-in default.
  // Set by pspec_tune or the PSPEC_EDGES_PER_LANE / PSPEC_EDGE_BLOCKS_PER_SM
  // environment variables.
  int edges_per_lane[3] = {0, 0, 0};
  int edge_blocks_per_sm[3] = {0, 0, 0};
  // workspace
  float* d_scratch = nullptr;        // n x 16 floats (HVP's Delta rows)
  size_t scratch_elems = 0;
  // Delta_p u kept by pspec_eval(PSPEC_KEEP_DELTA) for pspec_hvp(PSPEC_DELTA_KEPT)
  float* d_delta_keep = nullptr;     // n x k floats
  size_t delta_keep_elems = 0;
  bool keep_valid = false;
  const void* keep_U = nullptr;      // the U pointer as passed (host or device)
  unsigned keep_host = 0;            // PSPEC_HOST_PTRS of that call
  int keep_k = 0;
  double keep_p = 0.0;
  float* d_hub_part = nullptr;       // [max chunks][2*16] partial row sums
  size_t hub_part_elems = 0;
  float2* d_block_part = nullptr;    // [max blocks][64]
  float2* d_group_part = nullptr;    // [max groups][64]
  unsigned* d_counters = nullptr;    // [max groups + 1]
  double* d_scalars = nullptr;       // [512] per-call FP64 scalars
  double* d_red64 = nullptr;         // FP64 block partials of the plain path
  int* d_status = nullptr;           // kernel-recorded conditions
  int max_blocks = 0;
  // host staging for PSPEC_HOST_PTRS calls
  void* h_pinned = nullptr;
  size_t h_pinned_bytes = 0;
  void* d_io = nullptr;
  size_t d_io_bytes = 0;
  bool io_u_kept = false;  // d_io's first block holds U of the kept point (host-pointer calls)
  // solver workspace (allocated on first solve)
  void* d_solve = nullptr;
  size_t d_solve_bytes = 0;
  // pspec_solve runs on this private stream (joined to the caller's stream
  // by events), on which it can capture CUDA graphs whatever the caller's
  // stream is (capture is not possible on the legacy default stream)
  cudaStream_t solve_stream = nullptr;
  cudaEvent_t solve_event = nullptr;
  void* h_solve_rec = nullptr;  // pinned 512 bytes: the solve's per-step host record
  // batches: one single-graph handle per graph, built by the first
  // pspec_solve_batched call (columns rebased to the graph's own vertices)
  std::vector<pspec_graph*> subs;
  pspec::Timing timing;
};

namespace pspec {

// error plumbing -----------------------------------------------------------
pspec_status set_error(pspec_status s, const std::string& msg);
pspec_status cuda_error(cudaError_t e, const char* what);
#define PSPEC_CUDA(call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return ::pspec::cuda_error(e_, #call); \
  } while (0)
#define PSPEC_TRY(call)                    \
  do {                                     \
    pspec_status s_ = (call);              \
    if (s_ != PSPEC_OK) return s_;         \
  } while (0)

// timing: wrap a launch
void timing_begin(pspec_graph* g, const char* name, cudaStream_t s, int* slot);
void timing_end(pspec_graph* g, int slot, cudaStream_t s);

struct TimedScope {
  pspec_graph* g;
  cudaStream_t s;
  int slot = -1;
  TimedScope(pspec_graph* g_, const char* name, cudaStream_t s_) : g(g_), s(s_) {
    if (g && g->timing.enabled) timing_begin(g, name, s, &slot);
  }
  ~TimedScope() {
    if (slot >= 0) timing_end(g, slot, s);
  }
};

// task sets and workspace
pspec_status ensure_tasks(pspec_graph* g, int Q);
// the contiguous cost-balanced split of ts for nwarps warps (*out = NULL when
// it cannot be uploaded now, e.g. during a stream capture)
pspec_status ensure_split(TaskSet& ts, int nwarps, cudaStream_t s, const int32_t** out);
void free_tasks(TaskSet& ts);
inline int q_index(int Q) { return Q == 1 ? 0 : Q == 2 ? 1 : 2; }
pspec_status ensure_io(pspec_graph* g, size_t bytes);
int grid_blocks(pspec_graph* g, int blocks_per_sm);
pspec_status check_block(const void* ptr, int k, pspec_dtype dtype, const char* name);
pspec_status check_common(pspec_graph* g, int k, double p);
pspec_status take_status(pspec_graph* g, cudaStream_t s);
pspec_status status_error(int status_word);  // the error a status word reports (OK if 0)

// launchers (FP32 fast path), implemented per k in edge_*.cu
struct EdgeLaunch {
  const float* U;
  const float* V;      // HVP only
  float* out_a;        // eval: Delta; HVP: sparse part S
  float* out_b;        // HVP: Delta (NULL: not stored)
  double p;
  int k;
  const int* skip = nullptr;  // device flag: when nonzero the launch does nothing
  float* task_part = nullptr; // batches: per-task column sums (see edge_kernels.cuh)
  bool alg1 = false;          // HVP: Algorithm 1's form (no rank-two terms)
  const double* keep_nd = nullptr;  // HVP at a kept point: its N[16], D[16]
  // batches: graphs whose flag is nonzero are left out (their outputs and
  // task sums are not written)
  const int* graph_skip = nullptr;
};
pspec_status edge_occupancy(int k, bool hvp, int* blocks_per_sm, bool kept = false);
pspec_status launch_eval_edges(pspec_graph* g, const EdgeLaunch& a, cudaStream_t s);
pspec_status launch_hvp_edges(pspec_graph* g, const EdgeLaunch& a, cudaStream_t s);

// FP64 plain path
pspec_status eval_plain64(pspec_graph* g, const double* U, int k, double p, double* F_out,
                          double* grad, double* parts, cudaStream_t s);
pspec_status hvp_plain64(pspec_graph* g, const double* U, const double* V, int k, double p,
                         double* HV, cudaStream_t s, bool alg1 = false);

// FP32 fast path, device pointers only
// keep_delta: Delta_p u of U into keep_rows (n x k) and N, D into keep_nd
// (32 doubles), by default the handle's own kept point; delta_kept: the
// Hessian product at a point kept that way (the same buffers)
pspec_status eval_fast(pspec_graph* g, const float* U, int k, double p, double* F_out,
                       float* grad, double* parts, cudaStream_t s, bool keep_delta = false,
                       float* keep_rows = nullptr, double* keep_nd = nullptr);
pspec_status hvp_fast(pspec_graph* g, const float* U, const float* V, int k, double p, float* HV,
                      cudaStream_t s, const int* skip = nullptr, bool alg1 = false,
                      bool delta_kept = false, const float* keep_rows = nullptr,
                      const double* keep_nd = nullptr);
// the edge kernel of a Hessian product at a kept point alone (sparse part into S)
pspec_status hvp_kept_edges(pspec_graph* g, const float* U, const float* V, int k, double p, float* S,
                            const double* keep_nd, cudaStream_t s, const int* skip = nullptr,
                            bool alg1 = false);
// the epilogues over the handle's n_owned rows: grad from the Delta rows Dl
// (in place when Dl == grad), HV over the sparse part S held in HV; the
// coefficients come from d_scalars
pspec_status run_grad_epilogue(pspec_graph* g, const float* U, const float* Dl, float* grad, int k, double p,
                               cudaStream_t s);
pspec_status run_hvp_epilogue(pspec_graph* g, const float* U, const float* V, const float* Dl, float* HV,
                              int k, double p, cudaStream_t s, const int* skip = nullptr);
pspec_status ensure_scratch(pspec_graph* g, size_t elems);
// the edge kernel of hvp_fast alone: S (sparse part) into S, Delta_p u into
// the handle's scratch block, the epilogue coefficients into d_scalars
pspec_status hvp_edges_fast(pspec_graph* g, const float* U, const float* V, int k, double p, float* S,
                            cudaStream_t s, const int* skip = nullptr, bool alg1 = false);

// batches: per-graph scalars, 128 doubles per graph in d_graph_scalars
constexpr int kGsN = 0, kGsD = 16, kGsC0 = 32, kGsC1 = 48, kGsC2 = 64, kGsC3 = 80, kGsC4 = 96,
              kGsF = 112, kGsStride = 128;
pspec_status eval_batched(pspec_graph* g, const float* U, int k, double p, double* F_out,
                          float* grad, double* parts, cudaStream_t s);
pspec_status hvp_batched(pspec_graph* g, const float* U, const float* V, int k, double p,
                         float* HV, cudaStream_t s, bool alg1 = false);
int64_t task_count(pspec_graph* g, int k);
pspec_status check_solve_args(const double* p_schedule, int n_p, const pspec_solve_opts* opts,
                              pspec_solve_opts* o);
pspec_status solve_on_handle(pspec_graph* g, int k, const double* p_schedule, int n_p,
                             const pspec_solve_opts& o, pspec_dtype dtype, void* U_inout,
                             int32_t* labels_out, double* rcut_out, pspec_solve_stats* stats,
                             cudaStream_t caller);

// scalar slots in d_scalars
constexpr int kSlotN = 0;      // [16]
constexpr int kSlotD = 16;     // [16]
constexpr int kSlotCN = 32;    // [16] sum_i Delta_i V_i
constexpr int kSlotCD = 48;    // [16] sum_i phi_p(u_i) V_i
constexpr int kSlotF = 64;     // [1]
constexpr int kSlotCoef = 80;  // [6*16] epilogue coefficients
constexpr int kSlotKeep = 256; // [32] N, D of the last PSPEC_KEEP_DELTA evaluation

}  // namespace pspec
