// Graph handle: validation and upload of W, the warp-task partition of the
// rows, workspace management, kernel-status and timing plumbing, and the
// error/version entry points of the C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "edge_kernels.cuh"
#include "internal.h"

namespace pspec {

static thread_local std::string g_last_error;

pspec_status set_error(pspec_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

pspec_status cuda_error(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return set_error(e == cudaErrorMemoryAllocation ? PSPEC_ERR_OOM : PSPEC_ERR_CUDA, m);
}

// ---------------------------------------------------------------- timing ---
void timing_begin(pspec_graph* g, const char* name, cudaStream_t s, int* slot) {
  Timing& t = g->timing;
  Timing::Pending p;
  p.name = name;
  auto get = [&]() {
    cudaEvent_t e;
    if (!t.pool.empty()) {
      e = t.pool.back();
      t.pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  };
  p.a = get();
  p.b = get();
  cudaEventRecord(p.a, s);
  t.pending.push_back(p);
  *slot = (int)t.pending.size() - 1;
}

void timing_end(pspec_graph* g, int slot, cudaStream_t s) {
  cudaEventRecord(g->timing.pending[slot].b, s);
}

static void timing_collect(pspec_graph* g) {
  Timing& t = g->timing;
  for (auto& p : t.pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    auto& tot = t.totals[p.name];
    tot.first += 1;
    tot.second += ms;
    t.pool.push_back(p.a);
    t.pool.push_back(p.b);
  }
  t.pending.clear();
}

// ------------------------------------------------------------ workspace ---
int grid_blocks(pspec_graph* g, int blocks_per_sm) {
  int b = g->sm_count * std::max(1, blocks_per_sm);
  return std::min(b, g->max_blocks);
}

pspec_status ensure_io(pspec_graph* g, size_t bytes) {
  if (g->h_pinned_bytes < bytes) {
    if (g->h_pinned) cudaFreeHost(g->h_pinned);
    g->h_pinned = nullptr;
    g->h_pinned_bytes = 0;
    PSPEC_CUDA(cudaMallocHost(&g->h_pinned, bytes));
    g->h_pinned_bytes = bytes;
  }
  if (g->d_io_bytes < bytes) {
    g->io_u_kept = false;
    if (g->d_io) cudaFree(g->d_io);
    g->d_io = nullptr;
    g->d_io_bytes = 0;
    PSPEC_CUDA(cudaMalloc(&g->d_io, bytes));
    g->d_io_bytes = bytes;
  }
  return PSPEC_OK;
}

static int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : dflt;
}

// Build the warp-task partition for column split Q (see TaskSet) over the
// degree-sorted rows.  A row of degree d gets E edge slots, the smallest power
// of two with d <= L*E (L = target edges per lane); a task takes up to
// 32/(E*Q) consecutive sorted rows of the same E.  Rows longer than
// hub_deg are split into chunks of chunk_edges entries.
void free_tasks(TaskSet& ts) {
  cudaFree(ts.d_tasks);
  cudaFree(ts.d_hub_row);
  cudaFree(ts.d_hub_first);
  cudaFree(ts.d_hub_nchunk);
  cudaFree(ts.d_hub_ticket);
  cudaFree(ts.d_chunk_hub);
  cudaFree(ts.d_task_graph);
  cudaFree(ts.d_graph_task);
  for (auto& sp : ts.splits) cudaFree(sp.second);
  ts = TaskSet();
}

pspec_status ensure_split(TaskSet& ts, int nwarps, cudaStream_t s, const int32_t** out) {
  *out = nullptr;
  for (const auto& sp : ts.splits)
    if (sp.first == nwarps) {
      *out = sp.second;
      return PSPEC_OK;
    }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  PSPEC_CUDA(cudaStreamIsCapturing(s, &cs));
  if (cs != cudaStreamCaptureStatusNone) return PSPEC_OK;  // no upload inside a capture
  // warp w starts at the first task whose cost prefix reaches w/nwarps of the total
  const std::vector<int64_t>& c = ts.h_cost;
  const int64_t total = c.back();
  std::vector<int32_t> wb(nwarps + 1);
  for (int w = 0; w <= nwarps; ++w) {
    const int64_t target = (int64_t)((__int128)total * w / nwarps);
    wb[w] = (int32_t)(std::lower_bound(c.begin(), c.end(), target) - c.begin());
  }
  wb[nwarps] = (int32_t)ts.n_tasks;
  int32_t* d = nullptr;
  PSPEC_CUDA(cudaMalloc(&d, sizeof(int32_t) * (nwarps + 1)));
  ts.splits.emplace_back(nwarps, d);
  PSPEC_CUDA(cudaMemcpy(d, wb.data(), sizeof(int32_t) * (nwarps + 1), cudaMemcpyHostToDevice));
  PSPEC_CUDA(cudaStreamSynchronize(cudaStreamLegacy));  // uploaded before any stream's kernel reads it
  *out = d;
  return PSPEC_OK;
}

pspec_status ensure_tasks(pspec_graph* g, int Q) {
  int qi = Q == 1 ? 0 : Q == 2 ? 1 : 2;
  TaskSet& ts = g->tasks[qi];
  if (ts.built) return PSPEC_OK;
  // at most L entries per lane and row before the row gets more edge slots;
  // hub chunks give each lane that many entries.  L is the handle's (set by
  // pspec_tune), else PSPEC_EDGES_PER_LANE, else 16 Q: the largest of the
  // tuner's candidates, which it chose (or came within 4 % of) on the grid,
  // kNN, degree-corrected SBM and batch workloads.  Its tasks (32 L / Q
  // entries) are too long for the staged kernel, so the direct kernel runs;
  // 8 entries per lane would pick the staged kernel, 1.3x to 1.9x slower there.
  const int L = std::max(1, g->edges_per_lane[qi] > 0 ? g->edges_per_lane[qi]
                                                      : env_int("PSPEC_EDGES_PER_LANE", 16 * Q));
  const int max_slots = 32 / Q;
  int max_elog = 0;
  while ((1 << max_elog) < max_slots) ++max_elog;
  const int64_t hub_deg = (int64_t)L * max_slots;
  const int chunk = L * max_slots;
  const std::vector<int64_t>& rp = g->h_rowptr_s;
  const int64_t n = g->n_owned;  // a shard's halo rows (sorted last) get no tasks
  std::vector<int4> tasks;
  tasks.reserve((size_t)(n / 8 + 16));
  // a task's cost ~ the entries one lane walks plus a fixed part (descriptor,
  // vertex terms, sums, stores), in entry units
  constexpr int64_t kTaskCostFixed = 4;
  std::vector<int64_t> cost(1, 0);
  std::vector<int32_t> hub_row, hub_first, hub_nchunk, chunk_hub;
  int n_chunks = 0;
  auto elog_of = [&](int64_t d) {
    int e = 0;
    while (e < max_elog && d > (int64_t)L * (1 << e)) ++e;
    return e;
  };
  // plain task: x = first sorted row, y = nrows | degree << 8 (all rows of a
  // task have exactly this degree), z = elog, w = first entry of the task.
  // Rows are sorted within each graph of a batch, and no task crosses a graph.
  std::vector<int64_t> bounds = g->h_node_off;
  if (bounds.empty()) bounds = {0, n};
  std::vector<int32_t> task_graph;
  std::vector<int32_t> graph_task(bounds.size(), 0);  // first task of each graph
  size_t gi = 0;
  int64_t r = 0;
  while (r < n) {
    while (bounds[gi + 1] <= r) {
      ++gi;
      graph_task[gi] = (int32_t)tasks.size();
    }
    const int64_t gend = bounds[gi + 1];
    const int64_t deg = rp[r + 1] - rp[r];
    if (deg > hub_deg) {
      int nch = (int)((deg + chunk - 1) / chunk);
      hub_row.push_back((int32_t)r);
      hub_first.push_back(n_chunks);
      hub_nchunk.push_back(nch);
      // hub chunk: x = sorted row, y = chunk slot, z = elog | hub | first | len << 10,
      // w = first entry of the chunk
      for (int c = 0; c < nch; ++c) {
        const int64_t len = std::min<int64_t>(chunk, deg - (int64_t)c * chunk);
        tasks.push_back(make_int4((int)r, n_chunks + c,
                                  max_elog | (1 << 8) | ((c == 0 ? 1 : 0) << 9) | (int)(len << 10),
                                  (int)(rp[r] + (int64_t)c * chunk)));
        cost.push_back(cost.back() + (len + max_slots - 1) / max_slots + kTaskCostFixed);
        task_graph.push_back((int32_t)gi);
        chunk_hub.push_back((int32_t)hub_row.size() - 1);
      }
      n_chunks += nch;
      ++r;
      continue;
    }
    const int elog = elog_of(deg);
    const int R = 32 / ((1 << elog) * Q);
    int nrows = 0;
    while (nrows < R && r + nrows < gend && rp[r + nrows + 1] - rp[r + nrows] == deg) ++nrows;
    tasks.push_back(make_int4((int)r, nrows | (int)(deg << 8), elog, (int)rp[r]));
    cost.push_back(cost.back() + (deg + (1 << elog) - 1) / (1 << elog) + kTaskCostFixed);
    task_graph.push_back((int32_t)gi);
    r += nrows;
  }
  for (size_t q = gi + 1; q < graph_task.size(); ++q) graph_task[q] = (int32_t)tasks.size();
  ts.Q = Q;
  ts.L = L;
  ts.h_cost = std::move(cost);
  ts.chunk_edges = chunk;
  ts.n_tasks = (int64_t)tasks.size();
  ts.n_hubs = (int)hub_row.size();
  ts.n_chunks = n_chunks;
  PSPEC_CUDA(cudaMalloc(&ts.d_tasks, sizeof(int4) * std::max<size_t>(1, tasks.size())));
  PSPEC_CUDA(cudaMemcpy(ts.d_tasks, tasks.data(), sizeof(int4) * tasks.size(), cudaMemcpyHostToDevice));
  if (!g->h_node_off.empty()) {  // a batched handle, even of one graph
    PSPEC_CUDA(cudaMalloc(&ts.d_task_graph, sizeof(int32_t) * std::max<size_t>(1, task_graph.size())));
    PSPEC_CUDA(cudaMemcpy(ts.d_task_graph, task_graph.data(), sizeof(int32_t) * task_graph.size(),
                          cudaMemcpyHostToDevice));
    PSPEC_CUDA(cudaMalloc(&ts.d_graph_task, sizeof(int32_t) * graph_task.size()));
    PSPEC_CUDA(cudaMemcpy(ts.d_graph_task, graph_task.data(), sizeof(int32_t) * graph_task.size(),
                          cudaMemcpyHostToDevice));
  }
  if (ts.n_hubs > 0) {
    PSPEC_CUDA(cudaMalloc(&ts.d_hub_row, sizeof(int32_t) * ts.n_hubs));
    PSPEC_CUDA(cudaMalloc(&ts.d_hub_first, sizeof(int32_t) * ts.n_hubs));
    PSPEC_CUDA(cudaMalloc(&ts.d_hub_nchunk, sizeof(int32_t) * ts.n_hubs));
    PSPEC_CUDA(cudaMalloc(&ts.d_hub_ticket, sizeof(unsigned) * ts.n_hubs));
    PSPEC_CUDA(cudaMalloc(&ts.d_chunk_hub, sizeof(int32_t) * n_chunks));
    PSPEC_CUDA(cudaMemcpy(ts.d_hub_row, hub_row.data(), sizeof(int32_t) * ts.n_hubs, cudaMemcpyHostToDevice));
    PSPEC_CUDA(cudaMemcpy(ts.d_hub_first, hub_first.data(), sizeof(int32_t) * ts.n_hubs, cudaMemcpyHostToDevice));
    PSPEC_CUDA(cudaMemcpy(ts.d_hub_nchunk, hub_nchunk.data(), sizeof(int32_t) * ts.n_hubs, cudaMemcpyHostToDevice));
    PSPEC_CUDA(cudaMemcpy(ts.d_chunk_hub, chunk_hub.data(), sizeof(int32_t) * n_chunks, cudaMemcpyHostToDevice));
    PSPEC_CUDA(cudaMemset(ts.d_hub_ticket, 0, sizeof(unsigned) * ts.n_hubs));
    size_t need = (size_t)n_chunks * 2 * kMaxK;
    if (g->hub_part_elems < need) {
      if (g->d_hub_part) cudaFree(g->d_hub_part);
      g->d_hub_part = nullptr;
      PSPEC_CUDA(cudaMalloc(&g->d_hub_part, sizeof(float) * need));
      g->hub_part_elems = need;
    }
  }
  // The uploads above are ordered on the legacy default stream and a
  // cudaMemcpy from pageable memory (or a cudaMemset) may return before the
  // device holds the data; the kernels that read the task set run on other,
  // possibly non-blocking, streams.  Wait for them here.
  PSPEC_CUDA(cudaStreamSynchronize(cudaStreamLegacy));
  ts.built = true;
  return PSPEC_OK;
}

int64_t task_count(pspec_graph* g, int k) {
  const int Q = q_of(k);
  if (ensure_tasks(g, Q) != PSPEC_OK) return -1;
  return g->tasks[Q == 1 ? 0 : Q == 2 ? 1 : 2].n_tasks;
}

pspec_status check_block(const void* ptr, int k, pspec_dtype dtype, const char* name) {
  if (!ptr) return set_error(PSPEC_ERR_INVALID_ARG, std::string(name) + " is NULL");
  uintptr_t a = (uintptr_t)ptr;
  size_t need = dtype == PSPEC_F64 ? 8 : (k % 4 == 0 ? 16 : (k % 2 == 0 ? 8 : 4));
  if (a % need != 0)
    return set_error(PSPEC_ERR_INVALID_ARG, std::string(name) + " is not " + std::to_string(need) +
                                                "-byte aligned");
  return PSPEC_OK;
}

pspec_status check_common(pspec_graph* g, int k, double p) {
  if (!g) return set_error(PSPEC_ERR_INVALID_ARG, "graph is NULL");
  if (k < 1 || k > kMaxK) return set_error(PSPEC_ERR_INVALID_ARG, "k must be in [1, 16]");
  if (!(p > 1.0 && p <= 2.0)) return set_error(PSPEC_ERR_INVALID_ARG, "p must be in (1, 2]");
  return PSPEC_OK;
}

pspec_status take_status(pspec_graph* g, cudaStream_t s) {
  int st = 0;
  PSPEC_CUDA(cudaMemcpyAsync(&st, g->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaStreamSynchronize(s));
  if (st != 0) PSPEC_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(int), s));
  return status_error(st);
}

pspec_status status_error(int st) {
  if (st & kStatusNonFinite) return set_error(PSPEC_ERR_NONFINITE, "a NaN or Inf reached a sum");
  if (st & kStatusZeroColumn) return set_error(PSPEC_ERR_ZERO_COLUMN, "a column has zero p-norm");
  if (st & kStatusTimeout) return set_error(PSPEC_ERR_TIMEOUT, "a bounded device wait gave up");
  return PSPEC_OK;
}

// ---------------------------------------------------------------- create ---
template <typename T>
static bool weights_ok(const T* v, int64_t nnz, std::string* why) {
  for (int64_t e = 0; e < nnz; ++e) {
    double x = (double)v[e];
    if (!std::isfinite(x) || x < 0.0) {
      *why = "weight " + std::to_string(e) + " is negative or not finite";
      return false;
    }
  }
  return true;
}

static pspec_status create_impl(int64_t n, const int64_t* rowptr_in, const int32_t* col_in,
                                const void* val_in, pspec_dtype vt, unsigned flags, cudaStream_t s,
                                const std::vector<int64_t>& node_off, pspec_graph** out,
                                int64_t n_owned = -1) {
  if (!out) return set_error(PSPEC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n >= (int64_t)1 << 31) return set_error(PSPEC_ERR_INVALID_ARG, "n must be in [1, 2^31)");
  if (!rowptr_in || !col_in || !val_in) return set_error(PSPEC_ERR_INVALID_ARG, "NULL CSR array");
  if (vt != PSPEC_F32 && vt != PSPEC_F64) return set_error(PSPEC_ERR_INVALID_ARG, "bad val dtype");
  const bool host = (flags & PSPEC_HOST_PTRS) != 0;
  // stage everything on the host (validation and task building need it)
  std::vector<int64_t> rp(n + 1);
  if (host) {
    std::memcpy(rp.data(), rowptr_in, sizeof(int64_t) * (n + 1));
  } else {
    // the caller's work on `s` (which may have produced the arrays) first:
    // the copies below run on the legacy stream
    PSPEC_CUDA(cudaStreamSynchronize(s));
    PSPEC_CUDA(cudaMemcpy(rp.data(), rowptr_in, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
  }
  if (rp[0] != 0) return set_error(PSPEC_ERR_INVALID_ARG, "rowptr[0] must be 0");
  const bool shard = n_owned >= 0;
  if (!shard) n_owned = n;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return set_error(PSPEC_ERR_INVALID_ARG, "rowptr decreases at row " + std::to_string(i));
  const int64_t nnz = rp[n];
  if (nnz >= ((int64_t)1 << 31)) return set_error(PSPEC_ERR_INVALID_ARG, "nnz must be < 2^31");
  std::vector<int32_t> col(nnz);
  std::vector<float> v32(nnz);
  std::vector<double> v64(nnz);
  const size_t vbytes = (vt == PSPEC_F32 ? 4 : 8) * (size_t)nnz;
  std::vector<char> vraw(vbytes);
  if (host) {
    if (nnz) std::memcpy(col.data(), col_in, sizeof(int32_t) * nnz);
    if (nnz) std::memcpy(vraw.data(), val_in, vbytes);
  } else if (nnz) {
    PSPEC_CUDA(cudaMemcpy(col.data(), col_in, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost));
    PSPEC_CUDA(cudaMemcpy(vraw.data(), val_in, vbytes, cudaMemcpyDeviceToHost));
  }
  std::string why;
  if (vt == PSPEC_F32) {
    const float* f = reinterpret_cast<const float*>(vraw.data());
    if (!weights_ok(f, nnz, &why)) return set_error(PSPEC_ERR_INVALID_ARG, why);
    for (int64_t e = 0; e < nnz; ++e) { v32[e] = f[e]; v64[e] = (double)f[e]; }
  } else {
    const double* d = reinterpret_cast<const double*>(vraw.data());
    if (!weights_ok(d, nnz, &why)) return set_error(PSPEC_ERR_INVALID_ARG, why);
    for (int64_t e = 0; e < nnz; ++e) { v64[e] = d[e]; v32[e] = (float)d[e]; }
  }
  std::vector<int64_t> bounds = node_off;
  if (bounds.empty()) bounds = {0, n};
  {
    size_t gi = 0;
    for (int64_t i = 0; i < n; ++i) {
      while (bounds[gi + 1] <= i) ++gi;
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        int32_t c = col[e];
        if (c < 0 || c >= n)
          return set_error(PSPEC_ERR_INVALID_ARG, "col out of range at entry " + std::to_string(e));
        if (c < bounds[gi] || c >= bounds[gi + 1])
          return set_error(PSPEC_ERR_INVALID_ARG, "entry " + std::to_string(e) + " crosses graphs");
      }
    }
  }
  if (flags & PSPEC_CHECK_SYMMETRY) {
    std::vector<std::tuple<int32_t, int32_t, double>> a, b;
    a.reserve(nnz);
    b.reserve(nnz);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
        a.emplace_back((int32_t)i, col[e], v64[e]);
        b.emplace_back(col[e], (int32_t)i, v64[e]);
      }
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) return set_error(PSPEC_ERR_INVALID_ARG, "W is not symmetric");
  }

  pspec_graph* g = new pspec_graph();
  auto fail = [&](pspec_status st) {
    pspec_graph_destroy(g);
    return st;
  };
  cudaGetDevice(&g->device);
  cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
  g->n = n;
  g->n_owned = n_owned;
  g->is_shard = shard;
  g->nnz = nnz;
  g->h_rowptr = std::move(rp);
  g->h_node_off = node_off;
  g->n_graphs = node_off.empty() ? 1 : (int32_t)node_off.size() - 1;
  g->max_blocks = g->sm_count * 8;
  const int max_groups = (g->max_blocks + kGroup - 1) / kGroup;
  pspec_status st;
#define ALLOC(ptr, bytes)                                  \
  st = [&]() { PSPEC_CUDA(cudaMalloc(&(ptr), (bytes))); return PSPEC_OK; }(); \
  if (st != PSPEC_OK) return fail(st);
  ALLOC(g->d_rowptr, sizeof(int64_t) * (n + 1));
  ALLOC(g->d_col, sizeof(int32_t) * std::max<int64_t>(1, nnz));
  ALLOC(g->d_val32, sizeof(float) * std::max<int64_t>(1, nnz));
  ALLOC(g->d_val64, sizeof(double) * std::max<int64_t>(1, nnz));
  ALLOC(g->d_block_part, sizeof(float2) * g->max_blocks * 64);
  ALLOC(g->d_group_part, sizeof(float2) * max_groups * 64);
  ALLOC(g->d_counters, sizeof(unsigned) * (max_groups + 8));
  ALLOC(g->d_scalars, sizeof(double) * 1024);
  ALLOC(g->d_red64, sizeof(double) * (g->max_blocks + max_groups) * 64);
  ALLOC(g->d_status, sizeof(int));
  if (!node_off.empty()) ALLOC(g->d_node_off, sizeof(int64_t) * node_off.size());
#undef ALLOC
  auto copy = [&](void* dst, const void* src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? PSPEC_OK : cuda_error(e, "cudaMemcpyAsync(graph)");
  };
  if ((st = copy(g->d_rowptr, g->h_rowptr.data(), sizeof(int64_t) * (n + 1))) != PSPEC_OK) return fail(st);
  if (nnz) {
    if ((st = copy(g->d_col, col.data(), sizeof(int32_t) * nnz)) != PSPEC_OK) return fail(st);
    if ((st = copy(g->d_val32, v32.data(), sizeof(float) * nnz)) != PSPEC_OK) return fail(st);
    if ((st = copy(g->d_val64, v64.data(), sizeof(double) * nnz)) != PSPEC_OK) return fail(st);
  }
  if (!node_off.empty()) {
    if ((st = copy(g->d_node_off, node_off.data(), sizeof(int64_t) * node_off.size())) != PSPEC_OK)
      return fail(st);
    std::vector<int32_t> rg(n);
    for (size_t q = 0; q + 1 < node_off.size(); ++q)
      for (int64_t i = node_off[q]; i < node_off[q + 1]; ++i) rg[i] = (int32_t)q;
    cudaError_t e1 = cudaMalloc(&g->d_row_graph, sizeof(int32_t) * n);
    if (e1 != cudaSuccess) return fail(cuda_error(e1, "cudaMalloc(row_graph)"));
    e1 = cudaMalloc(&g->d_graph_scalars, sizeof(double) * 128 * (node_off.size() - 1));
    if (e1 != cudaSuccess) return fail(cuda_error(e1, "cudaMalloc(graph_scalars)"));
    if ((st = copy(g->d_row_graph, rg.data(), sizeof(int32_t) * n)) != PSPEC_OK) return fail(st);
    cudaError_t e2 = cudaStreamSynchronize(s);
    if (e2 != cudaSuccess) return fail(cuda_error(e2, "row_graph upload"));
  }
  // rows stably sorted by degree: the fast kernels' layout
  {
    std::vector<int32_t> perm(n);
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    const std::vector<int64_t>& rp0 = g->h_rowptr;
    // rows of each graph of a batch stay within the graph's range
    std::vector<int64_t> gb = node_off;
    if (gb.empty()) gb = {0, n};
    // (a shard's halo vertices, rows without entries, go after every owned
    // row, so the owned rows are the first n_owned sorted rows)
    for (size_t q = 0; q + 1 < gb.size(); ++q)
      std::stable_sort(perm.begin() + gb[q], perm.begin() + gb[q + 1], [&](int32_t a, int32_t b) {
        const bool ha = a >= n_owned, hb = b >= n_owned;
        if (ha != hb) return hb;
        return rp0[a + 1] - rp0[a] < rp0[b + 1] - rp0[b];
      });
    std::vector<int64_t> rps(n + 1, 0);
    for (int64_t r = 0; r < n; ++r) rps[r + 1] = rps[r] + (rp0[perm[r] + 1] - rp0[perm[r]]);
    // {column, log2 of the FP32 weight rounded to FP32}: the kernels form
    // w |d|^(p-2) as one power of two (a zero weight gives -inf, hence 0)
    std::vector<int2> cw(nnz);
    for (int64_t r = 0; r < n; ++r) {
      const int64_t src = rp0[perm[r]], len = rps[r + 1] - rps[r];
      for (int64_t q = 0; q < len; ++q) {
        const float lw = (float)std::log2((double)v32[src + q]);
        int bits;
        std::memcpy(&bits, &lw, sizeof(bits));
        cw[rps[r] + q] = make_int2(col[src + q], bits);
      }
    }
    auto alloc = [&](void** p, size_t bytes) {
      cudaError_t e = cudaMalloc(p, bytes);
      return e == cudaSuccess ? PSPEC_OK : cuda_error(e, "cudaMalloc(sorted CSR)");
    };
    if ((st = alloc((void**)&g->d_cw_s, sizeof(int2) * (nnz + 16))) != PSPEC_OK) return fail(st);
    if ((st = alloc((void**)&g->d_perm, sizeof(int32_t) * (n + 16))) != PSPEC_OK) return fail(st);
    if ((st = copy(g->d_perm, perm.data(), sizeof(int32_t) * n)) != PSPEC_OK) return fail(st);
    if (nnz)
      if ((st = copy(g->d_cw_s, cw.data(), sizeof(int2) * nnz)) != PSPEC_OK) return fail(st);
    cudaError_t e2 = cudaStreamSynchronize(s);  // the host vectors go out of scope
    if (e2 != cudaSuccess) return fail(cuda_error(e2, "sorted CSR upload"));
    g->h_rowptr_s = std::move(rps);
    g->h_perm = std::move(perm);
  }
  cudaMemsetAsync(g->d_counters, 0, sizeof(unsigned) * (max_groups + 8), s);
  cudaMemsetAsync(g->d_status, 0, sizeof(int), s);
  cudaMemsetAsync(g->d_scalars, 0, sizeof(double) * 1024, s);
  cudaError_t e = cudaStreamSynchronize(s);  // host buffers above are about to go away
  if (e != cudaSuccess) return fail(cuda_error(e, "graph upload"));
  *out = g;
  return PSPEC_OK;
}

}  // namespace pspec

using namespace pspec;

extern "C" {

pspec_status pspec_graph_create(int64_t n, const int64_t* rowptr, const int32_t* col,
                                const void* val, pspec_dtype val_dtype, unsigned flags,
                                void* stream, pspec_graph** out) {
  return create_impl(n, rowptr, col, val, val_dtype, flags, (cudaStream_t)stream, {}, out);
}

pspec_status pspec_graph_create_batched(int32_t n_graphs, const int64_t* node_off,
                                        const int64_t* rowptr, const int32_t* col,
                                        const void* val, pspec_dtype val_dtype, unsigned flags,
                                        void* stream, pspec_graph** out) {
  if (out) *out = nullptr;
  if (n_graphs < 1 || !node_off) return set_error(PSPEC_ERR_INVALID_ARG, "bad graph count or node_off");
  std::vector<int64_t> off(node_off, node_off + n_graphs + 1);
  if (off[0] != 0) return set_error(PSPEC_ERR_INVALID_ARG, "node_off[0] must be 0");
  for (int32_t i = 0; i < n_graphs; ++i)
    if (off[i + 1] <= off[i]) return set_error(PSPEC_ERR_INVALID_ARG, "empty or decreasing graph");
  return create_impl(off[n_graphs], rowptr, col, val, val_dtype, flags, (cudaStream_t)stream, off, out);
}

pspec_status pspec_graph_create_shard(int64_t n_owned, int64_t n_local, const int64_t* rowptr,
                                      const int32_t* col, const void* val, pspec_dtype val_dtype,
                                      unsigned flags, void* stream, pspec_graph** out) {
  if (out) *out = nullptr;
  if (!(flags & PSPEC_HOST_PTRS))
    return set_error(PSPEC_ERR_INVALID_ARG, "pspec_graph_create_shard takes host arrays (PSPEC_HOST_PTRS)");
  if (n_owned < 1 || n_local < n_owned) return set_error(PSPEC_ERR_INVALID_ARG, "need 1 <= n_owned <= n_local");
  if (!rowptr) return set_error(PSPEC_ERR_INVALID_ARG, "rowptr is NULL");
  // the halo rows carry no entries: extend the row offsets over them
  std::vector<int64_t> rp(rowptr, rowptr + n_owned + 1);
  rp.resize(n_local + 1, rp[n_owned]);
  return create_impl(n_local, rp.data(), col, val, val_dtype, flags, (cudaStream_t)stream, {}, out, n_owned);
}

void pspec_graph_destroy(pspec_graph* g) {
  if (!g) return;
  for (pspec_graph* sub : g->subs) pspec_graph_destroy(sub);
  g->subs.clear();
  for (auto& ts : g->tasks) {
    free_tasks(ts);
  }
  cudaFree(g->d_rowptr);
  cudaFree(g->d_col);
  cudaFree(g->d_cw_s);
  cudaFree(g->d_perm);
  cudaFree(g->d_val32);
  cudaFree(g->d_val64);
  cudaFree(g->d_node_off);
  cudaFree(g->d_row_graph);
  cudaFree(g->d_graph_scalars);
  cudaFree(g->d_task_part);
  cudaFree(g->d_scratch);
  cudaFree(g->d_delta_keep);
  cudaFree(g->d_hub_part);
  if (g->solve_stream) cudaStreamDestroy(g->solve_stream);
  if (g->h_solve_rec) cudaFreeHost(g->h_solve_rec);
  if (g->solve_event) cudaEventDestroy(g->solve_event);
  cudaFree(g->d_block_part);
  cudaFree(g->d_group_part);
  cudaFree(g->d_counters);
  cudaFree(g->d_scalars);
  cudaFree(g->d_red64);
  cudaFree(g->d_status);
  cudaFree(g->d_io);
  cudaFree(g->d_solve);
  if (g->h_pinned) cudaFreeHost(g->h_pinned);
  for (auto& p : g->timing.pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : g->timing.pool) cudaEventDestroy(e);
  delete g;
}

pspec_status pspec_graph_info(const pspec_graph* g, int64_t* n, int64_t* nnz, int32_t* n_graphs) {
  if (!g) return set_error(PSPEC_ERR_INVALID_ARG, "graph is NULL");
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (n_graphs) *n_graphs = g->n_graphs;
  return PSPEC_OK;
}

pspec_status pspec_graph_status(pspec_graph* g, void* stream) {
  if (!g) return set_error(PSPEC_ERR_INVALID_ARG, "graph is NULL");
  return take_status(g, (cudaStream_t)stream);
}

pspec_status pspec_set_timing(pspec_graph* g, int enable) {
  if (!g) return set_error(PSPEC_ERR_INVALID_ARG, "graph is NULL");
  g->timing.enabled = enable != 0;
  if (!enable) {
    timing_collect(g);
    g->timing.totals.clear();
  }
  return PSPEC_OK;
}

pspec_status pspec_kernel_times(pspec_graph* g, char* buf, size_t buf_len) {
  if (!g || !buf || buf_len == 0) return set_error(PSPEC_ERR_INVALID_ARG, "bad arguments");
  timing_collect(g);
  std::string s;
  char tmp[256];
  for (auto& kv : g->timing.totals) {
    std::snprintf(tmp, sizeof(tmp), "%s=%lld:%.6f;", kv.first.c_str(), kv.second.first, kv.second.second);
    s += tmp;
  }
  std::snprintf(buf, buf_len, "%s", s.c_str());
  g->timing.totals.clear();
  return s.size() < buf_len ? PSPEC_OK : set_error(PSPEC_ERR_INVALID_ARG, "buffer too small");
}

const char* pspec_last_error(void) { return g_last_error.c_str(); }

const char* pspec_version(void) { return "0.1.0 sm_103a"; }

}  // extern "C"
