// pspec_solve: the paper's solve (Section 2) -- F_p minimised on the
// Grassmann manifold by Newton's method with truncated-CG subproblems, with p
// lowered stage by stage from 2 toward 1 -- followed by k-means and RCut.
//
// Reading taken (the paper delegates these to ROPTLIB and prints no detail;
// the CPU oracle follows the same reading): the Riemannian trust-region
// Newton method of Absil, Baker & Gallivan with Steihaug-Toint truncated CG
// (no preconditioner, recurrences for <eta,delta> and <delta,delta>), the
// tangent projection P_U(G) = G - U U^T G, the Riemannian Hessian
// P_U(H eta) - eta U^T grad F, the retraction qf(U + eta) computed as
// Cholesky-QR twice, the radius update with the 1/4 and 3/4 rules, acceptance
// when the model decreased and rho > rho_prime, and rho regularised by
// rho_reg * max(1, |f|).
//
// Device / host split: every n x k operation is a kernel; the CG scalar
// recurrences run in the last block of the reduction kernels, so truncated CG
// proceeds on the device in chunks of iterations and the host reads one small
// state record per chunk (the kernels of iterations enqueued after CG stopped
// return immediately).  The host does the per-Newton-step trust-region
// arithmetic on a handful of FP64 scalars.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "solve_kernels.cuh"

namespace pspec {

namespace {

template <typename T>
struct SolveWork {
  // (H eta is not kept: it is r - rg when truncated CG stops)
  T *U, *Unew, *egrad, *egrad_new, *rg, *rg_new, *eta, *r, *delta, *He, *Hd, *tmp;
  // Delta_p u and N, D of the iterate and of the trial point (FP32: the
  // Hessian products of truncated CG reuse the iterate's; they swap with it)
  T *dk, *dk_new;
  double *nd, *nd_new;
  double *M, *Mnew, *G, *Gram, *Rinv, *dots, *gdot, *F;
  TcgState* st;
  int* bad;
  GridRed gr;
  int vblocks, gblocks, rblocks, tblocks;  // elementwise, Gram, row kernels, TMA Gram
};

template <typename T>
pspec_status carve(pspec_graph* g, int k, SolveWork<T>* w) {
  const size_t m = (size_t)g->n * k;
  const size_t vec = ((sizeof(T) * m + 255) / 256) * 256;
  w->vblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * 4, ((int64_t)m + kSolveBlock - 1) / kSolveBlock));
  w->gblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * 8,
                                                           (g->n + kGramTile - 1) / kGramTile));
  w->rblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * 4,
                                                           (g->n + kSolveBlock - 1) / kSolveBlock));
  w->tblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)g->sm_count * 3,
                                                           (g->n + kGramTile - 1) / kGramTile));
  const int maxb = std::max(w->vblocks, w->gblocks);
  const int groups = (maxb + kGroup - 1) / kGroup;
  const size_t red = sizeof(double) * 256 * (size_t)(maxb + groups);
  const size_t small = 4096 * sizeof(double);
  const size_t need = 14 * vec + 2 * red + small;
  if (g->d_solve_bytes < need) {
    if (g->d_solve) cudaFree(g->d_solve);
    g->d_solve = nullptr;
    g->d_solve_bytes = 0;
    PSPEC_CUDA(cudaMalloc(&g->d_solve, need));
    g->d_solve_bytes = need;
  }
  char* p = (char*)g->d_solve;
  T** vecs[14] = {&w->U, &w->Unew, &w->egrad, &w->egrad_new, &w->rg, &w->rg_new, &w->eta,
                  &w->r, &w->delta, &w->He, &w->Hd, &w->tmp, &w->dk, &w->dk_new};
  for (auto v : vecs) {
    *v = (T*)p;
    p += vec;
  }
  w->gr.block_part = p;
  w->gr.group_part = p + sizeof(double) * 256 * (size_t)maxb;
  p += 2 * red;
  double* sm = (double*)p;
  w->M = sm;
  w->G = sm + 256;
  w->Gram = sm + 512;
  w->Rinv = sm + 768;
  w->dots = sm + 1024;
  w->F = sm + 1040;
  w->st = (TcgState*)(sm + 1056);
  w->bad = (int*)(sm + 1100);
  w->Mnew = sm + 1280;
  w->gdot = sm + 1536;
  w->nd = sm + 1600;
  w->nd_new = sm + 1664;
  w->gr.counters = g->d_counters;
  return PSPEC_OK;
}

// CUDA graphs of a chunk of CG iterations, one per (iterate buffer, p): the
// solve alternates between two iterate buffers, so a stage needs at most two.
struct GraphCache {
  bool enabled = true;
  struct Entry {
    const void* U;
    double p;
    cudaGraphExec_t exec;
  };
  std::vector<Entry> entries;
  template <typename F>
  pspec_status get(const void* U, double p, cudaStream_t s, F&& body, cudaGraphExec_t* out) {
    for (const Entry& e : entries)
      if (e.U == U && e.p == p) {
        *out = e.exec;
        return PSPEC_OK;
      }
    PSPEC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    pspec_status st = body();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (st != PSPEC_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture(tCG chunk)");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate(tCG chunk)");
    entries.push_back({U, p, exec});
    *out = exec;
    return PSPEC_OK;
  }
  ~GraphCache() {
    for (const Entry& e : entries) cudaGraphExecDestroy(e.exec);
  }
};

template <typename T>
struct Solver {
  pspec_graph* g;
  int k;
  int64_t n, m;
  cudaStream_t s;
  SolveWork<T> w;
  int64_t evals = 0, hvps = 0;

  // F and the gradient at U; the FP32 path also keeps U's Delta_p u, N, D
  // in (dk, nd) for the Hessian products at U
  pspec_status eval(const T* U, double p, T* grad, T* dk, double* nd) {
    ++evals;
    if constexpr (sizeof(T) == 4)
      return eval_fast(g, U, k, p, w.F, grad, nullptr, s, true, dk, nd);
    else
      return eval_plain64(g, U, k, p, w.F, grad, nullptr, s);
  }
  bool alg1 = false;  // Algorithm 1's Hessian form instead of the exact one
  // the Hessian product at the iterate U (whose Delta_p u, N, D are w.dk, w.nd)
  pspec_status hvp(const T* U, const T* V, double p, T* out, const int* skip) {
    if constexpr (sizeof(T) == 4)
      return hvp_fast(g, U, V, k, p, out, s, skip, alg1, true, w.dk, w.nd);
    else
      return hvp_plain64(g, U, V, k, p, out, s, alg1);
  }
  // Hv = H[V] and Gm = U^T Hv: for FP32 with k a multiple of 4 the epilogue
  // and the Gram product run as one kernel (same bits as the two calls)
  pspec_status hvp_gram(const T* U, const T* V, double p, T* Hv, double* Gm, const int* done) {
    if constexpr (sizeof(T) == 4) {
      if (k % 4 == 0) {
        PSPEC_TRY(hvp_kept_edges(g, U, V, k, p, Hv, w.nd, s, done, alg1));
        TimedScope timer(g, "hvp_epi_gram", s);
        hvp_epi_gram_kernel<<<w.tblocks, kSolveBlock, 0, s>>>(U, V, w.dk, Hv, n, k, g->d_scalars,
                                                              (float)p - 2.0f, Gm, w.gr, done);
        PSPEC_CUDA(cudaGetLastError());
        return PSPEC_OK;
      }
    }
    PSPEC_TRY(hvp(U, V, p, Hv, done));
    return gram(U, Hv, Gm, done);
  }
  pspec_status gram(const T* A, const T* B, double* G, const int* done = nullptr) {
    TimedScope timer(g, "solve_gram", s);
    if constexpr (sizeof(T) == 4) {
      if (k % 4 != 0) {
        gram_kernel<T><<<w.gblocks, kSolveBlock, 0, s>>>(A, B, n, k, G, w.gr, done);
        PSPEC_CUDA(cudaGetLastError());
        return PSPEC_OK;
      }
      // once per process, thread-safe (batched solves run on several host threads)
      static const cudaError_t attr = cudaFuncSetAttribute(
          gram_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tma_smem_bytes());
      PSPEC_CUDA(attr);
      gram_tma_kernel<<<w.tblocks, kSolveBlock, gram_tma_smem_bytes(), s>>>(A, B, n, k, G, w.gr, done,
                                                                             g->d_status);
    } else {
      gram_kernel<T><<<w.gblocks, kSolveBlock, 0, s>>>(A, B, n, k, G, w.gr, done);
    }
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  pspec_status dots(DotPairs<T> dp, double* out) {
    TimedScope timer(g, "solve_dots", s);
    dots_kernel<T><<<w.vblocks, kSolveBlock, 0, s>>>(dp, m, out, w.gr, nullptr);
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  pspec_status combine(T* out, const T* X, double a, const T* Y, double b, const T* P,
                       const double* M1, const T* Q, const double* M2) {
    TimedScope timer(g, "solve_combine", s);
    switch (k_bucket(k)) {
      case 4: combine_kernel<T, 4><<<w.rblocks, kSolveBlock, 0, s>>>(out, X, a, Y, b, P, M1, Q, M2, n, k, nullptr); break;
      case 8: combine_kernel<T, 8><<<w.rblocks, kSolveBlock, 0, s>>>(out, X, a, Y, b, P, M1, Q, M2, n, k, nullptr); break;
      default: combine_kernel<T, 16><<<w.rblocks, kSolveBlock, 0, s>>>(out, X, a, Y, b, P, M1, Q, M2, n, k, nullptr);
    }
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  void rmul(T* out, const T* A) {
    switch (k_bucket(k)) {
      case 4: rmul_kernel<T, 4><<<w.rblocks, kSolveBlock, 0, s>>>(out, A, w.Rinv, n, k); break;
      case 8: rmul_kernel<T, 8><<<w.rblocks, kSolveBlock, 0, s>>>(out, A, w.Rinv, n, k); break;
      default: rmul_kernel<T, 16><<<w.rblocks, kSolveBlock, 0, s>>>(out, A, w.Rinv, n, k);
    }
  }
  void hess(TcgState* st) {
    switch (k_bucket(k)) {
      case 4: hess_kernel<T, 4><<<w.rblocks, kSolveBlock, 0, s>>>(w.Hd, w.He, w.U, w.G, w.delta, w.M, n, k, st, w.gr); break;
      case 8: hess_kernel<T, 8><<<w.rblocks, kSolveBlock, 0, s>>>(w.Hd, w.He, w.U, w.G, w.delta, w.M, n, k, st, w.gr); break;
      default: hess_kernel<T, 16><<<w.rblocks, kSolveBlock, 0, s>>>(w.Hd, w.He, w.U, w.G, w.delta, w.M, n, k, st, w.gr);
    }
  }
  // out = qf(A) by Cholesky-QR twice; A is overwritten
  pspec_status qf(T* A, T* out) {
    PSPEC_TRY(gram(A, A, w.Gram));
    chol_inv_kernel<<<1, 1, 0, s>>>(w.Gram, k, w.Rinv, w.bad);
    rmul(out, A);
    PSPEC_TRY(gram(out, out, w.Gram));
    chol_inv_kernel<<<1, 1, 0, s>>>(w.Gram, k, w.Rinv, w.bad);
    rmul(A, out);
    PSPEC_CUDA(cudaMemcpyAsync(out, A, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
    PSPEC_CUDA(cudaGetLastError());
    return PSPEC_OK;
  }
  // M = U^T egrad, rg = egrad - U M and <rg, rg> into *rr (enqueued only)
  pspec_status riemannian_grad(const T* U, const T* egrad, double* M, T* rg, double* rr) {
    PSPEC_TRY(gram(U, egrad, M));
    PSPEC_TRY(combine(rg, egrad, 1.0, nullptr, 0.0, U, M, nullptr, nullptr));
    DotPairs<T> dp{};
    dp.x[0] = rg;
    dp.y[0] = rg;
    dp.np = 1;
    return dots(dp, rr);
  }
  // One synchronisation per Newton step: F, the two model dots, <rg, rg> and
  // the status word land in a pinned host record together.
  struct Record {
    double dots[2];
    double rr;
    double F;
    int status;
  };
  Record* rec = nullptr;  // pinned, owned by the graph handle
  pspec_status fetch(bool with_dots) {
    if (with_dots) PSPEC_CUDA(cudaMemcpyAsync(rec->dots, w.dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    PSPEC_CUDA(cudaMemcpyAsync(&rec->rr, w.gdot, sizeof(double), cudaMemcpyDeviceToHost, s));
    PSPEC_CUDA(cudaMemcpyAsync(&rec->F, w.F, sizeof(double), cudaMemcpyDeviceToHost, s));
    PSPEC_CUDA(cudaMemcpyAsync(&rec->status, g->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    PSPEC_CUDA(cudaStreamSynchronize(s));
    if (rec->status != 0) PSPEC_CUDA(cudaMemsetAsync(g->d_status, 0, sizeof(int), s));
    return PSPEC_OK;
  }
};

}  // namespace

template <typename T>
static pspec_status solve_impl(pspec_graph* g, int k, const double* sched, int n_p,
                               const pspec_solve_opts& o, T* U_io, int32_t* labels,
                               double* rcut_out, pspec_solve_stats* stats, cudaStream_t s) {
  const auto t0 = std::chrono::steady_clock::now();
  Solver<T> S;
  S.g = g;
  S.k = k;
  S.n = g->n;
  S.m = g->n * k;
  S.s = s;
  S.alg1 = o.hessian_form == PSPEC_HESSIAN_ALG1;
  PSPEC_TRY(carve<T>(g, k, &S.w));
  SolveWork<T>& w = S.w;
  if (!g->h_solve_rec) PSPEC_CUDA(cudaMallocHost(&g->h_solve_rec, 512));
  S.rec = reinterpret_cast<typename Solver<T>::Record*>(g->h_solve_rec);
  TcgState* st_pinned = reinterpret_cast<TcgState*>(reinterpret_cast<char*>(g->h_solve_rec) + 256);
  const int64_t m = S.m;
  PSPEC_CUDA(cudaMemcpyAsync(w.U, U_io, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
  PSPEC_CUDA(cudaMemsetAsync(w.bad, 0, sizeof(int), s));
  const int chunk = sizeof(T) == 4 ? 6 : 2;  // CG iterations per host check
  GraphCache graphs;
  // per-kernel timing needs eager launches; PSPEC_SOLVE_EAGER=1 asks for them too
  graphs.enabled = !g->timing.enabled && !(std::getenv("PSPEC_SOLVE_EAGER") &&
                                           std::getenv("PSPEC_SOLVE_EAGER")[0] == '1');
  pspec_solve_stats st_local;
  std::memset(&st_local, 0, sizeof(st_local));
  bool all_converged = true;
  const double Delta_bar = o.delta_bar_scale * std::sqrt((double)k);
  for (int ip = 0; ip < n_p; ++ip) {
    const double p = sched[ip];
    double f = 0.0, gnorm = 0.0;
    PSPEC_TRY(S.eval(w.U, p, w.egrad, w.dk, w.nd));
    PSPEC_TRY(S.riemannian_grad(w.U, w.egrad, w.M, w.rg, w.gdot));
    PSPEC_TRY(S.fetch(false));
    PSPEC_TRY(status_error(S.rec->status));
    f = S.rec->F;
    gnorm = std::sqrt(std::max(S.rec->rr, 0.0));
    const double gnorm0 = gnorm;
    double Delta = o.delta0_scale * Delta_bar;
    int outer = 0, inner_total = 0;
    bool converged = false;
    while (true) {
      if (gnorm <= std::max(o.gtol_abs, o.gtol_rel * gnorm0)) {
        converged = true;
        break;
      }
      if (outer >= o.max_outer) break;
      ++outer;
      // ---- truncated CG on the device
      TcgState h{};
      h.Delta = Delta;
      h.rr = gnorm * gnorm;
      h.norm_r0 = gnorm;
      h.stop = gnorm * std::min(std::pow(gnorm, o.theta), o.kappa);
      h.e_Pe = 0.0;
      h.e_Pd = 0.0;
      h.d_Pd = h.rr;
      h.max_inner = o.max_inner;
      PSPEC_CUDA(cudaMemcpyAsync(w.st, &h, sizeof(TcgState), cudaMemcpyHostToDevice, s));
      PSPEC_CUDA(cudaMemsetAsync(w.eta, 0, sizeof(T) * m, s));
      PSPEC_CUDA(cudaMemcpyAsync(w.r, w.rg, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
      PSPEC_TRY(S.combine(w.delta, w.rg, -1.0, nullptr, 0.0, nullptr, nullptr, nullptr, nullptr));
      const int* done = &w.st->done;
      // one CG iteration: Hessian product, U^T (H delta), the Riemannian
      // Hessian and the CG updates, all decided on the device
      auto cg_iters = [&](int count) -> pspec_status {
        for (int c = 0; c < count; ++c) {
          PSPEC_TRY(S.hvp_gram(w.U, w.delta, p, w.He, w.G, done));
          TimedScope timer(g, "solve_tcg_vec", s);
          S.hess(w.st);
          cg_update_kernel<T><<<w.vblocks, kSolveBlock, 0, s>>>(w.eta, w.r, w.delta,
                                                                 w.Hd, m, w.st, w.gr);
          direction_kernel<T><<<w.vblocks, kSolveBlock, 0, s>>>(w.delta, w.r, m, w.st);
          PSPEC_CUDA(cudaGetLastError());
        }
        return PSPEC_OK;
      };
      TcgState hs{};
      for (int it = 0; it < o.max_inner; it += chunk) {
        // after the first chunk of a stage (which builds every lazily
        // allocated buffer), chunks replay a CUDA graph of `chunk` iterations
        // per (iterate buffer, p); iterations past the stop are no-ops
        if (graphs.enabled && (outer > 1 || it > 0)) {
          cudaGraphExec_t exec = nullptr;
          PSPEC_TRY(graphs.get(w.U, p, s, [&]() { return cg_iters(chunk); }, &exec));
          PSPEC_CUDA(cudaGraphLaunch(exec, s));
        } else {
          PSPEC_TRY(cg_iters(std::min(chunk, o.max_inner - it)));
        }
        PSPEC_CUDA(cudaMemcpyAsync(st_pinned, w.st, sizeof(TcgState), cudaMemcpyDeviceToHost, s));
        PSPEC_CUDA(cudaStreamSynchronize(s));
        hs = *st_pinned;
        if (hs.done) break;
      }
      S.hvps += hs.j;  // HVP launches enqueued after CG stopped were no-ops
      inner_total += hs.j;
      const bool on_boundary = hs.boundary != 0;
      // ---- trial point, model decrease, ratio
      PSPEC_TRY(S.combine(w.tmp, w.U, 1.0, w.eta, 1.0, nullptr, nullptr, nullptr, nullptr));
      PSPEC_TRY(S.qf(w.tmp, w.Unew));
      PSPEC_TRY(S.eval(w.Unew, p, w.egrad_new, w.dk_new, w.nd_new));
      DotPairs<T> dp{};
      dp.x[0] = w.rg;
      dp.y[0] = w.eta;
      dp.x[1] = w.eta;
      dp.y[1] = w.r;  // <eta, H eta> = <eta, r> - <eta, rg>
      dp.np = 2;
      PSPEC_TRY(S.dots(dp, w.dots));
      // the Riemannian gradient at the trial point, used if it is accepted
      PSPEC_TRY(S.riemannian_grad(w.Unew, w.egrad_new, w.Mnew, w.rg_new, w.gdot));
      PSPEC_TRY(S.fetch(true));
      const double dv[2] = {S.rec->dots[0], S.rec->dots[1] - S.rec->dots[0]};  // <rg, eta>, <eta, H eta>
      const double f_new = S.rec->F;
      // a trial point whose evaluation met a NaN/Inf or a zero column is rejected
      const bool trial_bad = S.rec->status != 0 || !std::isfinite(f_new);
      const double reg = o.rho_reg * std::max(1.0, std::fabs(f));
      const double num = f - f_new + reg;
      const double den = -(dv[0] + 0.5 * dv[1]) + reg;
      const bool model_decreased = den >= 0.0 && !trial_bad;
      const double rho = trial_bad ? NAN : (den != 0.0 ? num / den : -INFINITY);
      if (!model_decreased || rho < 0.25 || std::isnan(rho))
        Delta *= 0.25;
      else if (rho > 0.75 && on_boundary)
        Delta = std::min(2.0 * Delta, Delta_bar);
      const bool accept = model_decreased && rho > o.rho_prime;
      if (o.verbose)
        std::fprintf(stderr, "pspec p=%.3f it=%d f=%.10e |g|=%.3e tcg=%d(%d) rho=%.3f Delta=%.3e %s\n", p,
                     outer, f, gnorm, hs.j, hs.reason, rho, Delta, accept ? "acc" : "rej");
      if (accept) {  // the iterate, its gradient, U^T grad and Delta_p u move together
        std::swap(w.U, w.Unew);
        std::swap(w.egrad, w.egrad_new);
        std::swap(w.dk, w.dk_new);
        std::swap(w.nd, w.nd_new);
        std::swap(w.M, w.Mnew);
        std::swap(w.rg, w.rg_new);
        f = f_new;
        gnorm = std::sqrt(std::max(S.rec->rr, 0.0));
      }
    }
    if (!converged) all_converged = false;
    if (ip < 32) {
      st_local.outer[ip] = outer;
      st_local.inner[ip] = inner_total;
      st_local.f[ip] = f;
      st_local.gnorm[ip] = gnorm;
    }
  }
  st_local.n_stages = n_p;
  PSPEC_CUDA(cudaMemcpyAsync(U_io, w.U, sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
  int bad = 0;
  PSPEC_CUDA(cudaMemcpyAsync(&bad, w.bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  PSPEC_CUDA(cudaStreamSynchronize(s));
  if (bad) return set_error(PSPEC_ERR_NONFINITE, "Cholesky-QR met a Gram matrix that is not positive definite");
  // ---- k-means on the rows of U, then RCut
  if (labels || rcut_out) {
    int32_t* lab = labels;
    void* tmp_lab = nullptr;
    if (!lab) {
      PSPEC_CUDA(cudaMalloc(&tmp_lab, sizeof(int32_t) * g->n));
      lab = (int32_t*)tmp_lab;
    }
    double inertia = 0.0;
    pspec_status ks = pspec_kmeans(U_io, g->n, k, sizeof(T) == 4 ? PSPEC_F32 : PSPEC_F64, k, o.seed,
                                   o.kmeans_restarts, o.kmeans_max_iter, lab, nullptr, &inertia, s);
    st_local.kmeans_inertia = inertia;
    if (ks == PSPEC_OK && rcut_out) ks = pspec_rcut(g, lab, k, rcut_out, s);
    if (tmp_lab) cudaFree(tmp_lab);
    if (ks != PSPEC_OK) return ks;
  }
  st_local.eval_calls = S.evals;
  st_local.hvp_calls = S.hvps;
  st_local.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st_local;
  return all_converged ? PSPEC_OK : set_error(PSPEC_ERR_NOT_CONVERGED, "a stage reached max_outer");
}

// Validation shared by the solve entry points; *o gets the options (defaults
// where opts is NULL).
pspec_status check_solve_args(const double* p_schedule, int n_p, const pspec_solve_opts* opts,
                              pspec_solve_opts* o) {
  if (!p_schedule || n_p < 1) return set_error(PSPEC_ERR_INVALID_ARG, "empty p schedule");
  for (int i = 0; i < n_p; ++i) {
    if (!(p_schedule[i] > 1.0 && p_schedule[i] <= 2.0))
      return set_error(PSPEC_ERR_INVALID_ARG, "every p must be in (1, 2]");
    if (i > 0 && p_schedule[i] > p_schedule[i - 1])
      return set_error(PSPEC_ERR_INVALID_ARG, "the p schedule must be non-increasing");
  }
  pspec_solve_opts_default(o);
  if (opts) *o = *opts;
  if (o->max_inner < 1 || o->max_outer < 0 || o->kmeans_restarts < 1)
    return set_error(PSPEC_ERR_INVALID_ARG, "bad iteration caps");
  if (o->hessian_form != PSPEC_HESSIAN_EXACT && o->hessian_form != PSPEC_HESSIAN_ALG1)
    return set_error(PSPEC_ERR_INVALID_ARG, "hessian_form must be PSPEC_HESSIAN_EXACT or PSPEC_HESSIAN_ALG1");
  return PSPEC_OK;
}

// The solve of one single-graph handle on its private stream, joined to
// `caller` by events (validated arguments).
pspec_status solve_on_handle(pspec_graph* g, int k, const double* p_schedule, int n_p,
                             const pspec_solve_opts& o, pspec_dtype dtype, void* U_inout,
                             int32_t* labels_out, double* rcut_out, pspec_solve_stats* stats,
                             cudaStream_t caller) {
  if (!g->solve_stream) {
    PSPEC_CUDA(cudaStreamCreateWithFlags(&g->solve_stream, cudaStreamNonBlocking));
    PSPEC_CUDA(cudaEventCreateWithFlags(&g->solve_event, cudaEventDisableTiming));
  }
  cudaStream_t s = g->solve_stream;
  PSPEC_CUDA(cudaEventRecord(g->solve_event, caller));  // the caller's earlier work first
  PSPEC_CUDA(cudaStreamWaitEvent(s, g->solve_event, 0));
  const pspec_status st =
      dtype == PSPEC_F32
          ? solve_impl<float>(g, k, p_schedule, n_p, o, (float*)U_inout, labels_out, rcut_out, stats, s)
          : solve_impl<double>(g, k, p_schedule, n_p, o, (double*)U_inout, labels_out, rcut_out, stats, s);
  // whatever the solve left enqueued comes before the caller's later work
  cudaEventRecord(g->solve_event, s);
  cudaStreamWaitEvent(caller, g->solve_event, 0);
  return st;
}

}  // namespace pspec

using namespace pspec;

extern "C" void pspec_solve_opts_default(pspec_solve_opts* o) {
  if (!o) return;
  o->max_outer = 30;
  o->max_inner = 50;
  o->gtol_rel = 1e-6;
  o->gtol_abs = 0.0;
  o->theta = 1.0;
  o->kappa = 0.1;
  o->delta_bar_scale = 1.0;
  o->delta0_scale = 0.1;
  o->rho_prime = 0.1;
  o->rho_reg = 1e-10;
  o->kmeans_restarts = 10;
  o->kmeans_max_iter = 300;
  o->seed = 0;
  o->verbose = 0;
  o->hessian_form = PSPEC_HESSIAN_EXACT;
}

extern "C" pspec_status pspec_solve(pspec_graph* g, int k, const double* p_schedule, int n_p,
                                    const pspec_solve_opts* opts, pspec_dtype dtype, void* U_inout,
                                    int32_t* labels_out, double* rcut_out, pspec_solve_stats* stats,
                                    void* stream) {
  if (!g) return set_error(PSPEC_ERR_INVALID_ARG, "graph is NULL");
  if (g->n_graphs != 1) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_solve takes a single graph");
  if (g->is_shard) return set_error(PSPEC_ERR_INVALID_ARG, "pspec_solve takes a whole graph, not a shard");
  if (k < 1 || k > kMaxK) return set_error(PSPEC_ERR_INVALID_ARG, "k must be in [1, 16]");
  if (k > g->n) return set_error(PSPEC_ERR_INVALID_ARG, "k exceeds n");
  pspec_solve_opts o;
  PSPEC_TRY(check_solve_args(p_schedule, n_p, opts, &o));
  PSPEC_TRY(check_block(U_inout, k, dtype, "U_inout"));
  if (dtype != PSPEC_F32 && dtype != PSPEC_F64) return set_error(PSPEC_ERR_INVALID_ARG, "bad dtype");
  return solve_on_handle(g, k, p_schedule, n_p, o, dtype, U_inout, labels_out, rcut_out, stats,
                         (cudaStream_t)stream);
}
