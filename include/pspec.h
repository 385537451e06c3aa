/*
 * pspec.h -- C ABI of the GB300 (sm_103a) p-spectral clustering library.
 *
 * The library evaluates, on one GPU, the hot path of multiway p-spectral
 * clustering ("Nonlinear spectral clustering with C++ GraphBLAS", Section 2):
 *
 *   F_p(U) = sum_l sum_{i,j} w_ij |u_i^l - u_j^l|^p / (2 ||u^l||_p^p)   (Eq. 1)
 *   (Delta_p u)_i = sum_j w_ij phi_p(u_i - u_j),  phi_p(x) = |x|^(p-1) sign(x)
 *
 * its gradient (the paper's EucGrad), the exact Hessian-vector product (the
 * paper's EucHessianEta, Algorithm 1), the Newton / truncated-CG solve on the
 * Grassmann manifold with p continuation, the k-means discretisation and the
 * RCut score (Section 3.1).
 *
 * Conventions shared by every call
 *  - W is symmetric and non-negative, stored in CSR with BOTH triangles:
 *    rowptr int64[n+1] (rowptr[0] = 0, non-decreasing), col int32[nnz] in
 *    [0, n), val[nnz].  A stored diagonal entry contributes nothing.
 *  - Dense blocks (U, V, gradients, Hessian products) are n x k ROW-MAJOR
 *    (element (i, l) at offset i*k + l; the paper's k x n eta is the
 *    transpose).  1 <= k <= 16.  FP32 blocks must be 16-byte aligned when
 *    k % 4 == 0 and 8-byte aligned when k % 2 == 0 (cudaMalloc/torch
 *    allocations always are); FP64 blocks 8-byte aligned.
 *  - p lies in (1, 2] (Eq. 1).
 *  - Precision (pspec_dtype): PSPEC_F32 is the fast form (FP32 edge
 *    arithmetic, compensated FP32 per-thread sums, float-float cross-thread
 *    reductions, FP64 scalars); PSPEC_F64 is the plain form (FP64 everywhere,
 *    one thread per row, one column per pass, mirroring Algorithm 1's loop
 *    over columns).
 *  - Pointers are DEVICE pointers unless the call's flags contain
 *    PSPEC_HOST_PTRS.  The caller owns every pointer it passes; the graph
 *    handle owns its device copy of W and its workspace.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream ordered and return once the work is
 *    enqueued, except: calls with PSPEC_HOST_PTRS, pspec_solve,
 *    pspec_kmeans and pspec_rcut, which synchronise `stream` before they
 *    return.
 *  - Errors are returned as pspec_status; no C++ exception crosses the ABI.
 *    pspec_last_error() gives a message for the calling thread's last error.
 *    Conditions found by a kernel (a zero column norm, a non-finite result)
 *    are recorded in the graph's device status word: synchronous calls
 *    return them, asynchronous ones leave them for pspec_graph_status().
 *  - A graph handle may be used from one host thread at a time; calls on the
 *    same handle must be ordered on one stream (they share its workspace).
 */
#ifndef PSPEC_H
#define PSPEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PSPEC_OK = 0,
  PSPEC_ERR_INVALID_ARG = 1,   /* argument outside its documented domain   */
  PSPEC_ERR_CUDA = 2,          /* a CUDA runtime call failed               */
  PSPEC_ERR_OOM = 3,           /* device or pinned-host allocation failed  */
  PSPEC_ERR_ZERO_COLUMN = 4,   /* ||u^l||_p = 0 for some column            */
  PSPEC_ERR_NONFINITE = 5,     /* a NaN or Inf reached an objective sum    */
  PSPEC_ERR_NOT_CONVERGED = 6, /* iteration cap reached (informational)    */
  PSPEC_ERR_TIMEOUT = 7        /* a bounded device wait gave up            */
} pspec_status;

typedef enum { PSPEC_F32 = 0, PSPEC_F64 = 1 } pspec_dtype;

/* flags */
#define PSPEC_HOST_PTRS 0x1u      /* pointer arguments are host memory         */
#define PSPEC_CHECK_SYMMETRY 0x2u /* graph_create: verify w_ij == w_ji (host)  */
#define PSPEC_HVP_ALG1 0x4u       /* hvp: Algorithm 1's form (see pspec_hvp)   */
#define PSPEC_KEEP_DELTA 0x8u     /* eval: keep Delta_p u on the handle        */
#define PSPEC_DELTA_KEPT 0x10u    /* hvp: reuse the kept Delta_p u (same U)    */

typedef struct pspec_graph pspec_graph;

/* ---------------------------------------------------------------- graph ---
 * pspec_graph_create: copy W (CSR, both triangles; Section 2's weighted
 * adjacency of an undirected graph) to the device and build the row
 * partition the edge kernels walk.  rowptr/col/val are host pointers (or
 * device pointers without PSPEC_HOST_PTRS: they are then staged through the
 * host).  val_dtype gives val's type; the graph keeps an FP32 and an FP64
 * copy so either precision can run on it.
 * Errors: INVALID_ARG for n < 1, nnz >= 2^31, rowptr[0] != 0, a decreasing
 * rowptr, col outside [0, n), a negative or non-finite weight, or (with
 * PSPEC_CHECK_SYMMETRY) an entry without its mirror of equal weight; OOM;
 * CUDA.  On error *out is set to NULL. */
pspec_status pspec_graph_create(int64_t n, const int64_t* rowptr, const int32_t* col,
                                const void* val, pspec_dtype val_dtype, unsigned flags,
                                void* stream, pspec_graph** out);

/* pspec_graph_create_batched: G independent graphs concatenated into one
 * block-diagonal W.  node_off int64[G+1] (node_off[0] = 0) gives each
 * graph's vertex range; rowptr/col/val describe the concatenation with GLOBAL
 * column indices that must stay inside the row's own graph.  Batched eval
 * and HVP calls then treat every graph as its own problem (its own F, N_l,
 * D_l) in one launch.  Same errors as pspec_graph_create, plus INVALID_ARG
 * when an entry crosses graphs. */
pspec_status pspec_graph_create_batched(int32_t n_graphs, const int64_t* node_off,
                                        const int64_t* rowptr, const int32_t* col,
                                        const void* val, pspec_dtype val_dtype, unsigned flags,
                                        void* stream, pspec_graph** out);

/* Free the device copy and workspace.  NULL is accepted. */
void pspec_graph_destroy(pspec_graph* g);

/* n (vertices), nnz (stored entries), graph count of a handle. */
pspec_status pspec_graph_info(const pspec_graph* g, int64_t* n, int64_t* nnz, int32_t* n_graphs);

/* Synchronise `stream`, return the conditions kernels recorded since the
 * last call (ZERO_COLUMN, NONFINITE, TIMEOUT, or OK) and clear them. */
pspec_status pspec_graph_status(pspec_graph* g, void* stream);

/* ----------------------------------------------------------------- eval ---
 * pspec_eval: objective and Euclidean gradient (the paper's EucGrad).
 *   F_out[0]   = F_p(U) of Eq. 1                          (FP64, 1 value)
 *   grad_out   = dF/dU, column l = (p/D_l)(Delta_p u^l - lambda_l phi_p(u^l))
 *                with D_l = ||u^l||_p^p, N_l = (1/2) sum_ij w_ij |d_ij|^p,
 *                lambda_l = N_l / D_l                     (n x k, dtype)
 *   parts_out  = optional (NULL to skip) FP64[2k]: N_0..N_{k-1}, D_0..D_{k-1}
 * U and grad_out have type `dtype`; grad_out may not alias U.  F_out and
 * parts_out are device pointers (host with PSPEC_HOST_PTRS).  On a batched
 * graph every graph has k columns (group graphs of different k into
 * separate handles), F_out holds G values and parts_out G x 2k (graph g's
 * N then D at [g*2k]); the call runs the FP32 path only (dtype F32, else
 * INVALID_ARG).
 * With PSPEC_KEEP_DELTA in flags (FP32, single graph) the handle keeps the
 * rows Delta_p u of this call (n x k FP32 in its workspace) together with
 * the U pointer, k and p, for later pspec_hvp calls with PSPEC_DELTA_KEPT at
 * the same point: the Newton step of Section 2 evaluates the gradient once at
 * U and then applies the Hessian at U many times (truncated CG), and Delta_p u
 * depends on U alone.  A later KEEP call replaces what is kept.
 * Errors: INVALID_ARG (k, p, NULL, misalignment, KEEP on a batched graph or
 * with FP64), CUDA; ZERO_COLUMN and NONFINITE through the status word. */
pspec_status pspec_eval(pspec_graph* g, const void* U, int k, double p, pspec_dtype dtype,
                        double* F_out, void* grad_out, double* parts_out, unsigned flags,
                        void* stream);

/* ------------------------------------------------------------------ hvp ---
 * pspec_hvp: exact Euclidean Hessian of F_p at U applied to V (the paper's
 * EucHessianEta; block diagonal over columns):
 *   HV = (Hess N V - lambda Hess D V)/D
 *        - (g_N <g_D,V> + g_D <g_N,V> - 2 lambda g_D <g_D,V>)/D^2   per column,
 *   (Hess N V)_a = p(p-1) sum_j w_aj |d_aj|^(p-2) (V_a - V_j),
 *   (Hess D V)_a = p(p-1) |u_a|^(p-2) V_a,  g_N = p Delta_p u,  g_D = p phi_p(u).
 * A zero difference d_aj == 0 (or u_a == 0) contributes no curvature term.
 * The sparse-plus-diagonal part is what Algorithm 1 applies column by
 * column; the rank-two terms complete the Hessian of the quotient.
 * On a batched graph lambda, D, g_N and g_D are each graph's own (FP32
 * only, as pspec_eval).  With PSPEC_HVP_ALG1 in flags the rank-two terms
 * are left out: HV = (Hess N V - lambda Hess D V)/D per column, the sparse
 * (W's pattern) plus diagonal matrix that Algorithm 1 applies.  HV_out may
 * not alias U or V.
 * With PSPEC_DELTA_KEPT in flags (FP32, single graph) the call takes the rows
 * Delta_p u (needed by the rank-two terms) from the last pspec_eval with
 * PSPEC_KEEP_DELTA instead of writing them again: one n x k block less of
 * memory traffic per call.  That eval must have had the same U pointer
 * (host or device, as passed), k and p, else INVALID_ARG; the caller
 * guarantees that U's contents have not changed since, and orders both calls
 * on one stream.  The result equals the plain call's within rounding (the
 * objective's and the Hessian's kernels form phi_p by different power
 * formulas).  Errors as pspec_eval. */
pspec_status pspec_hvp(pspec_graph* g, const void* U, const void* V, int k, double p,
                       pspec_dtype dtype, void* HV_out, unsigned flags, void* stream);

/* ----------------------------------------------------------------- tune ---
 * pspec_tune: choose the launch shape of the fused edge kernels for this
 * handle and column count k by timing them.  Candidates: the edges-per-lane
 * target L in {Q, 2Q, 4Q, 8Q, 16Q} (Q = column lanes per row for this k; a
 * row of degree d gets the smallest power-of-two number of edge slots E with
 * d <= L*E, so L fixes how many rows a warp task holds, 32/(E*Q), and whether
 * the staged kernel -- for tasks short enough for its shared-memory buffers,
 * L <= 8 at k = 4, 8, 16 -- or the direct one runs) and the resident blocks per SM
 * (as many as each kernel fits, and one and two fewer than the direct HVP
 * kernel fits).  Each candidate runs one untimed eval + HVP and then `reps` timed
 * ones on U, V (device, n x k row-major FP32); the fastest is kept on the
 * handle for every later FP32 call with this k's column split (it changes
 * the summation order of the per-column sums, within the stated tolerance,
 * and results stay bit-reproducible for a fixed shape).  The paper has no
 * counterpart; the shape is a property of the hardware.  Allocates two n x k
 * FP32 outputs for the duration of the call and synchronises `stream`.
 * A single graph's candidates are timed on the pair a Newton step repeats
 * (pspec_eval keeping Delta_p u, then pspec_hvp reusing it; a batch: the
 * plain pair); the call drops whatever Delta_p u the handle kept.
 * report receives every candidate's mean eval + HVP time.  Errors:
 * INVALID_ARG (k, p, reps outside [1, 1000], NULL, misalignment), CUDA, OOM. */
#define PSPEC_TUNE_MAX 16
typedef struct {
  int32_t n_candidates;
  int32_t chosen;                         /* index into the arrays below */
  int32_t edges_per_lane[PSPEC_TUNE_MAX];
  int32_t blocks_per_sm[PSPEC_TUNE_MAX];
  double ms[PSPEC_TUNE_MAX];              /* mean device time of eval + HVP */
} pspec_tune_report;
pspec_status pspec_tune(pspec_graph* g, const float* U, const float* V, int k, double p, int reps,
                        pspec_tune_report* report, void* stream);

/* ------------------------------------------------------ hvp, no allocation ---
 * pspec_hvp_noalloc: the same Hessian-vector product as pspec_hvp (FP32,
 * device pointers), for callers that must not allocate device memory: code
 * whose device memory belongs to another runtime's allocator (a framework's
 * caching pool, an application that hands out fixed buffers), a section that
 * must not enter cudaMalloc because it can synchronise the device, or code
 * that cannot create a graph handle (creating one allocates).  The call
 * enqueues a memset and kernels on `stream`, so, like any CUDA call, it must
 * not be made from a host function running on a stream (cudaLaunchHostFunc,
 * stream callbacks).  The paper has no counterpart; this is an interface
 * convenience.
 *   rowptr/col/val: W in CSR (both triangles, FP32 weights), device memory
 *   U, V, HV_out:   n x k row-major FP32, device memory, HV_out not aliasing
 * Working memory (the rows of Delta_p u and the reduction partials) is one
 * fixed array in the library's device globals, about 2.6 MB, held on every
 * GPU that loads the library until the process exits; hence the limit
 * n * k <= 524288 (INVALID_ARG beyond it, with a message).  The arguments
 * are not validated on the device (col must lie in [0, n), weights >= 0).
 * The first call on a device, with that device current, looks up the
 * array's device address; make that first call before any stream capture.
 * Every call uses the same array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race and give wrong results.  The
 * looked-up address is kept for the life of the process: do not use the call
 * across a cudaDeviceReset of that device.  There is no handle and hence no
 * status word: a non-finite intermediate (NONFINITE for pspec_hvp) shows up
 * as a NaN or an infinity in HV_out, and a zero column norm as infinities.
 * Errors: INVALID_ARG, CUDA.  Enqueued on `stream`; does not synchronise. */
pspec_status pspec_hvp_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                               const float* val, const float* U, const float* V, int k, double p,
                               float* HV_out, void* stream);

/* ------------------------------------------------ row-partitioned runs ---
 * One rank of a run that partitions the rows of W over several GPUs (each
 * rank a process with its own GPU).  Every per-column quantity of Section 2
 * is a sum over rows, so a rank sums its owned rows, the ranks add their
 * sums, and each rank finishes its owned rows from the global sums:
 *   1. the caller copies the rows of U (and V) its owned rows read but other
 *      ranks own -- the halo -- into rows n_owned..n_local-1 of its block;
 *   2. pspec_eval_partial / pspec_hvp_partial sum the owned rows: FP64
 *      sums_out = N_r, D_r (2k values) or N_r, D_r, sigma_N_r, sigma_D_r (4k),
 *      with N_r = 1/2 sum over owned i, all j of w_ij |d_ij|^p, D_r = sum over
 *      owned i of |u_i|^p, sigma_N_r = sum over owned i of (Delta_p u)_i v_i,
 *      sigma_D_r = sum over owned i of phi_p(u_i) v_i;
 *   3. the caller adds sums_out over the ranks (an FP64 allreduce);
 *   4. pspec_eval_finish / pspec_hvp_finish form F, the gradient or the
 *      Hessian product (pspec_eval's and pspec_hvp's definitions) of the
 *      owned rows from the added sums (sums_in, same layout).
 * All blocks are device FP32, n_local x k row-major (owned rows first, then
 * halo rows); outputs are written on the owned rows only.  sums_out, sums_in
 * and F_out are device FP64.  The partial call leaves the rows Delta_p u of
 * the owned rows in grad_out (eval) or the handle (HVP) for its finish call;
 * a finish call must follow its partial call on the same stream.  Errors:
 * INVALID_ARG (k, p, NULL, misalignment, aliasing, a handle that is not a
 * shard, a finish without its partial), CUDA; ZERO_COLUMN and NONFINITE
 * through the status word.  The paper scales one graph over CPU threads
 * (Section 3.2); the row partition is this library's way to scale it over
 * GPUs.
 *
 * pspec_graph_create_shard: the owned rows of W on this rank with column
 * indices renumbered to local vertices: owned vertices 0..n_owned-1 (in
 * their global order), halo vertices n_owned..n_local-1.  rowptr has
 * n_owned + 1 entries; col in [0, n_local).  Host arrays only
 * (PSPEC_HOST_PTRS required).  Same validation as pspec_graph_create.  A
 * shard handle takes only the calls of this section and pspec_tune. */
pspec_status pspec_graph_create_shard(int64_t n_owned, int64_t n_local, const int64_t* rowptr,
                                      const int32_t* col, const void* val, pspec_dtype val_dtype,
                                      unsigned flags, void* stream, pspec_graph** out);
pspec_status pspec_eval_partial(pspec_graph* g, const float* U, int k, double p, float* grad_out,
                                double* sums_out, void* stream);
pspec_status pspec_eval_finish(pspec_graph* g, const float* U, int k, double p, const double* sums_in,
                               double* F_out, float* grad_out, void* stream);
pspec_status pspec_hvp_partial(pspec_graph* g, const float* U, const float* V, int k, double p,
                               float* HV_out, double* sums_out, void* stream);
/* flags: PSPEC_HVP_ALG1 for Algorithm 1's form (see pspec_hvp) */
pspec_status pspec_hvp_finish(pspec_graph* g, const float* U, const float* V, int k, double p,
                              const double* sums_in, float* HV_out, unsigned flags, void* stream);

/* ---------------------------------------------------------------- solve ---
 * pspec_solve: minimise Eq. 1 while p is continued from 2 toward 1
 * (Section 2): for each p of p_schedule (each in (1,2], non-increasing), a
 * trust-region Newton method on Gr(k, n) whose subproblems are solved by
 * truncated CG; tangent projection P_U(G) = G - U U^T G, Riemannian Hessian
 * P_U(H eta) - eta U^T grad F, retraction qf(U + eta) (thin QR with a
 * positive diagonal, computed as Cholesky-QR twice).  Then k-means on the
 * rows of U (k clusters, opts' seed/restarts) and the RCut of the labels.
 *   U_inout   device n x k (dtype): U0 in (orthonormal columns expected),
 *             final U out
 *   labels_out device int32[n] (may be NULL), rcut_out host double (may be
 *             NULL), stats host (may be NULL).
 * The solve runs on a private stream of the handle, after the work already
 * enqueued on `stream`, and returns once it is complete; `stream`'s later
 * work is ordered after it.  Chunks of truncated-CG iterations are replayed
 * as CUDA graphs (eagerly launched while kernel timing is on).  Returns OK,
 * or NOT_CONVERGED when a stage hit max_outer (the result is still
 * written).  Not for batched graphs; calls on one handle must not overlap. */
#define PSPEC_HESSIAN_EXACT 0 /* the exact Hessian of the quotient N/D        */
#define PSPEC_HESSIAN_ALG1 1  /* Algorithm 1's sparse-plus-diagonal form     */
typedef struct {
  int32_t max_outer;       /* Newton steps per p (default 30)                 */
  int32_t max_inner;       /* truncated-CG steps per Newton step (50)         */
  double gtol_rel;         /* stop: ||grad|| <= gtol_rel ||grad_stage0|| (1e-6) */
  double gtol_abs;         /* ... or ||grad|| <= gtol_abs (0)                  */
  double theta;            /* tCG exponent (1.0)                               */
  double kappa;            /* tCG linear factor (0.1)                          */
  double delta_bar_scale;  /* Delta_bar = scale * sqrt(k) (1.0)                */
  double delta0_scale;     /* Delta_0 = scale * Delta_bar (0.1)                */
  double rho_prime;        /* acceptance threshold (0.1)                       */
  double rho_reg;          /* ratio regularisation, times max(1,|f|) (1e-10)   */
  int32_t kmeans_restarts; /* (10)                                             */
  int32_t kmeans_max_iter; /* (300)                                            */
  uint64_t seed;           /* k-means seed (0)                                 */
  int32_t verbose;         /* print one line per Newton step to stderr (0)     */
  int32_t hessian_form;    /* PSPEC_HESSIAN_EXACT (default) or _ALG1: the
                              Euclidean Hessian the subproblems use           */
} pspec_solve_opts;

typedef struct {
  int32_t n_stages;
  int32_t outer[32];       /* Newton steps per stage (first 32 stages)        */
  int32_t inner[32];       /* truncated-CG steps per stage                    */
  double f[32];            /* F_p at the end of each stage                    */
  double gnorm[32];        /* ||Riemannian gradient|| at the end              */
  int64_t hvp_calls;       /* total Hessian-vector products                   */
  int64_t eval_calls;      /* total objective/gradient evaluations            */
  double seconds;          /* wall time of the solve (host clock)             */
  double kmeans_inertia;
} pspec_solve_stats;

void pspec_solve_opts_default(pspec_solve_opts* o);

pspec_status pspec_solve(pspec_graph* g, int k, const double* p_schedule, int n_p,
                         const pspec_solve_opts* opts, pspec_dtype dtype, void* U_inout,
                         int32_t* labels_out, double* rcut_out, pspec_solve_stats* stats,
                         void* stream);

/* ------------------------------------------------------ solve, batched ---
 * pspec_solve_batched: pspec_solve for every graph of a batched handle, each
 * graph its own problem (its own trust regions, truncated CG, k-means and
 * RCut), with the same k for all graphs.  The first call builds one
 * single-graph handle per graph (kept on the batched handle, freed with it);
 * the per-graph solves then run concurrently, n_threads host threads taking
 * graphs in turn, each solve on its graph handle's private stream.  Every
 * graph's result equals pspec_solve on that graph alone.
 *   U_inout     device n x k FP32 (the concatenation): each graph's U0 in,
 *               final U out
 *   labels_out  device int32[n]: each graph's k-means labels, 0..k-1
 *   rcut_out    host double[G]: each graph's RCut (NaN where the graph has
 *               fewer vertices than k, 0 for an empty graph)
 *   status_out  host int32[G]: each graph's pspec_status
 * Synchronises `stream` before and after.  Returns OK, NOT_CONVERGED when a
 * graph's stage hit max_outer, or the first graph error (INVALID_ARG when a
 * graph has fewer vertices than k, CUDA, OOM, NONFINITE), with its graph
 * named in pspec_last_error.  The paper solves one graph; batching is this
 * library's. */
pspec_status pspec_solve_batched(pspec_graph* g, int k, const double* p_schedule, int n_p,
                                 const pspec_solve_opts* opts, float* U_inout, int32_t* labels_out,
                                 double* rcut_out, int32_t* status_out, int n_threads, void* stream);

/* pspec_solve_lockstep: the same per-graph solves (Section 2's Newton/tCG on
 * the Grassmann manifold for every p of the schedule, then k-means and RCut)
 * with all graphs of a batched handle stepping together on the device: each
 * evaluation and each Hessian product is one launch of the edge kernel over
 * the concatenated CSR, every n x k operation one launch over all graphs'
 * rows, and every per-graph decision (truncated CG's recurrences, the
 * trust-region ratio, radius and acceptance, the stopping tests) is taken in
 * device memory; the host reads G flags per chunk of 6 CG iterations and per
 * Newton step for the whole batch, and replays each chunk as a CUDA graph.
 * A graph whose truncated CG or stage has ended waits, left out of every
 * launch, so each graph takes the iterates it would take alone; only the
 * reductions' summation order differs from pspec_solve, so results agree
 * with it to rounding (not bit for bit).  Stages are synchronous: the batch
 * moves to the next p when every graph has finished the current one.  The
 * final k-means runs per graph on n_threads host threads, each with its own
 * stream; RCut is one launch for all graphs.
 *   U_inout, labels_out, rcut_out, status_out: as pspec_solve_batched, except
 *               that rcut_out is NaN for a graph whose solve failed (labels
 *               of such a graph are left as they were)
 *   stats_out   host pspec_solve_stats[G] or NULL: each graph's counters
 *               (seconds = the whole call's wall time)
 * The FP32 path; opts->verbose = 1 prints one line per Newton step of the
 * batch, 2 also one line per graph that took the step (its F, ||grad||, CG
 * iterations and stop reason, ratio, radius and decision, as pspec_solve).
 * Synchronises the solve's own stream; joined to `stream` by events.
 * Returns OK, NOT_CONVERGED when a graph's stage hit max_outer, or the first
 * graph error in graph order (INVALID_ARG for a graph with fewer vertices
 * than k, NONFINITE, ZERO_COLUMN, CUDA, OOM).  Batching is this library's,
 * not the paper's. */
pspec_status pspec_solve_lockstep(pspec_graph* g, int k, const double* p_schedule, int n_p,
                                  const pspec_solve_opts* opts, float* U_inout, int32_t* labels_out,
                                  double* rcut_out, int32_t* status_out, pspec_solve_stats* stats_out,
                                  int n_threads, void* stream);


/* --------------------------------------------------------------- kmeans ---
 * pspec_kmeans: k-means of the n rows of X (n x dim, row-major, dtype,
 * device), the discretisation step of Section 1/2.  k-means++ seeding whose
 * uniforms come from SplitMix64(seed) (x >> 11) * 2^-53, consumed in order
 * across restarts; Lloyd iterations with squared distances accumulated in
 * FP64 dimension by dimension; ties to the smallest centre; an empty
 * cluster is re-seeded at the row farthest from its centre; stop when no
 * label changes or after max_iter updates; the restart with the smallest
 * inertia is kept.  1 <= dim <= 16, 1 <= n_clusters <= 64, n >= n_clusters.
 * The centres of FP32 rows are means of exact fixed-point sums at a scale
 * 2^q set from max |x| and n (within 2^-q of the exact mean, plus one
 * rounding); FP64 rows are summed in FP64.
 *   labels_out device int32[n]; centers_out device FP64[n_clusters*dim]
 *   (may be NULL); inertia_out host double (may be NULL).
 * Synchronises `stream`.  Returns INVALID_ARG for bad sizes or NULL X or
 * labels_out, and for FP32 rows holding a NaN or an infinity; CUDA or OOM
 * on device errors. */
pspec_status pspec_kmeans(const void* X, int64_t n, int dim, pspec_dtype dtype, int n_clusters,
                          uint64_t seed, int restarts, int max_iter, int32_t* labels_out,
                          double* centers_out, double* inertia_out, void* stream);

/* ----------------------------------------------------------------- rcut ---
 * pspec_rcut: RCut(C_1..C_c) = sum_c cut(C_c, complement)/|C_c| (Section
 * 3.1) with cut(C, C') = sum over i in C, j in C' of w_ij; empty clusters
 * contribute nothing.  labels device int32[n] in [0, n_clusters).
 * rcut_out host double.  Synchronises `stream`.  INVALID_ARG on a batched
 * handle (one RCut per graph: call it on each graph's own handle). */
pspec_status pspec_rcut(pspec_graph* g, const int32_t* labels, int n_clusters, double* rcut_out,
                        void* stream);

/* ------------------------------------------------------- instrumentation ---
 * Per-kernel timing: while enabled, every kernel the graph launches is
 * bracketed by CUDA events on its stream; pspec_kernel_times returns, per
 * kernel name, the number of launches and the summed device milliseconds
 * (it synchronises the recorded events).  Names are returned in a
 * caller-provided buffer as "name=launches:ms;..." */
pspec_status pspec_set_timing(pspec_graph* g, int enable);
pspec_status pspec_kernel_times(pspec_graph* g, char* buf, size_t buf_len);

/* Thread-local message of the last error on this thread ("" if none). */
const char* pspec_last_error(void);

/* Library version "major.minor.patch" and the arch it was built for. */
const char* pspec_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSPEC_H */
