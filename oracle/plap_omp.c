/*
 * plap_omp.c -- FP64 CPU oracle of the objective, the gradient and the exact
 * Hessian-vector product of multiway p-spectral clustering, on all host
 * cores (OpenMP over rows).  The paper runs its method on shared-memory CPU
 * threads in double (Section 3.2); this is the same arithmetic as plain
 * loops over the CSR in natural order, used as the timed all-core CPU
 * baseline.
 *
 * TEST INFRASTRUCTURE ONLY: nothing on the library's product path links or
 * loads this file; only the tests and the benchmark's CPU-baseline leg do.
 * It shares no code with the CUDA library.
 *
 * Definitions (paper, Section 2; both CSR triangles of the symmetric W stored):
 *   N_l = 1/2 sum_i sum_j w_ij |u_i - u_j|^p            (Eq. 1 numerator)
 *   D_l = sum_i |u_i|^p                                  (p-norm, per column)
 *   (Delta_p u)_i = sum_j w_ij phi_p(u_i - u_j),  phi_p(x) = |x|^(p-1) sign(x)
 *   grad = (p / D) (Delta_p u - lambda phi_p(u)),  lambda = N / D
 *   H v  = (S - lambda p(p-1) |u|^(p-2) v) / D
 *          - (g_N <g_D, v> + g_D <g_N, v> - 2 lambda g_D <g_D, v>) / D^2
 *     with S_i = p(p-1) sum_j w_ij |u_i - u_j|^(p-2) (v_i - v_j),
 *     g_N = p Delta_p u, g_D = p phi_p(u).
 * Readings: phi_p(0) = 0; |x|^(p-2) is 0 at x == 0 for p < 2 (a tie carries
 * no curvature) and 1 everywhere at p = 2.
 *
 * Blocks are n x k row-major.  Every function returns 0, or -1 for k outside
 * [1, 64].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KMAX 64

static double phi_p(double x, double p) {
  if (x == 0.0) return 0.0;
  return copysign(pow(fabs(x), p - 1.0), x);
}

static double abs_pow_pm2(double x, double p) {
  if (p == 2.0) return 1.0;
  if (x == 0.0) return 0.0;
  return pow(fabs(x), p - 2.0);
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads for the following calls (t >= 1); returns the count in effect. */
int oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t >= 1) omp_set_num_threads(t);
#endif
  return oracle_threads();
}

/* N_l and D_l of every column, and Delta_p u of every row (delta may be NULL). */
static void parts(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                  const double* U, int k, double p, double* N, double* D, double* delta) {
  double Ns[KMAX], Ds[KMAX];
  memset(Ns, 0, sizeof(Ns));
  memset(Ds, 0, sizeof(Ds));
#pragma omp parallel
  {
    double Nl[KMAX], Dl[KMAX];
    memset(Nl, 0, sizeof(Nl));
    memset(Dl, 0, sizeof(Dl));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      for (int l = 0; l < k; ++l) {
        const double ui = U[i * k + l];
        double dsum = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
          const double d = ui - U[(int64_t)col[e] * k + l];
          Nl[l] += val[e] * pow(fabs(d), p);
          dsum += val[e] * phi_p(d, p);
        }
        Dl[l] += pow(fabs(ui), p);
        if (delta) delta[i * k + l] = dsum;
      }
    }
#pragma omp critical
    for (int l = 0; l < k; ++l) {
      Ns[l] += Nl[l];
      Ds[l] += Dl[l];
    }
  }
  for (int l = 0; l < k; ++l) {
    N[l] = 0.5 * Ns[l];
    D[l] = Ds[l];
  }
}

/* F, N[k], D[k] and the gradient (grad may be NULL). */
int oracle_eval(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                const double* U, int k, double p, double* F, double* N, double* D,
                double* grad) {
  if (k < 1 || k > KMAX) return -1;
  parts(n, rowptr, col, val, U, k, p, N, D, grad);
  double f = 0.0;
  for (int l = 0; l < k; ++l) f += N[l] / D[l];
  *F = f;
  if (grad) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int l = 0; l < k; ++l) {
        const double lam = N[l] / D[l];
        grad[i * k + l] = (p / D[l]) * (grad[i * k + l] - lam * phi_p(U[i * k + l], p));
      }
  }
  return 0;
}

/* HV = exact Euclidean Hessian of F_p at U applied to V (delta: n x k
 * workspace for Delta_p u). */
int oracle_hvp(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
               const double* U, const double* V, int k, double p, double* HV, double* delta) {
  if (k < 1 || k > KMAX) return -1;
  double N[KMAX], D[KMAX];
  parts(n, rowptr, col, val, U, k, p, N, D, delta);
  const double c = p * (p - 1.0);
  /* column dots <g_N, v> and <g_D, v> */
  double cN[KMAX], cD[KMAX];
  memset(cN, 0, sizeof(cN));
  memset(cD, 0, sizeof(cD));
#pragma omp parallel
  {
    double a[KMAX], b[KMAX];
    memset(a, 0, sizeof(a));
    memset(b, 0, sizeof(b));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i)
      for (int l = 0; l < k; ++l) {
        a[l] += p * delta[i * k + l] * V[i * k + l];
        b[l] += p * phi_p(U[i * k + l], p) * V[i * k + l];
      }
#pragma omp critical
    for (int l = 0; l < k; ++l) {
      cN[l] += a[l];
      cD[l] += b[l];
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    for (int l = 0; l < k; ++l) {
      const double ui = U[i * k + l], vi = V[i * k + l];
      double s = 0.0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int64_t j = col[e];
        s += val[e] * abs_pow_pm2(ui - U[j * k + l], p) * (vi - V[j * k + l]);
      }
      const double lam = N[l] / D[l];
      const double gN = p * delta[i * k + l];
      const double gD = p * phi_p(ui, p);
      HV[i * k + l] = (c * s - lam * c * abs_pow_pm2(ui, p) * vi) / D[l] -
                      (gN * cD[l] + gD * cN[l] - 2.0 * lam * gD * cD[l]) / (D[l] * D[l]);
    }
  }
  return 0;
}
