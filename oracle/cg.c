/*
 * Plain FP64 Jacobi-preconditioned conjugate gradients on an assembled CSR
 * matrix, parallelised with OpenMP.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  It is used for grids too
 * large for the sparse direct solve (3D, 2D beyond ~1000^2) and as the timed
 * CPU baseline.  It shares no code with the CUDA path.
 *
 * The matrix is the reduced system of the finite-difference discretisation of
 * -hbar^2 Lap(phi) + f^2 phi = 0 (Sec. 4, Eq. (phiEquation); Sec. 6,
 * Eq. (sparse-system)), assembled by oracle/fd.py.  It is a symmetric
 * M-matrix, so phi > 0 and CG with the diagonal (Jacobi) preconditioner
 * converges.  The stopping rule is componentwise: max_i |r_i| / (a_ii x_i)
 * <= tol, which bounds the relative error of every unknown (the log-domain
 * residual of S), and at least min_iter iterations.  When the recurrence
 * residual meets the rule, the true residual b - A x is recomputed; if it does
 * not meet the rule, CG restarts from the true residual.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static void spmv(int64_t n, const int64_t *ip, const int64_t *ix,
                 const double *v, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = ip[i]; k < ip[i + 1]; ++k) s += v[k] * x[ix[k]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double *a, const double *b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* max_i |r_i| / (d_i x_i); +inf where x_i <= 0 */
static double cw_max(int64_t n, const double *r, const double *d,
                     const double *x) {
  double m = 0.0;
#pragma omp parallel for schedule(static) reduction(max : m)
  for (int64_t i = 0; i < n; ++i) {
    double v = (x[i] > 0.0) ? fabs(r[i]) / (d[i] * x[i]) : INFINITY;
    if (v > m) m = v;
  }
  return m;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/*
 * Solve A x = b.  x holds the initial guess on entry and the solution on exit.
 * Returns 0 on convergence, 1 if max_iter was reached, 2 on breakdown.
 * iters_out: iterations taken; cw_out: final componentwise residual of the
 * true residual.  nthreads <= 0 keeps the OpenMP default.
 */
int oracle_pcg(int64_t n, const int64_t *ip, const int64_t *ix, const double *v,
               const double *b, double *x, double tol, int64_t max_iter,
               int64_t min_iter, int nthreads, int64_t *iters_out,
               double *cw_out) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  double *d = (double *)malloc(sizeof(double) * n);
  double *r = (double *)malloc(sizeof(double) * n);
  double *z = (double *)malloc(sizeof(double) * n);
  double *p = (double *)malloc(sizeof(double) * n);
  double *q = (double *)malloc(sizeof(double) * n);
  int status = 1;
  int64_t it = 0;
  double cw = INFINITY;
  if (!d || !r || !z || !p || !q) {
    status = 3;
    goto done;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    d[i] = 0.0;
    for (int64_t k = ip[i]; k < ip[i + 1]; ++k)
      if (ix[k] == i) d[i] = v[k];
  }
  for (;;) {
    /* (re)start from the true residual */
    spmv(n, ip, ix, v, x, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      r[i] = b[i] - q[i];
      z[i] = r[i] / d[i];
      p[i] = z[i];
    }
    cw = cw_max(n, r, d, x);
    if (cw <= tol && it >= min_iter) {
      status = 0;
      break;
    }
    if (it >= max_iter) {
      status = 1;
      break;
    }
    double rho = dot(n, r, z);
    int restart = 0;
    while (it < max_iter) {
      spmv(n, ip, ix, v, p, q);
      double pq = dot(n, p, q);
      if (!(pq > 0.0) || !isfinite(pq)) {
        /* rho == 0 exactly means the residual vanished: let the true
           residual decide; otherwise it is a breakdown */
        if (rho == 0.0) {
          restart = 1;
          break;
        }
        status = 2;
        goto done;
      }
      double alpha = rho / pq;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
        z[i] = r[i] / d[i];
      }
      ++it;
      double rho_new = dot(n, r, z);
      if (it >= min_iter && cw_max(n, r, d, x) <= tol) {
        restart = 1;
        break;
      }
      double beta = rho_new / rho;
      rho = rho_new;
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    if (!restart) {
      /* max_iter reached inside the loop: report the true residual */
      spmv(n, ip, ix, v, x, q);
#pragma omp parallel for schedule(static)
      for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
      cw = cw_max(n, r, d, x);
      status = (cw <= tol) ? 0 : 1;
      break;
    }
  }
done:
  if (iters_out) *iters_out = it;
  if (cw_out) *cw_out = cw;
  free(d);
  free(r);
  free(z);
  free(p);
  free(q);
  return status;
}
