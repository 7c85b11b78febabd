// Gradient of S and backtracking of optimal paths (path-planning section,
// Eq. PathPlanning-backTrackOnS): a path from a target point solves
// dx/dt = -grad S / |grad S| and ends once it is within eps of a source.
//
// Discretisation (the paper gives none):
// * grad S at the nodes: (S[k+1] - S[k-1]) / (2h) inside, one-sided
//   (S[1] - S[0]) / h and (S[n-1] - S[n-2]) / h on the faces;
// * between nodes: multilinear interpolation of the nodal gradient in the
//   cell holding the point (cells clamped to the grid);
// * explicit Euler steps of fixed arc length, x <- clamp(x - step g/|g|),
//   preceded by the stop tests: distance to the nearest source < eps
//   (status 0), |g| zero or not finite (status 2); status 1 after max_steps.
// One thread per path.  The arithmetic is written with explicitly rounded
// operations (no fused multiply-add), in the order stated above, so a path
// is reproducible on any IEEE machine that evaluates the same steps.
#include <math.h>

#include "eik_internal.cuh"

namespace {

struct Dims3 {
  int n[3];
  int ndim;
  int64_t N;
};

__global__ void k_grad_S(Dims3 d, double h, const double *__restrict__ S,
                         double *__restrict__ G) {
  const int64_t sx = 1, sy = d.n[0], sz = (int64_t)d.n[0] * d.n[1];
  const int64_t st[3] = {sx, sy, sz};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k[3] = {(int)(i % d.n[0]), (int)((i / sy) % d.n[1]),
                      d.ndim == 3 ? (int)(i / sz) : 0};
    for (int a = 0; a < d.ndim; ++a) {
      double g;
      if (k[a] == 0)
        g = __ddiv_rn(__dsub_rn(S[i + st[a]], S[i]), h);
      else if (k[a] == d.n[a] - 1)
        g = __ddiv_rn(__dsub_rn(S[i], S[i - st[a]]), h);
      else
        g = __ddiv_rn(__dsub_rn(S[i + st[a]], S[i - st[a]]), __dmul_rn(2.0, h));
      G[a * d.N + i] = g;
    }
  }
}

__device__ double dist_to_sources(const double *x, int ndim, const int64_t *src, int64_t nsrc,
                                  Dims3 d, double h) {
  double best = INFINITY;
  for (int64_t s = 0; s < nsrc; ++s) {
    int64_t rem = src[s];
    double acc = 0.0;
    for (int a = 0; a < ndim; ++a) {
      const double y = __dmul_rn((double)(rem % d.n[a]), h);
      rem /= d.n[a];
      const double dx = __dsub_rn(x[a], y);
      acc = (a == 0) ? __dmul_rn(dx, dx) : __dadd_rn(acc, __dmul_rn(dx, dx));
    }
    const double r = __dsqrt_rn(acc);
    best = fmin(best, r);
  }
  return best;
}

__global__ void k_backtrack(Dims3 d, double h, const double *__restrict__ G,
                            const double *__restrict__ starts, int64_t npaths, double step,
                            int max_steps, const int64_t *__restrict__ src, int64_t nsrc,
                            double eps, double *__restrict__ paths, int *__restrict__ lengths,
                            int *__restrict__ status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npaths) return;
  const int nd = d.ndim;
  const int64_t stride_p = (int64_t)(max_steps + 1) * nd;
  double *out = paths + p * stride_p;
  double x[3] = {0.0, 0.0, 0.0}, hi[3];
  for (int a = 0; a < nd; ++a) {
    x[a] = starts[p * nd + a];
    hi[a] = __dmul_rn((double)(d.n[a] - 1), h);
    out[a] = x[a];
  }
  const int64_t strides[3] = {1, d.n[0], (int64_t)d.n[0] * d.n[1]};
  int len = 0, stat = 1;
  for (int k = 0; k < max_steps; ++k) {
    if (dist_to_sources(x, nd, src, nsrc, d, h) < eps) {
      stat = 0;
      break;
    }
    // multilinear interpolation of the nodal gradient
    int c[3];
    double t[3];
    for (int a = 0; a < nd; ++a) {
      const double u = __ddiv_rn(x[a], h);
      const double cf = fmin(fmax(floor(u), 0.0), (double)(d.n[a] - 2));
      c[a] = (int)cf;
      t[a] = __dsub_rn(u, cf);
    }
    double g[3] = {0.0, 0.0, 0.0};
    for (int corner = 0; corner < (1 << nd); ++corner) {
      double w = 1.0;
      int64_t idx = 0;
      for (int a = 0; a < nd; ++a) {
        const int bit = (corner >> a) & 1;
        w = __dmul_rn(w, bit ? t[a] : __dsub_rn(1.0, t[a]));
        idx += (int64_t)(c[a] + bit) * strides[a];
      }
      for (int a = 0; a < nd; ++a) g[a] = __dadd_rn(g[a], __dmul_rn(w, G[a * d.N + idx]));
    }
    double gg = __dmul_rn(g[0], g[0]);
    for (int a = 1; a < nd; ++a) gg = __dadd_rn(gg, __dmul_rn(g[a], g[a]));
    const double gn = __dsqrt_rn(gg);
    if (!(gn > 0.0)) {
      stat = 2;
      break;
    }
    ++len;
    for (int a = 0; a < nd; ++a) {
      const double xn = __dsub_rn(x[a], __ddiv_rn(__dmul_rn(step, g[a]), gn));
      x[a] = fmin(fmax(xn, 0.0), hi[a]);
      out[(int64_t)len * nd + a] = x[a];
    }
  }
  if (stat == 1 && dist_to_sources(x, nd, src, nsrc, d, h) < eps) stat = 0;
  for (int64_t k = (int64_t)(len + 1) * nd; k < stride_p; ++k) out[k] = NAN;
  lengths[p] = len;
  status[p] = stat;
}

bool make_dims(int ndim, const int64_t *dims, Dims3 &d) {
  if (ndim != 2 && ndim != 3) return false;
  d.ndim = ndim;
  d.N = 1;
  d.n[0] = d.n[1] = d.n[2] = 1;
  for (int a = 0; a < ndim; ++a) {
    if (dims[a] < 2 || dims[a] > (int64_t)1 << 30) return false;
    d.n[a] = (int)dims[a];
    d.N *= dims[a];
  }
  return true;
}

}  // namespace

extern "C" eik_status eik_grad_S(int ndim, const int64_t *dims, double h, const double *S,
                                 double *gradS, eik_stream_t stream) {
  Dims3 d{};
  if (!dims || !S || !gradS || !(h > 0) || !make_dims(ndim, dims, d)) return EIK_ERR_ARG;
  const int th = 256;
  const int nb = (int)std::min<int64_t>((d.N + th - 1) / th, 152 * 16);
  k_grad_S<<<nb, th, 0, stream>>>(d, h, S, gradS);
  return cudaGetLastError() == cudaSuccess ? EIK_OK : EIK_ERR_CUDA;
}

extern "C" eik_status eik_backtrack(int ndim, const int64_t *dims, double h, const double *gradS,
                                    const double *starts, int64_t npaths, double step,
                                    int max_steps, const int64_t *src_idx, int64_t nsrc,
                                    double eps, double *paths, int *lengths, int *status,
                                    eik_stream_t stream) {
  Dims3 d{};
  if (!dims || !(h > 0) || !make_dims(ndim, dims, d)) return EIK_ERR_ARG;
  if (npaths < 0 || nsrc < 0 || max_steps < 0 || !(step > 0) || !(eps >= 0)) return EIK_ERR_ARG;
  if (npaths == 0) return EIK_OK;
  if (!gradS || !starts || !paths || !lengths || !status || (nsrc > 0 && !src_idx))
    return EIK_ERR_ARG;
  const int th = 128;
  k_backtrack<<<(int)((npaths + th - 1) / th), th, 0, stream>>>(
      d, h, gradS, starts, npaths, step, max_steps, src_idx, nsrc, eps, paths, lengths, status);
  return cudaGetLastError() == cudaSuccess ? EIK_OK : EIK_ERR_CUDA;
}

// Shape-from-shading forcing (shape-from-shading section, Eq. SfS-forcingFunc):
// a Lambertian image under vertical light, P = 1/sqrt(|grad S|^2 + 1), gives
// the eikonal forcing f = sqrt(1/P^2 - 1), raised to f_min where smaller
// (flat regions would give f = 0, which eik_create rejects); P outside
// (0, 1] or not finite gives NaN (eik_create rejects it).  Explicitly
// rounded operations, as in the path kernels.
namespace {
__global__ void k_sfs_forcing(const double *__restrict__ P, int64_t n, double f_min,
                              double *__restrict__ f) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double p = P[i];
    double v = NAN;
    if (p > 0.0 && p <= 1.0) {
      const double g = __dsqrt_rn(__dsub_rn(__ddiv_rn(1.0, __dmul_rn(p, p)), 1.0));
      v = fmax(g, f_min);
    }
    f[i] = v;
  }
}
}  // namespace

extern "C" eik_status eik_sfs_forcing(const double *P, int64_t n, double f_min, double *f,
                                      eik_stream_t stream) {
  if (n < 0 || !(f_min >= 0.0) || (n > 0 && (!P || !f))) return EIK_ERR_ARG;
  if (n == 0) return EIK_OK;
  const int th = 256;
  const int nb = (int)std::min<int64_t>((n + th - 1) / th, 152 * 16);
  k_sfs_forcing<<<nb, th, 0, stream>>>(P, n, f_min, f);
  return cudaGetLastError() == cudaSuccess ? EIK_OK : EIK_ERR_CUDA;
}
