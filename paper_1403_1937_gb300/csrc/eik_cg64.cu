// FP64 kernels: setup of the scaled operator, true residual, the two CG
// passes, and the log epilogue.
//
// Operator (Sec. 4 Eq. phiEquation discretised as in Sec. 6 Eq.
// sparse-system, zero-flux half-cell faces) in Jacobi-scaled form, see
// eik_internal.cuh.  One CG iteration is two passes over the grid because CG
// needs two global inner products per iteration:
//   pass 1 (halo-staged stencil): ptil = rhat + beta*phat on the tile and its
//          halo, qhat = Ahat ptil, partial <ptil, qhat>; writes qhat.
//          The last block forms alpha = rho / <p, q>.
//   pass 2 (streaming): phat = rhat + beta*phat (same rounding as pass 1),
//          xh += alpha*phat, rhat -= alpha*qhat, partial <rhat, rhat> and the
//          componentwise test |rhat_i| <= tol*xh_i; the last block forms
//          beta and decides convergence.
// p is not written by pass 1 because neighbouring tiles still read the old p
// in their halos during that pass.
#include <math.h>

#include "eik_internal.cuh"
#include "eik_launch.h"

namespace eik {

constexpr int kCheckEvery = 4;   // iterations between componentwise tests

// ------------------------------------------------------------------ setup
__global__ void k_setup64(Grid g, const double *__restrict__ f,
                          double *__restrict__ sig, double *__restrict__ x,
                          int *__restrict__ err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
       i += stride) {
    const int ix = (int)(i % g.nx);
    const int64_t t = i / g.nx;
    const int iy = (int)(t % g.ny);
    const int iz = (int)(t / g.ny);
    const double hx = half_if(on_face(ix, g.nx, g.boundary));
    const double hy = half_if(on_face(iy, g.ny, g.boundary));
    const double hz = (g.ndim == 3) ? half_if(on_face(iz, g.nz, g.boundary)) : 1.0;
    const double sx = (double)((ix > 0) + (ix < g.nx - 1));
    const double sy = (double)((iy > 0) + (iy < g.ny - 1));
    const double sz = (g.ndim == 3) ? (double)((iz > 0) + (iz < g.nz - 1)) : 0.0;
    // sum of edge weights: x-edges carry hy*hz, y-edges hx*hz, z-edges hx*hy
    const double om = sx * hy * hz + sy * hx * hz + sz * hx * hy;
    const double fi = f[i];
    if (!(fi > 0.0) || !isfinite(fi)) atomicOr(err, 1);
    const double a = hx * hy * hz * fi * fi + g.c * om;
    sig[i] = sqrt(g.c / a);
    x[i] = 0.0;
  }
}

// Sources: sig = 0 and the slot holds sqrt(c) * exp(-(U - U_min)/hbar).
__global__ void k_sources64(Grid g, const int64_t *__restrict__ src,
                            const double *__restrict__ U, int64_t nsrc,
                            double *__restrict__ sig, double *__restrict__ x) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nsrc) {
    const int64_t j = src[k];
    sig[j] = 0.0;
    x[j] = g.sqrt_c * exp(-(U[k] - g.U_min) / g.hbar);
  }
}

// --------------------------------------------------------- tile utilities
template <int DIM>
__device__ __forceinline__ void tile_origin(const TileCount &tc, int64_t t,
                                            int &x0, int &y0, int &z0) {
  using T = Tile<DIM>;
  const int bx = (int)(t % tc.tx);
  const int64_t r = t / tc.tx;
  const int by = (int)(r % tc.ty);
  const int bz = (int)(r / tc.ty);
  x0 = bx * T::TX;
  y0 = by * T::TY;
  z0 = bz * T::TZ;
}

// Weighted neighbour sum for the interior node at halo index s.
template <int DIM>
__device__ __forceinline__ double nb_sum(const double *u, int s, const Grid &g,
                                         int gx, int gy, int gz) {
  using T = Tile<DIM>;
  const double hx = half_if(on_face(gx, g.nx, g.boundary));
  const double hy = half_if(on_face(gy, g.ny, g.boundary));
  if (DIM == 2) {
    return hy * (u[s - 1] + u[s + 1]) + hx * (u[s - T::HX] + u[s + T::HX]);
  } else {
    const double hz = half_if(on_face(gz, g.nz, g.boundary));
    constexpr int PL = T::HX * T::HY;
    return hy * hz * (u[s - 1] + u[s + 1]) + hx * hz * (u[s - T::HX] + u[s + T::HX]) +
           hx * hy * (u[s - PL] + u[s + PL]);
  }
}

// Unweighted neighbour sum (no node of the tile lies on a face).
template <int DIM>
__device__ __forceinline__ double nb_sum_plain(const double *u, int s) {
  using T = Tile<DIM>;
  if (DIM == 2) return (u[s - 1] + u[s + 1]) + (u[s - T::HX] + u[s + T::HX]);
  constexpr int PL = T::HX * T::HY;
  return ((u[s - 1] + u[s + 1]) + (u[s - T::HX] + u[s + T::HX])) + (u[s - PL] + u[s + PL]);
}

// ---------------------------------------------------------- true residual
// rhat = bhat - Ahat xh = sig_i sum_j omega_ij u_j - xh_i with
// u_j = sig_j xh_j (unknowns) or the source slot xh_j (sources).
// An optional extra right-hand side rhs (the adjoint solve) is added to
// bhat.  Also resets phat = 0, and reduces <rhat,rhat>, <bhat,bhat>, the
// unscaled ||r||^2, ||b||^2 and the componentwise max.
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_residual64(Grid g, TileCount tc, const double *__restrict__ sig,
             const double *__restrict__ x, const double *__restrict__ rhs,
             double *__restrict__ r,
             double *__restrict__ p, CgState *st, double *part, int nblk_part) {
  using T = Tile<DIM>;
  constexpr int HN = T::HX * T::HY * T::HZ;
  constexpr int TN = T::TX * T::TY * T::TZ;
  __shared__ double su[HN];
  __shared__ double sb[HN];
  __shared__ double red[32];
  __shared__ int flag;
  double a_rr = 0.0, a_bb = 0.0, a_r2 = 0.0, a_b2 = 0.0, a_cw = 0.0;
  for (int64_t t = blockIdx.x; t < tc.total; t += gridDim.x) {
    int x0, y0, z0;
    tile_origin<DIM>(tc, t, x0, y0, z0);
    for (int s = threadIdx.x; s < HN; s += blockDim.x) {
      const int hx = s % T::HX;
      const int hy = (s / T::HX) % T::HY;
      const int hz = s / (T::HX * T::HY);
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      const int gz = (DIM == 3) ? z0 - 1 + hz : 0;
      double u = 0.0, ub = 0.0;
      if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz) {
        const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
        const double sj = sig[gi], xj = x[gi];
        if (sj == 0.0) {
          u = xj;
          ub = xj;
        } else {
          u = sj * xj;
        }
      }
      su[s] = u;
      sb[s] = ub;
    }
    __syncthreads();
    for (int lin = threadIdx.x; lin < TN; lin += blockDim.x) {
      const int lx = lin % T::TX;
      const int ly = (lin / T::TX) % T::TY;
      const int lz = lin / (T::TX * T::TY);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      if (gx >= g.nx || gy >= g.ny || gz >= g.nz) continue;
      const int s = (DIM == 3 ? (lz + 1) * T::HX * T::HY : 0) + (ly + 1) * T::HX + lx + 1;
      const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
      const double si = sig[gi], xi = x[gi];
      double rh = 0.0, bh = 0.0, cw = 0.0;
      if (si != 0.0) {
        const double ex = rhs ? rhs[gi] : 0.0;
        rh = si * nb_sum<DIM>(su, s, g, gx, gy, gz) - xi + ex;
        bh = si * nb_sum<DIM>(sb, s, g, gx, gy, gz) + ex;
        const double sa = g.sqrt_c / si;   // sqrt(a_i)
        a_r2 += (rh * sa) * (rh * sa);
        a_b2 += (bh * sa) * (bh * sa);
        cw = (xi > 0.0) ? fabs(rh) / xi : INFINITY;
      }
      r[gi] = rh;
      p[gi] = 0.0;
      a_rr += rh * rh;
      a_bb += bh * bh;
      a_cw = fmax(a_cw, cw);
    }
    __syncthreads();
  }
  double v;
  v = block_sum(a_rr, red);
  if (threadIdx.x == 0) part[0 * nblk_part + blockIdx.x] = v;
  v = block_sum(a_bb, red);
  if (threadIdx.x == 0) part[1 * nblk_part + blockIdx.x] = v;
  v = block_sum(a_r2, red);
  if (threadIdx.x == 0) part[2 * nblk_part + blockIdx.x] = v;
  v = block_sum(a_b2, red);
  if (threadIdx.x == 0) part[3 * nblk_part + blockIdx.x] = v;
  v = block_max(a_cw, red);
  if (threadIdx.x == 0) part[4 * nblk_part + blockIdx.x] = v;
  if (!last_block(&st->counter[0], &flag)) return;
  const double rr = sum_partials(part + 0 * nblk_part, gridDim.x, red);
  const double bb = sum_partials(part + 1 * nblk_part, gridDim.x, red);
  const double r2 = sum_partials(part + 2 * nblk_part, gridDim.x, red);
  const double b2 = sum_partials(part + 3 * nblk_part, gridDim.x, red);
  const double cw = max_partials(part + 4 * nblk_part, gridDim.x, red);
  if (threadIdx.x == 0) {
    st->rho = rr;
    st->bnorm2 = bb;
    st->res_nw2_r = r2;
    st->res_nw2_b = b2;
    st->res_cw = cw;
    st->beta = 0.0;
    st->counter[0] = 0u;
  }
}

// --------------------------------------------------------------- pass 1
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_pass1_64(Grid g, TileCount tc, const double *__restrict__ sig,
           const double *__restrict__ r, const double *__restrict__ p,
           double *__restrict__ q, CgState *st, double *part, int nblk_part) {
  using T = Tile<DIM>;
  constexpr int HN = T::HX * T::HY * T::HZ;
  constexpr int TN = T::TX * T::TY * T::TZ;
  __shared__ double su[HN];
  __shared__ double sp[HN];
  __shared__ double red[32];
  __shared__ int flag;
  if (st->done) return;
  const double beta = st->beta;
  double acc = 0.0;
  for (int64_t t = blockIdx.x; t < tc.total; t += gridDim.x) {
    int x0, y0, z0;
    tile_origin<DIM>(tc, t, x0, y0, z0);
    // tiles that hold no face node need no face weights
    const bool interior = x0 >= 1 && x0 + T::TX <= g.nx - 1 && y0 >= 1 &&
                          y0 + T::TY <= g.ny - 1 &&
                          (DIM == 2 || (z0 >= 1 && z0 + T::TZ <= g.nz - 1));
    for (int s = threadIdx.x; s < HN; s += blockDim.x) {
      const int hx = s % T::HX;
      const int hy = (s / T::HX) % T::HY;
      const int hz = s / (T::HX * T::HY);
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      const int gz = (DIM == 3) ? z0 - 1 + hz : 0;
      double pt = 0.0, u = 0.0;
      if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz) {
        const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
        pt = fma(beta, p[gi], r[gi]);
        u = sig[gi] * pt;
      }
      sp[s] = pt;
      su[s] = u;
    }
    __syncthreads();
    for (int lin = threadIdx.x; lin < TN; lin += blockDim.x) {
      const int lx = lin % T::TX;
      const int ly = (lin / T::TX) % T::TY;
      const int lz = lin / (T::TX * T::TY);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      if (gx >= g.nx || gy >= g.ny || gz >= g.nz) continue;
      const int s = (DIM == 3 ? (lz + 1) * T::HX * T::HY : 0) + (ly + 1) * T::HX + lx + 1;
      const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
      const double pt = sp[s];
      const double nb = interior ? nb_sum_plain<DIM>(su, s) : nb_sum<DIM>(su, s, g, gx, gy, gz);
      const double qv = fma(-sig[gi], nb, pt);
      q[gi] = qv;
      acc = fma(pt, qv, acc);
    }
    __syncthreads();
  }
  const double v = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  if (!last_block(&st->counter[1], &flag)) return;
  const double pq = sum_partials(part, gridDim.x, red);
  if (threadIdx.x == 0) {
    const double rho = st->rho;
    if (pq > 0.0 && isfinite(pq)) {
      st->alpha = rho / pq;
    } else if (rho == 0.0) {
      st->alpha = 0.0;
      st->done = 1;
      st->status = EIK_OK;
    } else {
      st->alpha = 0.0;
      st->done = 1;
      st->status = EIK_ERR_BREAKDOWN;
    }
    st->counter[1] = 0u;
  }
}

// --------------------------------------------------------------- pass 2
__global__ void __launch_bounds__(kThreads)
k_pass2_64(int64_t n, double *__restrict__ x, double *__restrict__ r,
           double *__restrict__ p, const double *__restrict__ q,
           const double *__restrict__ cw_weight, CgState *st, double *part,
           int nblk_part) {
  __shared__ double red[32];
  __shared__ int flag;
  if (st->done) return;
  const double alpha = st->alpha, beta = st->beta, tol = st->tol;
  // the componentwise test costs three FP64 operations per node, so it is
  // evaluated on every kCheckEvery-th iteration only
  const bool check = ((st->iter + 1) % kCheckEvery) == 0;
  const bool cw_stop = (st->stop_norm == EIK_STOP_COMPONENTWISE) && check;
  double acc = 0.0, bad = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double ri = r[i];
    const double pt = fma(beta, p[i], ri);
    const double xn = fma(alpha, pt, x[i]);
    const double rn = fma(-alpha, q[i], ri);
    p[i] = pt;
    x[i] = xn;
    r[i] = rn;
    acc = fma(rn, rn, acc);
    if (cw_stop) {
      if (cw_weight) {
        // weighted absolute test |w_i r_i| <= tol (adjoint solve)
        if (!(fabs(cw_weight[i] * rn) <= tol)) bad = 1.0;
      } else if (!(fabs(rn) <= tol * fabs(xn))) {
        // |x| rather than x > 0: where rounding in the iterate left x <= 0
        // while the recurrence residual is already tiny, the loop ends and
        // the true residual (which counts x <= 0 as unconverged) restarts it
        bad = 1.0;
      }
    }
  }
  double v = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = v;
  v = block_max(bad, red);
  if (threadIdx.x == 0) part[nblk_part + blockIdx.x] = v;
  if (!last_block(&st->counter[2], &flag)) return;
  const double rr = sum_partials(part, gridDim.x, red);
  const double anybad = max_partials(part + nblk_part, gridDim.x, red);
  if (threadIdx.x == 0) {
    const double rho = st->rho;
    st->beta = (rho != 0.0) ? rr / rho : 0.0;
    st->rho = rr;
    st->iter += 1;
    bool conv;
    if (st->stop_norm == EIK_STOP_COMPONENTWISE)
      conv = cw_stop && (anybad == 0.0);
    else
      conv = (rr <= st->tol * st->tol * st->bnorm2);
    if (!isfinite(rr)) {
      st->done = 1;
      st->status = EIK_ERR_BREAKDOWN;
    } else if (conv) {
      st->done = 1;
      st->status = EIK_OK;
    } else if (st->iter >= st->max_iter) {
      st->done = 1;
      st->status = EIK_ERR_NOT_CONVERGED;
    }
    st->counter[2] = 0u;
  }
}

// -------------------------------------------------------------- epilogue
// S = U_min - hbar log(phi'), phi' = s_i xh_i = sig_i xh_i / sqrt(c)
// (Sec. 4 Eq. SfromPhi); sources are overwritten with U afterwards.
__global__ void k_epilogue64(Grid g, const double *__restrict__ sig,
                             const double *__restrict__ x, double *__restrict__ S,
                             double *__restrict__ phi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const double inv_sqrt_c = 1.0 / g.sqrt_c;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
    const double si = sig[i], xi = x[i];
    const double ph = ((si == 0.0) ? xi : si * xi) * inv_sqrt_c;
    S[i] = g.U_min - g.hbar * log(ph);
    if (phi) phi[i] = ph;
  }
}

__global__ void k_source_values(const int64_t *__restrict__ src,
                                const double *__restrict__ U, int64_t nsrc,
                                double *__restrict__ S) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nsrc) S[src[k]] = U[k];
}

// --------------------------------------------------------------- adjoint
// Right-hand side of the scaled adjoint system Ahat lamh = ghat with
// ghat_i = s_i g_i, g = dL/dphi = -hbar (dL/dS)/phi, phi_i = s_i xh_i, so
// ghat_i = -hbar (dL/dS)_i / xh_i (zero on the sources).  Each block also
// writes max_i |hbar (dL/dS)_i| over its unknowns (the scale of the
// right-hand side in the variables mu = xh * lamh).
__global__ void k_adjoint_rhs64(Grid g, const double *__restrict__ sig,
                                const double *__restrict__ x,
                                const double *__restrict__ dLdS,
                                double *__restrict__ ghat, double *gmax_part) {
  __shared__ double red[32];
  double m = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
    double v = 0.0;
    if (sig[i] != 0.0) {
      const double d = g.hbar * dLdS[i];
      v = -d / x[i];
      m = fmax(m, fabs(d));
    }
    ghat[i] = v;
  }
  m = block_max(m, red);
  if (threadIdx.x == 0) gmax_part[blockIdx.x] = m;
}

// dL/df_i = -2 w_i f_i phi_i lambda_i = -2 w_i f_i xh_i lamh_i / a_i,
// 1/a_i = sig_i^2 / c; zero on the sources.
__global__ void k_adjoint_grad64(Grid g, const double *__restrict__ f,
                                 const double *__restrict__ sig,
                                 const double *__restrict__ x,
                                 const double *__restrict__ lam,
                                 double *__restrict__ dLdf) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += stride) {
    const int ix = (int)(i % g.nx);
    const int64_t t = i / g.nx;
    const int iy = (int)(t % g.ny);
    const int iz = (int)(t / g.ny);
    const double w = half_if(on_face(ix, g.nx, g.boundary)) *
                     half_if(on_face(iy, g.ny, g.boundary)) *
                     ((g.ndim == 3) ? half_if(on_face(iz, g.nz, g.boundary)) : 1.0);
    const double si = sig[i];
    double v = 0.0;
    if (si != 0.0) v = -2.0 * w * f[i] * x[i] * lam[i] * (si * si / g.c);
    dLdf[i] = v;
  }
}

// -------------------------------------------------------- host launchers
static inline int blocks_for(int64_t n, int cap) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

TileCount tile_count(const Grid &g) {
  TileCount tc;
  if (g.ndim == 2) {
    tc.tx = (g.nx + Tile<2>::TX - 1) / Tile<2>::TX;
    tc.ty = (g.ny + Tile<2>::TY - 1) / Tile<2>::TY;
    tc.tz = 1;
  } else {
    tc.tx = (g.nx + Tile<3>::TX - 1) / Tile<3>::TX;
    tc.ty = (g.ny + Tile<3>::TY - 1) / Tile<3>::TY;
    tc.tz = (g.nz + Tile<3>::TZ - 1) / Tile<3>::TZ;
  }
  tc.total = (int64_t)tc.tx * tc.ty * tc.tz;
  return tc;
}

int stencil_grid_cap(int ndim, int num_sms) {
  int per_sm = 0;
  if (ndim == 2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass1_64<2>, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pass1_64<3>, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms;
}

void launch_setup64(const Grid &g, const double *f, double *sig, double *x, int *err,
                    cudaStream_t s, int cap) {
  k_setup64<<<blocks_for(g.n, cap), kThreads, 0, s>>>(g, f, sig, x, err);
}

void launch_sources64(const Grid &g, const int64_t *src, const double *U, int64_t nsrc,
                      double *sig, double *x, cudaStream_t s) {
  const int b = (int)((nsrc + kThreads - 1) / kThreads);
  k_sources64<<<b, kThreads, 0, s>>>(g, src, U, nsrc, sig, x);
}

void launch_residual64(const Grid &g, const TileCount &tc, int nblk, const double *sig,
                       const double *x, const double *rhs, double *r, double *p,
                       CgState *st, double *part, int nblk_part, cudaStream_t s) {
  if (g.ndim == 2)
    k_residual64<2><<<nblk, kThreads, 0, s>>>(g, tc, sig, x, rhs, r, p, st, part, nblk_part);
  else
    k_residual64<3><<<nblk, kThreads, 0, s>>>(g, tc, sig, x, rhs, r, p, st, part, nblk_part);
}

void launch_pass1_64(const Grid &g, const TileCount &tc, int nblk, const double *sig,
                     const double *r, const double *p, double *q, CgState *st,
                     double *part, int nblk_part, cudaStream_t s) {
  if (g.ndim == 2)
    k_pass1_64<2><<<nblk, kThreads, 0, s>>>(g, tc, sig, r, p, q, st, part, nblk_part);
  else
    k_pass1_64<3><<<nblk, kThreads, 0, s>>>(g, tc, sig, r, p, q, st, part, nblk_part);
}

void launch_pass2_64(int64_t n, int nblk, double *x, double *r, double *p, const double *q,
                     const double *cw_weight, CgState *st, double *part, int nblk_part,
                     cudaStream_t s) {
  k_pass2_64<<<nblk, kThreads, 0, s>>>(n, x, r, p, q, cw_weight, st, part, nblk_part);
}

void launch_epilogue64(const Grid &g, const double *sig, const double *x, double *S,
                       double *phi, cudaStream_t s, int cap) {
  k_epilogue64<<<blocks_for(g.n, cap), kThreads, 0, s>>>(g, sig, x, S, phi);
}

void launch_adjoint_rhs64(const Grid &g, const double *sig, const double *x,
                          const double *dLdS, double *ghat, double *gmax_part, int nblk,
                          cudaStream_t s) {
  k_adjoint_rhs64<<<nblk, kThreads, 0, s>>>(g, sig, x, dLdS, ghat, gmax_part);
}

void launch_adjoint_grad64(const Grid &g, const double *f, const double *sig,
                           const double *x, const double *lam, double *dLdf,
                           cudaStream_t s, int cap) {
  k_adjoint_grad64<<<blocks_for(g.n, cap), kThreads, 0, s>>>(g, f, sig, x, lam, dLdf);
}

void launch_source_values(const int64_t *src, const double *U, int64_t nsrc, double *S,
                          cudaStream_t s) {
  const int b = (int)((nsrc + kThreads - 1) / kThreads);
  k_source_values<<<b, kThreads, 0, s>>>(src, U, nsrc, S);
}

}  // namespace eik
