// Mixed-precision solve: FP32 inner CG in per-cell exponent units, FP64
// iterative refinement in relative (exponent-scaled) form.
//
// Why the scaling: phi = exp(-S/hbar) spans exp(-max S/hbar), far below the
// FP32 range (and, for S/hbar > ~700, below FP64).  A static power-of-two
// scale per cell of B^d nodes, kx(cell), rounded from a cheap distance
// estimate St ~ S (min-plus relaxation on the coarse cell grid, 16/26-
// neighbour stencil, edge cost = length x mean of the two cell-averaged f),
// keeps every stored number in range: solution-like vectors (the FP64 iterate
// x64, the FP32 correction d, and the inner CG's r and p) are stored as
// hat-value * 2^kx(cell).  All rescaling is by powers of two, so it is exact.
//
// The inner CG (eik_cg32.cu) is the single-reduction form of Jacobi-
// preconditioned CG in these units: one pass over the grid per iteration.  It
// yields accurate values near the sources but not in the far field: CG
// iterates there pass through transients many orders larger than the final
// values, whose cancellation FP32 cannot carry.  Refinement repairs this:
// each outer step forms the true FP64 residual in relative form and solves
// for a correction with a fresh inner CG.
//
// When kx spans more than a few hundred powers of two, no global CG (in any
// precision) resolves the far field: its transients there exceed even the
// FP32 exponent range of the correction.  The solve then sweeps level-set
// bands of kx, nearest first, each refined with the rest of the grid held as
// Dirichlet data (mixed_solve / refine).
#include <cuda.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "eik_batch.h"
#include "eik_cg32.h"
#include "eik_launch.h"
#include "eik_mg.h"
#include "eik_mixed.h"

namespace eik {

namespace {

constexpr int kInnerGraphIters = 32;   // even: the buffer sets alternate
constexpr int kMaxCells = 16384;
// level-set sweep (library choice): bands of kBandBits powers of two of phi,
// used when kx spans more than kSweepBits (measured on 2048^2: 40-bit bands
// took 2696 inner iterations, 48-bit ones 2845, 32-bit ones 3074)
constexpr int kBandBits = 40;
constexpr int kSweepBits = 96;
constexpr int kMaxSweeps = 4;
// first inner solve of a refinement step: reduce the kx-scaled max-norm
// residual by this factor (measured on the 2048^2 and 256^3 workloads:
// 1e-1 took the fewest total iterations among 1e-1 ... 1e-4)
constexpr double kInnerReduction = 1e-1;
constexpr int kMinOverlapBits = 32;    // band overlap (powers of two), at least
constexpr int kGlobalFinishBits = 160; // ranges that a global refinement still handles
// multigrid inner solves: sweep only beyond kMgSweepBits, in bands of
// kMgBandBits (measured: 2048^2 with a 216-bit range converges globally)
constexpr int kMgSweepBits = 256;
constexpr int kMgBandBits = 128;

thread_local std::string g_msg = "no error";   // per host thread (batches)

// ------------------------------------------------------------ exponents
__device__ __forceinline__ double pow2d(int n) {
  if (n < -1022) return 0.0;
  if (n > 1023) n = 1023;
  return __longlong_as_double((long long)(n + 1023) << 52);
}

// (mantissa, exponent) accumulator: value = m * 2^s.
struct Acc64 {
  double m;
  int s;
};
__device__ __forceinline__ void acc_add(Acc64 &a, double m, int t) {
  if (m == 0.0) return;
  if (a.m == 0.0) {
    a.m = m;
    a.s = t;
  } else if (t > a.s) {
    a.m = a.m * pow2d(a.s - t) + m;
    a.s = t;
  } else {
    a.m += m * pow2d(t - a.s);
  }
  // keep the mantissa near 1 so long sums cannot overflow
  if (a.m != 0.0) {
    int e;
    const double fr = frexp(a.m, &e);
    a.m = fr;
    a.s += e;
  }
}
// Deterministic block combine of Acc64 (valid in thread 0).
__device__ Acc64 block_acc(Acc64 v, double *shm, int *shs) {
  for (int o = 16; o > 0; o >>= 1) {
    const double m = __shfl_down_sync(0xffffffffu, v.m, o);
    const int s = __shfl_down_sync(0xffffffffu, v.s, o);
    acc_add(v, m, s);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    shm[w] = v.m;
    shs[w] = v.s;
  }
  __syncthreads();
  Acc64 r{0.0, 0};
  if (w == 0) {
    if (l < (int)(blockDim.x >> 5)) r = Acc64{shm[l], shs[l]};
    for (int o = 16; o > 0; o >>= 1) {
      const double m = __shfl_down_sync(0xffffffffu, r.m, o);
      const int s = __shfl_down_sync(0xffffffffu, r.s, o);
      acc_add(r, m, s);
    }
  }
  return r;
}
// Fixed-order combine of per-block Acc64 partials (m in pm, s in ps).
__device__ Acc64 sum_acc_partials(const double *pm, const double *ps, int nblk, double *shm,
                                  int *shs) {
  Acc64 v{0.0, 0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc_add(v, __ldcg(pm + b), (int)__ldcg(ps + b));
  return block_acc(v, shm, shs);
}


__device__ __forceinline__ int cell_of(const CellGrid &cg, int x, int y, int z) {
  return (x >> cg.lgB) + cg.cx * ((y >> cg.lgB) + cg.cy * (z >> cg.lgB));
}

template <int DIM>
__device__ __forceinline__ void tile_origin_m(const TileCount &tc, int64_t t, int &x0, int &y0,
                                              int &z0) {
  using T = Tile<DIM>;
  const int bx = (int)(t % tc.tx);
  const int64_t r = t / tc.tx;
  x0 = bx * T::TX;
  y0 = (int)(r % tc.ty) * T::TY;
  z0 = (int)(r / tc.ty) * T::TZ;
}

// ----------------------------------------------------------- setup kernels
// The FP32 / int16 inner-CG arrays use a row pitch px >= nx (a multiple of 8
// where the TMA kernels run, so their rows are 16-byte aligned); the FP64
// arrays are dense.  pidx maps a dense index to the pitched one.
__device__ __forceinline__ int64_t pidx(int64_t i, int nx, int px) {
  return (px == nx) ? i : (i / nx) * px + (i % nx);
}

__global__ void k_sig32(int64_t n, int nx, int px, const double *__restrict__ sig,
                        float *__restrict__ s32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s32[pidx(i, nx, px)] = (float)sig[i];
}

// s32 for one level-set band: sigma where band_lo <= kx(cell) < band_hi, 0
// elsewhere (those nodes then act as Dirichlet data in the inner CG).
__global__ void k_sig32_band(Grid g, int px, CellGrid cg, const int *__restrict__ kx, int lo,
                             int hi, const double *__restrict__ sig, float *__restrict__ s32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx);
    const int64_t t = i / g.nx;
    const int y = (int)(t % g.ny), z = (int)(t / g.ny);
    const int k = kx[cell_of(cg, x, y, z)];
    s32[t * px + x] = (k >= lo && k < hi) ? (float)sig[i] : 0.f;
  }
}

// Mean of f over each cell (one block per cell).
__global__ void k_cell_mean(Grid g, CellGrid cg, const double *__restrict__ f,
                            float *__restrict__ fb) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const int I = c % cg.cx, J = (c / cg.cx) % cg.cy, K = c / (cg.cx * cg.cy);
  const int x0 = I * cg.B, y0 = J * cg.B, z0 = K * cg.B;
  const int x1 = min(x0 + cg.B, g.nx), y1 = min(y0 + cg.B, g.ny);
  const int z1 = (g.ndim == 3) ? min(z0 + cg.B, g.nz) : 1;
  const int wx = x1 - x0, wy = y1 - y0, wz = z1 - z0;
  const int cnt = wx * wy * wz;
  double s = 0.0;
  for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
    const int lx = k % wx, ly = (k / wx) % wy, lz = k / (wx * wy);
    s += f[(x0 + lx) + (int64_t)g.nx * ((y0 + ly) + (int64_t)g.ny * (z0 + lz))];
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) fb[c] = (float)(s / cnt);
}

// Distance estimate St on the cell grid by min-plus relaxation, then the
// cell exponents kx = round(St / (hbar ln 2)).  One block; the cell grid is in
// shared memory.  Converges in at most ncell sweeps (Bellman-Ford bound).
__global__ void __launch_bounds__(1024)
k_coarse_exponents(Grid g, CellGrid cg, double h, const float *__restrict__ fb_g,
                   const int64_t *__restrict__ src, const double *__restrict__ U,
                   int64_t nsrc, int *__restrict__ kx, float *__restrict__ St_out) {
  extern __shared__ float smem[];
  float *St = smem;
  float *fb = smem + cg.ncell;
  const int nc = cg.ncell;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    St[c] = INFINITY;
    fb[c] = fb_g[c];
  }
  __syncthreads();
  const float H = (float)(h * cg.B);
  const int R = 2;
  const int span = (g.ndim == 3) ? (2 * R + 1) * (2 * R + 1) * (2 * R + 1) : (2 * R + 1) * (2 * R + 1);
  for (int64_t w = threadIdx.x; w < nsrc * span; w += blockDim.x) {
    const int64_t k = w / span;
    const int o = (int)(w % span);
    const int64_t j = src[k];
    const int sx = (int)(j % g.nx);
    const int sy = (int)((j / g.nx) % g.ny);
    const int sz = (int)(j / ((int64_t)g.nx * g.ny));
    const int dI = o % (2 * R + 1) - R, dJ = (o / (2 * R + 1)) % (2 * R + 1) - R;
    const int dK = (g.ndim == 3) ? o / ((2 * R + 1) * (2 * R + 1)) - R : 0;
    const int I = (sx >> cg.lgB) + dI, J = (sy >> cg.lgB) + dJ, K = (sz >> cg.lgB) + dK;
    if (I < 0 || I >= cg.cx || J < 0 || J >= cg.cy || K < 0 || K >= cg.cz) continue;
    const float cxp = fminf(I * cg.B + 0.5f * (cg.B - 1), (float)(g.nx - 1));
    const float cyp = fminf(J * cg.B + 0.5f * (cg.B - 1), (float)(g.ny - 1));
    const float czp = (g.ndim == 3) ? fminf(K * cg.B + 0.5f * (cg.B - 1), (float)(g.nz - 1)) : 0.f;
    const float dx = cxp - sx, dy = cyp - sy, dz = czp - sz;
    const int c = I + cg.cx * (J + cg.cy * K);
    const float v = (float)(U[k] - g.U_min) + fb[c] * (float)h * sqrtf(dx * dx + dy * dy + dz * dz);
    atomicMin((int *)&St[c], __float_as_int(fmaxf(v, 0.f)));
  }
  __syncthreads();
  // neighbour offsets: 2D axis + diagonal + knight (16); 3D the 26 of the cube
  for (int sweep = 0; sweep <= nc + 1; ++sweep) {
    int changed = 0;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      const int I = c % cg.cx, J = (c / cg.cx) % cg.cy, K = c / (cg.cx * cg.cy);
      float best = St[c];
      const float fc = fb[c];
      if (g.ndim == 2) {
        const int off[16][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {1, -1},
                                {-1, 1}, {-1, -1}, {1, 2}, {2, 1}, {-1, 2}, {-2, 1},
                                {1, -2}, {2, -1}, {-1, -2}, {-2, -1}};
        for (int q = 0; q < 16; ++q) {
          const int I2 = I + off[q][0], J2 = J + off[q][1];
          if (I2 < 0 || I2 >= cg.cx || J2 < 0 || J2 >= cg.cy) continue;
          const int c2 = I2 + cg.cx * J2;
          const float len = sqrtf((float)(off[q][0] * off[q][0] + off[q][1] * off[q][1]));
          best = fminf(best, St[c2] + H * len * 0.5f * (fc + fb[c2]));
        }
      } else {
        for (int q = 0; q < 27; ++q) {
          const int a = q % 3 - 1, b = (q / 3) % 3 - 1, d = q / 9 - 1;
          if (!a && !b && !d) continue;
          const int I2 = I + a, J2 = J + b, K2 = K + d;
          if (I2 < 0 || I2 >= cg.cx || J2 < 0 || J2 >= cg.cy || K2 < 0 || K2 >= cg.cz) continue;
          const int c2 = I2 + cg.cx * (J2 + cg.cy * K2);
          const float len = sqrtf((float)(a * a + b * b + d * d));
          best = fminf(best, St[c2] + H * len * 0.5f * (fc + fb[c2]));
        }
      }
      if (best < St[c]) {
        St[c] = best;
        changed = 1;
      }
    }
    if (!__syncthreads_or(changed)) break;
  }
  const float inv = (float)(1.0 / (g.hbar * 0.69314718055994530942));
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const float v = St[c];
    kx[c] = isfinite(v) ? (int)rintf(v * inv) : 0;
    if (St_out) St_out[c] = v;
  }
}

// FP64 iterate: 0 on the unknowns, the shifted source values in kx units on
// the sources: sqrt(c) phi_k 2^kx = sqrt(c) exp(kx ln2 - (U_k - U_min)/hbar).
__global__ void k_init_x64(Grid g, CellGrid cg, const int *__restrict__ kx,
                           const int64_t *__restrict__ src, const double *__restrict__ U,
                           int64_t nsrc, double *__restrict__ x64) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nsrc) return;
  const int64_t j = src[k];
  const int sx = (int)(j % g.nx), sy = (int)((j / g.nx) % g.ny);
  const int sz = (int)(j / ((int64_t)g.nx * g.ny));
  const int kk = kx[cell_of(cg, sx, sy, sz)];
  x64[j] = g.sqrt_c * exp(kk * 0.69314718055994530942 - (U[k] - g.U_min) / g.hbar);
}


// ----------------------------------------- FP64 residual in relative form
// rbar_i = sig_i sum_j omega_ij 2^(kx_i - kx_j) u_j - xbar_i (kx units),
// u_j = sig_j xbar_j (unknowns) or the source slot xbar_j.  Also starts the
// inner CG: r = rbar (FP32, frame 0) in buffer set 0, p = 0, d = 0, the FP32
// copy xref of the iterate, and reduces rho = <rbar, rbar> with the weights
// 2^(-2 kx), the componentwise residual max |rbar|/xbar, max |rbar| and
// max |xbar| (kx units).  Unknowns outside the level-set band
// [band_lo, band_hi) of kx are held as Dirichlet data (residual 0).
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_mixed_residual(Grid g, TileCount tc, CellGrid cg, const int *__restrict__ kx,
                 const double *__restrict__ sig, const double *__restrict__ x64,
                 float *__restrict__ r32, float *__restrict__ p32, float *__restrict__ d32,
                 float *__restrict__ xref, MixCtl *st, double *part, int nblk_part, int px) {
  using T = Tile<DIM>;
  constexpr int HN = T::HX * T::HY * T::HZ;
  constexpr int TN = T::TX * T::TY * T::TZ;
  __shared__ double su[HN];
  __shared__ int sk[HN];
  __shared__ double shm[32];
  __shared__ int shs[32];
  __shared__ int flag;
  Acc64 rho{0.0, 0};
  double cwm = 0.0, rinf = 0.0, xinf = 0.0;
  const int band_lo = st->band_lo, band_hi = st->band_hi;
  for (int64_t t = blockIdx.x; t < tc.total; t += gridDim.x) {
    int x0, y0, z0;
    tile_origin_m<DIM>(tc, t, x0, y0, z0);
    for (int s = threadIdx.x; s < HN; s += blockDim.x) {
      const int hx = s % T::HX, hy = (s / T::HX) % T::HY, hz = s / (T::HX * T::HY);
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = (DIM == 3) ? z0 - 1 + hz : 0;
      double u = 0.0;
      int kk = 0;
      if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz) {
        const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
        const double sj = sig[gi], xj = x64[gi];
        u = (sj == 0.0) ? xj : sj * xj;
        kk = kx[cell_of(cg, gx, gy, gz)];
      }
      su[s] = u;
      sk[s] = kk;
    }
    __syncthreads();
    for (int lin = threadIdx.x; lin < TN; lin += blockDim.x) {
      const int lx = lin % T::TX, ly = (lin / T::TX) % T::TY, lz = lin / (T::TX * T::TY);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      if (gx >= g.nx || gy >= g.ny || gz >= g.nz) continue;
      const int s = (DIM == 3 ? (lz + 1) * T::HX * T::HY : 0) + (ly + 1) * T::HX + lx + 1;
      const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
      const double si = sig[gi], xi = x64[gi];
      const int ki = sk[s];
      double rb = 0.0;
      if (si != 0.0 && ki >= band_lo && ki < band_hi) {
        const double hx = half_if(on_face(gx, g.nx, g.boundary));
        const double hy = half_if(on_face(gy, g.ny, g.boundary));
        double acc;
        if (DIM == 2) {
          acc = hy * (su[s - 1] * pow2d(ki - sk[s - 1]) + su[s + 1] * pow2d(ki - sk[s + 1])) +
                hx * (su[s - T::HX] * pow2d(ki - sk[s - T::HX]) +
                      su[s + T::HX] * pow2d(ki - sk[s + T::HX]));
        } else {
          const double hz = half_if(on_face(gz, g.nz, g.boundary));
          constexpr int PL = T::HX * T::HY;
          acc = hy * hz * (su[s - 1] * pow2d(ki - sk[s - 1]) + su[s + 1] * pow2d(ki - sk[s + 1])) +
                hx * hz * (su[s - T::HX] * pow2d(ki - sk[s - T::HX]) +
                           su[s + T::HX] * pow2d(ki - sk[s + T::HX])) +
                hx * hy * (su[s - PL] * pow2d(ki - sk[s - PL]) + su[s + PL] * pow2d(ki - sk[s + PL]));
        }
        rb = si * acc - xi;
        const double cw = (xi > 0.0) ? fabs(rb) / xi : INFINITY;
        cwm = fmax(cwm, cw);
        rinf = fmax(rinf, fabs(rb));
        xinf = fmax(xinf, fabs(xi));
        if (rb != 0.0) {
          // <rbar, rbar> with weight 2^(-2 ki): (rb 2^-ki)^2 as (mantissa, exponent)
          int ex;
          const double fr = frexp(rb, &ex);
          acc_add(rho, fr * fr, 2 * (ex - ki));
        }
      }
      const int64_t pi = gx + (int64_t)px * (gy + (int64_t)g.ny * gz);   // pitched
      r32[pi] = (float)rb;
      p32[pi] = 0.f;
      d32[pi] = 0.f;
      xref[pi] = (si != 0.0) ? (float)xi : 0.f;
    }
    __syncthreads();
  }
  const Acc64 tot = block_acc(rho, shm, shs);
  const double c1 = block_max(cwm, shm);
  const double c2 = block_max(rinf, shm);
  const double c3 = block_max(xinf, shm);
  if (threadIdx.x == 0) {
    part[0 * nblk_part + blockIdx.x] = tot.m;
    part[1 * nblk_part + blockIdx.x] = (double)tot.s;
    part[2 * nblk_part + blockIdx.x] = c1;
    part[3 * nblk_part + blockIdx.x] = c2;
    part[4 * nblk_part + blockIdx.x] = c3;
  }
  if (!last_block(&st->counter[0], &flag)) return;
  const Acc64 r = sum_acc_partials(part, part + nblk_part, gridDim.x, shm, shs);
  const double cw = max_partials(part + 2 * nblk_part, gridDim.x, shm);
  const double ri = max_partials(part + 3 * nblk_part, gridDim.x, shm);
  const double xi = max_partials(part + 4 * nblk_part, gridDim.x, shm);
  if (threadIdx.x == 0) {
    st->rho_m = r.m;
    st->rho_s = r.s;
    st->cw = cw;
    st->r_inf = ri;
    st->x_inf = xi;
    st->counter[0] = 0u;
  }
}

// x64 += d (kx units, unknowns only: d is zero on the sources).
__global__ void k_mixed_update(int64_t n, int nx, int px, const float *__restrict__ d32,
                               double *__restrict__ x64) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = d32[pidx(i, nx, px)];
    if (d != 0.f) x64[i] += (double)d;
  }
}

// S = U_min - hbar log(phi'), phi' = sig xbar 2^-kx / sqrt(c) (Eq. SfromPhi);
// sources are overwritten with U afterwards.
__global__ void k_mixed_epilogue(Grid g, CellGrid cg, const int *__restrict__ kx,
                                 const double *__restrict__ sig,
                                 const double *__restrict__ x64, double *__restrict__ S,
                                 double *__restrict__ phi) {
  const double ln2 = 0.69314718055994530942;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny);
    const int z = (int)(i / ((int64_t)g.nx * g.ny));
    const int kk = kx[cell_of(cg, x, y, z)];
    const double si = sig[i], xi = x64[i];
    const double v = ((si == 0.0) ? xi : si * xi) / g.sqrt_c;   // phi' 2^kx
    const double Sv = g.U_min - g.hbar * (log(v) - kk * ln2);
    S[i] = Sv;
    if (phi) phi[i] = exp(-(Sv - g.U_min) / g.hbar);
  }
}

// Hat-space FP64 solution xh = xbar 2^-kx (sources: sqrt(c) phi_k), for the
// FP64 adjoint after a mixed forward solve.
__global__ void k_mixed_export(Grid g, CellGrid cg, const int *__restrict__ kx,
                               const double *__restrict__ x64, double *__restrict__ xh) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny);
    const int z = (int)(i / ((int64_t)g.nx * g.ny));
    xh[i] = x64[i] * pow2d(-kx[cell_of(cg, x, y, z)]);
  }
}

}  // namespace

// ====================================================================== host
struct MixedState {
  Grid g;
  TileCount tc;
  CellGrid cg;
  int nblk_stencil = 0, nblk_part = 0, cap = 0;
  int px = 0;                        // row pitch of the FP32 arrays (multiple of 4)
  Cg32Plan plan;
  Cg32Buffers bufs;
  float *s32 = nullptr, *fb = nullptr, *St = nullptr, *d32 = nullptr, *xref = nullptr;
  float *r32[2] = {nullptr, nullptr}, *p32[2] = {nullptr, nullptr};
  int *kx = nullptr;
  double *x64 = nullptr, *part = nullptr;
  MixCtl *st = nullptr, *h_st = nullptr;
  // member of a packed batch: the FP32 arrays and st belong to the batch,
  // and inner solves run through it
  BatchExec *batch = nullptr;
  int bidx = -1;
  // multigrid-preconditioned inner solve (EIK_PRECOND_MULTIGRID), else null
  MgState *mg = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t launches[8] = {0};
  // per-launch CUDA-event timing of the inner passes when profiling
  bool profile = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  int64_t timed[8] = {0};
  double ms[8] = {0};
};

static const char *kMixedNames[] = {"mixed_setup", "coarse_exponents", "mixed_residual64",
                                    "mixed_cg_init", "mixed_cg", "mixed_update",
                                    "mixed_epilogue", "mixed_mg", nullptr};

const char *mixed_kernel_name(int k) {
  if (k < 0 || k >= 8) return nullptr;
  return kMixedNames[k];
}

int64_t mixed_kernel_launches(const MixedState *m, int k) {
  if (m && k == 7) return mg_launches(m->mg);
  return (m && k >= 0 && k < 8) ? m->launches[k] : 0;
}

void mixed_reset_launches(MixedState *m) {
  if (!m) return;
  mg_reset(m->mg);
  for (int k = 0; k < 8; ++k) {
    m->launches[k] = 0;
    m->timed[k] = 0;
    m->ms[k] = 0.0;
  }
}

void mixed_set_profiling(MixedState *m, bool on) {
  if (m) m->profile = on;
  if (m) mg_set_profiling(m->mg, on);
}

void mixed_kernel_time(const MixedState *m, int k, int64_t *timed, double *ms) {
  if (m && k == 7) {   // one multigrid-preconditioned iteration (all its kernels)
    mg_time(m->mg, timed, ms);
    return;
  }
  *timed = (m && k >= 0 && k < 8) ? m->timed[k] : 0;
  *ms = (m && k >= 0 && k < 8) ? m->ms[k] : 0.0;
}

const char *mixed_last_error() { return g_msg.c_str(); }

#define MCK(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      g_msg = std::string(#call) + ": " + cudaGetErrorString(e_);        \
      return EIK_ERR_CUDA;                                               \
    }                                                                    \
  } while (0)

template <class T>
static bool mal(T **p, size_t n) {
  return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)) == cudaSuccess;
}

// Cell grid, launch sizes and the FP64 / cell arrays of a solver.
static void mixed_layout(MixedState *m, const Grid &g, const TileCount &tc, int num_sms) {
  m->g = g;
  m->tc = tc;
  // cell edge: power of two >= 16 with at most kMaxCells cells
  for (int lg = 4;; ++lg) {
    const int B = 1 << lg;
    const int64_t cx = (g.nx + B - 1) / B, cy = (g.ny + B - 1) / B;
    const int64_t cz = (g.ndim == 3) ? (g.nz + B - 1) / B : 1;
    if (cx * cy * cz <= kMaxCells) {
      m->cg.B = B;
      m->cg.lgB = lg;
      m->cg.cx = (int)cx;
      m->cg.cy = (int)cy;
      m->cg.cz = (int)cz;
      m->cg.ncell = (int)(cx * cy * cz);
      break;
    }
  }
  int per_sm = 0;
  if (g.ndim == 2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mixed_residual<2>, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mixed_residual<3>, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  m->nblk_stencil = (int)std::min<int64_t>(tc.total, (int64_t)per_sm * num_sms);
  m->cap = num_sms * 8;
  m->nblk_part = std::max(std::max(m->nblk_stencil, m->cap), cg32_max_blocks(g.ndim, num_sms));
}

// The attribute belongs to the function, not to one solver: set it to the
// largest cell grid any solver can use, so concurrent solvers agree.
static bool coarse_smem_attr() {
  const size_t smem = 2 * sizeof(float) * kMaxCells;
  return cudaFuncSetAttribute(k_coarse_exponents, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem) == cudaSuccess;
}

eik_status mixed_create(MixedState **out, const Grid &g, const TileCount &tc, int num_sms,
                        int tile_override, int precond, cudaStream_t s) {
  MixedState *m = new MixedState();
  mixed_layout(m, g, tc, num_sms);
  // row pitch of the FP32 arrays: a multiple of 4 elements (16-byte rows for
  // the tensor maps and the float4 accesses of the inner passes)
  m->px = (g.nx + 3) / 4 * 4;
  const int64_t n = g.n;
  const int64_t np = (g.n / g.nx) * m->px;
  bool ok = mal(&m->s32, np) && mal(&m->d32, np) && mal(&m->xref, np) && mal(&m->r32[0], np) &&
            mal(&m->r32[1], np) && mal(&m->p32[0], np) && mal(&m->p32[1], np) &&
            mal(&m->x64, n) && mal(&m->fb, m->cg.ncell) && mal(&m->St, m->cg.ncell) &&
            mal(&m->kx, m->cg.ncell) && mal(&m->part, 8 * (size_t)m->nblk_part) &&
            mal(&m->st, 1);
  if (ok) ok = cudaMallocHost((void **)&m->h_st, sizeof(MixCtl)) == cudaSuccess;
  if (ok) {
    // padding columns are never read through the tensor maps; keep them finite
    float *arrs[] = {m->s32, m->d32, m->xref, m->r32[0], m->r32[1], m->p32[0], m->p32[1]};
    for (float *a : arrs) ok = ok && cudaMemsetAsync(a, 0, sizeof(float) * np, s) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    mixed_destroy(m);
    g_msg = "device allocation failed";
    return EIK_ERR_OOM;
  }
  Cg32Buffers &b = m->bufs;
  b.r[0] = m->r32[0];
  b.r[1] = m->r32[1];
  b.p[0] = m->p32[0];
  b.p[1] = m->p32[1];
  b.s32 = m->s32;
  b.d = m->d32;
  b.xref = m->xref;
  b.kx = m->kx;
  b.st = m->st;
  b.part = m->part;
  b.nblk_part = m->nblk_part;
  b.px = m->px;
  const char *why = "";
  if (!cg32_plan(&m->plan, g, m->cg, b, num_sms, tile_override, &why)) {
    mixed_destroy(m);
    g_msg = std::string("inner CG: ") + why;
    return EIK_ERR_CUDA;
  }
  if (!coarse_smem_attr()) {
    cudaGetLastError();
    mixed_destroy(m);
    g_msg = "cannot reserve shared memory for the coarse estimate";
    return EIK_ERR_CUDA;
  }
  if (precond == EIK_PRECOND_MULTIGRID) {
    const eik_status ms = mg_create(&m->mg, g, m->cg, m->px, num_sms, s);
    if (ms != EIK_OK) {
      g_msg = mg_last_error();
      mixed_destroy(m);
      return ms;
    }
  }
  *out = m;
  return EIK_OK;
}

eik_status mixed_create_member(MixedState **out, const Grid &g, const TileCount &tc,
                               int num_sms, BatchExec *batch, int idx, cudaStream_t s) {
  if (g.ndim != 2) {
    g_msg = "packed batches are two-dimensional";
    return EIK_ERR_ARG;
  }
  MixedState *m = new MixedState();
  mixed_layout(m, g, tc, num_sms);
  const BatchMember bm = batch_exec_member(batch, idx);
  m->batch = batch;
  m->bidx = idx;
  m->px = bm.P;
  m->s32 = bm.s32;
  m->d32 = bm.d;
  m->xref = bm.xref;
  m->r32[0] = bm.r0;
  m->p32[0] = bm.p0;
  m->st = bm.st;
  bool ok = mal(&m->x64, g.n) && mal(&m->fb, m->cg.ncell) && mal(&m->St, m->cg.ncell) &&
            mal(&m->kx, m->cg.ncell) && mal(&m->part, 8 * (size_t)m->nblk_part);
  if (ok) ok = cudaMallocHost((void **)&m->h_st, sizeof(MixCtl)) == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(m->kx, 0, sizeof(int) * m->cg.ncell, s) == cudaSuccess &&
               cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mixed_destroy(m);
    g_msg = "device allocation failed";
    return EIK_ERR_OOM;
  }
  if (!coarse_smem_attr()) {
    cudaGetLastError();
    mixed_destroy(m);
    g_msg = "cannot reserve shared memory for the coarse estimate";
    return EIK_ERR_CUDA;
  }
  batch_exec_set_cells(batch, idx, m->cg, m->kx);
  *out = m;
  return EIK_OK;
}

void mixed_destroy(MixedState *m) {
  if (!m) return;
  if (m->mg) mg_destroy(m->mg);
  if (m->graph) cudaGraphExecDestroy(m->graph);
  for (auto &e : m->ev)
    if (e) cudaEventDestroy(e);
  void *own[] = {m->fb, m->St, m->kx, m->x64, m->part};
  for (void *p : own)
    if (p) cudaFree(p);
  if (!m->batch) {   // a member's FP32 arrays and control block are the batch's
    void *fp32[] = {m->s32, m->xref, m->d32, m->r32[0], m->r32[1], m->p32[0], m->p32[1], m->st};
    for (void *p : fp32)
      if (p) cudaFree(p);
  }
  if (m->h_st) cudaFreeHost(m->h_st);
  delete m;
}

static void launch_residual(MixedState *m, const MixedArgs &a) {
  if (m->g.ndim == 2)
    k_mixed_residual<2><<<m->nblk_stencil, kThreads, 0, a.stream>>>(
        m->g, m->tc, m->cg, m->kx, a.sig, m->x64, m->r32[0], m->p32[0], m->d32, m->xref, m->st,
        m->part, m->nblk_part, m->px);
  else
    k_mixed_residual<3><<<m->nblk_stencil, kThreads, 0, a.stream>>>(
        m->g, m->tc, m->cg, m->kx, a.sig, m->x64, m->r32[0], m->p32[0], m->d32, m->xref, m->st,
        m->part, m->nblk_part, m->px);
  m->launches[2]++;
}

static eik_status build_graph(MixedState *m, cudaStream_t s) {
  if (m->graph) return EIK_OK;
  cudaGraph_t graph;
  MCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < kInnerGraphIters; ++k) cg32_iter(m->plan, m->g, m->cg, m->bufs, k & 1, s);
  MCK(cudaStreamEndCapture(s, &graph));
  MCK(cudaGraphInstantiate(&m->graph, graph, 0));
  MCK(cudaGraphDestroy(graph));
  return EIK_OK;
}

// Refinement steps restricted to the unknowns in cells with lo <= kx < hi
// (INT_MIN / INT_MAX: all): FP64 residual, FP32 inner CG on the correction,
// FP64 update, until the componentwise residual of the band is <= tol, the
// step limit, or no progress.  Iterations and steps are added to *total and
// *outer.  max_outer == 0: only the residual check.
static eik_status refine(MixedState *m, const MixedArgs &a, int lo, int hi, int max_outer,
                         int *total_io, int *outer_io, double *res_cw, bool trace) {
  const Grid &g = m->g;
  cudaStream_t s = a.stream;
  const int cap = m->cap;
  auto blocks = [&](int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, cap));
  };
  const double tol = a.opt.tol;
  const double red = (a.opt.inner_tol > 0) ? a.opt.inner_tol : kInnerReduction;
  int total = *total_io, outer = 0;
  double best_cw = INFINITY;
  int stall = 0;
  eik_status result = EIK_ERR_NOT_CONVERGED;
  for (;;) {
    MixCtl init{};
    init.band_lo = lo;
    init.band_hi = hi;
    *m->h_st = init;
    MCK(cudaMemcpyAsync(m->st, m->h_st, sizeof(MixCtl), cudaMemcpyHostToDevice, s));
    launch_residual(m, a);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(m->h_st, m->st, sizeof(MixCtl), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    const double cw = m->h_st->cw;
    *res_cw = cw;
    if (trace)
      fprintf(stderr, "[mixed] outer %d total %d cw %.3e r_inf %.3e x_inf %.3e\n", outer, total,
              cw, m->h_st->r_inf, m->h_st->x_inf);
    if (cw <= tol || m->h_st->rho_m == 0.0) {
      result = EIK_OK;
      break;
    }
    if (std::isnan(cw)) {
      g_msg = "mixed refinement produced a non-finite residual";
      result = EIK_ERR_BREAKDOWN;
      break;
    }
    if (outer >= max_outer || total >= a.opt.max_iter) {
      g_msg = "mixed refinement reached its step or iteration limit";
      break;
    }
    // (cw is infinite while some node of the iterate is not positive yet;
    // progress is then judged only once it is finite)
    if (!std::isfinite(cw) || cw < 0.5 * best_cw) {
      if (std::isfinite(cw)) best_cw = cw;
      stall = 0;
    } else if (++stall >= 2) {
      g_msg = "mixed refinement stopped making progress";
      break;
    }
    // inner solve on the correction.  First step (no iterate yet): reduce the
    // residual, in kx units, by `red`.  Later steps: componentwise test
    // |rhat_i| <= theta |x_i + d_i| with theta = max(tol/2, cw/1000).
    MixCtl st = *m->h_st;
    st.gam_m = st.rho_m;
    st.gam_s = st.rho_s;
    st.alpha = 0.0;
    st.beta = 0.0;
    st.F = 0;
    st.dF = 0;
    st.fd = st.rho_s;
    st.iter = 0;
    st.done = 0;
    st.status = 0;
    st.stalled = 0;
    st.fault = 0;
    st.max_iter = std::max(1, a.opt.max_iter - total);
    st.withhold = (a.opt.test_flags & 1) ? 1 : 0;
    st.mode = (outer == 0 || !std::isfinite(cw)) ? 0 : 1;
    st.thresh = (float)(red * st.r_inf);
    st.theta = (float)std::max(0.5 * tol, 1e-3 * cw);
    if (m->batch) {
      // the batch's passes make the first pass of this solve w = A r
      st.seq = batch_exec_ticket(m->batch, m->bidx);
      st.first = 1;
    }
    *m->h_st = st;
    MCK(cudaMemcpyAsync(m->st, m->h_st, sizeof(MixCtl), cudaMemcpyHostToDevice, s));
    if (m->mg) {
      const MgFine fine{m->r32[0], m->d32, m->xref, m->s32, m->kx, m->St};
      const eik_status ms = mg_inner(m->mg, fine, m->h_st, s);
      if (ms != EIK_OK) {
        g_msg = mg_last_error();
        result = ms;
        break;
      }
    } else if (m->batch) {
      // joins the batch's tile list at its next pass; returns when it ends
      MCK(cudaStreamSynchronize(s));
      const eik_status bs = batch_exec_inner(m->batch, m->bidx, st.seq, m->h_st);
      if (bs != EIK_OK) {
        g_msg = batch_exec_error(m->batch);
        result = bs;
        break;
      }
      m->launches[4] += m->h_st->iter + 1;
    } else {
      if (m->profile && !m->ev[0])
        for (auto &e : m->ev) MCK(cudaEventCreate(&e));
      if (m->profile) MCK(cudaEventRecord(m->ev[0], s));
      cg32_init(m->plan, g, m->cg, m->bufs, 0, s);
      m->launches[3]++;
      MCK(cudaGetLastError());
      if (m->profile) {
        MCK(cudaEventRecord(m->ev[1], s));
        MCK(cudaStreamSynchronize(s));
        float t = 0.f;
        MCK(cudaEventElapsedTime(&t, m->ev[0], m->ev[1]));
        m->ms[3] += t;
        m->timed[3] += 1;
      }
      for (int it = 0;; ++it) {
        if (m->profile) {
          // one timed iteration per host check: no launch runs past convergence
          MCK(cudaEventRecord(m->ev[1], s));
          cg32_iter(m->plan, g, m->cg, m->bufs, it & 1, s);
          MCK(cudaEventRecord(m->ev[2], s));
          m->launches[4] += 1;
        } else {
          MCK(cudaGraphLaunch(m->graph, s));
          m->launches[4] += kInnerGraphIters;
        }
        MCK(cudaMemcpyAsync(m->h_st, m->st, sizeof(MixCtl), cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        if (m->profile) {
          float t = 0.f;
          MCK(cudaEventElapsedTime(&t, m->ev[1], m->ev[2]));
          m->ms[4] += t;
          m->timed[4] += 1;
        }
        if (m->h_st->done) break;
      }
    }
    total += m->h_st->iter;
    ++outer;
    if (trace)
      fprintf(stderr,
              "[mixed]   inner end: iters %d status %d stalled %d alpha %.3e beta %.3e F %d\n",
              m->h_st->iter, m->h_st->status, m->h_st->stalled, m->h_st->alpha, m->h_st->beta,
              m->h_st->F);
    if (m->h_st->status == EIK_ERR_TIMEOUT) {
      g_msg = "a device-side wait for a tile copy timed out";
      result = EIK_ERR_TIMEOUT;
      break;
    }
    if (m->h_st->status == EIK_ERR_BREAKDOWN) {
      g_msg = "inner CG breakdown";
      result = EIK_ERR_BREAKDOWN;
      break;
    }
    k_mixed_update<<<blocks(g.n), kThreads, 0, s>>>(g.n, g.nx, m->px, m->d32, m->x64);
    m->launches[5]++;
    MCK(cudaGetLastError());
  }
  *total_io = total;
  *outer_io += outer;
  return result;
}

eik_status mixed_solve(MixedState *m, const MixedArgs &a, int *inner_iters, int *outer_iters,
                       double *res_cw, double *res_nw) {
  static const bool trace = getenv("EIK_TRACE_MIXED") != nullptr;
  const Grid &g = m->g;
  cudaStream_t s = a.stream;
  const int cap = m->cap;
  auto blocks = [&](int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, cap));
  };
  // setup: FP32 coefficients, cell means of f, coarse distance -> exponents
  k_sig32<<<blocks(g.n), kThreads, 0, s>>>(g.n, g.nx, m->px, a.sig, m->s32);
  k_cell_mean<<<m->cg.ncell, kThreads, 0, s>>>(g, m->cg, a.f, m->fb);
  const size_t smem = 2 * sizeof(float) * m->cg.ncell;
  k_coarse_exponents<<<1, 1024, smem, s>>>(g, m->cg, g.hbar / g.sqrt_c, m->fb, a.src, a.U,
                                           a.nsrc, m->kx, m->St);
  MCK(cudaMemsetAsync(m->x64, 0, sizeof(double) * g.n, s));
  k_init_x64<<<(int)((a.nsrc + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      g, m->cg, m->kx, a.src, a.U, a.nsrc, m->x64);
  m->launches[0] += 3;
  m->launches[1] += 1;
  MCK(cudaGetLastError());
  if (!m->batch && !m->mg) {
    eik_status gs = build_graph(m, s);
    if (gs != EIK_OK) return gs;
  }

  // multigrid inner solves take wider bands: one global refinement holds
  // ranges up to kMgSweepBits (its inner products lose the far field only
  // where their weights 2^(-2 kx) leave the FP64 range)
  const int band_bits = (a.opt.band_bits > 0) ? a.opt.band_bits : (m->mg ? kMgBandBits : kBandBits);
  int kmin = 0, kmax = 0;
  if (a.opt.band_bits >= 0 || m->mg) {
    std::vector<int> hk(m->cg.ncell);
    MCK(cudaMemcpyAsync(hk.data(), m->kx, sizeof(int) * hk.size(), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    kmin = *std::min_element(hk.begin(), hk.end());
    kmax = *std::max_element(hk.begin(), hk.end());
  }
  // the multigrid hierarchy follows the coefficients of the current band
  auto mg_rebuild = [&](int klo) -> eik_status {
    if (!m->mg) return EIK_OK;
    const MgFine fine{m->r32[0], m->d32, m->xref, m->s32, m->kx, m->St};
    const eik_status ms = mg_setup(m->mg, fine, std::max(klo, kmin), s);
    if (ms != EIK_OK) g_msg = mg_last_error();
    return ms;
  };
  const int max_outer = (a.opt.max_outer > 0) ? a.opt.max_outer : 30;
  int total = 0, outer = 0;
  eik_status result;
  const int sweep_bits = (a.opt.band_bits > 0) ? 2 * a.opt.band_bits
                                               : (m->mg ? kMgSweepBits : kSweepBits);
  if (a.opt.band_bits < 0 || kmax - kmin <= sweep_bits) {
    const eik_status ms = mg_rebuild(kmin);
    if (ms != EIK_OK) return ms;
    result = refine(m, a, INT_MIN, INT_MAX, max_outer, &total, &outer, res_cw, trace);
  } else {
    // Level-set sweep: bands of band_bits powers of two in kx (plus an outer
    // overlap), nearest first; everything nearer is held at its converged
    // values, everything farther at its current ones.  Then a check of the
    // whole grid; a further sweep where it fails.  The overlap is at least
    // kMinOverlapBits: kx comes from a coarse estimate whose error measured
    // up to ~20 powers of two, and the influence of the band's outer data
    // falls off like 2^(-2 x true overlap).
    const int ov = std::max(band_bits / 2, kMinOverlapBits);
    result = EIK_ERR_NOT_CONVERGED;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
      for (int lo = kmin;; lo += band_bits) {
        const int hi = std::min(lo + band_bits + ov, kmax + 1);
        k_sig32_band<<<blocks(g.n), kThreads, 0, s>>>(g, m->px, m->cg, m->kx, lo, hi, a.sig,
                                                      m->s32);
        m->launches[0]++;
        MCK(cudaGetLastError());
        const eik_status ms = mg_rebuild(lo);
        if (ms != EIK_OK) return ms;
        if (trace) fprintf(stderr, "[mixed] sweep %d band [%d, %d)\n", sweep, lo, hi);
        const eik_status bs = refine(m, a, lo, hi, max_outer, &total, &outer, res_cw, trace);
        if (bs != EIK_OK && bs != EIK_ERR_NOT_CONVERGED) return bs;   // breakdown, timeout, CUDA
        if (hi > kmax || total >= a.opt.max_iter) break;
      }
      k_sig32<<<blocks(g.n), kThreads, 0, s>>>(g.n, g.nx, m->px, a.sig, m->s32);
      m->launches[0]++;
      const eik_status ms = mg_rebuild(kmin);
      if (ms != EIK_OK) return ms;
      int checks = 0;
      result = refine(m, a, INT_MIN, INT_MAX, 0, &total, &checks, res_cw, trace);
      if (result == EIK_OK || total >= a.opt.max_iter) break;
    }
    if (result == EIK_ERR_NOT_CONVERGED && kmax - kmin <= kGlobalFinishBits &&
        total < a.opt.max_iter) {
      // a moderate range: finish with refinement steps over the whole grid
      result = refine(m, a, INT_MIN, INT_MAX, max_outer, &total, &outer, res_cw, trace);
    }
    if (result == EIK_ERR_NOT_CONVERGED) g_msg = "level-set sweeps did not converge";
  }
  *inner_iters = total;
  *outer_iters = outer;
  *res_nw = 0.0;
  return result;
}

eik_status mixed_export_hat(MixedState *m, const MixedArgs &a, double *xh) {
  const Grid &g = m->g;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + kThreads - 1) / kThreads, m->cap));
  k_mixed_export<<<nb, kThreads, 0, a.stream>>>(g, m->cg, m->kx, m->x64, xh);
  MCK(cudaGetLastError());
  return EIK_OK;
}

eik_status mixed_write_outputs(MixedState *m, const MixedArgs &a, double *S, double *phi) {
  const Grid &g = m->g;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((g.n + kThreads - 1) / kThreads, m->cap));
  k_mixed_epilogue<<<nb, kThreads, 0, a.stream>>>(g, m->cg, m->kx, a.sig, m->x64, S, phi);
  m->launches[6]++;
  MCK(cudaGetLastError());
  return EIK_OK;
}

}  // namespace eik
