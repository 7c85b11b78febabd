// Mixed-precision solve: FP32 inner CG with per-node block floating point,
// FP64 iterative refinement in relative (exponent-scaled) form.
//
// Why the scaling: phi = exp(-S/hbar) spans exp(-max S/hbar), far below the
// FP32 range (and, for S/hbar > ~700, below FP64).  Two exponents keep every
// stored number in range:
//   * kx(cell): a static power-of-two scale per cell of B^d nodes, rounded
//     from a cheap distance estimate St ~ S (min-plus relaxation on the
//     coarse cell grid, 16/26-neighbour stencil, edge cost = length x mean of
//     the two cell-averaged f).  Solution-like vectors (the FP64 iterate xk and
//     the FP32 correction d) are stored as hat-value * 2^kx(cell).
//   * e(node): a per-node exponent shared by the FP32 residual r and search
//     direction p of the inner CG, renormalised in every pass 2 so the larger
//     of |r|, |p| lies in [1, 2).  Hat values are stored * 2^-e ... i.e.
//     rhat = r * 2^-e.  This follows the residual's own decay, which spans far
//     more than the FP32 range over an inner solve.
// All rescaling is by powers of two, so it is exact; CG arithmetic is that of
// Jacobi-preconditioned CG on the scaled operator Ahat (see eik_internal.cuh)
// rounded to FP32 mantissas.  Inner products are accumulated as
// (mantissa, exponent) pairs (or, in the TMA kernels, in FP32 relative to the
// previous <rhat, rhat>) so they cannot underflow or overflow.
//
// The inner FP32 CG yields accurate values near the sources but not in the
// far field: CG iterates there pass through transients many orders larger
// than the final values, whose cancellation FP32 cannot carry.  Refinement
// repairs this: each outer step forms the true FP64 residual in relative
// form and solves for a correction with a fresh inner CG.
//
// When kx spans more than a few hundred powers of two, no global CG (in any
// precision) resolves the far field: its transients there exceed even the
// FP32 exponent range of the correction.  The solve then sweeps level-set
// bands of kx, nearest first, each refined with the rest of the grid held as
// Dirichlet data (mixed_solve / refine).
//
// Inner-CG kernels: TMA-staged tiles with mbarrier pipelines on sm_103a
// (k_mixed2d_tma, k_mixed3d_tma) where the row pitch allows 16-byte aligned
// tensor maps, warp-marched rows (k_mixed2d) or generic halo tiles
// (k_mixed_pass1/2) elsewhere.
#include <cuda.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "eik_launch.h"
#include "eik_mixed.h"

namespace eik {

namespace {

constexpr int kInnerGraphIters = 32;   // even: the buffer sets alternate
constexpr int kNoExp = 30000;          // exponent of an all-zero node
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

thread_local std::string g_msg = "no error";   // per host thread (batches)

// ------------------------------------------------------------ exponents
// 2^n as a float; 0 below the normal range, 2^127 above it.
__device__ __forceinline__ float pow2f(int n) {
  return __int_as_float(min(max(n + 127, 0), 254) << 23);
}
__device__ __forceinline__ double pow2d(int n) {
  if (n < -1022) return 0.0;
  if (n > 1023) n = 1023;
  return __longlong_as_double((long long)(n + 1023) << 52);
}
// floor(log2 |m|) for a finite non-zero normal float
__device__ __forceinline__ int expof(float m) {
  return ((__float_as_int(m) >> 23) & 0xff) - 127;
}

// (mantissa, exponent) accumulators: value = m * 2^s.
struct Acc32 {
  float m;
  int s;
};
struct Acc64 {
  double m;
  int s;
};
__device__ __forceinline__ void acc_add(Acc32 &a, float m, int t) {
  if (m == 0.f) return;
  if (a.m == 0.f) {
    a.m = m;
    a.s = t;
  } else if (t > a.s) {
    a.m = a.m * pow2f(a.s - t) + m;
    a.s = t;
  } else {
    a.m += m * pow2f(t - a.s);
  }
}
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
__device__ __forceinline__ Acc64 to64(const Acc32 &a) {
  Acc64 r{0.0, 0};
  acc_add(r, (double)a.m, a.s);
  return r;
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
__device__ float block_maxf(float v, float *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.f;
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  }
  return v;
}
// Fixed-order combine of per-block Acc64 partials (m in pm, s in ps).
__device__ Acc64 sum_acc_partials(const double *pm, const double *ps, int nblk, double *shm,
                                  int *shs) {
  Acc64 v{0.0, 0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc_add(v, __ldcg(pm + b), (int)__ldcg(ps + b));
  return block_acc(v, shm, shs);
}
__device__ __forceinline__ double acc_ratio(const Acc64 &a, const Acc64 &b) {
  if (b.m == 0.0) return 0.0;
  return (a.m / b.m) * pow2d(a.s - b.s);
}

// Inner-CG control block (device resident).
struct MixState {
  double rho_m;      // <rhat, rhat> = rho_m * 2^rho_s
  int rho_s;
  int iter;          // inner iterations of the current solve
  double alpha, beta;
  float thresh;      // mode 0: stop when max_i |rhat_i| 2^kx(i) <= thresh
  float theta;       // mode 1: stop when |rhat_i| 2^kx(i) <= theta |xref_i + d_i| for all i
  int mode;
  int max_iter;
  int done;
  int status;
  int total_iter;
  int fault;         // a bounded device-side wait expired (see k_mixed2d_tma)
  unsigned int counter[4];
  // outputs of the relative-form FP64 residual
  double cw;         // max |r|/(a phi) over the unknowns
  double r_inf;      // max |rbar64| (kx units)
  double x_inf;      // max |xbar64| (kx units)
  // level-set band of the refinement step: unknowns in cells with
  // band_lo <= kx < band_hi take part, all others are held as Dirichlet data
  int band_lo, band_hi;
  // test hook (eik_options.test_flags bit 0): block 0 of the 2D TMA pass 1
  // does not issue its first tile, so its bounded wait expires
  int withhold;
};

struct CellGrid {
  int B, lgB;        // cell edge in nodes (power of two) and its log2
  int cx, cy, cz;    // cells per axis
  int ncell;
};

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
// u_j = sig_j xbar_j (unknowns) or the source slot xbar_j.  Also initialises
// the inner CG: BFP residual (mantissa + exponent) in buffer set 0, p = 0,
// d = 0, and reduces rho = <rhat, rhat>, the componentwise residual
// max |rbar|/xbar, max |rbar| and max |xbar| (kx units).
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_mixed_residual(Grid g, TileCount tc, CellGrid cg, const int *__restrict__ kx,
                 const double *__restrict__ sig, const double *__restrict__ x64,
                 float *__restrict__ r32, float *__restrict__ p32, short *__restrict__ e16,
                 float *__restrict__ d32, float *__restrict__ xref, MixState *st, double *part,
                 int nblk_part, int px) {
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
      }
      // BFP initial residual: rhat = rb 2^-ki = m 2^-e with m in [1, 2)
      float m = 0.f;
      int e = kNoExp;
      if (rb != 0.0) {
        int ex;
        const double fr = frexp(rb, &ex);      // rb = fr 2^ex, |fr| in [0.5, 1)
        m = (float)(2.0 * fr);
        e = ki - (ex - 1);
        acc_add(rho, (double)m * (double)m, -2 * e);
      }
      const int64_t pi = gx + (int64_t)px * (gy + (int64_t)g.ny * gz);   // pitched
      r32[pi] = m;
      p32[pi] = 0.f;
      e16[pi] = (short)max(-32000, min(e, 32000));
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
    st->beta = 0.0;
    st->counter[0] = 0u;
  }
}

// ------------------------------------------------------------ inner CG
// Stages ptil = r + beta p (per-node exponent e) with sig for the tile and
// its halo; zero nodes carry e = kNoExp.
template <int DIM>
__device__ __forceinline__ void stage_p(const Grid &g, int x0, int y0, int z0, float beta,
                                        const float *__restrict__ r32,
                                        const float *__restrict__ p32,
                                        const short *__restrict__ e16,
                                        const float *__restrict__ s32, float *sp, int *se,
                                        float *ss) {
  using T = Tile<DIM>;
  constexpr int HN = T::HX * T::HY * T::HZ;
  for (int s = threadIdx.x; s < HN; s += blockDim.x) {
    const int hx = s % T::HX, hy = (s / T::HX) % T::HY, hz = s / (T::HX * T::HY);
    const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = (DIM == 3) ? z0 - 1 + hz : 0;
    float pv = 0.f, sv = 0.f;
    int ev = kNoExp;
    if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz) {
      const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
      pv = fmaf(beta, p32[gi], r32[gi]);
      ev = e16[gi];   // exponent of r and p at this node (kNoExp if both are 0)
      sv = s32[gi];
    }
    sp[s] = pv;
    se[s] = ev;
    ss[s] = sv * pv;   // u = sig * ptil
  }
}

// q in units of E = min exponent of the stencil (the largest scale), so no
// term can overflow: q = ptil_i 2^(E-e_i) - sig_i sum_j omega u_j 2^(E-e_j),
// u = sig * ptil (staged in su).  sig_i is passed by the caller.
template <int DIM>
__device__ __forceinline__ float stencil_q(const Grid &g, const float *sp, const int *se,
                                           const float *ss, int s, int gx, int gy, int gz,
                                           float sig_i, bool interior, int &E) {
  using T = Tile<DIM>;
  constexpr int PL = T::HX * T::HY;
  const int ei = se[s];
  int m = min(ei, min(min(se[s - 1], se[s + 1]), min(se[s - T::HX], se[s + T::HX])));
  if (DIM == 3) m = min(m, min(se[s - PL], se[s + PL]));
  E = m;
  const float a1 = ss[s - 1] * pow2f(m - se[s - 1]) + ss[s + 1] * pow2f(m - se[s + 1]);
  const float a2 = ss[s - T::HX] * pow2f(m - se[s - T::HX]) + ss[s + T::HX] * pow2f(m - se[s + T::HX]);
  float acc;
  if (DIM == 2) {
    if (interior) {
      acc = a1 + a2;
    } else {
      const float hx = on_face(gx, g.nx, g.boundary) ? 0.5f : 1.f;
      const float hy = on_face(gy, g.ny, g.boundary) ? 0.5f : 1.f;
      acc = fmaf(hy, a1, hx * a2);
    }
  } else {
    const float a3 = ss[s - PL] * pow2f(m - se[s - PL]) + ss[s + PL] * pow2f(m - se[s + PL]);
    if (interior) {
      acc = (a1 + a2) + a3;
    } else {
      const float hx = on_face(gx, g.nx, g.boundary) ? 0.5f : 1.f;
      const float hy = on_face(gy, g.ny, g.boundary) ? 0.5f : 1.f;
      const float hz = on_face(gz, g.nz, g.boundary) ? 0.5f : 1.f;
      acc = hy * hz * a1 + hx * hz * a2 + hx * hy * a3;
    }
  }
  return fmaf(-sig_i, acc, sp[s] * pow2f(m - ei));
}

template <int DIM>
__device__ __forceinline__ bool tile_interior(const Grid &g, int x0, int y0, int z0) {
  using T = Tile<DIM>;
  return x0 >= 1 && x0 + T::TX <= g.nx - 1 && y0 >= 1 && y0 + T::TY <= g.ny - 1 &&
         (DIM == 2 || (z0 >= 1 && z0 + T::TZ <= g.nz - 1));
}

// Pass 1: <ptil, Ahat ptil>; the last block forms alpha.
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_mixed_pass1(Grid g, TileCount tc, const float *__restrict__ r32,
              const float *__restrict__ p32, const short *__restrict__ e16,
              const float *__restrict__ s32, MixState *st, double *part, int nblk_part) {
  using T = Tile<DIM>;
  constexpr int HN = T::HX * T::HY * T::HZ;
  constexpr int TN = T::TX * T::TY * T::TZ;
  __shared__ float sp[HN];
  __shared__ int se[HN];
  __shared__ float ss[HN];
  __shared__ double shm[32];
  __shared__ int shs[32];
  __shared__ int flag;
  if (st->done) return;
  const float beta = (float)st->beta;
  Acc32 acc{0.f, 0};
  for (int64_t t = blockIdx.x; t < tc.total; t += gridDim.x) {
    int x0, y0, z0;
    tile_origin_m<DIM>(tc, t, x0, y0, z0);
    stage_p<DIM>(g, x0, y0, z0, beta, r32, p32, e16, s32, sp, se, ss);
    const bool interior = tile_interior<DIM>(g, x0, y0, z0);
    __syncthreads();
    for (int lin = threadIdx.x; lin < TN; lin += blockDim.x) {
      const int lx = lin % T::TX, ly = (lin / T::TX) % T::TY, lz = lin / (T::TX * T::TY);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      if (gx >= g.nx || gy >= g.ny || gz >= g.nz) continue;
      const int s = (DIM == 3 ? (lz + 1) * T::HX * T::HY : 0) + (ly + 1) * T::HX + lx + 1;
      if (sp[s] == 0.f) continue;
      const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
      int E;
      const float q = stencil_q<DIM>(g, sp, se, ss, s, gx, gy, gz, s32[gi], interior, E);
      // phat*qhat = ptil 2^-e * q 2^-E
      acc_add(acc, sp[s] * q, -(se[s] + E));
    }
    __syncthreads();
  }
  const Acc64 tot = block_acc(to64(acc), shm, shs);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = tot.m;
    part[nblk_part + blockIdx.x] = (double)tot.s;
  }
  if (!last_block(&st->counter[1], &flag)) return;
  const Acc64 pq = sum_acc_partials(part, part + nblk_part, gridDim.x, shm, shs);
  if (threadIdx.x == 0) {
    const Acc64 rho{st->rho_m, st->rho_s};
    if (pq.m > 0.0 && isfinite(pq.m)) {
      st->alpha = acc_ratio(rho, pq);
    } else if (rho.m == 0.0) {
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

// Pass 2: d += alpha ptil (kx units), r -= alpha q, renormalise (r, p) per
// node, write buffer set B; reduce <rhat, rhat> and the scaled residual max.
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_mixed_pass2(Grid g, TileCount tc, CellGrid cg, const int *__restrict__ kx,
              const float *__restrict__ r32, const float *__restrict__ p32,
              const short *__restrict__ e16, const float *__restrict__ s32,
              float *__restrict__ r32o, float *__restrict__ p32o, short *__restrict__ e16o,
              float *__restrict__ d32, const float *__restrict__ xref, MixState *st,
              double *part, int nblk_part) {
  using T = Tile<DIM>;
  constexpr int HN = T::HX * T::HY * T::HZ;
  constexpr int TN = T::TX * T::TY * T::TZ;
  __shared__ float sp[HN];
  __shared__ int se[HN];
  __shared__ float ss[HN];
  __shared__ double shm[32];
  __shared__ int shs[32];
  __shared__ float shf[32];
  __shared__ int flag;
  if (st->done) return;
  const float beta = (float)st->beta, alpha = (float)st->alpha;
  const int mode = st->mode;
  const float theta = st->theta;
  Acc32 acc{0.f, 0};
  float rmax = 0.f;
  for (int64_t t = blockIdx.x; t < tc.total; t += gridDim.x) {
    int x0, y0, z0;
    tile_origin_m<DIM>(tc, t, x0, y0, z0);
    stage_p<DIM>(g, x0, y0, z0, beta, r32, p32, e16, s32, sp, se, ss);
    const bool interior = tile_interior<DIM>(g, x0, y0, z0);
    __syncthreads();
    for (int lin = threadIdx.x; lin < TN; lin += blockDim.x) {
      const int lx = lin % T::TX, ly = (lin / T::TX) % T::TY, lz = lin / (T::TX * T::TY);
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      if (gx >= g.nx || gy >= g.ny || gz >= g.nz) continue;
      const int s = (DIM == 3 ? (lz + 1) * T::HX * T::HY : 0) + (ly + 1) * T::HX + lx + 1;
      const int64_t gi = gx + (int64_t)g.nx * (gy + (int64_t)g.ny * gz);
      const float pt = sp[s];
      const int ei = se[s];
      float rn = 0.f, pn = 0.f;
      int en = kNoExp;
      {
        int E;
        const float q = stencil_q<DIM>(g, sp, se, ss, s, gx, gy, gz, s32[gi], interior, E);
        const int ki = kx[cell_of(cg, gx, gy, gz)];
        float dn = d32[gi];
        if (pt != 0.f) {
          dn = fmaf(alpha * pt, pow2f(ki - ei), dn);
          d32[gi] = dn;
        }
        const float f = pow2f(E - ei);
        const float rE = fmaf(-alpha, q, r32[gi] * f);   // r in E units
        const float pE = pt * f;
        const float mx = fmaxf(fabsf(rE), fabsf(pE));
        if (mx > 0.f && isfinite(mx)) {
          const int sh = expof(mx);
          const float sc = pow2f(-sh);
          rn = rE * sc;
          pn = pE * sc;
          en = E - sh;
          acc_add(acc, rn * rn, -2 * en);
          const float rk = fabsf(rn) * pow2f(ki - en);   // |rhat| in kx units
          if (mode == 0)
            rmax = fmaxf(rmax, rk);
          else if (rk > theta * fabsf(xref[gi] + dn))
            rmax = 1.f;                                   // not yet converged here
        } else if (!isfinite(mx)) {
          rmax = INFINITY;
        }
      }
      r32o[gi] = rn;
      p32o[gi] = pn;
      e16o[gi] = (short)max(-32000, min(en, 32000));
    }
    __syncthreads();
  }
  const Acc64 tot = block_acc(to64(acc), shm, shs);
  const float bm = block_maxf(rmax, shf);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = tot.m;
    part[nblk_part + blockIdx.x] = (double)tot.s;
    part[2 * nblk_part + blockIdx.x] = (double)bm;
  }
  if (!last_block(&st->counter[2], &flag)) return;
  const Acc64 rr = sum_acc_partials(part, part + nblk_part, gridDim.x, shm, shs);
  const double rm = max_partials(part + 2 * nblk_part, gridDim.x, shm);
  if (threadIdx.x == 0) {
    const Acc64 rho{st->rho_m, st->rho_s};
    st->beta = acc_ratio(rr, rho);
    st->rho_m = rr.m;
    st->rho_s = rr.s;
    st->iter += 1;
    st->total_iter += 1;
    if (!isfinite(rr.m) || !isfinite(st->beta)) {
      st->done = 1;
      st->status = EIK_ERR_BREAKDOWN;
    } else if ((st->mode == 0 ? rm <= (double)st->thresh : rm == 0.0) || rr.m == 0.0) {
      st->done = 1;
      st->status = EIK_OK;
    } else if (st->iter >= st->max_iter) {
      st->done = 1;
      st->status = EIK_ERR_NOT_CONVERGED;
    }
    st->counter[2] = 0u;
  }
}

// ------------------------------------------- 2D inner CG, warp-marched rows
// Specialisation for 2D grids with nx % VEC == 0: a warp owns 32*VEC
// consecutive columns (VEC = 2 or 4 per lane, vector loads) and marches down
// kRowsPerWarp rows, keeping the rows above and below in registers and taking
// the x neighbours
// by warp shuffle (lanes 0 and 31 load the column beyond the warp).  No shared
// memory and no block barrier on the data path; the next row's loads are
// issued before the current row is computed.  Arithmetic is that of
// stencil_q / k_mixed_pass1 / k_mixed_pass2 above; inner-product terms are
// accumulated node by node, as there.
constexpr int kRowsPerWarp = 4;
constexpr int kWarpsPerBlock = 8;
constexpr int kRowTile = kRowsPerWarp * kWarpsPerBlock;   // rows per block tile

// Row of a warp: VEC consecutive columns per lane (VEC = 2 or 4), plus the
// u/e of the column left of the lane's first and right of its last.
template <int VEC>
struct Row {
  float r[VEC], pt[VEC], s[VEC], u[VEC];
  int e[VEC];
  float uL, uR;
  int eL, eR;
};

template <int VEC>
__device__ __forceinline__ void ldv(const float *p, float (&v)[VEC]) {
  if (VEC == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    v[0] = t.x; v[1] = t.y;
  }
}
template <int VEC>
__device__ __forceinline__ void stv(float *p, const float (&v)[VEC]) {
  if (VEC == 4)
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}
template <int VEC>
__device__ __forceinline__ void lde(const short *p, int (&v)[VEC]) {
  if (VEC == 4) {
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    v[0] = (short)(t.x & 0xffff); v[1] = (short)(t.x >> 16);
    v[2] = (short)(t.y & 0xffff); v[3] = (short)(t.y >> 16);
  } else {
    const unsigned int t = *reinterpret_cast<const unsigned int *>(p);
    v[0] = (short)(t & 0xffff); v[1] = (short)(t >> 16);
  }
}
__device__ __forceinline__ uint32_t pack2(int a, int b) {
  return (uint32_t)(uint16_t)(short)max(-32000, min(a, 32000)) |
         ((uint32_t)(uint16_t)(short)max(-32000, min(b, 32000)) << 16);
}
template <int VEC>
__device__ __forceinline__ void ste(short *p, const int (&v)[VEC]) {
  if (VEC == 4)
    *reinterpret_cast<uint2 *>(p) = make_uint2(pack2(v[0], v[1]), pack2(v[2], v[3]));
  else
    *reinterpret_cast<unsigned int *>(p) = pack2(v[0], v[1]);
}

template <int VEC>
__device__ __forceinline__ void load_row(const Grid &g, int x, int xw, int y, float beta,
                                         const float *__restrict__ r32,
                                         const float *__restrict__ p32,
                                         const short *__restrict__ e16,
                                         const float *__restrict__ s32, Row<VEC> &R) {
  const int lane = threadIdx.x & 31;
  const bool in = (y >= 0) && (y < g.ny) && (x < g.nx);
  if (in) {
    const int64_t o = (int64_t)y * g.nx + x;
    float p[VEC];
    ldv<VEC>(r32 + o, R.r);
    ldv<VEC>(p32 + o, p);
    ldv<VEC>(s32 + o, R.s);
    lde<VEC>(e16 + o, R.e);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      R.pt[j] = fmaf(beta, p[j], R.r[j]);
      R.u[j] = R.s[j] * R.pt[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      R.r[j] = R.pt[j] = R.s[j] = R.u[j] = 0.f;
      R.e[j] = kNoExp;
    }
  }
  R.uL = __shfl_up_sync(0xffffffffu, R.u[VEC - 1], 1);
  R.eL = __shfl_up_sync(0xffffffffu, R.e[VEC - 1], 1);
  R.uR = __shfl_down_sync(0xffffffffu, R.u[0], 1);
  R.eR = __shfl_down_sync(0xffffffffu, R.e[0], 1);
  if (lane == 0 || lane == 31) {
    const int xn = (lane == 0) ? xw - 1 : xw + 32 * VEC;
    float uu = 0.f;
    int ee = kNoExp;
    if (y >= 0 && y < g.ny && xn >= 0 && xn < g.nx) {
      const int64_t o = (int64_t)y * g.nx + xn;
      uu = s32[o] * fmaf(beta, p32[o], r32[o]);
      ee = e16[o];
    }
    if (lane == 0) {
      R.uL = uu;
      R.eL = ee;
    } else {
      R.uR = uu;
      R.eR = ee;
    }
  }
}

// q for one column: u/e of the x neighbours, the row above (a) and below (b).
__device__ __forceinline__ float q_node(float pt, float sg, int ei, float uL, int eL, float uR,
                                        int eR, float ua, int ea, float ub, int eb, float hx,
                                        float hy, int &E) {
  const int m = min(min(ei, min(eL, eR)), min(ea, eb));
  E = m;
  const float a1 = uL * pow2f(m - eL) + uR * pow2f(m - eR);
  const float a2 = ua * pow2f(m - ea) + ub * pow2f(m - eb);
  return fmaf(-sg, fmaf(hy, a1, hx * a2), pt * pow2f(m - ei));
}

// End of an inner pass: block partials of the inner product (and, in pass
// 2, of the residual maximum), then the last block forms alpha (pass 1) or
// beta and the stopping decision (pass 2).
template <bool PASS2>
__device__ void inner_pass_tail(const Acc32 &acc, float rmax, MixState *st, double *part,
                                int nblk_part) {
  __shared__ double shm[32];
  __shared__ int shs[32];
  __shared__ float shf[32];
  __shared__ int flag;
  const Acc64 tot = block_acc(to64(acc), shm, shs);
  float bm = 0.f;
  if (PASS2) bm = block_maxf(rmax, shf);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = tot.m;
    part[nblk_part + blockIdx.x] = (double)tot.s;
    if (PASS2) part[2 * nblk_part + blockIdx.x] = (double)bm;
  }
  if (!last_block(&st->counter[PASS2 ? 2 : 1], &flag)) return;
  const Acc64 sum = sum_acc_partials(part, part + nblk_part, gridDim.x, shm, shs);
  if (!PASS2) {
    if (threadIdx.x == 0) {
      const Acc64 rho{st->rho_m, st->rho_s};
      if (st->fault) {
        st->alpha = 0.0;
        st->done = 1;
        st->status = EIK_ERR_TIMEOUT;
      } else if (sum.m > 0.0 && isfinite(sum.m)) {
        st->alpha = acc_ratio(rho, sum);
      } else if (rho.m == 0.0) {
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
  } else {
    const double rm = max_partials(part + 2 * nblk_part, gridDim.x, shm);
    if (threadIdx.x == 0) {
      const Acc64 rho{st->rho_m, st->rho_s};
      st->beta = acc_ratio(sum, rho);
      st->rho_m = sum.m;
      st->rho_s = sum.s;
      st->iter += 1;
      st->total_iter += 1;
      if (st->fault) {
        st->done = 1;
        st->status = EIK_ERR_TIMEOUT;
      } else if (!isfinite(sum.m) || !isfinite(st->beta)) {
        st->done = 1;
        st->status = EIK_ERR_BREAKDOWN;
      } else if ((st->mode == 0 ? rm <= (double)st->thresh : rm == 0.0) || sum.m == 0.0) {
        st->done = 1;
        st->status = EIK_OK;
      } else if (st->iter >= st->max_iter) {
        st->done = 1;
        st->status = EIK_ERR_NOT_CONVERGED;
      }
      st->counter[2] = 0u;
    }
  }
}

// 2^n for n <= 0 (0 below the normal range): one clamp and one multiply-add.
__device__ __forceinline__ float pow2f_le0(int n) {
  return __int_as_float(max(n, -127) * (1 << 23) + (127 << 23));
}

// q_node for the TMA kernels: the same value, with the scale factors (all
// 2^(m - e) with m the minimum exponent, so never above 1) formed by
// pow2f_le0.
__device__ __forceinline__ float q_node_le0(float pt, float sg, int ei, float uL, int eL,
                                            float uR, int eR, float ua, int ea, float ub, int eb,
                                            float hx, float hy, int &E) {
  const int m = min(min(ei, min(eL, eR)), min(ea, eb));
  E = m;
  const float a1 = uL * pow2f_le0(m - eL) + uR * pow2f_le0(m - eR);
  const float a2 = ua * pow2f_le0(m - ea) + ub * pow2f_le0(m - eb);
  return fmaf(-sg, fmaf(hy, a1, hx * a2), pt * pow2f_le0(m - ei));
}

template <bool PASS2, int VEC>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_mixed2d(Grid g, CellGrid cg, int tiles_x, int ntiles, const int *__restrict__ kx,
          const float *__restrict__ r32, const float *__restrict__ p32,
          const short *__restrict__ e16, const float *__restrict__ s32,
          float *__restrict__ r32o, float *__restrict__ p32o, short *__restrict__ e16o,
          float *__restrict__ d32, const float *__restrict__ xref, MixState *st, double *part,
          int nblk_part) {
  constexpr int W = 32 * VEC;   // columns per warp
  if (st->done) return;
  const float beta = (float)st->beta, alpha = (float)st->alpha;
  const int mode = st->mode;
  const float theta = st->theta;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool half = g.boundary == EIK_BOUNDARY_HALF_CELL;
  Acc32 acc{0.f, 0};
  float rmax = 0.f;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int xw = (t % tiles_x) * W;
    const int x = xw + VEC * lane;
    const int y0 = (t / tiles_x) * kRowTile + warp * kRowsPerWarp;
    if (y0 >= g.ny) continue;   // whole warp: uniform
    // face weights of the columns (x edges carry hy, y edges hx)
    float hx[VEC];
#pragma unroll
    for (int j = 0; j < VEC; ++j)
      hx[j] = (half && (x + j == 0 || x + j == g.nx - 1)) ? 0.5f : 1.f;
    Row<VEC> A, C, B;   // above, current, below
    load_row<VEC>(g, x, xw, y0 - 1, beta, r32, p32, e16, s32, A);
    load_row<VEC>(g, x, xw, y0, beta, r32, p32, e16, s32, C);
    for (int k = 0; k < kRowsPerWarp; ++k) {
      const int y = y0 + k;
      load_row<VEC>(g, x, xw, y + 1, beta, r32, p32, e16, s32, B);
      if (y < g.ny && x < g.nx) {
        const float hy = (half && (y == 0 || y == g.ny - 1)) ? 0.5f : 1.f;
        float q[VEC];
        int E[VEC];
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          const float uL = (j == 0) ? C.uL : C.u[j - 1];
          const int eL = (j == 0) ? C.eL : C.e[j - 1];
          const float uR = (j == VEC - 1) ? C.uR : C.u[j + 1];
          const int eR = (j == VEC - 1) ? C.eR : C.e[j + 1];
          q[j] = q_node(C.pt[j], C.s[j], C.e[j], uL, eL, uR, eR, A.u[j], A.e[j], B.u[j], B.e[j],
                        hx[j], hy, E[j]);
        }
        if (!PASS2) {
          // <phat, qhat>: terms pt*q 2^-(e+E)
#pragma unroll
          for (int j = 0; j < VEC; ++j) acc_add(acc, C.pt[j] * q[j], -(C.e[j] + E[j]));
        } else {
          const int64_t o = (int64_t)y * g.nx + x;
          const int ki = kx[(x >> cg.lgB) + cg.cx * (y >> cg.lgB)];
          float dd[VEC], rn[VEC], pn[VEC], xr[VEC];
          int en[VEC];
          ldv<VEC>(d32 + o, dd);
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            const float pt = C.pt[j];
            if (pt != 0.f) dd[j] = fmaf(alpha * pt, pow2f(ki - C.e[j]), dd[j]);
            const float f = pow2f(E[j] - C.e[j]);
            const float rE = fmaf(-alpha, q[j], C.r[j] * f);
            const float pE = pt * f;
            const float mx = fmaxf(fabsf(rE), fabsf(pE));
            if (mx > 0.f && mx <= 3.4e38f) {
              const int sh = expof(mx);
              const float sc = pow2f(-sh);
              rn[j] = rE * sc;
              pn[j] = pE * sc;
              en[j] = E[j] - sh;
            } else {
              rn[j] = 0.f;
              pn[j] = 0.f;
              en[j] = kNoExp;
              if (!(mx <= 3.4e38f)) rmax = INFINITY;
            }
            acc_add(acc, rn[j] * rn[j], -2 * en[j]);   // <rhat, rhat>
          }
          if (mode != 0) ldv<VEC>(xref + o, xr);
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            if (rn[j] == 0.f) continue;
            const float rk = fabsf(rn[j]) * pow2f(ki - en[j]);
            if (mode == 0)
              rmax = fmaxf(rmax, rk);
            else if (rk > theta * fabsf(xr[j] + dd[j]))
              rmax = 1.f;
          }
          stv<VEC>(d32 + o, dd);
          stv<VEC>(r32o + o, rn);
          stv<VEC>(p32o + o, pn);
          ste<VEC>(e16o + o, en);
        }
      }
      A = C;
      C = B;
    }
  }
  inner_pass_tail<PASS2>(acc, rmax, st, part, nblk_part);
}

// ------------------------------------ 2D inner CG, TMA-staged tiles (sm_103a)
// A block owns tiles of kTmaTX x TY nodes.  For each tile one thread issues
// tensor-memory-accelerator copies of r, p, sigma and e with a one-node halo
// (and, in pass 2, of d and xref without halo) into a shared-memory stage and
// the block waits on that stage's mbarrier; two stages alternate, so the
// copies of the next tile are in flight while the current one is computed.
// Every copy lands whole: nothing on the data path waits on a single global
// load.  Inside a tile a warp owns 64 columns (2 per lane) and marches down
// TY/RG rows, computing u = sigma (r + beta p) of each row once and taking
// the x neighbours by warp shuffle.  The arithmetic per node is that of
// q_node / k_mixed2d above.
//
// Requirements (checked on the host): 2D, nx a multiple of 8 (the row pitch
// of the int16 exponents must be a multiple of 16 bytes).  Nodes outside the
// grid arrive as zeros (TMA fill); a neighbour with u = 0 is left out of the
// exponent minimum, so the zero fill needs no special case.
constexpr int kTmaTX = 128;                 // tile columns
constexpr int kTmaStages = 2;               // default stage count (2D)
constexpr unsigned long long kTmaWaitNs = 200ull * 1000 * 1000;   // 0.2 s

template <int TY>
struct TmaTile {
  static constexpr int H = TY + 2;                         // rows incl. halo
  static constexpr int FW = kTmaTX + 8;                    // floats: x0-4 .. x0+TX+3
  static constexpr int EW = kTmaTX + 16;                   // shorts: x0-8 .. x0+TX+7
  static constexpr int F_BYTES = ((FW * H * 4 + 127) / 128) * 128;
  static constexpr int E_BYTES = ((EW * H * 2 + 127) / 128) * 128;
  static constexpr int C_BYTES = kTmaTX * TY * 4;          // d / xref tiles (no halo)
  static constexpr int OFF_R = 0, OFF_P = F_BYTES, OFF_S = 2 * F_BYTES;
  static constexpr int OFF_E = 3 * F_BYTES;
  static constexpr int OFF_D = OFF_E + E_BYTES, OFF_X = OFF_D + C_BYTES;
  static constexpr int STAGE1 = OFF_D;                     // pass 1 stage bytes
  static constexpr int STAGE2 = OFF_X + C_BYTES;           // pass 2 stage bytes
  static constexpr int smem(bool pass2, int ns = kTmaStages) {
    return ns * (pass2 ? STAGE2 : STAGE1) + 128;
  }
};

struct TmaMaps {
  CUtensorMap r, p, e;   // one buffer set (halo boxes)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `parity` of the barrier for at most kTmaWaitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *b, uint32_t parity) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(b, parity)) return true;
    if (global_ns() - t0 > kTmaWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// One TMA row of the tile, as seen by one lane (2 columns).
struct TRow {
  float r0, r1, pt0, pt1, s0, s1, u0, u1;
  int e0, e1;    // stored exponents (centre use)
  int n0, n1;    // exponents for neighbour use: kNoExp where u == 0
};

template <int TY>
__device__ __forceinline__ void trow_load(const unsigned char *stage, int j, int lc, float beta,
                                          TRow &R) {
  using T = TmaTile<TY>;
  const float *sr = reinterpret_cast<const float *>(stage + T::OFF_R);
  const float *sp = reinterpret_cast<const float *>(stage + T::OFF_P);
  const float *ss = reinterpret_cast<const float *>(stage + T::OFF_S);
  const short *se = reinterpret_cast<const short *>(stage + T::OFF_E);
  const int fo = j * T::FW + lc + 4, eo = j * T::EW + lc + 8;
  const float2 r = *reinterpret_cast<const float2 *>(sr + fo);
  const float2 p = *reinterpret_cast<const float2 *>(sp + fo);
  const float2 sg = *reinterpret_cast<const float2 *>(ss + fo);
  const unsigned int ee = *reinterpret_cast<const unsigned int *>(se + eo);
  R.r0 = r.x;
  R.r1 = r.y;
  R.pt0 = fmaf(beta, p.x, r.x);
  R.pt1 = fmaf(beta, p.y, r.y);
  R.s0 = sg.x;
  R.s1 = sg.y;
  R.u0 = sg.x * R.pt0;
  R.u1 = sg.y * R.pt1;
  R.e0 = (short)(ee & 0xffffu);
  R.e1 = (short)(ee >> 16);
  R.n0 = (R.u0 != 0.f) ? R.e0 : kNoExp;
  R.n1 = (R.u1 != 0.f) ? R.e1 : kNoExp;
}

// u and neighbour exponent of a single tile-local column c of smem row j.
template <int TY>
__device__ __forceinline__ void tcol_load(const unsigned char *stage, int j, int c, float beta,
                                          float &u, int &n) {
  using T = TmaTile<TY>;
  const float *sr = reinterpret_cast<const float *>(stage + T::OFF_R);
  const float *sp = reinterpret_cast<const float *>(stage + T::OFF_P);
  const float *ss = reinterpret_cast<const float *>(stage + T::OFF_S);
  const short *se = reinterpret_cast<const short *>(stage + T::OFF_E);
  const int fo = j * T::FW + c + 4;
  u = ss[fo] * fmaf(beta, sp[fo], sr[fo]);
  n = (u != 0.f) ? (int)se[j * T::EW + c + 8] : kNoExp;
}

template <bool PASS2, int TY, int RG, int NS>
__global__ void __launch_bounds__(64 * RG, 1)
k_mixed2d_tma(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_p,
              const __grid_constant__ CUtensorMap tm_e, const __grid_constant__ CUtensorMap tm_s,
              const __grid_constant__ CUtensorMap tm_d, const __grid_constant__ CUtensorMap tm_x,
              Grid g, CellGrid cg, int tiles_x, int ntiles, const int *__restrict__ kx,
              float *__restrict__ r32o, float *__restrict__ p32o, short *__restrict__ e16o,
              float *__restrict__ d32, MixState *st, double *part, int nblk_part, int px) {
  using T = TmaTile<TY>;
  constexpr int RW = TY / RG;   // rows marched by one warp
  static_assert(TY % RG == 0, "rows per warp");
  extern __shared__ unsigned char tma_smem_raw[];
  __shared__ __align__(8) uint64_t bar[NS];
  if (st->done) return;
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tma_smem_raw) + 127) & ~uintptr_t(127));
  constexpr int STAGE = PASS2 ? T::STAGE2 : T::STAGE1;
  const float beta = (float)st->beta, alpha = (float)st->alpha;
  const int mode = st->mode;
  const float theta = st->theta;
  const bool want_x = PASS2 && mode != 0;
  const uint32_t tx_bytes =
      3 * (T::FW * T::H * 4) + T::EW * T::H * 2 + (PASS2 ? T::C_BYTES : 0) +
      (want_x ? T::C_BYTES : 0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cw = warp & 1, rg = warp >> 1;
  const bool half = g.boundary == EIK_BOUNDARY_HALF_CELL;

  int last_k = -1;   // thread 0: index (in this block's tile sequence) of the last tile issued
  auto issue = [&](int t, int stg) {
    last_k = (t - (int)blockIdx.x) / (int)gridDim.x;
    unsigned char *dst = smem + stg * STAGE;
    const int x0 = (t % tiles_x) * kTmaTX, y0 = (t / tiles_x) * TY;
    mbar_expect_tx(&bar[stg], tx_bytes);
    tma_load_2d(dst + T::OFF_R, &tm_r, x0 - 4, y0 - 1, &bar[stg]);
    tma_load_2d(dst + T::OFF_P, &tm_p, x0 - 4, y0 - 1, &bar[stg]);
    tma_load_2d(dst + T::OFF_S, &tm_s, x0 - 4, y0 - 1, &bar[stg]);
    tma_load_2d(dst + T::OFF_E, &tm_e, x0 - 8, y0 - 1, &bar[stg]);
    if (PASS2) tma_load_2d(dst + T::OFF_D, &tm_d, x0, y0, &bar[stg]);
    if (want_x) tma_load_2d(dst + T::OFF_X, &tm_x, x0, y0, &bar[stg]);
  };

  if (tid == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  const int first = blockIdx.x, step = gridDim.x;
  if (tid == 0)
    for (int k = 0; k < NS; ++k)
      if (first + k * step < ntiles && !(k == 0 && !PASS2 && blockIdx.x == 0 && st->withhold))
        issue(first + k * step, k);

  // Inner-product terms are summed in FP32 relative to 2^frame, the scale of
  // the previous <rhat, rhat>: terms more than 2^126 below it (far-field
  // nodes with negligible weight) flush to zero, none can overflow.
  const int frame = st->rho_s;
  float accf = 0.f;
  float rmax = 0.f;
  bool fault = false;
  int k = 0;
  for (int t = first; t < ntiles; t += step, ++k) {
    const int stg = k % NS;
    const uint32_t parity = (uint32_t)(k / NS) & 1u;
    // pass 2: the cell exponent of the warp's first row, loaded before the
    // wait so its latency hides behind it (reloaded below only when the row
    // crosses into the next cell row)
    int kcy = -1, kyi = 0;
    if (PASS2) {
      const int xq = min((t % tiles_x) * kTmaTX + 64 * cw + 2 * lane, g.nx - 1);
      const int yq = min((t / tiles_x) * TY + rg * RW, g.ny - 1);
      kcy = yq >> cg.lgB;
      kyi = kx[(xq >> cg.lgB) + cg.cx * kcy];
    }
    const bool ok = mbar_wait_bounded(&bar[stg], parity);
    if (__syncthreads_or(!ok)) {
      fault = true;
      break;
    }
    // every thread is past tile k - 1: its stage takes tile k - 1 + NS
    if (tid == 0 && k >= 1 && t + (NS - 1) * step < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + (NS - 1) * step, (k - 1) % NS);
    }
    const unsigned char *S = smem + stg * STAGE;
    const int x0 = (t % tiles_x) * kTmaTX, y0 = (t / tiles_x) * TY;
    const int lc = 64 * cw + 2 * lane;          // tile-local column of node 0
    const int x = x0 + lc;
    const int hc = (lane == 0) ? lc - 1 : lc + 2;   // halo column (lanes 0, 31)
    const float hx0 = (half && (x == 0 || x == g.nx - 1)) ? 0.5f : 1.f;   // odd nx: x = nx-1
    const float hx1 = (half && x + 1 == g.nx - 1) ? 0.5f : 1.f;
    TRow A, C, B;
    const int j0 = rg * RW + 1;                 // smem row of the first centre row
    trow_load<TY>(S, j0 - 1, lc, beta, A);
    trow_load<TY>(S, j0, lc, beta, C);
#pragma unroll 2
    for (int i = 0; i < RW; ++i) {
      const int j = j0 + i;
      const int y = y0 + j - 1;
      trow_load<TY>(S, j + 1, lc, beta, B);
      float uh = 0.f;
      int nh = kNoExp;
      if (lane == 0 || lane == 31) tcol_load<TY>(S, j, hc, beta, uh, nh);
      float uL = __shfl_up_sync(0xffffffffu, C.u1, 1);
      int nL = __shfl_up_sync(0xffffffffu, C.n1, 1);
      float uR = __shfl_down_sync(0xffffffffu, C.u0, 1);
      int nR = __shfl_down_sync(0xffffffffu, C.n0, 1);
      if (lane == 0) {
        uL = uh;
        nL = nh;
      }
      if (lane == 31) {
        uR = uh;
        nR = nh;
      }
      if (y < g.ny && x < g.nx) {
        const float hy = (half && (y == 0 || y == g.ny - 1)) ? 0.5f : 1.f;
        int E0, E1;
        const float q0 = q_node_le0(C.pt0, C.s0, C.e0, uL, nL, C.u1, C.n1, A.u0, A.n0, B.u0,
                                    B.n0, hx0, hy, E0);
        const float q1 = q_node_le0(C.pt1, C.s1, C.e1, C.u0, C.n0, uR, nR, A.u1, A.n1, B.u1,
                                    B.n1, hx1, hy, E1);
        if (!PASS2) {
          accf = fmaf(C.pt0 * q0, pow2f(-(C.e0 + E0) - frame), accf);
          accf = fmaf(C.pt1 * q1, pow2f(-(C.e1 + E1) - frame), accf);
        } else {
          const int li = (j - 1) * kTmaTX + lc;   // tile-local index, no halo
          const float2 dd = *reinterpret_cast<const float2 *>(S + T::OFF_D + 4 * li);
          float2 xr = make_float2(0.f, 0.f);
          if (want_x) xr = *reinterpret_cast<const float2 *>(S + T::OFF_X + 4 * li);
          if ((y >> cg.lgB) != kcy) {   // x, x+1: one cell
            kcy = y >> cg.lgB;
            kyi = kx[(x >> cg.lgB) + cg.cx * kcy];
          }
          float d[2] = {dd.x, dd.y}, rn[2], pn[2];
          int en[2];
          const float pt[2] = {C.pt0, C.pt1}, rr[2] = {C.r0, C.r1}, q[2] = {q0, q1};
          const int ee[2] = {C.e0, C.e1}, EE[2] = {E0, E1};
          const float xx[2] = {xr.x, xr.y};
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (pt[c] != 0.f) d[c] = fmaf(alpha * pt[c], pow2f(kyi - ee[c]), d[c]);
            const float f = pow2f_le0(EE[c] - ee[c]);
            const float rE = fmaf(-alpha, q[c], rr[c] * f);
            const float pE = pt[c] * f;
            const float mx = fmaxf(fabsf(rE), fabsf(pE));
            if (mx > 0.f && mx <= 3.4e38f) {
              const int sh = expof(mx);
              const float sc = __int_as_float((127 - sh) << 23);   // 2^-sh, sh in [-127, 127]
              rn[c] = rE * sc;
              pn[c] = pE * sc;
              en[c] = EE[c] - sh;
              accf = fmaf(rn[c] * rn[c], pow2f(-2 * en[c] - frame), accf);
              const float rk = fabsf(rn[c]) * pow2f(kyi - en[c]);
              if (mode == 0)
                rmax = fmaxf(rmax, rk);
              else if (rk > theta * fabsf(xx[c] + d[c]))
                rmax = 1.f;
            } else {
              rn[c] = 0.f;
              pn[c] = 0.f;
              en[c] = kNoExp;
              if (!(mx <= 3.4e38f)) rmax = INFINITY;
            }
          }
          const int64_t o = (int64_t)y * px + x;   // pitched row
          *reinterpret_cast<float2 *>(d32 + o) = make_float2(d[0], d[1]);
          *reinterpret_cast<float2 *>(r32o + o) = make_float2(rn[0], rn[1]);
          *reinterpret_cast<float2 *>(p32o + o) = make_float2(pn[0], pn[1]);
          *reinterpret_cast<unsigned int *>(e16o + o) = pack2(en[0], en[1]);
        }
      }
      A = C;
      C = B;
    }
  }
  if (fault) {
    // leave no copy in flight: wait (bounded) for every stage still pending
    if (tid == 0) {
      atomicExch(&st->fault, 1);
      for (int kk = k; kk <= last_k; ++kk)
        mbar_wait_bounded(&bar[kk % NS], (uint32_t)(kk / NS) & 1u);
    }
    __syncthreads();
  }
  inner_pass_tail<PASS2>(Acc32{accf, frame}, rmax, st, part, nblk_part);
}

// ------------------------------------ 3D inner CG, TMA-staged z-marching
// A tile is 128 columns x TY rows x zc planes.  The block streams the tile's
// zc + 2 planes (with their x/y halo, box 136 x (TY + 2) x 1, and the
// int16 exponents with 144 x (TY + 2)) through a ring of kTma3Stages
// shared-memory stages, each guarded by an mbarrier with a bounded wait.
// One warp owns one row y of 64 columns (2 per lane) and marches in z: the
// rows at z - 1 and z (u, exponents) stay in registers, the row at z + 1 and
// the y neighbours at z come from shared memory, the x neighbours by warp
// shuffle.  Plane q of the block's stream goes to stage q % kTma3Stages;
// once a block barrier shows every thread done with a plane, the plane
// kTma3Stages further on is issued into its stage (one barrier per plane).
// Arithmetic per node as in k_mixed2d_tma.
constexpr int kTma3Stages = 4;

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// u and neighbour exponents of the lane's two columns in smem row j.
template <int TY>
__device__ __forceinline__ void urow_load(const unsigned char *stage, int j, int lc, float beta,
                                          float &u0, float &u1, int &n0, int &n1) {
  using T = TmaTile<TY>;
  const float *sr = reinterpret_cast<const float *>(stage + T::OFF_R);
  const float *sp = reinterpret_cast<const float *>(stage + T::OFF_P);
  const float *ss = reinterpret_cast<const float *>(stage + T::OFF_S);
  const short *se = reinterpret_cast<const short *>(stage + T::OFF_E);
  const int fo = j * T::FW + lc + 4;
  const float2 r = *reinterpret_cast<const float2 *>(sr + fo);
  const float2 p = *reinterpret_cast<const float2 *>(sp + fo);
  const float2 sg = *reinterpret_cast<const float2 *>(ss + fo);
  const unsigned int ee = *reinterpret_cast<const unsigned int *>(se + j * T::EW + lc + 8);
  u0 = sg.x * fmaf(beta, p.x, r.x);
  u1 = sg.y * fmaf(beta, p.y, r.y);
  n0 = (u0 != 0.f) ? (int)(short)(ee & 0xffffu) : kNoExp;
  n1 = (u1 != 0.f) ? (int)(short)(ee >> 16) : kNoExp;
}

__device__ __forceinline__ float q_node3_le0(float pt, float sg, int ei, float uL, int eL,
                                             float uR, int eR, float uS, int eS, float uN, int eN,
                                             float uD, int eD, float uU, int eU, float wx,
                                             float wy, float wz, int &E) {
  const int m = min(min(ei, min(eL, eR)), min(min(eS, eN), min(eD, eU)));
  E = m;
  const float a1 = uL * pow2f_le0(m - eL) + uR * pow2f_le0(m - eR);
  const float a2 = uS * pow2f_le0(m - eS) + uN * pow2f_le0(m - eN);
  const float a3 = uD * pow2f_le0(m - eD) + uU * pow2f_le0(m - eU);
  return fmaf(-sg, fmaf(wx, a1, fmaf(wy, a2, wz * a3)), pt * pow2f_le0(m - ei));
}

template <bool PASS2, int TY>
__global__ void __launch_bounds__(64 * TY, 1)
k_mixed3d_tma(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_p,
              const __grid_constant__ CUtensorMap tm_e, const __grid_constant__ CUtensorMap tm_s,
              const __grid_constant__ CUtensorMap tm_d, const __grid_constant__ CUtensorMap tm_x,
              Grid g, CellGrid cg, int tiles_x, int tiles_y, int zc, int ntiles,
              const int *__restrict__ kx, float *__restrict__ r32o, float *__restrict__ p32o,
              short *__restrict__ e16o, float *__restrict__ d32, MixState *st, double *part,
              int nblk_part, int px) {
  using T = TmaTile<TY>;
  constexpr int NS = kTma3Stages;
  static_assert(NS >= 4, "the plane ring needs four stages (two read, two ahead)");
  extern __shared__ unsigned char tma_smem_raw[];
  __shared__ __align__(8) uint64_t bar[NS];
  if (st->done) return;
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tma_smem_raw) + 127) & ~uintptr_t(127));
  constexpr int STAGE = PASS2 ? T::STAGE2 : T::STAGE1;
  const float beta = (float)st->beta, alpha = (float)st->alpha;
  const int mode = st->mode;
  const float theta = st->theta;
  const bool want_x = PASS2 && mode != 0;
  const uint32_t tx_bytes =
      3 * (T::FW * T::H * 4) + T::EW * T::H * 2 + (PASS2 ? T::C_BYTES : 0) +
      (want_x ? T::C_BYTES : 0);
  const int frame = st->rho_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cw = warp & 1, ry = warp >> 1;
  const bool half = g.boundary == EIK_BOUNDARY_HALF_CELL;
  const int PL = zc + 2;   // planes per tile
  const int my_tiles =
      (blockIdx.x < ntiles) ? (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const int nq = my_tiles * PL;
  int nissued = 0;   // planes issued so far (thread 0)

  auto issue = [&](int q) {
    nissued = q + 1;
    const int k = q / PL, j = q % PL;
    const int t = blockIdx.x + k * gridDim.x;
    const int stg = q % NS;
    const int xt = t % tiles_x, rest = t / tiles_x;
    const int x0 = xt * kTmaTX, y0 = (rest % tiles_y) * TY, zp = (rest / tiles_y) * zc - 1 + j;
    unsigned char *dst = smem + stg * STAGE;
    mbar_expect_tx(&bar[stg], tx_bytes);
    tma_load_3d(dst + T::OFF_R, &tm_r, x0 - 4, y0 - 1, zp, &bar[stg]);
    tma_load_3d(dst + T::OFF_P, &tm_p, x0 - 4, y0 - 1, zp, &bar[stg]);
    tma_load_3d(dst + T::OFF_S, &tm_s, x0 - 4, y0 - 1, zp, &bar[stg]);
    tma_load_3d(dst + T::OFF_E, &tm_e, x0 - 8, y0 - 1, zp, &bar[stg]);
    if (PASS2) tma_load_3d(dst + T::OFF_D, &tm_d, x0, y0, zp, &bar[stg]);
    if (want_x) tma_load_3d(dst + T::OFF_X, &tm_x, x0, y0, zp, &bar[stg]);
  };
  auto wait = [&](int q) {
    return mbar_wait_bounded(&bar[q % NS], (uint32_t)(q / NS) & 1u);
  };
  auto stage = [&](int q) -> const unsigned char * { return smem + (q % NS) * STAGE; };
  // Called right after a block barrier: every thread is done with all planes
  // below `safe`, so (thread 0) each of them hands its stage to the plane NS
  // further on.
  int rel = 0;   // thread 0: next plane to release
  auto release_below = [&](int safe) {
    if (tid != 0) return;
    bool fenced = false;
    for (; rel < safe; ++rel) {
      if (rel + NS >= nq) continue;
      if (!fenced) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fenced = true;
      }
      issue(rel + NS);
    }
  };

  if (tid == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int q = 0; q < NS && q < nq; ++q) issue(q);

  float accf = 0.f, rmax = 0.f;
  bool fault = false;
  int qwait = 0;   // first plane not yet waited for
  const int lc = 64 * cw + 2 * lane;
  const int hc = (lane == 0) ? lc - 1 : lc + 2;
  for (int k = 0; k < my_tiles && !fault; ++k) {
    const int t = blockIdx.x + k * gridDim.x;
    const int xt = t % tiles_x, rest = t / tiles_x;
    const int x = xt * kTmaTX + lc, y = (rest % tiles_y) * TY + ry;
    const int z0 = (rest / tiles_y) * zc;
    const int q0 = k * PL;
    int kcz = -1, kyi = 0;   // cell exponent of (x, y, z), cached per cell in z
    const float wyz = (half && (y == 0 || y == g.ny - 1)) ? 0.5f : 1.f;   // hy
    const float hx0 = (half && (x == 0 || x == g.nx - 1)) ? 0.5f : 1.f;   // odd nx: x = nx-1
    const float hx1 = (half && x + 1 == g.nx - 1) ? 0.5f : 1.f;
    // prologue: rows at z0 - 1 (u, exponents) and z0 (full)
    bool ok = wait(q0);
    ok = wait(q0 + 1) && ok;
    qwait = q0 + 2;
    if (__syncthreads_or(!ok)) {
      fault = true;
      qwait = q0;
      break;
    }
    release_below(q0);
    float uA0, uA1;
    int nA0, nA1;
    urow_load<TY>(stage(q0), ry + 1, lc, beta, uA0, uA1, nA0, nA1);
    TRow C, B;
    trow_load<TY>(stage(q0 + 1), ry + 1, lc, beta, C);
    for (int i = 0; i < zc; ++i) {
      const int qb = q0 + i + 2;
      const bool okb = wait(qb);
      qwait = qb + 1;
      if (__syncthreads_or(!okb)) {
        fault = true;
        qwait = qb;
        break;
      }
      release_below(qb - 1);   // this step reads planes qb - 1 and qb
      const unsigned char *Sc = stage(qb - 1);
      trow_load<TY>(stage(qb), ry + 1, lc, beta, B);
      float uS0, uS1, uN0, uN1;
      int nS0, nS1, nN0, nN1;
      urow_load<TY>(Sc, ry, lc, beta, uS0, uS1, nS0, nS1);       // y - 1
      urow_load<TY>(Sc, ry + 2, lc, beta, uN0, uN1, nN0, nN1);   // y + 1
      float uh = 0.f;
      int nh = kNoExp;
      if (lane == 0 || lane == 31) tcol_load<TY>(Sc, ry + 1, hc, beta, uh, nh);
      float uL = __shfl_up_sync(0xffffffffu, C.u1, 1);
      int nL = __shfl_up_sync(0xffffffffu, C.n1, 1);
      float uR = __shfl_down_sync(0xffffffffu, C.u0, 1);
      int nR = __shfl_down_sync(0xffffffffu, C.n0, 1);
      if (lane == 0) {
        uL = uh;
        nL = nh;
      }
      if (lane == 31) {
        uR = uh;
        nR = nh;
      }
      const int z = z0 + i;
      if (x < g.nx && y < g.ny && z < g.nz) {
        const float hz = (half && (z == 0 || z == g.nz - 1)) ? 0.5f : 1.f;
        // x edges carry hy hz, y edges hx hz, z edges hx hy
        int E0, E1;
        const float q0v = q_node3_le0(C.pt0, C.s0, C.e0, uL, nL, C.u1, C.n1, uS0, nS0, uN0, nN0,
                                      uA0, nA0, B.u0, B.n0, wyz * hz, hx0 * hz, hx0 * wyz, E0);
        const float q1v = q_node3_le0(C.pt1, C.s1, C.e1, C.u0, C.n0, uR, nR, uS1, nS1, uN1, nN1,
                                      uA1, nA1, B.u1, B.n1, wyz * hz, hx1 * hz, hx1 * wyz, E1);
        if (!PASS2) {
          accf = fmaf(C.pt0 * q0v, pow2f(-(C.e0 + E0) - frame), accf);
          accf = fmaf(C.pt1 * q1v, pow2f(-(C.e1 + E1) - frame), accf);
        } else {
          const int li = ry * kTmaTX + lc;   // tile-local index, no halo
          const float2 dd = *reinterpret_cast<const float2 *>(Sc + T::OFF_D + 4 * li);
          float2 xr = make_float2(0.f, 0.f);
          if (want_x) xr = *reinterpret_cast<const float2 *>(Sc + T::OFF_X + 4 * li);
          if ((z >> cg.lgB) != kcz) {   // x, x+1: one cell; y fixed per warp
            kcz = z >> cg.lgB;
            kyi = kx[cell_of(cg, x, y, z)];
          }
          float d[2] = {dd.x, dd.y}, rn[2], pn[2];
          int en[2];
          const float pt[2] = {C.pt0, C.pt1}, rr[2] = {C.r0, C.r1}, qq[2] = {q0v, q1v};
          const int ee[2] = {C.e0, C.e1}, EE[2] = {E0, E1};
          const float xx[2] = {xr.x, xr.y};
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            if (pt[c] != 0.f) d[c] = fmaf(alpha * pt[c], pow2f(kyi - ee[c]), d[c]);
            const float f = pow2f_le0(EE[c] - ee[c]);
            const float rE = fmaf(-alpha, qq[c], rr[c] * f);
            const float pE = pt[c] * f;
            const float mx = fmaxf(fabsf(rE), fabsf(pE));
            if (mx > 0.f && mx <= 3.4e38f) {
              const int sh = expof(mx);
              const float sc = __int_as_float((127 - sh) << 23);
              rn[c] = rE * sc;
              pn[c] = pE * sc;
              en[c] = EE[c] - sh;
              accf = fmaf(rn[c] * rn[c], pow2f(-2 * en[c] - frame), accf);
              const float rk = fabsf(rn[c]) * pow2f(kyi - en[c]);
              if (mode == 0)
                rmax = fmaxf(rmax, rk);
              else if (rk > theta * fabsf(xx[c] + d[c]))
                rmax = 1.f;
            } else {
              rn[c] = 0.f;
              pn[c] = 0.f;
              en[c] = kNoExp;
              if (!(mx <= 3.4e38f)) rmax = INFINITY;
            }
          }
          const int64_t o = ((int64_t)z * g.ny + y) * px + x;   // pitched rows
          *reinterpret_cast<float2 *>(d32 + o) = make_float2(d[0], d[1]);
          *reinterpret_cast<float2 *>(r32o + o) = make_float2(rn[0], rn[1]);
          *reinterpret_cast<float2 *>(p32o + o) = make_float2(pn[0], pn[1]);
          *reinterpret_cast<unsigned int *>(e16o + o) = pack2(en[0], en[1]);
        }
      }
      uA0 = C.u0;
      uA1 = C.u1;
      nA0 = C.n0;
      nA1 = C.n1;
      C = B;
    }
  }
  if (fault) {
    // leave no copy in flight: wait (bounded) for every plane issued and not
    // yet waited for
    if (tid == 0) {
      atomicExch(&st->fault, 1);
      for (int q = qwait; q < nissued; ++q)
        mbar_wait_bounded(&bar[q % NS], (uint32_t)(q / NS) & 1u);
    }
    __syncthreads();
  }
  inner_pass_tail<PASS2>(Acc32{accf, frame}, rmax, st, part, nblk_part);
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
  bool rows2d = false;           // warp-marched 2D kernels (nx % vec == 0)
  int vec = 2;                   // columns per lane
  int tiles_x = 0, ntiles2d = 0, nblk2d = 0;
  int tma = 0;                   // TMA-staged 2D kernels: variant index (0 = off)
  int tma_tiles_x = 0, tma_ntiles = 0, tma_nblk1 = 0, tma_nblk2 = 0;
  int tma_tiles_y = 0, tma_zc = 0;   // 3D: rows per tile come from the variant
  int px = 0;                        // row pitch of the FP32 / int16 arrays
  CUtensorMap tm_r[2], tm_p[2], tm_e[2], tm_s, tm_d, tm_x;
  float *s32 = nullptr, *fb = nullptr, *St = nullptr, *d32 = nullptr, *xref = nullptr;
  float *r32[2] = {nullptr, nullptr}, *p32[2] = {nullptr, nullptr};
  short *e16[2] = {nullptr, nullptr};
  int *kx = nullptr;
  double *x64 = nullptr, *part = nullptr;
  MixState *st = nullptr, *h_st = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t launches[8] = {0};
  // per-launch CUDA-event timing of the inner passes when profiling
  bool profile = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  int64_t timed[8] = {0};
  double ms[8] = {0};
};

static const char *kMixedNames[] = {"mixed_setup", "coarse_exponents", "mixed_residual64",
                                    "mixed_pass1", "mixed_pass2", "mixed_update",
                                    "mixed_epilogue", nullptr};

const char *mixed_kernel_name(int k) {
  if (k < 0 || k >= 7) return nullptr;
  return kMixedNames[k];
}

int64_t mixed_kernel_launches(const MixedState *m, int k) {
  return (m && k >= 0 && k < 8) ? m->launches[k] : 0;
}

void mixed_reset_launches(MixedState *m) {
  if (!m) return;
  for (int k = 0; k < 8; ++k) {
    m->launches[k] = 0;
    m->timed[k] = 0;
    m->ms[k] = 0.0;
  }
}

void mixed_set_profiling(MixedState *m, bool on) {
  if (m) m->profile = on;
}

void mixed_kernel_time(const MixedState *m, int k, int64_t *timed, double *ms) {
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

// TMA variants: (rows per tile, row groups per block); 2 warps per row
// group.  Variant 3 (16 rows, 8 warps) is the library default: it measured
// fastest on the 2048^2 workload.
constexpr int kTmaVariantCount = 9;
// rows per tile.  2D (row groups, stages): 1 (2, 2), 2 (4, 2), 3 (4, 2),
// 4 (2, 2), 7 (4, 4), 8 (4, 3), 9 (2, 4); variants 5, 6 are the 3D kernels.
constexpr int kTmaTYs[kTmaVariantCount] = {16, 32, 16, 32, 4, 8, 8, 16, 8};

template <int TY, int RG, int NS>
static bool tma_setup_t(MixedState *m, int num_sms) {
  using T = TmaTile<TY>;
  const int s1 = T::smem(false, NS), s2 = T::smem(true, NS);
  if (cudaFuncSetAttribute(k_mixed2d_tma<false, TY, RG, NS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, s1) != cudaSuccess ||
      cudaFuncSetAttribute(k_mixed2d_tma<true, TY, RG, NS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, s2) != cudaSuccess)
    return false;
  int per1 = 0, per2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_mixed2d_tma<false, TY, RG, NS>, 64 * RG,
                                                    s1) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_mixed2d_tma<true, TY, RG, NS>, 64 * RG,
                                                    s2) != cudaSuccess)
    return false;
  if (per1 < 1 || per2 < 1) return false;
  m->tma_tiles_x = (m->g.nx + kTmaTX - 1) / kTmaTX;
  m->tma_ntiles = m->tma_tiles_x * ((m->g.ny + TY - 1) / TY);
  m->tma_nblk1 = std::min(m->tma_ntiles, per1 * num_sms);
  m->tma_nblk2 = std::min(m->tma_ntiles, per2 * num_sms);
  return true;
}

// 3D variants 5 / 6: TY = 4 / 8 rows per tile (2 warps per row).  The
// number of planes per tile, zc, is chosen to balance the tiles over the
// resident blocks.
template <int TY>
static bool tma3_setup_t(MixedState *m, int num_sms) {
  using T = TmaTile<TY>;
  const int s1 = kTma3Stages * T::STAGE1 + 128, s2 = kTma3Stages * T::STAGE2 + 128;
  if (cudaFuncSetAttribute(k_mixed3d_tma<false, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           s1) != cudaSuccess ||
      cudaFuncSetAttribute(k_mixed3d_tma<true, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           s2) != cudaSuccess)
    return false;
  int per1 = 0, per2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_mixed3d_tma<false, TY>, 64 * TY,
                                                    s1) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_mixed3d_tma<true, TY>, 64 * TY,
                                                    s2) != cudaSuccess)
    return false;
  if (per1 < 1 || per2 < 1) return false;
  const Grid &g = m->g;
  m->tma_tiles_x = (g.nx + kTmaTX - 1) / kTmaTX;
  m->tma_tiles_y = (g.ny + TY - 1) / TY;
  const int64_t plane_tiles = (int64_t)m->tma_tiles_x * m->tma_tiles_y;
  int best_zc = 8;
  int64_t best_cost = INT64_MAX;
  for (int zc : {8, 16, 32, 64}) {
    const int64_t nt = plane_tiles * ((g.nz + zc - 1) / zc);
    const int64_t nb = std::min<int64_t>(nt, (int64_t)per2 * num_sms);
    const int64_t cost = ((nt + nb - 1) / nb) * (zc + 2);
    if (cost <= best_cost) {
      best_cost = cost;
      best_zc = zc;
    }
  }
  const int64_t nt = plane_tiles * ((g.nz + best_zc - 1) / best_zc);
  if (nt > INT_MAX / (best_zc + 2)) return false;
  m->tma_zc = best_zc;
  m->tma_ntiles = (int)nt;
  m->tma_nblk1 = (int)std::min<int64_t>(nt, (int64_t)per1 * num_sms);
  m->tma_nblk2 = (int)std::min<int64_t>(nt, (int64_t)per2 * num_sms);
  return true;
}

static bool tma_setup(MixedState *m, int v, int num_sms) {
  m->tma = v;
  switch (v) {
    case 1: return tma_setup_t<16, 2, 2>(m, num_sms);
    case 2: return tma_setup_t<32, 4, 2>(m, num_sms);
    case 3: return tma_setup_t<16, 4, 2>(m, num_sms);
    case 4: return tma_setup_t<32, 2, 2>(m, num_sms);
    case 5: return tma3_setup_t<4>(m, num_sms);
    case 6: return tma3_setup_t<8>(m, num_sms);
    case 7: return tma_setup_t<8, 4, 4>(m, num_sms);
    case 8: return tma_setup_t<16, 4, 3>(m, num_sms);
    case 9: return tma_setup_t<8, 2, 4>(m, num_sms);
  }
  return false;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tiled tensor map over a row-major nx x ny (x nz) array, box bw x bh (x 1)
// elements; nz == 0 gives a 2D map.
static bool encode_map(CUtensorMap *map, void *base, bool is_short, int nx, int px, int ny,
                       int nz, int bw, int bh) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const size_t es = is_short ? 2 : 4;
  const cuuint32_t rank = nz > 0 ? 3 : 2;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)(nz > 0 ? nz : 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)px * es, (cuuint64_t)px * ny * es};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, is_short ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
            rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool tma_encode(MixedState *m) {
  const int ty = kTmaTYs[m->tma - 1];
  const int nx = m->g.nx, px = m->px, ny = m->g.ny, nz = (m->g.ndim == 3) ? m->g.nz : 0;
  const int fw = kTmaTX + 8, ew = kTmaTX + 16, h = ty + 2;
  bool ok = true;
  for (int k = 0; k < 2; ++k) {
    ok = ok && encode_map(&m->tm_r[k], m->r32[k], false, nx, px, ny, nz, fw, h);
    ok = ok && encode_map(&m->tm_p[k], m->p32[k], false, nx, px, ny, nz, fw, h);
    ok = ok && encode_map(&m->tm_e[k], m->e16[k], true, nx, px, ny, nz, ew, h);
  }
  ok = ok && encode_map(&m->tm_s, m->s32, false, nx, px, ny, nz, fw, h);
  ok = ok && encode_map(&m->tm_d, m->d32, false, nx, px, ny, nz, kTmaTX, ty);
  ok = ok && encode_map(&m->tm_x, m->xref, false, nx, px, ny, nz, kTmaTX, ty);
  return ok;
}

template <class T>
static bool mal(T **p, size_t n) {
  return cudaMalloc((void **)p, sizeof(T) * (n ? n : 1)) == cudaSuccess;
}

eik_status mixed_create(MixedState **out, const Grid &g, const TileCount &tc, int num_sms,
                        int tile_override, cudaStream_t s) {
  MixedState *m = new MixedState();
  m->g = g;
  m->tc = tc;
  // cell edge: power of two >= 16 with at most kMaxCells cells
  int lg = 4;
  for (;; ++lg) {
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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mixed_pass2<2>, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mixed_pass2<3>, kThreads, 0);
  if (per_sm < 1) per_sm = 1;
  m->nblk_stencil = (int)std::min<int64_t>(tc.total, (int64_t)per_sm * num_sms);
  m->cap = num_sms * 8;
  // tile_override: 0 library choice, 1 generic halo tiles, 2 / 3 warp-marched
  // rows with 4 / 2 columns per lane, 4..7 TMA-staged tiles (variants 1..4
  // listed at kTmaTYs)
  const int vec = (tile_override == 2) ? 4 : 2;
  // Library choice: TMA tiles where the row pitch is already a multiple of 8
  // or the grid is large (>= 2^20 nodes; its FP32 arrays are then padded);
  // small odd-width grids measured faster on the register-marched or generic
  // kernels (few tiles per block leave the TMA pipeline no depth).  An
  // explicit TMA variant always pads.
  const bool tma_default = g.nx % 8 == 0 || g.n >= (int64_t(1) << 20);
  const bool tma_ok = g.ndim == 2 &&
                      ((tile_override == 0 && tma_default) ||
                       (tile_override >= 4 && tile_override <= 7) ||
                       (tile_override >= 10 && tile_override <= 12));
  const bool tma3_ok = g.ndim == 3 && ((tile_override == 0 && tma_default) ||
                                       tile_override == 8 || tile_override == 9);
  const bool march_ok = g.ndim == 2 && g.nx % vec == 0 &&
                        (tile_override == 0 || tile_override == 2 || tile_override == 3);
  if (march_ok) {
    int per = 0;
    if (vec == 4)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mixed2d<true, 4>, kWarpsPerBlock * 32, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mixed2d<true, 2>, kWarpsPerBlock * 32, 0);
    if (per < 1) per = 1;
    m->rows2d = true;
    m->vec = vec;
    m->tiles_x = (g.nx + 32 * vec - 1) / (32 * vec);
    m->ntiles2d = m->tiles_x * ((g.ny + kRowTile - 1) / kRowTile);
    m->nblk2d = std::min(m->ntiles2d, per * num_sms);
  }
  if (tma_ok) {
    // tile_override 4..7 -> variants 1..4, 10..12 -> variants 7..9
    const int v = (tile_override >= 4) ? tile_override - 3 : 3;   // default: 16 rows, 8 warps
    if (v <= kTmaVariantCount && tma_setup(m, v, num_sms)) {
      m->rows2d = false;
    } else {
      m->tma = 0;
      cudaGetLastError();
    }
  }
  if (tma3_ok) {
    const int v = (tile_override == 9) ? 6 : 5;   // default: 4 rows per tile
    if (!tma_setup(m, v, num_sms)) {
      m->tma = 0;
      cudaGetLastError();
    }
  }
  m->nblk_part = std::max(std::max(m->nblk_stencil, m->cap), m->nblk2d);
  m->nblk_part = std::max(m->nblk_part, std::max(m->tma_nblk1, m->tma_nblk2));
  // row pitch of the FP32 / int16 arrays: a multiple of 8 for the TMA
  // kernels (16-byte aligned rows for the tensor maps), nx otherwise
  m->px = m->tma ? (g.nx + 7) / 8 * 8 : g.nx;
  const int64_t n = g.n;
  const int64_t np = (g.n / g.nx) * m->px;
  bool ok = mal(&m->s32, np) && mal(&m->d32, np) && mal(&m->xref, np) && mal(&m->r32[0], np) &&
            mal(&m->r32[1], np) && mal(&m->p32[0], np) && mal(&m->p32[1], np) &&
            mal(&m->e16[0], np) && mal(&m->e16[1], np) && mal(&m->x64, n) &&
            mal(&m->fb, m->cg.ncell) &&
            mal(&m->St, m->cg.ncell) && mal(&m->kx, m->cg.ncell) &&
            mal(&m->part, 8 * (size_t)m->nblk_part) && mal(&m->st, 1);
  if (ok) ok = cudaMallocHost((void **)&m->h_st, sizeof(MixState)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    mixed_destroy(m);
    g_msg = "device allocation failed";
    return EIK_ERR_OOM;
  }
  if (m->tma && !tma_encode(m)) {
    mixed_destroy(m);
    g_msg = "cannot encode the TMA tensor maps";
    return EIK_ERR_CUDA;
  }
  // the attribute belongs to the function, not to this solver: set it to the
  // largest cell grid any solver can use, so concurrent solvers agree
  const size_t smem = 2 * sizeof(float) * kMaxCells;
  if (cudaFuncSetAttribute(k_coarse_exponents, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    mixed_destroy(m);
    g_msg = "cannot reserve shared memory for the coarse estimate";
    return EIK_ERR_CUDA;
  }
  (void)s;
  *out = m;
  return EIK_OK;
}

void mixed_destroy(MixedState *m) {
  if (!m) return;
  if (m->graph) cudaGraphExecDestroy(m->graph);
  for (auto &e : m->ev)
    if (e) cudaEventDestroy(e);
  void *ptrs[] = {m->s32, m->xref, m->fb, m->St, m->d32, m->r32[0], m->r32[1], m->p32[0],
                  m->p32[1], m->e16[0], m->e16[1], m->kx, m->x64, m->part, m->st};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (m->h_st) cudaFreeHost(m->h_st);
  delete m;
}

static void launch_residual(MixedState *m, const MixedArgs &a) {
  if (m->g.ndim == 2)
    k_mixed_residual<2><<<m->nblk_stencil, kThreads, 0, a.stream>>>(
        m->g, m->tc, m->cg, m->kx, a.sig, m->x64, m->r32[0], m->p32[0], m->e16[0], m->d32,
        m->xref, m->st, m->part, m->nblk_part, m->px);
  else
    k_mixed_residual<3><<<m->nblk_stencil, kThreads, 0, a.stream>>>(
        m->g, m->tc, m->cg, m->kx, a.sig, m->x64, m->r32[0], m->p32[0], m->e16[0], m->d32,
        m->xref, m->st, m->part, m->nblk_part, m->px);
  m->launches[2]++;
}

static void launch_iteration(MixedState *m, int set, cudaStream_t s, bool timed = false) {
  const int a = set, b = 1 - set;
  double *p1 = m->part;
  double *p2 = m->part + 3 * (size_t)m->nblk_part;
  if (m->tma) {
#define EIK_LAUNCH_TMA(TY, RG, NS)                                                              \
  do {                                                                                          \
    if (timed) cudaEventRecord(m->ev[0], s);                                                    \
    k_mixed2d_tma<false, TY, RG, NS>                                                            \
        <<<m->tma_nblk1, 64 * RG, TmaTile<TY>::smem(false, NS), s>>>(                           \
        m->tm_r[a], m->tm_p[a], m->tm_e[a], m->tm_s, m->tm_d, m->tm_x, m->g, m->cg,             \
        m->tma_tiles_x, m->tma_ntiles, m->kx, nullptr, nullptr, nullptr, m->d32, m->st, p1,     \
        m->nblk_part, m->px);                                                                   \
    if (timed) cudaEventRecord(m->ev[1], s);                                                    \
    k_mixed2d_tma<true, TY, RG, NS>                                                             \
        <<<m->tma_nblk2, 64 * RG, TmaTile<TY>::smem(true, NS), s>>>(                            \
        m->tm_r[a], m->tm_p[a], m->tm_e[a], m->tm_s, m->tm_d, m->tm_x, m->g, m->cg,             \
        m->tma_tiles_x, m->tma_ntiles, m->kx, m->r32[b], m->p32[b], m->e16[b], m->d32, m->st,   \
        p2, m->nblk_part, m->px);                                                               \
    if (timed) cudaEventRecord(m->ev[2], s);                                                    \
  } while (0)
#define EIK_LAUNCH_TMA3(TY)                                                                     \
  do {                                                                                          \
    using T3 = TmaTile<TY>;                                                                     \
    if (timed) cudaEventRecord(m->ev[0], s);                                                    \
    k_mixed3d_tma<false, TY><<<m->tma_nblk1, 64 * TY, kTma3Stages * T3::STAGE1 + 128, s>>>(     \
        m->tm_r[a], m->tm_p[a], m->tm_e[a], m->tm_s, m->tm_d, m->tm_x, m->g, m->cg,             \
        m->tma_tiles_x, m->tma_tiles_y, m->tma_zc, m->tma_ntiles, m->kx, nullptr, nullptr,      \
        nullptr, m->d32, m->st, p1, m->nblk_part, m->px);                                       \
    if (timed) cudaEventRecord(m->ev[1], s);                                                    \
    k_mixed3d_tma<true, TY><<<m->tma_nblk2, 64 * TY, kTma3Stages * T3::STAGE2 + 128, s>>>(      \
        m->tm_r[a], m->tm_p[a], m->tm_e[a], m->tm_s, m->tm_d, m->tm_x, m->g, m->cg,             \
        m->tma_tiles_x, m->tma_tiles_y, m->tma_zc, m->tma_ntiles, m->kx, m->r32[b], m->p32[b],  \
        m->e16[b], m->d32, m->st, p2, m->nblk_part, m->px);                                     \
    if (timed) cudaEventRecord(m->ev[2], s);                                                    \
  } while (0)
    switch (m->tma) {
      case 1: EIK_LAUNCH_TMA(16, 2, 2); break;
      case 2: EIK_LAUNCH_TMA(32, 4, 2); break;
      case 3: EIK_LAUNCH_TMA(16, 4, 2); break;
      case 4: EIK_LAUNCH_TMA(32, 2, 2); break;
      case 5: EIK_LAUNCH_TMA3(4); break;
      case 6: EIK_LAUNCH_TMA3(8); break;
      case 7: EIK_LAUNCH_TMA(8, 4, 4); break;
      case 8: EIK_LAUNCH_TMA(16, 4, 3); break;
      default: EIK_LAUNCH_TMA(8, 2, 4); break;
    }
#undef EIK_LAUNCH_TMA
#undef EIK_LAUNCH_TMA3
    return;
  }
  if (m->rows2d) {
#define EIK_LAUNCH_2D(V)                                                                        \
  do {                                                                                          \
    if (timed) cudaEventRecord(m->ev[0], s);                                                    \
    k_mixed2d<false, V><<<m->nblk2d, kWarpsPerBlock * 32, 0, s>>>(                              \
        m->g, m->cg, m->tiles_x, m->ntiles2d, m->kx, m->r32[a], m->p32[a], m->e16[a], m->s32,   \
        nullptr, nullptr, nullptr, m->d32, m->xref, m->st, p1, m->nblk_part);                   \
    if (timed) cudaEventRecord(m->ev[1], s);                                                    \
    k_mixed2d<true, V><<<m->nblk2d, kWarpsPerBlock * 32, 0, s>>>(                               \
        m->g, m->cg, m->tiles_x, m->ntiles2d, m->kx, m->r32[a], m->p32[a], m->e16[a], m->s32,   \
        m->r32[b], m->p32[b], m->e16[b], m->d32, m->xref, m->st, p2, m->nblk_part);             \
    if (timed) cudaEventRecord(m->ev[2], s);                                                    \
  } while (0)
    if (m->vec == 4)
      EIK_LAUNCH_2D(4);
    else
      EIK_LAUNCH_2D(2);
#undef EIK_LAUNCH_2D
    return;
  }
  if (timed) cudaEventRecord(m->ev[0], s);
  if (m->g.ndim == 2)
    k_mixed_pass1<2><<<m->nblk_stencil, kThreads, 0, s>>>(m->g, m->tc, m->r32[a], m->p32[a],
                                                         m->e16[a], m->s32, m->st, p1,
                                                         m->nblk_part);
  else
    k_mixed_pass1<3><<<m->nblk_stencil, kThreads, 0, s>>>(m->g, m->tc, m->r32[a], m->p32[a],
                                                         m->e16[a], m->s32, m->st, p1,
                                                         m->nblk_part);
  if (timed) cudaEventRecord(m->ev[1], s);
  if (m->g.ndim == 2) {
    k_mixed_pass2<2><<<m->nblk_stencil, kThreads, 0, s>>>(
        m->g, m->tc, m->cg, m->kx, m->r32[a], m->p32[a], m->e16[a], m->s32, m->r32[b],
        m->p32[b], m->e16[b], m->d32, m->xref, m->st, p2, m->nblk_part);
  } else {
    k_mixed_pass2<3><<<m->nblk_stencil, kThreads, 0, s>>>(
        m->g, m->tc, m->cg, m->kx, m->r32[a], m->p32[a], m->e16[a], m->s32, m->r32[b],
        m->p32[b], m->e16[b], m->d32, m->xref, m->st, p2, m->nblk_part);
  }
  if (timed) cudaEventRecord(m->ev[2], s);
}

static eik_status build_graph(MixedState *m, cudaStream_t s) {
  if (m->graph) return EIK_OK;
  cudaGraph_t graph;
  MCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < kInnerGraphIters; ++k) launch_iteration(m, k & 1, s);
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
    MixState init{};
    init.band_lo = lo;
    init.band_hi = hi;
    *m->h_st = init;
    MCK(cudaMemcpyAsync(m->st, m->h_st, sizeof(MixState), cudaMemcpyHostToDevice, s));
    launch_residual(m, a);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(m->h_st, m->st, sizeof(MixState), cudaMemcpyDeviceToHost, s));
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
    MixState st = *m->h_st;
    st.iter = 0;
    st.done = 0;
    st.status = 0;
    st.beta = 0.0;
    st.max_iter = a.opt.max_iter - total;
    st.withhold = (a.opt.test_flags & 1) ? 1 : 0;
    st.mode = (outer == 0 || !std::isfinite(cw)) ? 0 : 1;
    st.thresh = (float)(red * st.r_inf);
    st.theta = (float)std::max(0.5 * tol, 1e-3 * cw);
    *m->h_st = st;
    MCK(cudaMemcpyAsync(m->st, m->h_st, sizeof(MixState), cudaMemcpyHostToDevice, s));
    if (m->profile && !m->ev[0])
      for (auto &e : m->ev) MCK(cudaEventCreate(&e));
    for (int it = 0;; ++it) {
      if (trace && it < 6) {
        launch_iteration(m, it & 1, s);
        MCK(cudaMemcpyAsync(m->h_st, m->st, sizeof(MixState), cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        fprintf(stderr, "[mixed]   it %d alpha %.9e beta %.9e rho %.9e*2^%d\n", m->h_st->iter,
                m->h_st->alpha, m->h_st->beta, m->h_st->rho_m, m->h_st->rho_s);
        if (m->h_st->done) break;
        continue;   // six traced iterations: the graph resumes on buffer set 0
      }
      if (m->profile) {
        // one timed iteration per host check: no launch runs past convergence
        launch_iteration(m, it & 1, s, true);
        m->launches[3] += 1;
        m->launches[4] += 1;
      } else {
        MCK(cudaGraphLaunch(m->graph, s));
        m->launches[3] += kInnerGraphIters;
        m->launches[4] += kInnerGraphIters;
      }
      MCK(cudaMemcpyAsync(m->h_st, m->st, sizeof(MixState), cudaMemcpyDeviceToHost, s));
      MCK(cudaStreamSynchronize(s));
      if (m->profile) {
        float t1 = 0.f, t2 = 0.f;
        MCK(cudaEventElapsedTime(&t1, m->ev[0], m->ev[1]));
        MCK(cudaEventElapsedTime(&t2, m->ev[1], m->ev[2]));
        m->ms[3] += t1;
        m->ms[4] += t2;
        m->timed[3] += 1;
        m->timed[4] += 1;
      }
      if (m->h_st->done) break;
    }
    total += m->h_st->iter;
    ++outer;
    if (trace)
      fprintf(stderr, "[mixed]   inner end: iters %d status %d alpha %.3e beta %.3e rho %.3e*2^%d\n",
              m->h_st->iter, m->h_st->status, m->h_st->alpha, m->h_st->beta, m->h_st->rho_m,
              m->h_st->rho_s);
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
  eik_status gs = build_graph(m, s);
  if (gs != EIK_OK) return gs;

  const int band_bits = (a.opt.band_bits > 0) ? a.opt.band_bits : kBandBits;
  int kmin = 0, kmax = 0;
  if (a.opt.band_bits >= 0) {
    std::vector<int> hk(m->cg.ncell);
    MCK(cudaMemcpyAsync(hk.data(), m->kx, sizeof(int) * hk.size(), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    kmin = *std::min_element(hk.begin(), hk.end());
    kmax = *std::max_element(hk.begin(), hk.end());
  }
  const int max_outer = (a.opt.max_outer > 0) ? a.opt.max_outer : 30;
  int total = 0, outer = 0;
  eik_status result;
  const int sweep_bits = (a.opt.band_bits > 0) ? 2 * a.opt.band_bits : kSweepBits;
  if (a.opt.band_bits < 0 || kmax - kmin <= sweep_bits) {
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
        if (trace) fprintf(stderr, "[mixed] sweep %d band [%d, %d)\n", sweep, lo, hi);
        const eik_status bs = refine(m, a, lo, hi, max_outer, &total, &outer, res_cw, trace);
        if (bs != EIK_OK && bs != EIK_ERR_NOT_CONVERGED) return bs;   // breakdown, timeout, CUDA
        if (hi > kmax || total >= a.opt.max_iter) break;
      }
      k_sig32<<<blocks(g.n), kThreads, 0, s>>>(g.n, g.nx, m->px, a.sig, m->s32);
      m->launches[0]++;
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
