// Multigrid-preconditioned inner solve of the mixed-precision path (2D, 3D).
//
// The paper names multigrid as the O(N) route for the sparse system of
// Sec. 6 (Eq. sparse-system); this file builds one that keeps the relative
// accuracy the method needs.  phi = exp(-S/hbar) spans hundreds of powers of
// two, and a componentwise tolerance asks for the far field as precisely as
// the near field, so the coarse spaces are built in relative form:
//
// * Level 0 is the Jacobi-scaled operator of the correction equation in kx
//   units, (A v)_i = v_i - sig_i sum_j omega_ij sig_j 2^(kx_i - kx_j) v_j,
//   exactly as in the Jacobi-preconditioned inner CG.
// * Coarse node C of level l + 1 aggregates a 2 x 2 (x 2) box of level-l
//   nodes.  Its basis function is, on level 0, the estimated solution shape
//   w_i = exp(kx_i ln 2 - St_i / hbar) / sig_i on the box (St_i: the cell
//   distance estimate interpolated (bi/tri)linearly between cell centres), so a
//   coarse unknown is a relative correction, constant on its box, of the
//   estimated phi.  Coarser levels take unit weights, so every coarse basis
//   function keeps that level-0 shape.
// * Every level l holds its Galerkin operator A^l = P^T A^(l-1) P (true,
//   symmetric) for vectors stored as value * 2^k, k a power-of-two exponent
//   per node: (A y)_C = a_C y_C + sum_D c_CD y_D with the row-relative
//   coefficients c_CD = A_CD 2^(k_C - k_D), one per neighbour (west, east,
//   south, north, below, above), formed in FP64.  Between an aggregate and its upstream
//   neighbour (nearer the sources) c is O(1); downstream it is tiny or 0.
//   (Storing A_CD and the factor separately would overflow FP32 on coarse
//   levels, where neighbouring exponents differ by over a hundred.)  The
//   transfers in these units: restriction g_C = sum_{i in C} P_i 2^(k_C -
//   k_i) t_i, prolongation y_i += P_i 2^(k_i - k_C) y_C, with P_i = w_i on
//   level 0 (one exponent per box there) and P_i = 2^(k_C - k_i), k_C = min
//   over the box, above; so c^(l+1)_CD = sum_{i in C, j in D} 2^(2(k_C -
//   k_i)) c_ij and a^(l+1)_C = sum_{i in C} 2^(2(k_C - k_i)) (a_i + sum_{j in
//   C} c_ij).
// * The cycle is a symmetric V-cycle down to one node: one damped-Jacobi
//   sweep (omega = 8/9) before and after each coarse correction, the single
//   node solved exactly.  Sources (sig = 0) take no part in any transfer.
//
// The outer iteration is preconditioned CG on level 0 in kx units with the
// true inner product, <u, v> = sum u_i v_i 2^(-2 kx_i) (per-thread FP32
// sums, weights relative to the smallest exponent, 0 past the FP32 range;
// FP64 across threads and blocks in a fixed order),
// one graph launch per two iterations:
//   z = M r, rho = <r, z>, beta = rho / rho_old, p = z + beta p, q = A p,
//   alpha = rho / <p, q>, d += alpha p, r -= alpha q,
// and the inner solve stops on the mixed solve's tests (scaled max norm of r
// or the componentwise test against the iterate).  Measured on a CPU model of
// this scheme (FP32 inner vectors, FP64 refinement): 56 inner iterations
// instead of 998 for Jacobi-PCG on a 513^2 workload with hbar = 10.2 h, and
// 72 / 79 with hbar = 4 h / 2 h (phi down to e^-128, no level-set bands).
#include <cuda.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <climits>
#include <string>
#include <vector>

#include "eik_mg.h"

namespace eik {

namespace {

constexpr float kOmega = 8.0f / 9.0f;   // Chebyshev-optimal single step on [1/4, 2]
constexpr int kGraphIters = 2;          // even: the direction buffers alternate
// an inner solve that has not met its test after this many iterations ends
// (the refinement step then judges progress from the true residual)
constexpr int kMaxInnerIters = 1000;
thread_local std::string g_msg = "no error";

enum { kW = 0, kE = 1, kS = 2, kN = 3, kB = 4, kT = 5, kDirs = 6 };

struct MgLevel {
  int nx = 0, ny = 0, nz = 1;
  float *a = nullptr;            // diagonal; a < 0 marks a node with no unknowns
  float *ia = nullptr;           // 1 / a (0 on nodes with no unknowns)
  float *c = nullptr;            // kDirs x m row-relative coefficients (W, E, S, N, B, T)
  int *k = nullptr;
  float *g = nullptr, *y = nullptr;
};

struct MgCtl {
  double rho;        // <r, z> of the current residual
  double alpha, beta;
  int iter, max_iter, done, status, stalled, mode, first, kmin;
  float thresh, theta;
  unsigned int counter[4];
};

__device__ __forceinline__ int kx_at(const CellGrid &cg, int x, int y, int z, const int *kx) {
  return kx[(x >> cg.lgB) + cg.cx * ((y >> cg.lgB) + cg.cy * (z >> cg.lgB))];
}
__device__ __forceinline__ float face(int i, int n, int boundary) {
  return (boundary == EIK_BOUNDARY_HALF_CELL && (i == 0 || i == n - 1)) ? 0.5f : 1.f;
}
// the face factor of the z axis (1 in 2D, which has no z faces)
__device__ __forceinline__ float facez(const Grid &g, int z) {
  return (g.nz > 1) ? face(z, g.nz, g.boundary) : 1.f;
}

// 2^e from its bit pattern; 0 below the normal range (such factors only
// scale terms that are negligible), e capped at 127.
__device__ __forceinline__ float p2f(int e) {
  e = min(e, 127);
  return (e < -126) ? 0.f : __int_as_float((e + 127) << 23);
}

// Grid-stride loops over the rows (y, z) of a level (blockIdx.y) and its
// columns x: no 64-bit division per node.
#define MG_ROWS(ny_, nz_)                                              \
  for (int rr = blockIdx.y; rr < (ny_) * (nz_); rr += gridDim.y)      \
    for (int y = rr % (ny_), z = rr / (ny_), once_ = 1; once_; once_ = 0)
#define MG_COLS(nx_) \
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < (nx_); x += gridDim.x * blockDim.x)

// Level-0 off-diagonal sum  sig_i sum_j omega_ij sig_j 2^(k_i - k_j) v(j)
// for the node (x, y, z); v(j, xj, yj, zj) gives the vector at pitched
// index j.  The exponent is looked up only where the neighbour lies in
// another cell.  Edge weights: the product of the face factors of the other
// axes (Sec. 6 with zero-flux faces, half cells on the faces).
// Linear index of (x, y, z) on a level of pitch nx and ny rows per plane
// (DIM = 2: z is 0).
template <int DIM>
__device__ __forceinline__ int64_t lin(int x, int y, int z, int nx, int ny) {
  if constexpr (DIM == 3) return x + (int64_t)nx * (y + (int64_t)ny * z);
  else return x + (int64_t)nx * y;
}

template <int DIM, class V>
__device__ __forceinline__ float nb0(const Grid &g, const CellGrid &cg, int px,
                                     const float *__restrict__ s32, const int *__restrict__ kx,
                                     int x, int y, int z, int ki, V v) {
  float acc = 0.f;
  const int mask = cg.B - 1;
  const float hx = face(x, g.nx, g.boundary), hy = face(y, g.ny, g.boundary);
  const float hz = (DIM == 3) ? facez(g, z) : 1.f;
  const int64_t i = lin<DIM>(x, y, z, px, g.ny);
  if (x > 0) {
    const float f = ((x & mask) == 0) ? p2f(ki - kx_at(cg, x - 1, y, z, kx)) : 1.f;
    acc = fmaf(hy * hz * s32[i - 1] * f, v(i - 1, x - 1, y, z), acc);
  }
  if (x + 1 < g.nx) {
    const float f = (((x + 1) & mask) == 0) ? p2f(ki - kx_at(cg, x + 1, y, z, kx)) : 1.f;
    acc = fmaf(hy * hz * s32[i + 1] * f, v(i + 1, x + 1, y, z), acc);
  }
  if (y > 0) {
    const float f = ((y & mask) == 0) ? p2f(ki - kx_at(cg, x, y - 1, z, kx)) : 1.f;
    acc = fmaf(hx * hz * s32[i - px] * f, v(i - px, x, y - 1, z), acc);
  }
  if (y + 1 < g.ny) {
    const float f = (((y + 1) & mask) == 0) ? p2f(ki - kx_at(cg, x, y + 1, z, kx)) : 1.f;
    acc = fmaf(hx * hz * s32[i + px] * f, v(i + px, x, y + 1, z), acc);
  }
  if constexpr (DIM == 3) {
    const int64_t pz = (int64_t)px * g.ny;
    if (z > 0) {
      const float f = ((z & mask) == 0) ? p2f(ki - kx_at(cg, x, y, z - 1, kx)) : 1.f;
      acc = fmaf(hx * hy * s32[i - pz] * f, v(i - pz, x, y, z - 1), acc);
    }
    if (z + 1 < g.nz) {
      const float f = (((z + 1) & mask) == 0) ? p2f(ki - kx_at(cg, x, y, z + 1, kx)) : 1.f;
      acc = fmaf(hx * hy * s32[i + pz] * f, v(i + pz, x, y, z + 1), acc);
    }
  }
  return s32[i] * acc;
}

// Coarse-level operator (A u)_t for node (x, y, z) of a level; u(j, xj, yj,
// zj) by dense index and coordinates.
template <int DIM, class V>
__device__ __forceinline__ float apply_l(const MgLevel &L, int x, int y, int z, V u) {
  const int64_t pl = (int64_t)L.nx * L.ny;
  const int64_t m = (DIM == 3) ? pl * L.nz : pl;
  const int64_t i = lin<DIM>(x, y, z, L.nx, L.ny);
  float acc = fabsf(L.a[i]) * u(i, x, y, z);
  if (x > 0) acc = fmaf(L.c[kW * m + i], u(i - 1, x - 1, y, z), acc);
  if (x + 1 < L.nx) acc = fmaf(L.c[kE * m + i], u(i + 1, x + 1, y, z), acc);
  if (y > 0) acc = fmaf(L.c[kS * m + i], u(i - L.nx, x, y - 1, z), acc);
  if (y + 1 < L.ny) acc = fmaf(L.c[kN * m + i], u(i + L.nx, x, y + 1, z), acc);
  if constexpr (DIM == 3) {
    if (z > 0) acc = fmaf(L.c[kB * m + i], u(i - pl, x, y, z - 1), acc);
    if (z + 1 < L.nz) acc = fmaf(L.c[kT * m + i], u(i + pl, x, y, z + 1), acc);
  }
  return acc;
}

// ------------------------------------------------------------- setup
// w_i = exp(kx_i ln 2 - St_i / hbar) / sig_i (0 on the sources); St_i
// interpolated linearly along each axis between the cell centres (flat
// beyond the outer ones).
__global__ void k_mg_weights(Grid g, CellGrid cg, int px, const float *__restrict__ s32,
                             const int *__restrict__ kx, const float *__restrict__ St,
                             float *__restrict__ w) {
  const float B = (float)cg.B, half = 0.5f * (B - 1.f);
  auto axis = [&](int c, int ncell, int nn, int &I0, int &I1, float &tt) {
    I0 = min(max((int)floorf(((float)c - half) / B), 0), ncell - 1);
    I1 = min(I0 + 1, ncell - 1);
    const float c0 = fminf(I0 * B + half, (float)(nn - 1));
    const float c1 = fminf(I1 * B + half, (float)(nn - 1));
    tt = (c1 > c0) ? fminf(fmaxf(((float)c - c0) / (c1 - c0), 0.f), 1.f) : 0.f;
  };
  MG_ROWS(g.ny, g.nz) MG_COLS(g.nx) {
    const int64_t i = x + (int64_t)px * rr;
    const float s = s32[i];
    if (s == 0.f) {
      w[i] = 0.f;
      continue;
    }
    int I0, I1, J0, J1, K0, K1;
    float tx, ty, tz;
    axis(x, cg.cx, g.nx, I0, I1, tx);
    axis(y, cg.cy, g.ny, J0, J1, ty);
    axis(z, cg.cz, g.nz, K0, K1, tz);
    auto Sc = [&](int I, int J, int K) { return St[I + cg.cx * (J + cg.cy * K)]; };
    const float v[8] = {Sc(I0, J0, K0), Sc(I1, J0, K0), Sc(I0, J1, K0), Sc(I1, J1, K0),
                        Sc(I0, J0, K1), Sc(I1, J0, K1), Sc(I0, J1, K1), Sc(I1, J1, K1)};
    bool fin = true;
    for (int q = 0; q < 8; ++q) fin = fin && isfinite(v[q]);
    const int ki = kx_at(cg, x, y, z, kx);
    float ex = 0.f;
    if (fin) {
      const float b0 = (1.f - ty) * ((1.f - tx) * v[0] + tx * v[1]) + ty * ((1.f - tx) * v[2] + tx * v[3]);
      const float b1 = (1.f - ty) * ((1.f - tx) * v[4] + tx * v[5]) + ty * ((1.f - tx) * v[6] + tx * v[7]);
      const float Sb = (1.f - tz) * b0 + tz * b1;
      ex = (float)((double)ki * 0.69314718055994530942 - (double)Sb / g.hbar);
      ex = fminf(fmaxf(ex, -30.f), 30.f);   // w^2 stays in the FP32 range
    }
    w[i] = expf(ex) / s;
  }
}

// Level 1 from level 0: P_i = w_i (one exponent per box: boxes lie inside
// one cell), true A_ij = -sig_i sig_j omega_ij; c_CD = 2^(k_C - k_D) sum
// w_i w_j A_ij over the edges between the two boxes.  Sums in FP64.
__global__ void k_mg_coarsen0(Grid g, CellGrid cg, int px, const float *__restrict__ s32,
                              const int *__restrict__ kx, const float *__restrict__ w, MgLevel L) {
  const int64_t m = (int64_t)L.nx * L.ny * L.nz;
  MG_ROWS(L.ny, L.nz) MG_COLS(L.nx) {
    const int64_t t = x + (int64_t)L.nx * rr;
    const int x0 = 2 * x, y0 = 2 * y, z0 = 2 * z;
    const int x1 = min(x0 + 1, g.nx - 1), y1 = min(y0 + 1, g.ny - 1), z1 = min(z0 + 1, g.nz - 1);
    auto at = [&](int a, int b, int c) { return a + (int64_t)px * (b + (int64_t)g.ny * c); };
    auto W = [&](int a, int b, int c) { return (double)w[at(a, b, c)]; };
    auto S = [&](int a, int b, int c) { return (double)s32[at(a, b, c)]; };
    // A_ij of the edges (a, b, c)-(a + 1, b, c), (a, b, c)-(a, b + 1, c), (a, b, c)-(a, b, c + 1)
    auto ax = [&](int a, int b, int c) {
      return -S(a, b, c) * S(a + 1, b, c) * (double)(face(b, g.ny, g.boundary) * facez(g, c));
    };
    auto ay = [&](int a, int b, int c) {
      return -S(a, b, c) * S(a, b + 1, c) * (double)(face(a, g.nx, g.boundary) * facez(g, c));
    };
    auto az = [&](int a, int b, int c) {
      return -S(a, b, c) * S(a, b, c + 1) *
             (double)(face(a, g.nx, g.boundary) * face(b, g.ny, g.boundary));
    };
    const int kc = kx_at(cg, x0, y0, z0, kx);
    double A = 0.0, cd[kDirs] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool live = false;
    for (int c = z0; c <= z1; ++c)
      for (int b = y0; b <= y1; ++b)
        for (int a = x0; a <= x1; ++a) {
          const double wi = W(a, b, c);
          if (wi != 0.0) live = true;
          A += wi * wi;
        }
    for (int c = z0; c <= z1; ++c)
      for (int b = y0; b <= y1; ++b) {
        if (x1 > x0) A += 2.0 * W(x0, b, c) * W(x1, b, c) * ax(x0, b, c);
        if (x > 0) cd[kW] += W(x0, b, c) * W(x0 - 1, b, c) * ax(x0 - 1, b, c);
        if (x + 1 < L.nx && x0 + 2 < g.nx) cd[kE] += W(x1, b, c) * W(x0 + 2, b, c) * ax(x1, b, c);
      }
    for (int c = z0; c <= z1; ++c)
      for (int a = x0; a <= x1; ++a) {
        if (y1 > y0) A += 2.0 * W(a, y0, c) * W(a, y1, c) * ay(a, y0, c);
        if (y > 0) cd[kS] += W(a, y0, c) * W(a, y0 - 1, c) * ay(a, y0 - 1, c);
        if (y + 1 < L.ny && y0 + 2 < g.ny) cd[kN] += W(a, y1, c) * W(a, y0 + 2, c) * ay(a, y1, c);
      }
    for (int b = y0; b <= y1; ++b)
      for (int a = x0; a <= x1; ++a) {
        if (z1 > z0) A += 2.0 * W(a, b, z0) * W(a, b, z1) * az(a, b, z0);
        if (z > 0) cd[kB] += W(a, b, z0) * W(a, b, z0 - 1) * az(a, b, z0 - 1);
        if (z + 1 < L.nz && z0 + 2 < g.nz) cd[kT] += W(a, b, z1) * W(a, b, z0 + 2) * az(a, b, z1);
      }
    // row-relative: times 2^(k_C - k_D), k_D the neighbouring box's cell exponent
    if (x > 0) cd[kW] *= ldexp(1.0, kc - kx_at(cg, x0 - 2, y0, z0, kx));
    if (x + 1 < L.nx && x0 + 2 < g.nx) cd[kE] *= ldexp(1.0, kc - kx_at(cg, x0 + 2, y0, z0, kx));
    if (y > 0) cd[kS] *= ldexp(1.0, kc - kx_at(cg, x0, y0 - 2, z0, kx));
    if (y + 1 < L.ny && y0 + 2 < g.ny) cd[kN] *= ldexp(1.0, kc - kx_at(cg, x0, y0 + 2, z0, kx));
    if (z > 0) cd[kB] *= ldexp(1.0, kc - kx_at(cg, x0, y0, z0 - 2, kx));
    if (z + 1 < L.nz && z0 + 2 < g.nz) cd[kT] *= ldexp(1.0, kc - kx_at(cg, x0, y0, z0 + 2, kx));
    L.a[t] = live ? (float)A : -1.f;
    L.ia[t] = live ? (float)(1.0 / A) : 0.f;
    for (int d = 0; d < kDirs; ++d) L.c[d * m + t] = live ? (float)cd[d] : 0.f;
    L.k[t] = kc;
  }
}

// Smallest exponent over the live nodes of the box (X, Y, Z) of level F;
// INT_MAX when it has none.
__device__ __forceinline__ int box_k(const MgLevel &F, int X, int Y, int Z) {
  int k = INT_MAX;
  for (int z = 2 * Z; z <= min(2 * Z + 1, F.nz - 1); ++z)
    for (int y = 2 * Y; y <= min(2 * Y + 1, F.ny - 1); ++y)
      for (int x = 2 * X; x <= min(2 * X + 1, F.nx - 1); ++x) {
        const int64_t i = x + (int64_t)F.nx * (y + (int64_t)F.ny * z);
        if (F.a[i] >= 0.f) k = min(k, F.k[i]);
      }
  return k;
}

// Level l + 1 (C) from level l (F): rows restricted with 2^(2(k_C - k_i)),
// columns prolonged with unit weight (live nodes only).
__global__ void k_mg_coarsen(MgLevel F, MgLevel C) {
  const int64_t m = (int64_t)C.nx * C.ny * C.nz;
  const int64_t mf = (int64_t)F.nx * F.ny * F.nz;
  MG_ROWS(C.ny, C.nz) MG_COLS(C.nx) {
    const int64_t t = x + (int64_t)C.nx * rr;
    const int kc = box_k(F, x, y, z);
    if (kc == INT_MAX) {
      C.a[t] = -1.f;
      C.ia[t] = 0.f;
      for (int d = 0; d < kDirs; ++d) C.c[d * m + t] = 0.f;
      C.k[t] = F.k[2 * x + (int64_t)F.nx * (2 * y + (int64_t)F.ny * 2 * z)];
      continue;
    }
    const int x0 = 2 * x, y0 = 2 * y, z0 = 2 * z;
    const int x1 = min(x0 + 1, F.nx - 1), y1 = min(y0 + 1, F.ny - 1), z1 = min(z0 + 1, F.nz - 1);
    double A = 0.0, cd[kDirs] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int c = z0; c <= z1; ++c)
      for (int b = y0; b <= y1; ++b)
        for (int a = x0; a <= x1; ++a) {
          const int64_t i = a + (int64_t)F.nx * (b + (int64_t)F.ny * c);
          if (F.a[i] < 0.f) continue;
          const double r = ldexp(1.0, 2 * (kc - F.k[i]));
          double row = (double)F.a[i];
          // neighbours inside the box join the diagonal, the others the links
          auto add = [&](bool exists, bool inside, int d) {
            if (!exists) return;
            const double cij = (double)F.c[d * mf + i];
            if (inside) row += cij;
            else cd[d] += r * cij;
          };
          add(a > 0, a - 1 >= x0, kW);
          add(a + 1 < F.nx, a + 1 <= x1, kE);
          add(b > 0, b - 1 >= y0, kS);
          add(b + 1 < F.ny, b + 1 <= y1, kN);
          add(c > 0, c - 1 >= z0, kB);
          add(c + 1 < F.nz, c + 1 <= z1, kT);
          A += r * row;
        }
    C.a[t] = (float)A;
    C.ia[t] = (float)(1.0 / A);
    C.c[kW * m + t] = (x > 0) ? (float)cd[kW] : 0.f;
    C.c[kE * m + t] = (x + 1 < C.nx) ? (float)cd[kE] : 0.f;
    C.c[kS * m + t] = (y > 0) ? (float)cd[kS] : 0.f;
    C.c[kN * m + t] = (y + 1 < C.ny) ? (float)cd[kN] : 0.f;
    C.c[kB * m + t] = (z > 0) ? (float)cd[kB] : 0.f;
    C.c[kT * m + t] = (z + 1 < C.nz) ? (float)cd[kT] : 0.f;
    C.k[t] = kc;
  }
}

// ------------------------------------------------------------- V-cycle
// Level 0 down: y = omega r, t = r - A y, g1 = sum over the box of w_i t_i.
template <int DIM>
__global__ void k_mg_down0(Grid g, CellGrid cg, int px, const float *__restrict__ s32,
                           const int *__restrict__ kx, const float *__restrict__ w,
                           const float *__restrict__ r, MgLevel L1, const MgCtl *ctl) {
  if (ctl->done) return;
  auto rv = [&](int64_t j, int, int, int) { return r[j]; };
  MG_ROWS(L1.ny, L1.nz) MG_COLS(L1.nx) {
    float sum = 0.f;
    const int zt = (DIM == 3) ? min(2 * z + 1, g.nz - 1) : 0;
    for (int cz = 2 * z; cz <= zt; ++cz)
      for (int cy = 2 * y; cy <= min(2 * y + 1, g.ny - 1); ++cy)
        for (int cx = 2 * x; cx <= min(2 * x + 1, g.nx - 1); ++cx) {
          const int64_t i = lin<DIM>(cx, cy, cz, px, g.ny);
          const float wi = w[i];
          if (wi == 0.f) continue;
          const int ki = kx_at(cg, cx, cy, cz, kx);
          const float off = nb0<DIM>(g, cg, px, s32, kx, cx, cy, cz, ki, rv);
          // (A (omega r))_i = omega (r_i - off)
          const float ti = r[i] - kOmega * (r[i] - off);
          sum = fmaf(wi, ti, sum);
        }
    L1.g[x + (int64_t)L1.nx * rr] = sum;
  }
}

// Level l down (l >= 1) at coarse node (x, y, z): y = omega g / a on the
// box, t = g - A y, restricted to level l + 1.
template <int DIM>
__device__ __forceinline__ void down_node(const MgLevel &F, const MgLevel &C, int x, int y, int z) {
  auto yv = [&](int64_t j, int, int, int) { return kOmega * F.g[j] * F.ia[j]; };
  const int64_t t = lin<DIM>(x, y, z, C.nx, C.ny);
  const int kc = C.k[t];
  float sum = 0.f;
  if (C.a[t] >= 0.f) {
    const int zt = (DIM == 3) ? min(2 * z + 1, F.nz - 1) : 0;
    for (int cz = 2 * z; cz <= zt; ++cz)
      for (int cy = 2 * y; cy <= min(2 * y + 1, F.ny - 1); ++cy)
        for (int cx = 2 * x; cx <= min(2 * x + 1, F.nx - 1); ++cx) {
          const int64_t i = lin<DIM>(cx, cy, cz, F.nx, F.ny);
          if (F.a[i] < 0.f) continue;
          const float ti = F.g[i] - apply_l<DIM>(F, cx, cy, cz, yv);
          sum = fmaf(p2f(2 * (kc - F.k[i])), ti, sum);
        }
  }
  C.g[t] = sum;
}

template <int DIM>
__global__ void k_mg_down(MgLevel F, MgLevel C, const MgCtl *ctl) {
  if (ctl->done) return;
  MG_ROWS(C.ny, C.nz) MG_COLS(C.nx) down_node<DIM>(F, C, x, y, z);
}

// Level l up (l >= 1) at node (x, y, z): u = omega g / a + y(parent);
// y = u + omega (g - A u) / a.
template <int DIM>
__device__ __forceinline__ void up_node(const MgLevel &F, const MgLevel &C, int x, int y, int z) {
  const int64_t t = lin<DIM>(x, y, z, F.nx, F.ny);
  if (F.a[t] < 0.f) {
    F.y[t] = 0.f;
    return;
  }
  auto uat = [&](int64_t j, int xj, int yj, int zj) {
    const float par = (F.a[j] >= 0.f) ? C.y[lin<DIM>(xj >> 1, yj >> 1, zj >> 1, C.nx, C.ny)] : 0.f;
    return fmaf(kOmega * F.g[j], F.ia[j], par);
  };
  const float ut = uat(t, x, y, z);
  const float Au = apply_l<DIM>(F, x, y, z, uat);
  F.y[t] = fmaf(kOmega * (F.g[t] - Au), F.ia[t], ut);
}

template <int DIM>
__global__ void k_mg_up(MgLevel F, MgLevel C, const MgCtl *ctl) {
  if (ctl->done) return;
  MG_ROWS(F.ny, F.nz) MG_COLS(F.nx) up_node<DIM>(F, C, x, y, z);
}

// The small levels s .. L of the V-cycle in one block: down sweeps, the
// single-node solve, up sweeps, a block barrier between levels.
constexpr int kMaxLevels = 24;
constexpr int kTailNodes = 256;    // levels of at most this many nodes run in the tail
constexpr int kTailThreads = 1024;
struct MgTail {
  MgLevel lv[kMaxLevels];
  int s, L;
};
template <int DIM>
__global__ void __launch_bounds__(kTailThreads) k_mg_tail(MgTail T, const MgCtl *ctl) {
  if (ctl->done) return;
  for (int l = T.s; l < T.L; ++l) {
    const MgLevel &F = T.lv[l], &C = T.lv[l + 1];
    const int m = C.nx * C.ny * C.nz;
    for (int t = threadIdx.x; t < m; t += blockDim.x)
      down_node<DIM>(F, C, t % C.nx, (t / C.nx) % C.ny, t / (C.nx * C.ny));
    __syncthreads();
  }
  {
    const MgLevel &B = T.lv[T.L];
    const int m = B.nx * B.ny * B.nz;
    for (int t = threadIdx.x; t < m; t += blockDim.x) B.y[t] = B.g[t] * B.ia[t];
    __syncthreads();
  }
  for (int l = T.L - 1; l >= T.s; --l) {
    const MgLevel &F = T.lv[l], &C = T.lv[l + 1];
    const int m = F.nx * F.ny * F.nz;
    for (int t = threadIdx.x; t < m; t += blockDim.x)
      up_node<DIM>(F, C, t % F.nx, (t / F.nx) % F.ny, t / (F.nx * F.ny));
    __syncthreads();
  }
}

// ------------------------------------------------------------- PCG passes
// Inner-product weight 2^(-2 (k - kmin)); 0 past the FP32 range, where a
// term is below 2^-126 of the nearest ones.  Per-thread sums are FP32, the
// block and grid sums FP64.
__device__ __forceinline__ float wdot(int k, int kmin) { return p2f(2 * (kmin - k)); }

__device__ __forceinline__ int block_id() { return blockIdx.y * gridDim.x + blockIdx.x; }
__device__ __forceinline__ int block_count() { return gridDim.x * gridDim.y; }

// Last-block-done over a 2D grid (all gridDim.x * gridDim.y blocks): true in
// the block that arrives last, after every block has written its partials.
__device__ __forceinline__ bool last_block_2d(unsigned int *ticket, int *sh_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    *sh_flag = (t == (unsigned int)block_count() - 1u);
  }
  __syncthreads();
  const bool last = *sh_flag != 0;
  if (last) __threadfence();
  return last;
}

// Level 0 up: u = omega r + w y1(parent), z = u + omega (r - A u); rho = <r, z>.
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_mg_up0(Grid g, CellGrid cg, int px, const float *__restrict__ s32, const int *__restrict__ kx,
         const float *__restrict__ w, const float *__restrict__ r, MgLevel L1,
         float *__restrict__ zv, MgCtl *ctl, double *part) {
  __shared__ double sh[32];
  __shared__ int flag;
  if (ctl->done) return;
  const int kmin = ctl->kmin;
  float rz = 0.f;
  auto u = [&](int64_t j, int xj, int yj, int zj) {
    return fmaf(w[j], L1.y[lin<DIM>(xj >> 1, yj >> 1, zj >> 1, L1.nx, L1.ny)], kOmega * r[j]);
  };
  MG_ROWS(g.ny, g.nz) MG_COLS(g.nx) {
    const int64_t i = x + (int64_t)px * rr;
    if (s32[i] == 0.f) {
      zv[i] = 0.f;
      continue;
    }
    const int ki = kx_at(cg, x, y, z, kx);
    const float ui = u(i, x, y, z);
    const float Au = ui - nb0<DIM>(g, cg, px, s32, kx, x, y, z, ki, u);
    const float zi = fmaf(kOmega, r[i] - Au, ui);
    zv[i] = zi;
    rz = fmaf(r[i] * zi, wdot(ki, kmin), rz);
  }
  const double bs = block_sum((double)rz, sh);
  if (threadIdx.x == 0) part[block_id()] = bs;
  if (!last_block_2d(&ctl->counter[0], &flag)) return;
  const double tot = sum_partials(part, block_count(), sh);
  if (threadIdx.x == 0) {
    ctl->beta = ctl->first ? 0.0 : tot / ctl->rho;
    ctl->rho = tot;
    ctl->counter[0] = 0u;
    if (!(tot > 0.0) || !isfinite(tot)) {   // z = M r lost positivity: stop here
      ctl->stalled = 1;
      ctl->done = 1;
    }
  }
}

// p = z + beta p_old, q = A p, <p, q>; alpha = rho / <p, q>.
template <int DIM>
__global__ void __launch_bounds__(kThreads)
k_mg_dir(Grid g, CellGrid cg, int px, const float *__restrict__ s32, const int *__restrict__ kx,
         const float *__restrict__ zv, const float *__restrict__ p_old, float *__restrict__ p_new,
         float *__restrict__ q, MgCtl *ctl, double *part) {
  __shared__ double sh[32];
  __shared__ int flag;
  if (ctl->done) return;
  const int kmin = ctl->kmin;
  const float beta = (float)ctl->beta;
  const bool first = ctl->first != 0;
  float pq = 0.f;
  auto pv = [&](int64_t j, int, int, int) { return first ? zv[j] : fmaf(beta, p_old[j], zv[j]); };
  MG_ROWS(g.ny, g.nz) MG_COLS(g.nx) {
    const int64_t i = x + (int64_t)px * rr;
    const float pi = pv(i, x, y, z);
    float qi = 0.f;
    if (s32[i] != 0.f) {
      const int ki = kx_at(cg, x, y, z, kx);
      qi = pi - nb0<DIM>(g, cg, px, s32, kx, x, y, z, ki, pv);
      pq = fmaf(pi * qi, wdot(ki, kmin), pq);
    }
    p_new[i] = pi;
    q[i] = qi;
  }
  const double bs = block_sum((double)pq, sh);
  if (threadIdx.x == 0) part[block_id()] = bs;
  if (!last_block_2d(&ctl->counter[1], &flag)) return;
  const double tot = sum_partials(part, block_count(), sh);
  if (threadIdx.x == 0) {
    ctl->counter[1] = 0u;
    ctl->first = 0;
    if (!(tot > 0.0) || !isfinite(tot)) {
      ctl->alpha = 0.0;
      ctl->stalled = 1;
      ctl->done = 1;
    } else {
      ctl->alpha = ctl->rho / tot;
    }
  }
}

// d += alpha p, r -= alpha q, and the stopping tests.
__global__ void __launch_bounds__(kThreads)
k_mg_step(Grid g, int px, const float *__restrict__ p, const float *__restrict__ q,
          const float *__restrict__ xref, float *__restrict__ d, float *__restrict__ r, MgCtl *ctl,
          double *part, int nblk_part) {
  __shared__ double sh[32];
  __shared__ int flag;
  if (ctl->done) return;
  const float alpha = (float)ctl->alpha;
  const int mode = ctl->mode;
  const float theta = ctl->theta;
  float rmax = 0.f, viol = 0.f;
  for (int rr = blockIdx.y; rr < g.ny * g.nz; rr += gridDim.y) MG_COLS(g.nx) {
    const int64_t i = x + (int64_t)px * rr;
    const float di = fmaf(alpha, p[i], d[i]);
    const float ri = fmaf(-alpha, q[i], r[i]);
    d[i] = di;
    r[i] = ri;
    rmax = fmaxf(rmax, fabsf(ri));
    if (mode == 1 && fabsf(ri) > theta * fabsf(xref[i] + di)) viol = 1.f;
  }
  const double b1 = block_max((double)rmax, sh);
  const double b2 = block_max((double)viol, sh);
  if (threadIdx.x == 0) {
    part[block_id()] = b1;
    part[nblk_part + block_id()] = b2;
  }
  if (!last_block_2d(&ctl->counter[2], &flag)) return;
  const double rm = max_partials(part, block_count(), sh);
  const double vi = max_partials(part + nblk_part, block_count(), sh);
  if (threadIdx.x == 0) {
    ctl->counter[2] = 0u;
    ctl->iter += 1;
    const bool conv = (mode == 0) ? (rm <= (double)ctl->thresh) : (vi == 0.0);
    if (!isfinite(rm)) {
      ctl->status = EIK_ERR_BREAKDOWN;
      ctl->done = 1;
    } else if (conv || ctl->iter >= ctl->max_iter) {
      ctl->done = 1;
    }
  }
}

}  // namespace

// ====================================================================== host
struct MgState {
  Grid g;
  CellGrid cg;
  int px = 0, cap = 0;
  std::vector<MgLevel> lv;   // lv[0]: level-0 sizes only
  float *w = nullptr, *z = nullptr, *p[2] = {nullptr, nullptr}, *q = nullptr;
  MgCtl *ctl = nullptr, *h_ctl = nullptr;
  double *part = nullptr;
  cudaGraphExec_t graph = nullptr;
  MgFine bound{};            // arrays the graph was captured with
  int64_t launches = 0;
  bool profile = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int64_t timed_iters = 0;
  double ms = 0.0;
};

const char *mg_last_error() { return g_msg.c_str(); }
int mg_levels(const MgState *mg) { return mg ? (int)mg->lv.size() : 0; }
int64_t mg_launches(const MgState *mg) { return mg ? mg->launches : 0; }
void mg_set_profiling(MgState *mg, bool on) {
  if (mg) mg->profile = on;
}
void mg_time(const MgState *mg, int64_t *iters, double *ms) {
  *iters = mg ? mg->timed_iters : 0;
  *ms = mg ? mg->ms : 0.0;
}
void mg_reset(MgState *mg) {
  if (!mg) return;
  mg->launches = 0;
  mg->timed_iters = 0;
  mg->ms = 0.0;
}

#define GCK(call)                                                       \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      g_msg = std::string(#call) + ": " + cudaGetErrorString(e_);       \
      return EIK_ERR_CUDA;                                              \
    }                                                                   \
  } while (0)

void mg_destroy(MgState *mg) {
  if (!mg) return;
  if (mg->graph) cudaGraphExecDestroy(mg->graph);
  for (auto &e : mg->ev)
    if (e) cudaEventDestroy(e);
  for (size_t l = 1; l < mg->lv.size(); ++l) {
    MgLevel &L = mg->lv[l];
    void *arr[] = {L.a, L.ia, L.c, L.k, L.g, L.y};
    for (void *p : arr)
      if (p) cudaFree(p);
  }
  void *arr[] = {mg->w, mg->z, mg->p[0], mg->p[1], mg->q, mg->ctl, mg->part};
  for (void *p : arr)
    if (p) cudaFree(p);
  if (mg->h_ctl) cudaFreeHost(mg->h_ctl);
  delete mg;
}

eik_status mg_create(MgState **out, const Grid &g, const CellGrid &cg, int px, int num_sms,
                     cudaStream_t s) {
  *out = nullptr;
  MgState *mg = new MgState();
  mg->g = g;
  mg->cg = cg;
  mg->px = px;
  mg->cap = num_sms * 8;
  MgLevel L0;
  L0.nx = g.nx;
  L0.ny = g.ny;
  L0.nz = g.nz;
  mg->lv.push_back(L0);
  bool ok = true;
  int nx = g.nx, ny = g.ny, nz = g.nz;
  while (ok && (nx > 1 || ny > 1 || nz > 1) && (int)mg->lv.size() < kMaxLevels) {
    nx = (nx + 1) / 2;
    ny = (ny + 1) / 2;
    nz = (nz + 1) / 2;
    MgLevel L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    const size_t m = (size_t)nx * ny * nz;
    ok = cudaMalloc(&L.a, 4 * m) == cudaSuccess && cudaMalloc(&L.ia, 4 * m) == cudaSuccess &&
         cudaMalloc(&L.c, 4 * kDirs * m) == cudaSuccess &&
         cudaMalloc(&L.k, 4 * m) == cudaSuccess && cudaMalloc(&L.g, 4 * m) == cudaSuccess &&
         cudaMalloc(&L.y, 4 * m) == cudaSuccess;
    mg->lv.push_back(L);
  }
  const size_t np = (size_t)g.ny * g.nz * px;
  ok = ok && cudaMalloc(&mg->w, 4 * np) == cudaSuccess && cudaMalloc(&mg->z, 4 * np) == cudaSuccess &&
       cudaMalloc(&mg->p[0], 4 * np) == cudaSuccess && cudaMalloc(&mg->p[1], 4 * np) == cudaSuccess &&
       cudaMalloc(&mg->q, 4 * np) == cudaSuccess &&
       cudaMalloc(&mg->ctl, sizeof(MgCtl)) == cudaSuccess &&
       cudaMalloc(&mg->part, 2 * sizeof(double) * mg->cap) == cudaSuccess &&
       cudaMallocHost(&mg->h_ctl, sizeof(MgCtl)) == cudaSuccess;
  if (ok) {
    // padding columns of the pitched arrays are read by no kernel; keep them finite
    float *arr[] = {mg->w, mg->z, mg->p[0], mg->p[1], mg->q};
    for (float *a : arr) ok = ok && cudaMemsetAsync(a, 0, 4 * np, s) == cudaSuccess;
    ok = ok && cudaMemsetAsync(mg->ctl, 0, sizeof(MgCtl), s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    mg_destroy(mg);
    g_msg = "multigrid: device allocation failed";
    return EIK_ERR_OOM;
  }
  *out = mg;
  return EIK_OK;
}

// Row-strided launch grid of a level: columns by blockIdx.x, rows by
// blockIdx.y, at most cap blocks.
static dim3 grid2(const MgState *mg, int nx, int64_t rows) {
  const int gx = std::max(1, std::min((nx + kThreads - 1) / kThreads, mg->cap));
  const int gy = (int)std::max<int64_t>(1, std::min<int64_t>(rows, mg->cap / gx));
  return dim3((unsigned)gx, (unsigned)gy, 1);
}
static dim3 grid_of(const MgState *mg, const MgLevel &L) {
  return grid2(mg, L.nx, (int64_t)L.ny * L.nz);
}

eik_status mg_setup(MgState *mg, const MgFine &f, int kmin, cudaStream_t s) {
  const Grid &g = mg->g;
  k_mg_weights<<<grid_of(mg, mg->lv[0]), kThreads, 0, s>>>(g, mg->cg, mg->px, f.s32, f.kx, f.St,
                                                            mg->w);
  MgLevel &L1 = mg->lv[1];
  k_mg_coarsen0<<<grid_of(mg, L1), kThreads, 0, s>>>(g, mg->cg, mg->px, f.s32, f.kx, mg->w, L1);
  mg->launches += 2;
  for (size_t l = 1; l + 1 < mg->lv.size(); ++l) {
    MgLevel &C = mg->lv[l + 1];
    k_mg_coarsen<<<grid_of(mg, C), kThreads, 0, s>>>(mg->lv[l], C);
    mg->launches++;
  }
  GCK(cudaGetLastError());
  mg->h_ctl->kmin = kmin;
  return EIK_OK;
}

// One PCG iteration (direction buffers: read p[set], write p[1 - set]).
// First level handled by the tail kernel: the first of at most kTailNodes
// nodes, level 1 at the earliest.
static int tail_start(const MgState *mg) {
  int l = 1;
  while (l < (int)mg->lv.size() - 1 &&
         (int64_t)mg->lv[l].nx * mg->lv[l].ny * mg->lv[l].nz > kTailNodes)
    ++l;
  return l;
}

template <int DIM>
static void launch_iter_d(MgState *mg, const MgFine &f, int set, cudaStream_t s) {
  const Grid &g = mg->g;
  const int L = (int)mg->lv.size() - 1;   // coarsest level index
  const dim3 g0 = grid_of(mg, mg->lv[0]);
  k_mg_down0<DIM><<<grid_of(mg, mg->lv[1]), kThreads, 0, s>>>(
      g, mg->cg, mg->px, f.s32, f.kx, mg->w, f.r, mg->lv[1], mg->ctl);
  // levels 1 .. ts - 1 one launch each way; ts .. L in the single-block tail
  const int ts = tail_start(mg);
  for (int l = 1; l < ts; ++l)
    k_mg_down<DIM><<<grid_of(mg, mg->lv[l + 1]), kThreads, 0, s>>>(mg->lv[l], mg->lv[l + 1],
                                                                     mg->ctl);
  MgTail T{};
  for (int l = ts; l <= L; ++l) T.lv[l] = mg->lv[l];
  T.s = ts;
  T.L = L;
  k_mg_tail<DIM><<<1, kTailThreads, 0, s>>>(T, mg->ctl);
  for (int l = ts - 1; l >= 1; --l)
    k_mg_up<DIM><<<grid_of(mg, mg->lv[l]), kThreads, 0, s>>>(mg->lv[l], mg->lv[l + 1], mg->ctl);
  k_mg_up0<DIM><<<g0, kThreads, 0, s>>>(g, mg->cg, mg->px, f.s32, f.kx, mg->w, f.r, mg->lv[1], mg->z,
                                   mg->ctl, mg->part);
  k_mg_dir<DIM><<<g0, kThreads, 0, s>>>(g, mg->cg, mg->px, f.s32, f.kx, mg->z, mg->p[set],
                                   mg->p[1 - set], mg->q, mg->ctl, mg->part);
  k_mg_step<<<g0, kThreads, 0, s>>>(g, mg->px, mg->p[1 - set], mg->q, f.xref, f.d, f.r, mg->ctl,
                                    mg->part, mg->cap);
}

// One PCG iteration with the kernels specialised to the grid's dimension.
static void launch_iter(MgState *mg, const MgFine &f, int set, cudaStream_t s) {
  if (mg->g.ndim == 3)
    launch_iter_d<3>(mg, f, set, s);
  else
    launch_iter_d<2>(mg, f, set, s);
}

static int launches_per_iter(const MgState *mg) { return 2 * (tail_start(mg) - 1) + 5; }

eik_status mg_inner(MgState *mg, const MgFine &f, MixCtl *h_st, cudaStream_t s) {
  if (mg->graph && (f.r != mg->bound.r || f.d != mg->bound.d || f.xref != mg->bound.xref ||
                    f.s32 != mg->bound.s32 || f.kx != mg->bound.kx)) {
    cudaGraphExecDestroy(mg->graph);
    mg->graph = nullptr;
  }
  if (!mg->graph) {
    cudaGraph_t graph;
    GCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    for (int it = 0; it < kGraphIters; ++it) launch_iter(mg, f, it & 1, s);
    GCK(cudaStreamEndCapture(s, &graph));
    GCK(cudaGraphInstantiate(&mg->graph, graph, 0));
    GCK(cudaGraphDestroy(graph));
    mg->bound = f;
  }
  MgCtl c{};
  c.kmin = mg->h_ctl->kmin;
  c.max_iter = std::max(1, std::min(h_st->max_iter, kMaxInnerIters));
  c.mode = h_st->mode;
  c.thresh = h_st->thresh;
  c.theta = h_st->theta;
  c.first = 1;
  *mg->h_ctl = c;
  GCK(cudaMemcpyAsync(mg->ctl, mg->h_ctl, sizeof(MgCtl), cudaMemcpyHostToDevice, s));
  if (mg->profile && !mg->ev[0])
    for (auto &e : mg->ev) GCK(cudaEventCreate(&e));
  int before = 0;
  for (;;) {
    if (mg->profile) GCK(cudaEventRecord(mg->ev[0], s));
    GCK(cudaGraphLaunch(mg->graph, s));
    if (mg->profile) GCK(cudaEventRecord(mg->ev[1], s));
    GCK(cudaMemcpyAsync(mg->h_ctl, mg->ctl, sizeof(MgCtl), cudaMemcpyDeviceToHost, s));
    GCK(cudaStreamSynchronize(s));
    // every kernel of the graph launches (those past the end return at once)
    mg->launches += (int64_t)kGraphIters * launches_per_iter(mg);
    const int done_iters = mg->h_ctl->iter - before;
    before = mg->h_ctl->iter;
    if (mg->profile && done_iters == kGraphIters) {
      float t = 0.f;
      GCK(cudaEventElapsedTime(&t, mg->ev[0], mg->ev[1]));
      mg->ms += t;
      mg->timed_iters += done_iters;
    }
    if (mg->h_ctl->done) break;
  }
  h_st->iter = mg->h_ctl->iter;
  h_st->status = mg->h_ctl->status;
  h_st->stalled = mg->h_ctl->stalled;
  h_st->done = 1;
  return EIK_OK;
}

}  // namespace eik
