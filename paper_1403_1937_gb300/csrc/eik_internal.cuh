// Internal definitions shared by the CUDA translation units of libeik.
//
// Discretisation (Sec. 4 Eq. phiEquation, Sec. 6 Eq. sparse-system): on a
// vertex-centred grid, every non-source node i satisfies
//   a_i phi_i - c sum_{j~i} omega_ij phi_j = 0,   a_i = w_i f_i^2 + c sum_j omega_ij
// with c = hbar^2/h^2 and half-cell face weights w_i, omega_ij.
//
// The solver works in Jacobi-scaled ("hat") variables: phi_i = s_i xh_i with
// s_i = a_i^{-1/2}.  The scaled operator has unit diagonal,
//   (Ahat v)_i = v_i - sig_i * sum_{j~i} omega_ij sig_j v_j,  sig_i = sqrt(c/a_i),
// so Jacobi-preconditioned CG on A is plain CG on Ahat with unweighted inner
// products.  Source nodes carry sig = 0 (their rows and columns vanish from
// Ahat); the slot xh_k of a source holds sqrt(c)*phi_k, which is the value
// sig_j*xh_j would take in the right-hand side  bhat_i = sig_i sum_{k in Y}
// omega_ik sqrt(c) phi_k.  The componentwise residual |r_i|/(a_i phi_i) equals
// |rhat_i| / xh_i.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/eik.h"

namespace eik {

constexpr int kThreads = 256;

// Geometry and constants of one grid.  nz = 1 in 2D.
struct Grid {
  int nx, ny, nz;
  int ndim;
  int64_t n;
  double c;        // hbar^2 / h^2
  double sqrt_c;
  double hbar;
  double U_min;
  int boundary;    // EIK_BOUNDARY_*
};

// Device-resident CG control block.  Written only by the last block of a
// pass (or by single-thread kernels), read by every block of the next pass.
struct CgState {
  double rho;        // <rhat, rhat>
  double alpha;
  double beta;
  double bnorm2;     // <bhat, bhat> (normwise stop)
  double res_cw;     // componentwise max from the last residual kernel
  double res_nw2_r;  // unscaled ||r||^2 from the last residual kernel
  double res_nw2_b;  // unscaled ||b||^2
  double tol;
  int iter;          // CG iterations done
  int max_iter;
  int done;          // 1: stop iterating (see status)
  int status;        // eik_status of the iteration
  int stop_norm;
  int pad0;
  unsigned int counter[4];   // last-block-done tickets, one per pass kind
};

// Reduction slots per block.
enum { kSlotA = 0, kSlotB = 1, kSlotC = 2, kSlots = 3 };

// --------------------------------------------------------------- helpers
__device__ __forceinline__ bool on_face(int i, int n, int boundary) {
  return boundary == EIK_BOUNDARY_HALF_CELL && (i == 0 || i == n - 1);
}

__device__ __forceinline__ double half_if(bool b) { return b ? 0.5 : 1.0; }

// Deterministic block sum of a double: warp shuffles, then warp 0.
__device__ __forceinline__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  }
  return v;
}

// Last-block-done protocol.  Thread 0 of every block has written its
// partials; returns true in the single block that arrives last (all threads
// of that block see the same answer).  The ticket is reset by that block.
__device__ __forceinline__ bool last_block(unsigned int *ticket, int *sh_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    *sh_flag = (t == gridDim.x - 1);
  }
  __syncthreads();
  const bool last = *sh_flag != 0;
  if (last) __threadfence();
  return last;
}

// Fixed-order sum of nblk partials (deterministic for a fixed grid size).
__device__ __forceinline__ double sum_partials(const double *part, int nblk, double *sh) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v += __ldcg(part + b);
  return block_sum(v, sh);
}

__device__ __forceinline__ double max_partials(const double *part, int nblk, double *sh) {
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) v = fmax(v, __ldcg(part + b));
  return block_max(v, sh);
}

// Tile geometry for the halo-staged stencil kernels.
template <int DIM> struct Tile;
template <> struct Tile<2> {
  static constexpr int TX = 64, TY = 32, TZ = 1;
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = 1;
};
template <> struct Tile<3> {
  static constexpr int TX = 32, TY = 8, TZ = 4;
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
};

struct TileCount {
  int tx, ty, tz;
  int64_t total;
};

}  // namespace eik
