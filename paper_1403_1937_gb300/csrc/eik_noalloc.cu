// Allocation-free componentwise residual of a given S (eik_residual_noalloc).
//
// Some callers cannot allocate device memory at the point where they want to
// check a solution: code running inside a memory pool or arena that must not
// grow, allocator-hook or plugin code that is forbidden to call back into the
// allocator, and real-time loops where cudaMalloc's implicit device
// synchronisation is not acceptable.  This entry point therefore takes all of
// its working memory from one file-scope device array, sized at build time,
// and calls no cudaMalloc, cudaFree or allocating library routine.
//
// What it computes is the componentwise residual that eik_solve reports as
// eik_stats.res_cw, but from S instead of from the solver's internal state:
// for every non-source node i,
//   rho_i = | (c / a_i) sum_{j~i} omega_ij exp((S_i - S_j)/hbar) - 1 |,
// which equals |r_i| / (a_i phi_i) for phi = exp(-S/hbar) (divide row i of
// the discrete system by a_i phi_i), and 0 on the sources.  The result is
// max_i rho_i.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "eik_internal.cuh"

namespace {
constexpr int64_t kNoAllocMaxNodes = int64_t(1) << 20;   // largest grid accepted
constexpr int kNoAllocBlocks = 1024;                      // reduction blocks
// layout of the scratch array (in doubles)
constexpr int64_t kRhoOff = 0;                            // per-node residuals
constexpr int64_t kPartOff = kNoAllocMaxNodes;            // per-block maxima
constexpr int64_t kFlagOff = kPartOff + kNoAllocBlocks;   // ticket, bad-index flag
constexpr int64_t kScratchLen = kFlagOff + 2;
}  // namespace

// Working memory of eik_residual_noalloc (about 8.4 MB).  Every GPU that loads
// the library holds it until the process exits.  All calls share it.
static __device__ __align__(256) double g_noalloc_scratch[kScratchLen];

namespace {

// Host copies of the scratch's device address, one per device, filled by the
// first call made with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

using eik::Grid;
using eik::half_if;
using eik::on_face;

__global__ void k_rho(Grid g, const double *__restrict__ f, const double *__restrict__ S,
                      double *__restrict__ sc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % g.nx);
    const int64_t t = i / g.nx;
    const int iy = (int)(t % g.ny);
    const int iz = (int)(t / g.ny);
    const double hx = half_if(on_face(ix, g.nx, g.boundary));
    const double hy = half_if(on_face(iy, g.ny, g.boundary));
    const double hz = (g.ndim == 3) ? half_if(on_face(iz, g.nz, g.boundary)) : 1.0;
    const double Si = S[i];
    double sum = 0.0, om = 0.0;
    const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
    // x edges carry hy*hz, y edges hx*hz, z edges hx*hy
    if (ix > 0) { sum += hy * hz * exp((Si - S[i - 1]) / g.hbar); om += hy * hz; }
    if (ix < g.nx - 1) { sum += hy * hz * exp((Si - S[i + 1]) / g.hbar); om += hy * hz; }
    if (iy > 0) { sum += hx * hz * exp((Si - S[i - sy]) / g.hbar); om += hx * hz; }
    if (iy < g.ny - 1) { sum += hx * hz * exp((Si - S[i + sy]) / g.hbar); om += hx * hz; }
    if (g.ndim == 3) {
      if (iz > 0) { sum += hx * hy * exp((Si - S[i - sz]) / g.hbar); om += hx * hy; }
      if (iz < g.nz - 1) { sum += hx * hy * exp((Si - S[i + sz]) / g.hbar); om += hx * hy; }
    }
    const double fi = f[i];
    const double a = hx * hy * hz * fi * fi + g.c * om;
    sc[kRhoOff + i] = fabs(g.c * sum / a - 1.0);
  }
}

// Sources carry no residual.  An index outside the grid is not written; it
// sets the flag that turns the result into NaN.
__global__ void k_rho_sources(int64_t n, const int64_t *__restrict__ src, int64_t nsrc,
                              double *__restrict__ sc) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nsrc) return;
  const int64_t j = src[k];
  if (j >= 0 && j < n)
    sc[kRhoOff + j] = 0.0;
  else
    sc[kFlagOff + 1] = 1.0;
}

__global__ void k_rho_max(int64_t n, double *__restrict__ sc, double *out) {
  __shared__ double red[32];
  __shared__ int flag;
  double m = 0.0;
  bool nan_seen = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = sc[kRhoOff + i];
    if (v != v)
      nan_seen = true;   // fmax in the reductions below would drop it
    else
      m = fmax(m, v);
  }
  // A NaN residual (NaN in S, or inf - inf between two +inf neighbours) must
  // not come back as a small finite maximum: the block's partial becomes NaN
  // and the last block turns the result into NaN.  The partial travels
  // through the same fence and ticket as the maxima.
  nan_seen = __syncthreads_or(nan_seen) != 0;
  m = eik::block_max(m, red);
  if (threadIdx.x == 0) sc[kPartOff + blockIdx.x] = nan_seen ? NAN : m;
  unsigned int *ticket = reinterpret_cast<unsigned int *>(sc + kFlagOff);
  if (!eik::last_block(ticket, &flag)) return;
  double tot = 0.0;
  bool any_nan = false;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double v = __ldcg(sc + kPartOff + b);
    if (v != v)
      any_nan = true;
    else
      tot = fmax(tot, v);
  }
  any_nan = __syncthreads_or(any_nan) != 0;
  tot = eik::block_max(tot, red);
  if (threadIdx.x == 0) {
    *out = (any_nan || sc[kFlagOff + 1] != 0.0) ? NAN : tot;
    *ticket = 0u;
  }
}

}  // namespace

extern "C" eik_status eik_residual_noalloc(int ndim, const int64_t *dims, double h, double hbar,
                                           const double *f, const double *S,
                                           const int64_t *src_idx, int64_t nsrc, int boundary,
                                           double *res_max, eik_stream_t stream) {
  if (ndim != 2 && ndim != 3) return EIK_ERR_ARG;
  if (!dims || !f || !S || !res_max || (nsrc > 0 && !src_idx)) return EIK_ERR_ARG;
  if (!(h > 0) || !(hbar > 0) || !isfinite(h) || !isfinite(hbar)) return EIK_ERR_ARG;
  if (boundary != EIK_BOUNDARY_HALF_CELL && boundary != EIK_BOUNDARY_DROP_EDGE) return EIK_ERR_ARG;
  int64_t d[3] = {1, 1, 1}, n = 1;
  for (int a = 0; a < ndim; ++a) {
    d[a] = dims[a];
    // each extent is bounded before it is multiplied in, so the product
    // cannot wrap around (and every extent fits an int)
    if (d[a] < 2 || d[a] > kNoAllocMaxNodes) return EIK_ERR_ARG;
    n *= d[a];
    if (n > kNoAllocMaxNodes) return EIK_ERR_ARG;   // larger than the scratch array
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EIK_ERR_CUDA;
  double *sc = nullptr;
  {
    // one-time set-up per device: the address of the file-scope scratch array
    // as seen by this device (the host-side symbol is not a device address)
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return EIK_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    sc = g_scratch_ptr[dev];
  }
  Grid g{};
  g.nx = (int)d[0];
  g.ny = (int)d[1];
  g.nz = (int)d[2];
  g.ndim = ndim;
  g.n = n;
  g.c = hbar * hbar / (h * h);
  g.sqrt_c = hbar / h;
  g.hbar = hbar;
  g.U_min = 0.0;
  g.boundary = boundary;
  cudaStream_t s = stream;
  // the ticket and the bad-index flag must start at zero whatever a previous
  // (possibly failed) call left behind
  if (cudaMemsetAsync(sc + kFlagOff, 0, 2 * sizeof(double), s) != cudaSuccess)
    return EIK_ERR_CUDA;
  const int th = eik::kThreads;
  const int nb = (int)std::min<int64_t>((n + th - 1) / th, kNoAllocBlocks);
  k_rho<<<nb, th, 0, s>>>(g, f, S, sc);
  if (nsrc > 0) k_rho_sources<<<(int)((nsrc + th - 1) / th), th, 0, s>>>(n, src_idx, nsrc, sc);
  k_rho_max<<<nb, th, 0, s>>>(n, sc, res_max);
  return cudaGetLastError() == cudaSuccess ? EIK_OK : EIK_ERR_CUDA;
}
