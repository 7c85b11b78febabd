// FFT perturbation series of Sec. 5 (Table 1) on a 2D grid.
//
// With a constant f~, phi = phi_0 - phi_1 + phi_2 - ... + (-1)^T phi_T,
// phi_0 = G~ * delta_kron (G~ = exp(-f~|x|/hbar), Sec. 3.2), and
// phi_i = h^2 G * [(f^2 - f~^2) phi_{i-1}] (Eq. phi_i_Solution) with G the 2D
// Green's function K_0(f~|x|/hbar) / (2 pi hbar^2) (Eq. GreensFunction2D);
// S = -hbar log phi.  Every convolution is the linear one over the grid,
// computed by complex FP64 transforms of arrays zero-padded to P_a >= 2 n_a - 1
// points per axis (powers of two) with the kernel sampled at the offsets
// -(n_a - 1) .. n_a - 1 and wrapped; G's sample at the origin is its average
// over the grid cell.
//
// Transforms: a 2D transform is a pass of 1D transforms along the rows, a
// tiled transpose, and a second row pass; the spectrum stays in the
// transposed layout, where the pointwise products are taken, and the inverse
// retraces the same steps.  A row transform runs in one block, in shared
// memory, as the Stockham self-sorting form of the mixed-radix FFT: lengths
// P = 2^a 3^b 5^c (the smallest >= 2n - 1), stages of radix 4, 2, 3 and 5,
// each reading one buffer and writing the other in natural order.
//
// K_0 and K_1 come from their integral representation
// K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9), summed by
// the trapezoidal rule, which converges geometrically for this analytic,
// doubly exponentially decaying integrand; the step shrinks like 1/sqrt(x)
// for large x, where the integrand is a narrow Gaussian around t = 0.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "eik_internal.cuh"

namespace eik {
namespace {

constexpr int kMaxFft = 7200;   // largest transform length per axis (two buffers
                                // of P complex doubles in shared memory)
constexpr int kMaxStages = 16;

__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Twiddles w_q = exp(-2 pi i q / P), q < P.
__global__ void k_twiddles(double2 *tw, int P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  double s, c;
  sincospi(2.0 * q / P, &s, &c);
  tw[q] = make_double2(c, -s);
}

// The radices of one transform length, in stage order.
struct Radices {
  int n;
  int r[kMaxStages];
};

// Multiplication by -i (forward) or +i (inverse).
template <bool INV>
__device__ __forceinline__ double2 rot(double2 a) {
  return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// In-place DFT of R points, forward (exp(-2 pi i q r / R)) or inverse.
// Radix-3 and -5 constants: cos/sin of 2 pi / R multiples (passed in).
struct DftConst {
  double c3, s3;            // cos(2pi/3), sin(2pi/3)
  double c51, c52, s51, s52;  // cos(2pi/5), cos(4pi/5), sin(2pi/5), sin(4pi/5)
};

template <int R, bool INV>
__device__ __forceinline__ void dft(double2 *v, const DftConst &k) {
  if constexpr (R == 2) {
    const double2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const double2 t2 = cadd(v[1], v[3]), t3 = rot<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else if constexpr (R == 3) {
    const double2 a = v[0], t = cadd(v[1], v[2]);
    const double2 m = make_double2(a.x + k.c3 * t.x, a.y + k.c3 * t.y);
    const double2 d = rot<INV>(csub(v[1], v[2]));
    v[0] = cadd(a, t);
    v[1] = make_double2(m.x + k.s3 * d.x, m.y + k.s3 * d.y);
    v[2] = make_double2(m.x - k.s3 * d.x, m.y - k.s3 * d.y);
  } else {   // R == 5
    const double2 a = v[0];
    const double2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const double2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    const double2 m1 = make_double2(a.x + k.c51 * t1.x + k.c52 * t2.x,
                                    a.y + k.c51 * t1.y + k.c52 * t2.y);
    const double2 m2 = make_double2(a.x + k.c52 * t1.x + k.c51 * t2.x,
                                    a.y + k.c52 * t1.y + k.c51 * t2.y);
    const double2 n1 = rot<INV>(make_double2(k.s51 * t3.x + k.s52 * t4.x,
                                             k.s51 * t3.y + k.s52 * t4.y));
    const double2 n2 = rot<INV>(make_double2(k.s52 * t3.x - k.s51 * t4.x,
                                             k.s52 * t3.y - k.s51 * t4.y));
    v[0] = cadd(a, cadd(t1, t2));
    v[1] = cadd(m1, n1);
    v[4] = csub(m1, n1);
    v[2] = cadd(m2, n2);
    v[3] = csub(m2, n2);
  }
}

// One 1D transform of length P per block (rows of `a`, pitch P); INV uses
// the conjugate twiddles and butterflies (no 1/P scaling).  Stockham stage of
// radix R over span Ns: for j < P/R, with k = j mod Ns, the R inputs
// x[j + r P/R] are twiddled by w^(r k P/(Ns R)), transformed, and written to
// y[(j / Ns) Ns R + k + r Ns]; Ns grows by R each stage.
template <int R, bool INV>
__device__ __forceinline__ void stockham_stage(const double2 *x, double2 *y, int P, int Ns,
                                               const double2 *__restrict__ tw,
                                               const DftConst &kc) {
  const int m = P / R;
  const int tstep = P / (Ns * R);   // w_{Ns R}^(r k) = w_P^(r k tstep)
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const int k = j % Ns;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double2 t = x[j + r * m];
      if (r > 0 && k > 0) {
        double2 w = tw[(r * k * tstep) % P];
        if (INV) w.y = -w.y;
        t = cmul(w, t);
      }
      v[r] = t;
    }
    dft<R, INV>(v, kc);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) y[base + r * Ns] = v[r];
  }
}

template <bool INV>
__global__ void k_fft_rows(double2 *a, int P, Radices rad, DftConst kc,
                           const double2 *__restrict__ tw) {
  extern __shared__ double2 fsm[];
  double2 *x = fsm, *y = fsm + P;
  double2 *row = a + (size_t)blockIdx.x * P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) x[i] = row[i];
  __syncthreads();
  int Ns = 1;
  for (int st = 0; st < rad.n; ++st) {
    const int R = rad.r[st];
    switch (R) {
      case 4: stockham_stage<4, INV>(x, y, P, Ns, tw, kc); break;
      case 2: stockham_stage<2, INV>(x, y, P, Ns, tw, kc); break;
      case 3: stockham_stage<3, INV>(x, y, P, Ns, tw, kc); break;
      default: stockham_stage<5, INV>(x, y, P, Ns, tw, kc); break;
    }
    __syncthreads();
    double2 *tmp = x;
    x = y;
    y = tmp;
    Ns *= R;
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) row[i] = x[i];
}

// out (cols x rows) = transpose of in (rows x cols), 32 x 32 tiles.
__global__ void k_transpose(const double2 *__restrict__ in, double2 *__restrict__ out, int rows,
                            int cols) {
  __shared__ double2 t[32][33];
  const int x = blockIdx.x * 32 + threadIdx.x;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int y = blockIdx.y * 32 + k;
    if (x < cols && y < rows) t[k][threadIdx.x] = in[(size_t)y * cols + x];
  }
  __syncthreads();
  const int ox = blockIdx.y * 32 + threadIdx.x;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int oy = blockIdx.x * 32 + k;
    if (ox < rows && oy < cols) out[(size_t)oy * rows + ox] = t[threadIdx.x][k];
  }
}

// K_nu(x), nu = 0 or 1, x > 0 (integral representation, trapezoidal rule).
// The nodes' c_k = cosh(k eta) come from the recurrence c_{k+1} =
// 2 cosh(eta) c_k - c_{k-1} (one exponential per node instead of three; the
// rounding it adds grows like k eps over the few dozen nodes summed).
__device__ double bessel_k(int nu, double x) {
  if (!(x > 0.0)) return INFINITY;
  if (x > 745.0) return 0.0;
  const double eta = fmin(0.25, 0.7 / sqrt(x));
  const double ex = exp(-x);
  const double ce = cosh(eta);
  // exp(-x cosh t) = exp(-x) exp(-x (cosh t - 1)); half weight at t = 0
  double sum = 0.5, cprev = 1.0, c = ce;
  for (int k = 1; k < 4000; ++k) {
    const double term = exp(-x * (c - 1.0)) * (nu ? c : 1.0);
    sum += term;
    if (term < 1e-18 * sum) break;
    const double cn = 2.0 * ce * c - cprev;
    cprev = c;
    c = cn;
  }
  return eta * ex * sum;
}

// Wrapped offset of index i of a transform of length P for an axis of n
// nodes: offsets 0 .. n-1 at i = 0 .. n-1, -1 .. -(n-1) at P-1 .. P-n+1.
__device__ __forceinline__ bool wrapped(int i, int P, int n, int *o) {
  if (i < n) {
    *o = i;
    return true;
  }
  if (i >= P - (n - 1)) {
    *o = i - P;
    return true;
  }
  return false;
}

// G at the offsets 0 <= b <= a < m, packed as tab[a (a + 1) / 2 + b] (G
// depends on |offset| only, so one octant serves all); the origin takes *g0.
__global__ void k_green_table(double *tab, int m, double h, double ft, double hbar,
                              const double *g0) {
  const int64_t tot = (int64_t)m * (m + 1) / 2;
  const double inv2pi = 1.0 / (2.0 * M_PI * hbar * hbar);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
    while ((int64_t)a * (a + 1) / 2 > e) --a;
    while ((int64_t)(a + 1) * (a + 2) / 2 <= e) ++a;
    const int b = (int)(e - (int64_t)a * (a + 1) / 2);
    tab[e] = (a == 0) ? *g0 : bessel_k(0, ft * h * hypot((double)a, (double)b) / hbar) * inv2pi;
  }
}

// Kernel sampled at the wrapped offsets into a (Py x Px, pitch Px) complex
// array: mode 0 G~ = exp(-f~ r / hbar); mode 1 G from the octant table.
__global__ void k_fill_kernel(double2 *a, int Px, int Py, int nx, int ny, double h, double ft,
                              double hbar, int mode, const double *__restrict__ tab) {
  const int64_t tot = (int64_t)Px * Py;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(e % Px), iy = (int)(e / Px);
    int ox, oy;
    double v = 0.0;
    if (wrapped(ix, Px, nx, &ox) && wrapped(iy, Py, ny, &oy)) {
      if (mode == 0) {
        v = exp(-ft * h * hypot((double)ox, (double)oy) / hbar);
      } else {
        const int p = max(abs(ox), abs(oy)), q = min(abs(ox), abs(oy));
        v = tab[(int64_t)p * (p + 1) / 2 + q];
      }
    }
    a[e] = make_double2(v, 0.0);
  }
}

// G's average over the cell [-h/2, h/2]^2: 8 rays' triangles, along each
// int_0^R r K_0(a r) dr = (1 - a R K_1(a R)) / a^2, R = (h/2) / cos(theta),
// over theta in [0, pi/4] by Simpson's rule: the weighted samples first,
// spread over the GPU, then their fixed-order sum in one block.
constexpr int kSimpson = 2048;   // intervals (even)

__global__ void k_cell_samples(double h, double ft, double hbar, double *val) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kSimpson) return;
  const double a = ft / hbar;
  const double th = (M_PI / 4) * k / kSimpson;
  const double R = 0.5 * h / cos(th);
  const double v = (1.0 - a * R * bessel_k(1, a * R)) / (a * a);
  const double w = (k == 0 || k == kSimpson) ? 1.0 : ((k & 1) ? 4.0 : 2.0);
  val[k] = w * v;
}

__global__ void k_cell_average(const double *__restrict__ val, double h, double hbar,
                               double *g0) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int k = threadIdx.x; k <= kSimpson; k += blockDim.x) acc += val[k];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    const double integral = 8.0 * acc * (M_PI / 4) / (3.0 * kSimpson);
    *g0 = integral / (h * h) / (2.0 * M_PI * hbar * hbar);
  }
}

// Pointwise spectral product b *= k.
__global__ void k_cmul(double2 *b, const double2 *__restrict__ k, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    b[e] = cmul(b[e], k[e]);
}

// Zero-padded complex array of psi = (f^2 - f~^2) g for the grid function g
// (Table 1 step 9), zero outside the grid.
__global__ void k_embed(double2 *a, int Px, int Py, int nx, int ny, const double *__restrict__ f,
                        double ft2, const double *__restrict__ g) {
  const int64_t tot = (int64_t)Px * Py;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(e % Px), iy = (int)(e / Px);
    double v = 0.0;
    if (ix < nx && iy < ny) {
      const int64_t i = (int64_t)iy * nx + ix;
      const double fi = f[i];
      v = (fi * fi - ft2) * g[i];   // psi_i = (f^2 - f~^2) phi_{i-1}
    }
    a[e] = make_double2(v, 0.0);
  }
}

__global__ void k_delta(double2 *a, int Px, const int64_t *__restrict__ src, int64_t nsrc, int nx) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nsrc) return;
  const int64_t j = src[k];
  const int x = (int)(j % nx), y = (int)(j / nx);
  a[(size_t)y * Px + x] = make_double2(1.0, 0.0);
}

// Grid values of an inverse transform: term = scale * Re(a); phi += sign term.
__global__ void k_extract(const double2 *__restrict__ a, int Px, int nx, int64_t n, double scale,
                          double sign, double *__restrict__ term, double *__restrict__ phi,
                          int first) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)(i / nx);
    const double v = scale * a[(size_t)y * Px + x].x;
    term[i] = v;
    phi[i] = first ? v : phi[i] + sign * v;
  }
}

__global__ void k_log(const double *__restrict__ phi, int64_t n, double hbar, double *S) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    S[i] = -hbar * log(phi[i]);
}

// min and max of f, and a flag for values that are not finite and positive.
__global__ void k_fminmax(const double *__restrict__ f, int64_t n, double *out, int *bad) {
  double lo = INFINITY, hi = 0.0;
  int b = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = f[i];
    if (!(v > 0.0) || !isfinite(v)) b = 1;
    lo = fmin(lo, v);
    hi = fmax(hi, v);
  }
  if (b) atomicExch(bad, 1);
  // per warp, then one atomic per warp: positive doubles order like their bits
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (hi > 0.0)
      atomicMax(reinterpret_cast<unsigned long long *>(out + 1),
                (unsigned long long)__double_as_longlong(hi));
    if (lo > 0.0 && lo < INFINITY)
      atomicMin(reinterpret_cast<unsigned long long *>(out),
                (unsigned long long)__double_as_longlong(lo));
  }
}

struct Fft2 {
  int Px, Py;
  Radices rx, ry;
  DftConst kc;
  double2 *twx, *twy;
  double2 *A, *B;   // A: Py x Px (grid layout); B: Px x Py (transposed)
  cudaStream_t s;
};

// Smallest 2^a 3^b 5^c >= n (0 if above kMaxFft).
int fft_length(int n) {
  for (int p = std::max(n, 2); p <= kMaxFft; ++p) {
    int q = p;
    for (int f : {2, 3, 5})
      while (q % f == 0) q /= f;
    if (q == 1) return p;
  }
  return 0;
}

// Stage radices of P: fours first, then a two, threes and fives.
Radices radices(int P) {
  Radices r{};
  int q = P;
  while (q % 4 == 0 && r.n < kMaxStages) {
    r.r[r.n++] = 4;
    q /= 4;
  }
  for (int f : {2, 3, 5})
    while (q % f == 0 && r.n < kMaxStages) {
      r.r[r.n++] = f;
      q /= f;
    }
  return r;
}

void rows(const Fft2 &F, double2 *a, int count, int P, const Radices &rad, const double2 *tw,
          bool inv) {
  const int th = std::min(512, std::max(32, P / 2));
  const size_t sm = 2 * sizeof(double2) * P;
  if (inv)
    k_fft_rows<true><<<count, th, sm, F.s>>>(a, P, rad, F.kc, tw);
  else
    k_fft_rows<false><<<count, th, sm, F.s>>>(a, P, rad, F.kc, tw);
}

void transpose(const Fft2 &F, const double2 *in, double2 *out, int r, int c) {
  dim3 g((c + 31) / 32, (r + 31) / 32), b(32, 8);
  k_transpose<<<g, b, 0, F.s>>>(in, out, r, c);
}

// A (grid layout) -> B (spectrum, transposed layout).  Rows of A at and past
// `rows_in` are zero (grid functions), so their transforms are zero and are
// skipped.
void forward(const Fft2 &F, int rows_in) {
  rows(F, F.A, rows_in, F.Px, F.rx, F.twx, false);
  transpose(F, F.A, F.B, F.Py, F.Px);
  rows(F, F.B, F.Px, F.Py, F.ry, F.twy, false);
}

// B (spectrum) -> A (grid layout), unscaled; only the first `rows_out` rows
// of A (the grid's) are transformed back.
void inverse(const Fft2 &F, int rows_out) {
  rows(F, F.B, F.Px, F.Py, F.ry, F.twy, true);
  transpose(F, F.B, F.A, F.Px, F.Py);
  rows(F, F.A, rows_out, F.Px, F.rx, F.twx, true);
}

// Work arrays from the stream-ordered allocator (the device's memory pool):
// after the first call, allocating and freeing them costs no synchronisation.
struct Buf {
  cudaStream_t s;
  std::vector<void *> p;
  explicit Buf(cudaStream_t st) : s(st) {}
  ~Buf() {
    for (void *q : p) cudaFreeAsync(q, s);
  }
  template <class T>
  bool get(T **out, size_t n) {
    void *q = nullptr;
    if (cudaMallocAsync(&q, sizeof(T) * std::max<size_t>(n, 1), s) != cudaSuccess) return false;
    p.push_back(q);
    *out = static_cast<T *>(q);
    return true;
  }
};

}  // namespace
}  // namespace eik

using namespace eik;

extern "C" eik_status eik_fft_series(const int64_t *dims, double h, double hbar, const double *f,
                                     const int64_t *src_idx, int64_t nsrc, int terms,
                                     double f_tilde, double *S_out, double *phi_out,
                                     double *f_tilde_out, eik_stream_t stream) {
  if (!dims || !f || !src_idx || !S_out || nsrc < 1 || terms < 0 || terms > 64)
    return EIK_ERR_ARG;
  if (!(h > 0.0) || !std::isfinite(h) || !(hbar > 0.0) || !std::isfinite(hbar) ||
      !(f_tilde >= 0.0) || !std::isfinite(f_tilde))
    return EIK_ERR_ARG;
  const int64_t nx64 = dims[0], ny64 = dims[1];
  if (nx64 < 2 || ny64 < 2 || 2 * nx64 - 1 > kMaxFft || 2 * ny64 - 1 > kMaxFft)
    return EIK_ERR_ARG;
  const int nx = (int)nx64, ny = (int)ny64;
  const int64_t n = nx64 * ny64;
  std::vector<int64_t> hs(nsrc);
  if (cudaMemcpy(hs.data(), src_idx, sizeof(int64_t) * nsrc, cudaMemcpyDefault) != cudaSuccess)
    return EIK_ERR_ARG;
  for (int64_t s : hs)
    if (s < 0 || s >= n) return EIK_ERR_ARG;
  cudaStream_t s = stream;
  Fft2 F;
  F.Px = fft_length(2 * nx - 1);
  F.Py = fft_length(2 * ny - 1);
  if (F.Px == 0 || F.Py == 0) return EIK_ERR_ARG;
  F.rx = radices(F.Px);
  F.ry = radices(F.Py);
  F.kc = DftConst{-0.5, 0.5 * std::sqrt(3.0),
                  0.25 * (std::sqrt(5.0) - 1.0), -0.25 * (std::sqrt(5.0) + 1.0),
                  std::sqrt(0.125 * (5.0 + std::sqrt(5.0))),
                  std::sqrt(0.125 * (5.0 - std::sqrt(5.0)))};
  F.s = s;
  const int64_t np = (int64_t)F.Px * F.Py;
  Buf buf(s);
  double2 *K = nullptr;
  double *fd = nullptr, *phi = nullptr, *t0 = nullptr, *t1 = nullptr, *mm = nullptr, *g0 = nullptr;
  double *gtab = nullptr, *cval = nullptr;
  const int m = std::max(nx, ny);
  int64_t *src = nullptr;
  int *bad = nullptr;
  if (!buf.get(&F.twx, F.Px) || !buf.get(&F.twy, F.Py) || !buf.get(&F.A, np) ||
      !buf.get(&F.B, np) || !buf.get(&K, np) || !buf.get(&fd, n) || !buf.get(&phi, n) ||
      !buf.get(&t0, n) || !buf.get(&t1, n) || !buf.get(&mm, 2) || !buf.get(&g0, 1) ||
      !buf.get(&src, nsrc) || !buf.get(&bad, 1) ||
      !buf.get(&gtab, (size_t)m * (m + 1) / 2) || !buf.get(&cval, kSimpson + 1)) {
    cudaGetLastError();
    return EIK_ERR_OOM;
  }
  for (int P : {F.Px, F.Py}) {
    const size_t sm = 2 * sizeof(double2) * P;
    if (cudaFuncSetAttribute(k_fft_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max<size_t>(sm, 48 * 1024)) != cudaSuccess ||
        cudaFuncSetAttribute(k_fft_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max<size_t>(sm, 48 * 1024)) != cudaSuccess)
      return EIK_ERR_CUDA;
  }
  const int nb = 152 * 8;
  if (cudaMemcpyAsync(fd, f, sizeof(double) * n, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(src, hs.data(), sizeof(int64_t) * nsrc, cudaMemcpyHostToDevice, s) !=
          cudaSuccess)
    return EIK_ERR_ARG;
  // f validation and f~ (Eq. fTildeValue when not given)
  const double init[2] = {INFINITY, 0.0};
  if (cudaMemcpyAsync(mm, init, sizeof init, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(bad, 0, sizeof(int), s) != cudaSuccess)
    return EIK_ERR_CUDA;
  k_fminmax<<<nb, kThreads, 0, s>>>(fd, n, mm, bad);
  double hmm[2];
  int hbad = 0;
  if (cudaMemcpyAsync(hmm, mm, sizeof hmm, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return EIK_ERR_CUDA;
  if (hbad) return EIK_ERR_ARG;
  const double ft = (f_tilde > 0.0) ? f_tilde : std::sqrt(0.5 * (hmm[0] * hmm[0] + hmm[1] * hmm[1]));
  k_twiddles<<<(F.Px + 255) / 256, 256, 0, s>>>(F.twx, F.Px);
  k_twiddles<<<(F.Py + 255) / 256, 256, 0, s>>>(F.twy, F.Py);
  const double inv = 1.0 / ((double)F.Px * F.Py);
  // Table 1 steps 1-5: phi_0 = G~ * delta_kron
  k_fill_kernel<<<nb, kThreads, 0, s>>>(F.A, F.Px, F.Py, nx, ny, h, ft, hbar, 0, gtab);
  forward(F, F.Py);
  cudaMemcpyAsync(K, F.B, sizeof(double2) * np, cudaMemcpyDeviceToDevice, s);
  cudaMemsetAsync(F.A, 0, sizeof(double2) * np, s);
  k_delta<<<(int)((nsrc + 255) / 256), 256, 0, s>>>(F.A, F.Px, src, nsrc, nx);
  forward(F, ny);
  k_cmul<<<nb, kThreads, 0, s>>>(F.B, K, np);
  inverse(F, ny);
  // step 6: phi = phi_0 (t0 holds phi_{i-1})
  k_extract<<<nb, kThreads, 0, s>>>(F.A, F.Px, nx, n, inv, 1.0, t0, phi, 1);
  // step 7: transform of G
  if (terms > 0) {
    k_cell_samples<<<(kSimpson + 1 + 63) / 64, 64, 0, s>>>(h, ft, hbar, cval);
    k_cell_average<<<1, kThreads, 0, s>>>(cval, h, hbar, g0);
    k_green_table<<<nb, kThreads, 0, s>>>(gtab, m, h, ft, hbar, g0);
    k_fill_kernel<<<nb, kThreads, 0, s>>>(F.A, F.Px, F.Py, nx, ny, h, ft, hbar, 1, gtab);
    forward(F, F.Py);
    cudaMemcpyAsync(K, F.B, sizeof(double2) * np, cudaMemcpyDeviceToDevice, s);
  }
  // steps 8-14
  double *prev = t0, *cur = t1;
  for (int i = 1; i <= terms; ++i) {
    k_embed<<<nb, kThreads, 0, s>>>(F.A, F.Px, F.Py, nx, ny, fd, ft * ft, prev);
    forward(F, ny);
    k_cmul<<<nb, kThreads, 0, s>>>(F.B, K, np);
    inverse(F, ny);
    k_extract<<<nb, kThreads, 0, s>>>(F.A, F.Px, nx, n, inv * h * h, (i & 1) ? -1.0 : 1.0, cur,
                                      phi, 0);
    std::swap(prev, cur);
  }
  // step 15 (into the buffer no longer needed)
  double *Sd = cur;
  k_log<<<nb, kThreads, 0, s>>>(phi, n, hbar, Sd);
  if (cudaGetLastError() != cudaSuccess) return EIK_ERR_CUDA;
  if (cudaMemcpyAsync(S_out, Sd, sizeof(double) * n, cudaMemcpyDefault, s) != cudaSuccess)
    return EIK_ERR_ARG;
  if (phi_out &&
      cudaMemcpyAsync(phi_out, phi, sizeof(double) * n, cudaMemcpyDefault, s) != cudaSuccess)
    return EIK_ERR_ARG;
  if (cudaStreamSynchronize(s) != cudaSuccess) return EIK_ERR_CUDA;
  if (f_tilde_out) *f_tilde_out = ft;
  return EIK_OK;
}
