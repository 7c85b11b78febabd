// C ABI of libeik (declared in include/eik.h): argument checking, device
// memory, stream ordering, the CG driver loop (captured in a CUDA graph),
// restarts from the true residual, epilogue and adjoint.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "eik_batch.h"
#include "eik_internal.cuh"
#include "eik_launch.h"
#include "eik_mixed.h"

using namespace eik;

namespace {

thread_local std::string g_last_error = "no error";

eik_status fail(eik_status st, const std::string &msg) {
  g_last_error = msg;
  return st;
}

struct CudaError {
  cudaError_t err;
  const char *what;
};

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) throw CudaError{e_, #call};        \
  } while (0)

bool is_device_pointer(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

constexpr int kGraphIters = 32;     // CG iterations per graph launch
constexpr int kMaxRestarts = 3;     // restarts in a row without progress

// Kernels counted per handle (eik_kernel_stats).
enum KernelId {
  K_SETUP64 = 0, K_SOURCES64, K_RESIDUAL64, K_PASS1_64, K_PASS2_64, K_EPILOGUE64,
  K_SOURCE_VALUES, K_ADJ_RHS64, K_ADJ_GRAD64, K_MIXED_FIRST
};
constexpr int kMaxKernels = 32;
const char *const kKernelNames[K_MIXED_FIRST] = {
    "setup64", "sources64", "residual64", "cg_pass1_64", "cg_pass2_64", "epilogue64",
    "source_values", "adjoint_rhs64", "adjoint_grad64"};

struct KernelStat {
  int64_t launches = 0, timed = 0;
  double ms = 0.0;
};

}  // namespace

struct eik_handle {
  int device = 0;
  int num_sms = 0;
  Grid g{};
  TileCount tc{};
  int nblk_stencil = 0, nblk_stream = 0, nblk_part = 0, cap_elem = 0;
  eik_options opt{};
  cudaStream_t user = nullptr, stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  // FP64 state
  double *f = nullptr, *sig = nullptr, *x = nullptr, *r = nullptr, *p = nullptr,
         *q = nullptr, *aux = nullptr, *lam = nullptr, *grhs = nullptr;
  int64_t *src = nullptr;
  double *U = nullptr;
  int64_t nsrc = 0;
  CgState *st = nullptr;
  CgState *h_st = nullptr;     // pinned mirror
  double *part = nullptr;
  int *err = nullptr;
  int *h_err = nullptr;
  // graph of kGraphIters CG iterations for (x, r, p, q, weight)
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    double *x = nullptr, *w = nullptr;
  } graphs[2];
  bool have_solution = false;
  MixedState *mixed = nullptr;
  // diagnostics
  KernelStat kstat[kMaxKernels];
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> pending;   // (kernel id, event pair index)
};

namespace {

void free_handle(eik_handle *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto &gr : h->graphs)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  if (h->mixed) mixed_destroy(h->mixed);
  double *ptrs[] = {h->f,   h->sig, h->x, h->r,    h->p,
                    h->q,   h->aux, h->lam, h->grhs, h->U, h->part};
  for (double *d : ptrs)
    if (d) cudaFree(d);
  if (h->src) cudaFree(h->src);
  if (h->st) cudaFree(h->st);
  if (h->err) cudaFree(h->err);
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->h_err) cudaFreeHost(h->h_err);
  cudaEvent_t evs[] = {h->ev_in, h->ev_out, h->ev_t0, h->ev_t1};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

void count_launch(eik_handle *h, int id, int64_t n = 1) { h->kstat[id].launches += n; }

// Resolves the event pairs of timed launches (call after a stream sync).
void flush_timed(eik_handle *h) {
  for (auto &pr : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[2 * pr.second], h->ev_pool[2 * pr.second + 1]) ==
        cudaSuccess) {
      h->kstat[pr.first].ms += ms;
      h->kstat[pr.first].timed += 1;
    }
  }
  h->pending.clear();
}

// Launches fn() on the internal stream, counting it and, when profiling,
// bracketing it with CUDA events.
template <class F>
void launch_k(eik_handle *h, int id, F fn) {
  count_launch(h, id);
  if (!h->profiling) {
    fn();
    return;
  }
  const int pair = (int)h->pending.size();
  while ((int)h->ev_pool.size() < 2 * (pair + 1)) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    h->ev_pool.push_back(e);
  }
  CK(cudaEventRecord(h->ev_pool[2 * pair], h->stream));
  fn();
  CK(cudaEventRecord(h->ev_pool[2 * pair + 1], h->stream));
  h->pending.push_back({id, pair});
}

template <class T>
void dalloc(T **p, size_t count) {
  cudaError_t e = cudaMalloc((void **)p, sizeof(T) * std::max<size_t>(count, 1));
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw std::bad_alloc();
  }
}

// Orders the internal stream after the user's stream.
void enter(eik_handle *h) {
  CK(cudaSetDevice(h->device));
  CK(cudaEventRecord(h->ev_in, h->user));
  CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));
}

// Orders the user's stream after the internal stream.
void leave(eik_handle *h) {
  CK(cudaEventRecord(h->ev_out, h->stream));
  CK(cudaStreamWaitEvent(h->user, h->ev_out, 0));
}

// Copies a grid array (host or device) into device buffer dst.
void copy_in(eik_handle *h, double *dst, const double *src, int64_t n) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDefault, h->stream));
  if (!is_device_pointer(src)) CK(cudaStreamSynchronize(h->stream));
}

eik_status upload_f(eik_handle *h, const double *f) {
  copy_in(h, h->f, f, h->g.n);
  CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
  launch_k(h, K_SETUP64,
           [&] { launch_setup64(h->g, h->f, h->sig, h->x, h->err, h->stream, h->cap_elem); });
  launch_k(h, K_SOURCES64,
           [&] { launch_sources64(h->g, h->src, h->U, h->nsrc, h->sig, h->x, h->stream); });
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->h_err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->have_solution = false;
  if (*h->h_err) return fail(EIK_ERR_ARG, "f must be finite and > 0 at every node");
  return EIK_OK;
}

// Captures kGraphIters CG iterations (pass 1 + pass 2) on the internal
// stream for the given solution vector and optional weight.
cudaGraphExec_t graph_for(eik_handle *h, double *x, const double *w) {
  for (auto &gr : h->graphs)
    if (gr.exec && gr.x == x && gr.w == w) return gr.exec;
  auto &slot = (x == h->x) ? h->graphs[0] : h->graphs[1];
  if (slot.exec) {
    CK(cudaGraphExecDestroy(slot.exec));
    slot.exec = nullptr;
  }
  cudaGraph_t graph;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < kGraphIters; ++k) {
    launch_pass1_64(h->g, h->tc, h->nblk_stencil, h->sig, h->r, h->p, h->q, h->st, h->part,
                    h->nblk_part, h->stream);
    launch_pass2_64(h->g.n, h->nblk_stream, x, h->r, h->p, h->q, w, h->st,
                    h->part + 8 * (size_t)h->nblk_part, h->nblk_part, h->stream);
  }
  CK(cudaStreamEndCapture(h->stream, &graph));
  cudaGraphExec_t exec;
  CK(cudaGraphInstantiate(&exec, graph, 0));
  CK(cudaGraphDestroy(graph));
  slot.exec = exec;
  slot.x = x;
  slot.w = const_cast<double *>(w);
  return exec;
}

// Runs CG on Ahat xs = bhat (+ rhs) from the current xs until the stopping
// rule holds on the true residual, restarting from the true residual when
// the recurrence has drifted.  Fills iterations and the final residuals.
eik_status run_cg64(eik_handle *h, double *xs, const double *rhs, const double *weight,
                    double tol, int stop_norm, int max_iter, int *iters, double *res_cw,
                    double *res_nw) {
  CgState init{};
  init.tol = tol;
  init.max_iter = max_iter;
  init.stop_norm = stop_norm;
  *iters = 0;
  eik_status status = EIK_OK;
  double last_res = INFINITY;
  int stalled = 0;
  for (int restart = 0;; ++restart) {
    init.iter = *iters;
    *h->h_st = init;
    CK(cudaMemcpyAsync(h->st, h->h_st, sizeof(CgState), cudaMemcpyHostToDevice, h->stream));
    launch_k(h, K_RESIDUAL64, [&] {
      launch_residual64(h->g, h->tc, h->nblk_stencil, h->sig, xs, rhs, h->r, h->p, h->st,
                        h->part, h->nblk_part, h->stream);
    });
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(CgState), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    // weighted mode: the stop test of the true residual is done on the host
    // side of the next iteration; here the residual kernel's figures decide
    bool ok_now;
    if (stop_norm == EIK_STOP_NORMWISE)
      ok_now = h->h_st->rho <= tol * tol * h->h_st->bnorm2;
    else if (weight)
      ok_now = false;
    else
      ok_now = h->h_st->res_cw <= tol;
    *res_cw = h->h_st->res_cw;
    *res_nw = (h->h_st->res_nw2_b > 0) ? std::sqrt(h->h_st->res_nw2_r / h->h_st->res_nw2_b)
                                       : std::sqrt(h->h_st->res_nw2_r);
    if (ok_now || h->h_st->rho == 0.0) return EIK_OK;
    if (*iters >= max_iter) return fail(EIK_ERR_NOT_CONVERGED, "maximum number of CG iterations reached");
    // restarts continue while each one at least halves the true residual
    const double now = (stop_norm == EIK_STOP_NORMWISE || weight) ? h->h_st->rho : h->h_st->res_cw;
    if (restart > 0 && !(now < 0.5 * last_res)) {
      if (++stalled >= kMaxRestarts)
        return fail(EIK_ERR_NOT_CONVERGED, "restarts from the true residual stopped making progress");
    } else {
      stalled = 0;
    }
    last_res = std::min(last_res, now);
    cudaGraphExec_t exec = h->profiling ? nullptr : graph_for(h, xs, weight);
    for (;;) {
      if (exec) {
        CK(cudaGraphLaunch(exec, h->stream));
        count_launch(h, K_PASS1_64, kGraphIters);
        count_launch(h, K_PASS2_64, kGraphIters);
      } else {
        // profiled: one iteration per host check, so no launch runs past
        // convergence and every timed launch does the full pass
        for (int k = 0; k < 1; ++k) {
          launch_k(h, K_PASS1_64, [&] {
            launch_pass1_64(h->g, h->tc, h->nblk_stencil, h->sig, h->r, h->p, h->q, h->st,
                            h->part, h->nblk_part, h->stream);
          });
          launch_k(h, K_PASS2_64, [&] {
            launch_pass2_64(h->g.n, h->nblk_stream, xs, h->r, h->p, h->q, weight, h->st,
                            h->part + 8 * (size_t)h->nblk_part, h->nblk_part, h->stream);
          });
        }
        CK(cudaGetLastError());
      }
      CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(CgState), cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
      flush_timed(h);
      if (h->h_st->done) break;
    }
    *iters = h->h_st->iter;
    status = (eik_status)h->h_st->status;
    if (status == EIK_ERR_BREAKDOWN) return fail(status, "CG breakdown (p.Ap <= 0)");
    if (weight && status == EIK_OK) {
      // the recurrence met the weighted test; accept (the adjoint has no
      // componentwise true-residual form)
      return EIK_OK;
    }
    if (status == EIK_ERR_NOT_CONVERGED) {
      // report the true residual of the last iterate
      launch_k(h, K_RESIDUAL64, [&] {
        launch_residual64(h->g, h->tc, h->nblk_stencil, h->sig, xs, rhs, h->r, h->p, h->st,
                          h->part, h->nblk_part, h->stream);
      });
      CK(cudaMemcpyAsync(h->h_st, h->st, sizeof(CgState), cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
      *res_cw = h->h_st->res_cw;
      *res_nw = (h->h_st->res_nw2_b > 0)
                    ? std::sqrt(h->h_st->res_nw2_r / h->h_st->res_nw2_b)
                    : std::sqrt(h->h_st->res_nw2_r);
      return fail(EIK_ERR_NOT_CONVERGED, "maximum number of CG iterations reached");
    }
  }
}

// Writes S (and phi) from the solution xh in h->x to the outputs, which may
// be host or device pointers.
void write_outputs(eik_handle *h, double *S_out, double *phi_out,
                   const MixedArgs *ma = nullptr) {
  const bool S_dev = is_device_pointer(S_out);
  const bool P_dev = phi_out ? is_device_pointer(phi_out) : true;
  double *S_d = S_dev ? S_out : h->aux;
  double *P_d = phi_out ? (P_dev ? phi_out : h->q) : nullptr;
  if (ma) {
    if (mixed_write_outputs(h->mixed, *ma, S_d, P_d) != EIK_OK)
      throw CudaError{cudaErrorUnknown, "mixed epilogue"};
  } else {
    launch_k(h, K_EPILOGUE64,
             [&] { launch_epilogue64(h->g, h->sig, h->x, S_d, P_d, h->stream, h->cap_elem); });
  }
  launch_k(h, K_SOURCE_VALUES,
           [&] { launch_source_values(h->src, h->U, h->nsrc, S_d, h->stream); });
  CK(cudaGetLastError());
  if (!S_dev)
    CK(cudaMemcpyAsync(S_out, S_d, sizeof(double) * h->g.n, cudaMemcpyDeviceToHost,
                       h->stream));
  if (phi_out && !P_dev)
    CK(cudaMemcpyAsync(phi_out, P_d, sizeof(double) * h->g.n, cudaMemcpyDeviceToHost,
                       h->stream));
}

}  // namespace

// ===================================================================== ABI
extern "C" {

void eik_default_options(eik_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = EIK_PREC_FP64;
  opt->tol = 1e-12;
  opt->stop_norm = EIK_STOP_COMPONENTWISE;
  opt->max_iter = 200000;
  opt->boundary = EIK_BOUNDARY_HALF_CELL;
  opt->tile_override = 0;
  opt->inner_tol = 0.0;
  opt->max_outer = 0;
  opt->band_bits = 0;
}

const char *eik_last_error(void) { return g_last_error.c_str(); }

int eik_abi_version(void) { return EIK_ABI_VERSION; }

int eik_cuda_arch(void) {
#ifdef EIK_ARCH
  return EIK_ARCH;
#else
  return 0;
#endif
}

// Creates one solver; with exec, a member of a packed batch whose FP32
// inner-CG arrays live in the batch's atlas (instance `member`).
static eik_status create_impl(eik_handle **out, int ndim, const int64_t *dims, double hsp,
                              double hbar, const double *f, const int64_t *src_idx,
                              const double *src_U, int64_t nsrc, const eik_options *opt,
                              eik_stream_t stream, BatchExec *exec, int member) {
  if (!out) return fail(EIK_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (ndim != 2 && ndim != 3) return fail(EIK_ERR_ARG, "ndim must be 2 or 3");
  if (!dims || !f || !src_idx) return fail(EIK_ERR_ARG, "NULL dims, f or src_idx");
  if (!(hsp > 0) || !std::isfinite(hsp) || !(hbar > 0) || !std::isfinite(hbar))
    return fail(EIK_ERR_ARG, "h and hbar must be finite and > 0");
  if (nsrc < 1) return fail(EIK_ERR_ARG, "at least one source is required");
  int64_t d[3] = {1, 1, 1};
  int64_t n = 1;
  for (int a = 0; a < ndim; ++a) {
    d[a] = dims[a];
    if (d[a] < 2 || d[a] > (int64_t)1 << 30) return fail(EIK_ERR_ARG, "each extent must be >= 2");
    n *= d[a];
    if (n > ((int64_t)1 << 40)) return fail(EIK_ERR_ARG, "grid too large");
  }
  eik_options o;
  eik_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != EIK_PREC_FP64 && o.precision != EIK_PREC_MIXED)
    return fail(EIK_ERR_ARG, "unknown precision mode");
  if (o.boundary != EIK_BOUNDARY_HALF_CELL && o.boundary != EIK_BOUNDARY_DROP_EDGE)
    return fail(EIK_ERR_ARG, "unknown boundary mode");
  if (o.stop_norm != EIK_STOP_COMPONENTWISE && o.stop_norm != EIK_STOP_NORMWISE)
    return fail(EIK_ERR_ARG, "unknown stop_norm");
  if (!(o.tol > 0) || o.max_iter < 1) return fail(EIK_ERR_ARG, "tol and max_iter must be > 0");
  if (o.tile_override < 0 || o.tile_override > 4)
    return fail(EIK_ERR_ARG, "tile_override must be in 0..4");
  if (o.batch_pack < -1 || o.batch_pack > 1)
    return fail(EIK_ERR_ARG, "batch_pack must be -1, 0 or 1");
  if (o.batch_tile_rows < 0 || o.batch_tile_rows > 1024)
    return fail(EIK_ERR_ARG, "batch_tile_rows must be in 0..1024");
  if (o.precond != EIK_PRECOND_JACOBI && o.precond != EIK_PRECOND_MULTIGRID)
    return fail(EIK_ERR_ARG, "unknown precond");
  if (o.precond == EIK_PRECOND_MULTIGRID && o.precision != EIK_PREC_MIXED)
    return fail(EIK_ERR_ARG, "the multigrid preconditioner needs mixed precision");

  eik_handle *h = new (std::nothrow) eik_handle();
  if (!h) return fail(EIK_ERR_OOM, "host allocation failed");
  try {
    CK(cudaGetDevice(&h->device));
    CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    h->opt = o;
    h->user = stream;
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    CK(cudaEventCreate(&h->ev_t0));
    CK(cudaEventCreate(&h->ev_t1));
    CK(cudaEventRecord(h->ev_in, h->user));
    CK(cudaStreamWaitEvent(h->stream, h->ev_in, 0));

    // sources: validate and de-duplicate on the host
    std::vector<int64_t> hs(nsrc);
    std::vector<double> hu(nsrc, 0.0);
    CK(cudaMemcpy(hs.data(), src_idx, sizeof(int64_t) * nsrc, cudaMemcpyDefault));
    if (src_U) CK(cudaMemcpy(hu.data(), src_U, sizeof(double) * nsrc, cudaMemcpyDefault));
    std::vector<std::pair<int64_t, double>> sv(nsrc);
    for (int64_t k = 0; k < nsrc; ++k) {
      if (hs[k] < 0 || hs[k] >= n) {
        free_handle(h);
        return fail(EIK_ERR_ARG, "source index out of range");
      }
      if (!std::isfinite(hu[k])) {
        free_handle(h);
        return fail(EIK_ERR_ARG, "source value not finite");
      }
      sv[k] = {hs[k], hu[k]};
    }
    std::sort(sv.begin(), sv.end(),
              [](const std::pair<int64_t, double> &a, const std::pair<int64_t, double> &b) {
                return a.first < b.first;
              });
    std::vector<int64_t> us;
    std::vector<double> uu;
    for (auto &e : sv) {
      if (!us.empty() && us.back() == e.first) {
        if (uu.back() != e.second) {
          free_handle(h);
          return fail(EIK_ERR_ARG, "duplicate source with conflicting values");
        }
        continue;
      }
      us.push_back(e.first);
      uu.push_back(e.second);
    }
    const double U_min = *std::min_element(uu.begin(), uu.end());
    for (double u : uu)
      if ((u - U_min) / hbar > 690.0) {
        free_handle(h);
        return fail(EIK_ERR_ARG,
                    "source values differ by more than 690*hbar (phi would underflow)");
      }
    h->nsrc = (int64_t)us.size();

    Grid &g = h->g;
    g.nx = (int)d[0];
    g.ny = (int)d[1];
    g.nz = (int)d[2];
    g.ndim = ndim;
    g.n = n;
    g.c = hbar * hbar / (hsp * hsp);
    g.sqrt_c = hbar / hsp;
    g.hbar = hbar;
    g.U_min = U_min;
    g.boundary = o.boundary;
    h->tc = tile_count(g);
    const int cap = stencil_grid_cap(ndim, h->num_sms);
    h->nblk_stencil = (int)std::min<int64_t>(h->tc.total, cap);
    h->cap_elem = h->num_sms * 8;
    h->nblk_stream = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, h->cap_elem);
    h->nblk_part = std::max(h->nblk_stencil, h->nblk_stream);

    try {
      dalloc(&h->f, n);
      dalloc(&h->sig, n);
      dalloc(&h->x, n);
      dalloc(&h->r, n);
      dalloc(&h->p, n);
      dalloc(&h->q, n);
      dalloc(&h->aux, n);
      dalloc(&h->src, h->nsrc);
      dalloc(&h->U, h->nsrc);
      dalloc(&h->st, 1);
      dalloc(&h->part, 16 * (size_t)h->nblk_part);
      dalloc(&h->err, 1);
    } catch (std::bad_alloc &) {
      free_handle(h);
      return fail(EIK_ERR_OOM, "device allocation failed");
    }
    CK(cudaMallocHost((void **)&h->h_st, sizeof(CgState)));
    CK(cudaMallocHost((void **)&h->h_err, sizeof(int)));
    CK(cudaMemsetAsync(h->st, 0, sizeof(CgState), h->stream));
    CK(cudaMemcpyAsync(h->src, us.data(), sizeof(int64_t) * h->nsrc, cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaMemcpyAsync(h->U, uu.data(), sizeof(double) * h->nsrc, cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (o.precision == EIK_PREC_MIXED) {
      eik_status ms = exec ? mixed_create_member(&h->mixed, g, h->tc, h->num_sms, exec, member,
                                                 h->stream)
                           : mixed_create(&h->mixed, g, h->tc, h->num_sms, o.tile_override,
                                          o.precond, h->stream);
      if (ms != EIK_OK) {
        free_handle(h);
        return fail(ms, "mixed-precision workspace allocation failed");
      }
    }
    eik_status s = upload_f(h, f);
    if (s != EIK_OK) {
      free_handle(h);
      return s;
    }
    leave(h);
  } catch (CudaError &e) {
    std::string msg = std::string("CUDA error in ") + e.what + ": " + cudaGetErrorString(e.err);
    free_handle(h);
    return fail(EIK_ERR_CUDA, msg);
  } catch (std::bad_alloc &) {
    free_handle(h);
    return fail(EIK_ERR_OOM, "allocation failed");
  }
  *out = h;
  return EIK_OK;
}

eik_status eik_create(eik_handle **out, int ndim, const int64_t *dims, double hsp,
                      double hbar, const double *f, const int64_t *src_idx,
                      const double *src_U, int64_t nsrc, const eik_options *opt,
                      eik_stream_t stream) {
  return create_impl(out, ndim, dims, hsp, hbar, f, src_idx, src_U, nsrc, opt, stream, nullptr,
                     -1);
}

eik_status eik_set_f(eik_handle *h, const double *f) {
  if (!h || !f) return fail(EIK_ERR_ARG, "NULL handle or f");
  try {
    enter(h);
    eik_status s = upload_f(h, f);
    leave(h);
    return s;
  } catch (CudaError &e) {
    return fail(EIK_ERR_CUDA, std::string("CUDA error in ") + e.what + ": " +
                                  cudaGetErrorString(e.err));
  }
}

eik_status eik_solve(eik_handle *h, double *S_out, double *phi_out, eik_stats *stats) {
  if (!h || !S_out) return fail(EIK_ERR_ARG, "NULL handle or S_out");
  try {
    enter(h);
    CK(cudaEventRecord(h->ev_t0, h->stream));
    int iters = 0, outer = 1;
    double res_cw = 0, res_nw = 0;
    eik_status s;
    MixedArgs ma{};
    const bool mixed = h->opt.precision == EIK_PREC_MIXED;
    if (mixed) {
      ma.g = h->g;
      ma.tc = h->tc;
      ma.stream = h->stream;
      ma.sig = h->sig;
      ma.x = h->x;
      ma.r = h->r;
      ma.aux = h->aux;
      ma.part = h->part;
      ma.nblk_part = h->nblk_part;
      ma.nblk_stencil = h->nblk_stencil;
      ma.st = h->st;
      ma.h_st = h->h_st;
      ma.f = h->f;
      ma.src = h->src;
      ma.U = h->U;
      ma.nsrc = h->nsrc;
      ma.opt = h->opt;
      s = mixed_solve(h->mixed, ma, &iters, &outer, &res_cw, &res_nw);
      if (s != EIK_OK) g_last_error = mixed_last_error();
    } else {
      // reset the solution (sources keep their slots)
      CK(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream));
      launch_k(h, K_SETUP64,
               [&] { launch_setup64(h->g, h->f, h->sig, h->x, h->err, h->stream, h->cap_elem); });
      launch_k(h, K_SOURCES64,
               [&] { launch_sources64(h->g, h->src, h->U, h->nsrc, h->sig, h->x, h->stream); });
      s = run_cg64(h, h->x, nullptr, nullptr, h->opt.tol, h->opt.stop_norm, h->opt.max_iter,
                   &iters, &res_cw, &res_nw);
    }
    if (s == EIK_OK || s == EIK_ERR_NOT_CONVERGED)
      write_outputs(h, S_out, phi_out, mixed ? &ma : nullptr);
    // the adjoint works on the hat-space FP64 solution in h->x
    if (mixed && s == EIK_OK && mixed_export_hat(h->mixed, ma, h->x) != EIK_OK)
      throw CudaError{cudaErrorUnknown, "mixed export"};
    CK(cudaEventRecord(h->ev_t1, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    flush_timed(h);
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
    if (stats) {
      stats->outer_iters = outer;
      stats->inner_iters = iters;
      stats->res_cw = res_cw;
      stats->res_nw = res_nw;
      stats->ms = ms;
    }
    h->have_solution = (s == EIK_OK);
    leave(h);
    return s;
  } catch (CudaError &e) {
    return fail(EIK_ERR_CUDA, std::string("CUDA error in ") + e.what + ": " +
                                  cudaGetErrorString(e.err));
  }
}

eik_status eik_grad(eik_handle *h, const double *dLdS, double *dLdf, eik_stats *stats) {
  if (!h || !dLdS || !dLdf) return fail(EIK_ERR_ARG, "NULL handle, dLdS or dLdf");
  if (!h->have_solution) return fail(EIK_ERR_STATE, "eik_grad needs a successful eik_solve");
  try {
    enter(h);
    CK(cudaEventRecord(h->ev_t0, h->stream));
    if (!h->lam) {
      try {
        dalloc(&h->lam, h->g.n);
        dalloc(&h->grhs, h->g.n);
      } catch (std::bad_alloc &) {
        leave(h);
        return fail(EIK_ERR_OOM, "device allocation failed");
      }
    }
    // dLdS -> aux (device)
    CK(cudaMemcpyAsync(h->aux, dLdS, sizeof(double) * h->g.n, cudaMemcpyDefault, h->stream));
    if (!is_device_pointer(dLdS)) CK(cudaStreamSynchronize(h->stream));
    double *rhs = h->grhs;
    double *gmax_part = h->part + 12 * (size_t)h->nblk_part;
    launch_k(h, K_ADJ_RHS64, [&] {
      launch_adjoint_rhs64(h->g, h->sig, h->x, h->aux, rhs, gmax_part, h->nblk_stream,
                           h->stream);
    });
    std::vector<double> gm(h->nblk_stream);
    CK(cudaMemcpyAsync(gm.data(), gmax_part, sizeof(double) * h->nblk_stream,
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemsetAsync(h->lam, 0, sizeof(double) * h->g.n, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double gmax = 0.0;
    for (double v : gm) gmax = std::max(gmax, v);
    int iters = 0;
    double res_cw = 0, res_nw = 0;
    eik_status s = EIK_OK;
    if (gmax > 0.0) {
      // stop when |xh_i * rhat_i| <= tol * max|hbar dL/dS| (residual of the
      // variables mu = xh * lamh, whose right-hand side is -hbar dL/dS)
      const double tol = std::max(h->opt.tol, 1e-14) * gmax;
      s = run_cg64(h, h->lam, rhs, h->x, tol, EIK_STOP_COMPONENTWISE, h->opt.max_iter, &iters,
                   &res_cw, &res_nw);
    }
    const bool out_dev = is_device_pointer(dLdf);
    double *out_d = out_dev ? dLdf : h->aux;
    launch_k(h, K_ADJ_GRAD64, [&] {
      launch_adjoint_grad64(h->g, h->f, h->sig, h->x, h->lam, out_d, h->stream, h->cap_elem);
    });
    CK(cudaGetLastError());
    if (!out_dev)
      CK(cudaMemcpyAsync(dLdf, out_d, sizeof(double) * h->g.n, cudaMemcpyDeviceToHost,
                         h->stream));
    CK(cudaEventRecord(h->ev_t1, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    flush_timed(h);
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev_t0, h->ev_t1));
    if (stats) {
      stats->outer_iters = 1;
      stats->inner_iters = iters;
      stats->res_cw = res_cw;
      stats->res_nw = res_nw;
      stats->ms = ms;
    }
    leave(h);
    return s;
  } catch (CudaError &e) {
    return fail(EIK_ERR_CUDA, std::string("CUDA error in ") + e.what + ": " +
                                  cudaGetErrorString(e.err));
  }
}

eik_status eik_set_profiling(eik_handle *h, int enable) {
  if (!h) return fail(EIK_ERR_ARG, "NULL handle");
  h->profiling = enable != 0;
  mixed_set_profiling(h->mixed, h->profiling);
  return EIK_OK;
}

eik_status eik_kernel_stats(eik_handle *h, eik_kernel_stat *out, int max, int *count) {
  if (!h || !count) return fail(EIK_ERR_ARG, "NULL handle or count");
  int n = 0;
  for (int id = 0; id < kMaxKernels; ++id) {
    const char *name = id < K_MIXED_FIRST ? kKernelNames[id] : mixed_kernel_name(id - K_MIXED_FIRST);
    if (!name) continue;
    if (out && n < max) {
      std::memset(out[n].name, 0, sizeof(out[n].name));
      std::strncpy(out[n].name, name, sizeof(out[n].name) - 1);
      out[n].launches = h->kstat[id].launches +
                        (id >= K_MIXED_FIRST ? mixed_kernel_launches(h->mixed, id - K_MIXED_FIRST) : 0);
      out[n].timed_launches = h->kstat[id].timed;
      out[n].total_ms = h->kstat[id].ms;
      if (id >= K_MIXED_FIRST) {
        int64_t t = 0;
        double ms = 0.0;
        mixed_kernel_time(h->mixed, id - K_MIXED_FIRST, &t, &ms);
        out[n].timed_launches += t;
        out[n].total_ms += ms;
      }
    }
    ++n;
  }
  *count = n;
  return EIK_OK;
}

eik_status eik_reset_kernel_stats(eik_handle *h) {
  if (!h) return fail(EIK_ERR_ARG, "NULL handle");
  for (auto &k : h->kstat) k = KernelStat{};
  mixed_reset_launches(h->mixed);
  return EIK_OK;
}

eik_status eik_destroy(eik_handle *h) {
  free_handle(h);
  return EIK_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batch
struct eik_batch {
  int count = 0;
  int ndim = 2;
  int workers = 0;
  std::vector<eik_handle *> hs;
  std::vector<int64_t> off;   // node offsets, count+1
  BatchExec *exec = nullptr;  // packed 2D mixed batches
};

namespace {

// Runs fn(i) for every instance on a pool of host threads; each thread keeps
// its own CUDA calls on the instance's internal stream.  Returns the first
// non-OK status (by instance order) and its message.
template <class F>
eik_status run_pool(eik_batch *b, F fn) {
  const int n = b->count;
  int workers = b->workers > 0 ? b->workers : 16;
  workers = std::max(1, std::min(workers, n));
  std::vector<eik_status> st(n, EIK_OK);
  std::vector<std::string> msg(n);
  std::atomic<int> next{0};
  int dev = 0;
  cudaGetDevice(&dev);
  auto work = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      st[i] = fn(i);
      if (st[i] != EIK_OK) msg[i] = eik_last_error();
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < workers; ++w) th.emplace_back(work);
  work();
  for (auto &t : th) t.join();
  for (int i = 0; i < n; ++i)
    if (st[i] != EIK_OK) {
      g_last_error = "instance " + std::to_string(i) + ": " + msg[i];
      return st[i];
    }
  return EIK_OK;
}

}  // namespace

extern "C" {

eik_status eik_create_batch(eik_batch **out, int count, int ndim, const int64_t *dims,
                            const double *h, const double *hbar, const double *f,
                            const int64_t *src_offsets, const int64_t *src_idx,
                            const double *src_U, const eik_options *opt,
                            eik_stream_t stream) {
  if (!out) return fail(EIK_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || (ndim != 2 && ndim != 3) || !dims || !h || !hbar || !f || !src_offsets ||
      !src_idx)
    return fail(EIK_ERR_ARG, "invalid batch arguments");
  eik_batch *b = new (std::nothrow) eik_batch();
  if (!b) return fail(EIK_ERR_OOM, "host allocation failed");
  b->count = count;
  b->ndim = ndim;
  b->off.assign(count + 1, 0);
  std::vector<int64_t> so(count + 1);
  if (cudaMemcpy(so.data(), src_offsets, sizeof(int64_t) * (count + 1), cudaMemcpyDefault) !=
      cudaSuccess) {
    delete b;
    return fail(EIK_ERR_ARG, "cannot read src_offsets");
  }
  for (int i = 0; i < count; ++i) {
    int64_t n = 1;
    for (int a = 0; a < ndim; ++a) n *= dims[(int64_t)i * ndim + a];
    b->off[i + 1] = b->off[i] + n;
    if (so[i + 1] < so[i]) {
      delete b;
      return fail(EIK_ERR_ARG, "src_offsets must be non-decreasing");
    }
  }
  eik_options o;
  eik_default_options(&o);
  if (opt) o = *opt;
  if (ndim == 2 && o.precision == EIK_PREC_MIXED && o.batch_pack >= 0 &&
      o.precond == EIK_PRECOND_JACOBI) {
    // packed: one atlas for the FP32 arrays of every instance
    std::vector<int> nx(count), ny(count);
    for (int i = 0; i < count; ++i) {
      const int64_t ex = dims[2 * (int64_t)i], ey = dims[2 * (int64_t)i + 1];
      if (ex < 2 || ey < 2 || ex > (1 << 20) || ey > (1 << 20)) {
        delete b;
        return fail(EIK_ERR_ARG, "packed batch: each extent must be in 2 .. 2^20");
      }
      nx[i] = (int)ex;
      ny[i] = (int)ey;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (o.tile_override < 0 || o.tile_override > 4 || o.batch_tile_rows < 0 ||
        o.batch_tile_rows > 1024) {
      delete b;
      return fail(EIK_ERR_ARG, "invalid tile_override or batch_tile_rows");
    }
    const eik_status es = batch_exec_create(&b->exec, count, nx.data(), ny.data(), o.boundary,
                                            nsm, o.tile_override, o.batch_tile_rows);
    if (es != EIK_OK) {
      delete b;
      return fail(es, "packed batch: atlas allocation failed");
    }
  }
  b->hs.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    eik_status st = create_impl(&b->hs[i], ndim, dims + (int64_t)i * ndim, h[i], hbar[i],
                                f + b->off[i], src_idx + so[i], src_U ? src_U + so[i] : nullptr,
                                so[i + 1] - so[i], opt, stream, b->exec, i);
    if (st != EIK_OK) {
      const std::string m = "instance " + std::to_string(i) + ": " + g_last_error;
      eik_destroy_batch(b);
      return fail(st, m);
    }
  }
  *out = b;
  return EIK_OK;
}

eik_status eik_batch_set_concurrency(eik_batch *b, int workers) {
  if (!b) return fail(EIK_ERR_ARG, "NULL batch");
  b->workers = workers;
  return EIK_OK;
}

eik_status eik_set_f_batch(eik_batch *b, const double *f) {
  if (!b || !f) return fail(EIK_ERR_ARG, "NULL batch or f");
  return run_pool(b, [&](int i) { return eik_set_f(b->hs[i], f + b->off[i]); });
}

eik_status eik_solve_batch(eik_batch *b, double *S_out, eik_stats *stats) {
  if (!b || !S_out) return fail(EIK_ERR_ARG, "NULL batch or S_out");
  if (!b->exec)
    return run_pool(b, [&](int i) {
      return eik_solve(b->hs[i], S_out + b->off[i], nullptr, stats ? stats + i : nullptr);
    });
  // packed: every instance's program on its own host thread; their inner
  // solves meet in the batch executor
  const eik_status bs = batch_exec_begin(b->exec, b->count);
  if (bs != EIK_OK) return fail(bs, "packed batch: " + batch_exec_error(b->exec));
  const int n = b->count;
  std::vector<eik_status> st(n, EIK_OK);
  std::vector<std::string> msg(n);
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::thread> th;
  th.reserve(n);
  for (int i = 0; i < n; ++i)
    th.emplace_back([&, i]() {
      cudaSetDevice(dev);
      st[i] = eik_solve(b->hs[i], S_out + b->off[i], nullptr, stats ? stats + i : nullptr);
      if (st[i] != EIK_OK) msg[i] = eik_last_error();
      batch_exec_leave(b->exec, i);
    });
  for (auto &t : th) t.join();
  const eik_status es = batch_exec_end(b->exec);
  for (int i = 0; i < n; ++i)
    if (st[i] != EIK_OK) {
      g_last_error = "instance " + std::to_string(i) + ": " + msg[i];
      return st[i];
    }
  if (es != EIK_OK) return fail(es, "packed batch: " + batch_exec_error(b->exec));
  return EIK_OK;
}

eik_status eik_batch_info(const eik_batch *b, int *packed, int *variant, int *tile_rows,
                          int *tuned, int64_t *passes, int64_t *node_passes, double *pass_ms) {
  if (!b) return fail(EIK_ERR_ARG, "NULL batch");
  int v = 0, ty = 0, how = 0;
  int64_t work = 0;
  double ms = 0.0;
  if (b->exec) {
    batch_exec_plan(b->exec, &v, &ty, &how);
    batch_exec_work(b->exec, &work, &ms);
  }
  if (packed) *packed = b->exec ? 1 : 0;
  if (variant) *variant = v;
  if (tile_rows) *tile_rows = ty;
  if (tuned) *tuned = how;
  if (passes) *passes = b->exec ? batch_exec_passes(b->exec) : 0;
  if (node_passes) *node_passes = work;
  if (pass_ms) *pass_ms = ms;
  return EIK_OK;
}

eik_status eik_grad_batch(eik_batch *b, const double *dLdS, double *dLdf, eik_stats *stats) {
  if (!b || !dLdS || !dLdf) return fail(EIK_ERR_ARG, "NULL batch, dLdS or dLdf");
  return run_pool(b, [&](int i) {
    return eik_grad(b->hs[i], dLdS + b->off[i], dLdf + b->off[i], stats ? stats + i : nullptr);
  });
}

eik_status eik_destroy_batch(eik_batch *b) {
  if (!b) return EIK_OK;
  for (eik_handle *h : b->hs)
    if (h) free_handle(h);
  batch_exec_destroy(b->exec);   // after the members, whose arrays it holds
  delete b;
  return EIK_OK;
}

}  // extern "C"
