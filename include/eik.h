/*
 * eik.h -- C ABI of the GB300 screened-Poisson eikonal solver.
 *
 * Method (Gurumoorthy et al., "A fast eikonal equation solver using the
 * Schroedinger wave equation", arXiv 1403.1937):
 *
 *   The eikonal equation |grad S| = f (Sec. 1, Eq. eikonalEq) with S = U_k at
 *   source nodes y_k (Sec. 3.2, after Eq. forcedPhiEquation) is replaced by the
 *   linear equation  -hbar^2 Lap(phi) + f^2 phi = 0  (Sec. 4, Eq. phiEquation)
 *   for phi = exp(-S/hbar), discretised with the 5-point (2D) / 7-point (3D)
 *   finite-difference Laplacian (Sec. 6, Eq. sparse-system), and S is
 *   recovered as S = -hbar log(phi) (Sec. 4, Eq. SfromPhi).
 *
 *   Discrete system solved here, for every non-source node i of a vertex-
 *   centred grid with spacing h (nodes on the outer faces), c = hbar^2/h^2:
 *
 *     sum_{j~i} c*omega_ij*(phi_i - phi_j) + w_i*f_i^2*phi_i = 0,
 *     phi_k = exp(-U_k/hbar) on the sources,
 *
 *   with zero flux on the outer faces in half-cell form (w_i = product over
 *   axes b of 1/2 if i lies on a b-face; omega_ij = the same product over the
 *   axes other than the edge's).  The matrix is a symmetric M-matrix; it is
 *   solved matrix-free by Jacobi-preconditioned conjugate gradients.
 *
 * Conventions (all entry points):
 *   - Grid arrays are dense, C order, x fastest: node (ix, iy[, iz]) is at
 *     flat index ix + nx*(iy + ny*iz).  Values are float64.
 *   - Pointer arguments may be device pointers or host pointers (pageable or
 *     pinned); the library tells them apart through unified addressing.  Device
 *     pointers must be on the device that is current at eik_create.
 *   - Inputs are copied at eik_create / eik_set_f; the caller may free them on
 *     return.  Output buffers are owned by the caller.
 *   - All device work runs on an internal stream ordered after, and before,
 *     the stream passed to eik_create: work already queued on that stream is
 *     seen, and work queued on it after a call returns sees the results.
 *     eik_solve and eik_grad return after the solve has finished (they must
 *     read the convergence status).
 *   - Errors are returned as eik_status; C++ exceptions never cross the ABI.
 *     eik_last_error() returns a thread-local description of the last error.
 *     After EIK_ERR_CUDA the handle should only be destroyed.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef EIK_H_
#define EIK_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EIK_ABI_VERSION 1

typedef struct eik_handle eik_handle;          /* opaque, library-owned */
typedef struct CUstream_st *eik_stream_t;      /* same type as cudaStream_t */

typedef enum {
  EIK_OK = 0,
  EIK_ERR_ARG = 1,            /* invalid argument (sizes, h, hbar, f, sources) */
  EIK_ERR_CUDA = 2,           /* CUDA runtime error; handle unusable */
  EIK_ERR_OOM = 3,            /* device allocation failed */
  EIK_ERR_NOT_CONVERGED = 4,  /* max_iter reached; outputs hold the iterate */
  EIK_ERR_BREAKDOWN = 5,      /* CG breakdown (p.Ap <= 0 or non-finite) */
  EIK_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired */
  EIK_ERR_STATE = 7           /* call out of order (e.g. eik_grad before a solve) */
} eik_status;

enum {
  EIK_PREC_FP64 = 0,          /* plain FP64 Jacobi-PCG */
  EIK_PREC_MIXED = 1          /* FP32 inner CG on the rescaled system + FP64
                                 iterative refinement (see eik_options) */
};

enum {
  EIK_PRECOND_JACOBI = 0,     /* Jacobi-PCG, one fused pass per iteration */
  EIK_PRECOND_MULTIGRID = 1   /* PCG with a V-cycle of relative-form
                                 aggregation multigrid (Sec. 6 names
                                 multigrid as the O(N) route for the sparse
                                 system): coarse basis functions are the
                                 estimated phi = exp(-S/hbar) on 2 x 2
                                 (x 2) boxes, so coarse corrections are relative
                                 ones and the far field converges with the
                                 near field */
};

enum {
  EIK_STOP_COMPONENTWISE = 0, /* max_i |r_i| / (a_ii phi_i) <= tol */
  EIK_STOP_NORMWISE = 1       /* ||r_hat||_2 / ||b_hat||_2 <= tol (Jacobi-scaled) */
};

enum {
  EIK_BOUNDARY_HALF_CELL = 0, /* second-order zero flux (default) */
  EIK_BOUNDARY_DROP_EDGE = 1  /* first-order zero flux: missing edges dropped */
};

typedef struct {
  int precision;      /* EIK_PREC_*; default EIK_PREC_FP64 */
  double tol;         /* stopping tolerance; default 1e-12 */
  int stop_norm;      /* EIK_STOP_*; default EIK_STOP_COMPONENTWISE */
  int max_iter;       /* CG iterations (total over refinement steps); default
                         200000 */
  int boundary;       /* EIK_BOUNDARY_*; default half cell */
  int tile_override;  /* mixed-mode inner-CG kernel variant (results agree
                         to rounding; for tuning and tests):
                         0 = library choice (variant 1);
                         2D (every warp an independent pipeline over tiles
                         of 128 columns): 1..4 = (row stages per warp,
                         warps per block) = (5, 5), (6, 4), (7, 4), (6, 7);
                         3D (a block marches 128 x TY rows through z):
                         1..4 = (TY, plane stages) = (12, 5), (8, 6),
                         (16, 4), (8, 8).  Other values return
                         EIK_ERR_ARG. */
  double inner_tol;   /* mixed mode: factor by which the first FP32 inner
                         solve of a refinement step reduces the residual
                         (scaled max norm); 0 = library choice (1e-1) */
  int max_outer;      /* mixed mode: refinement steps (per level-set band);
                         0 = library choice (30) */
  int band_bits;      /* mixed mode: when the coarse distance estimate puts
                         phi over more than 2 * band_bits powers of two, the
                         solve sweeps level-set bands of band_bits powers of
                         two (nearest first, an overlap of at least 32),
                         holding the rest as Dirichlet data; 0 = library
                         choice (bands of 40 when the range exceeds 96),
                         negative = never sweep */
  int test_flags;     /* test hook, 0 in normal use.  Bit 0 (mixed mode): in
                         the first inner-CG iteration one pipeline (a warp
                         in 2D, a block in 3D) never gets its first copy,
                         so its bounded wait (0.2 s) expires and the solve
                         returns EIK_ERR_TIMEOUT; exercises the timeout path
                         without any fault. */
  int batch_pack;     /* eik_create_batch of 2D mixed-precision instances:
                         0 (default) or 1 = packed: the instances share one
                         set of FP32 inner-CG arrays and every inner-CG pass
                         is one launch over a tile list spanning all of them
                         (see eik_create_batch); -1 = each instance solves on
                         its own stream.  Ignored for FP64 and 3D batches
                         (always per-instance). */
  int batch_tile_rows;/* packed batches: rows per tile of the packed pass
                         (1..1024); 0 = autotuned.  tile_override (1..4)
                         fixes the pass's 2D variant; 0 = autotuned. */
  int precond;        /* EIK_PRECOND_*: preconditioner of the FP32 inner
                         solve in mixed mode; default EIK_PRECOND_JACOBI.
                         EIK_PRECOND_MULTIGRID needs EIK_PREC_MIXED (else
                         EIK_ERR_ARG); its solves sweep level-set
                         bands only when phi spans more than 256 powers of
                         two (bands of 128; band_bits overrides both as for
                         Jacobi), and a batch of such instances solves per
                         instance (batch_pack is ignored).  2D and 3D. */
  int reserved[2];
} eik_options;

typedef struct {
  int outer_iters;    /* refinement steps (1 for plain FP64 without restart) */
  int inner_iters;    /* CG iterations in total */
  double res_cw;      /* final componentwise residual max_i |r_i|/(a_ii phi_i) */
  double res_nw;      /* final ||r||_2 / ||b||_2 of the unscaled system */
  double ms;          /* device time of the solve in milliseconds */
} eik_stats;

/* Fills *opt with the defaults listed above. */
void eik_default_options(eik_options *opt);

/*
 * Creates a solver for one grid (Sec. 6, Eq. sparse-system; Sec. 3.2 sources).
 *   ndim     2 or 3.
 *   dims     ndim extents (nx, ny[, nz]), each >= 2.
 *   h, hbar  grid spacing and the Schroedinger parameter hbar (> 0).
 *   f        N = prod(dims) forcing values, finite and > 0 (checked on the
 *            device; failure returns EIK_ERR_ARG).
 *   src_idx  nsrc flat node indices in [0, N) (nsrc >= 1).  Duplicates with
 *            equal values are merged; duplicates with different values, or
 *            indices out of range, return EIK_ERR_ARG.
 *   src_U    nsrc prescribed values of S at the sources, or NULL for zeros.
 *   opt      options, or NULL for eik_default_options().
 *   stream   CUDA stream whose work orders the library's work (may be NULL for
 *            the legacy default stream).
 * Allocates device memory proportional to N (about 7 float64 vectors; the
 * mixed mode adds one float64 and 7 float32 vectors).  Returns EIK_ERR_OOM if that
 * fails.
 */
eik_status eik_create(eik_handle **out, int ndim, const int64_t *dims,
                      double h, double hbar, const double *f,
                      const int64_t *src_idx, const double *src_U,
                      int64_t nsrc, const eik_options *opt,
                      eik_stream_t stream);

/* Replaces the forcing field (same validation as eik_create).  Sources, h
 * and hbar are kept.  Invalidates the state kept for eik_grad. */
eik_status eik_set_f(eik_handle *h, const double *f);

/*
 * Solves the system and writes S = -hbar log(phi) (Sec. 4, Eq. SfromPhi) to
 * S_out (N values; S = U exactly on the sources).  phi_out, if not NULL,
 * receives phi * exp(U_min/hbar) with U_min = min_k U_k (equal to phi when all
 * U_k = 0), which lies in (0, 1].  stats may be NULL.  On
 * EIK_ERR_NOT_CONVERGED the outputs hold the last iterate.
 */
eik_status eik_solve(eik_handle *h, double *S_out, double *phi_out,
                     eik_stats *stats);

/*
 * Adjoint gradient of a loss L(S) with respect to f, after a successful
 * eik_solve with the current f: dLdS (N values) in, dLdf (N values) out.
 * With A(f) phi = b and A_ii = w_i f_i^2 + ..., dL/df_i = -2 w_i f_i phi_i
 * lambda_i where A lambda = dL/dphi = -hbar (dL/dS)/phi; dLdf is 0 on the
 * sources.  Returns EIK_ERR_STATE if no solve result is held.
 */
eik_status eik_grad(eik_handle *h, const double *dLdS, double *dLdf,
                    eik_stats *stats);

/*
 * Batched solves: many independent instances (own grid, h, hbar, f and
 * sources; Sec. 6 system per instance) solved together, each with its own
 * refinement and convergence test; instances stop independently.  All
 * instances share ndim and the options.
 *
 * Packed (2D mixed precision, the default there; eik_options.batch_pack):
 * the FP32 inner-CG arrays of all instances are stacked in one pitched
 * array, and an inner solve runs for every instance that needs one at once:
 * each CG iteration is ONE kernel launch over a tile list spanning all those
 * instances, with per-instance recurrence scalars and stopping tests, and an
 * instance whose inner solve has ended leaves the list.  The iterations run
 * as a captured CUDA graph.  The tile shape (kernel variant, rows per tile)
 * is autotuned at the first solve: each candidate is timed on the batch's
 * own geometry and the fastest is cached in a JSON file, keyed by GPU name,
 * dimension, precision and size class (log2 of the node and instance
 * counts); the file is $EIK_TUNE_CACHE if set ("" or "off": no file), else
 * $XDG_CACHE_HOME/eik/tune.json or $HOME/.cache/eik/tune.json.  The FP64
 * refinement steps of each instance run on its own stream, one host thread
 * per instance.
 * Per-instance (FP64, 3D, or batch_pack = -1): each instance runs on its own
 * internal stream, and host worker threads drive them concurrently.
 *   count        number of instances (>= 1)
 *   dims         count*ndim extents, instance-major
 *   h, hbar      count values each
 *   f            sum_i N_i values, instances concatenated in order
 *   src_offsets  count+1 offsets into src_idx / src_U (src_offsets[0] = 0)
 *   src_idx      flat node indices within each instance's grid
 *   src_U        values or NULL for zeros
 * Outputs of eik_solve_batch / eik_grad_batch are concatenated the same way;
 * stats (nullable) receives count entries.  The first failing instance's
 * status is returned (all instances are still attempted).
 */
typedef struct eik_batch eik_batch;
eik_status eik_create_batch(eik_batch **out, int count, int ndim, const int64_t *dims,
                            const double *h, const double *hbar, const double *f,
                            const int64_t *src_offsets, const int64_t *src_idx,
                            const double *src_U, const eik_options *opt,
                            eik_stream_t stream);
eik_status eik_set_f_batch(eik_batch *b, const double *f);
eik_status eik_solve_batch(eik_batch *b, double *S_out, eik_stats *stats);
eik_status eik_grad_batch(eik_batch *b, const double *dLdS, double *dLdf, eik_stats *stats);
eik_status eik_destroy_batch(eik_batch *b);
/* Instances solved concurrently (host worker threads) in per-instance
 * batches; 0 = library choice.  No effect on packed batches. */
eik_status eik_batch_set_concurrency(eik_batch *b, int workers);
/*
 * How the batch runs: *packed = 1 for a packed batch, else 0; for a packed
 * batch the pass's 2D variant (1..4), its rows per tile, and how they were
 * chosen (*tuned: 0 fixed by the options, 1 measured by the autotuner, 2
 * read from the cache file; all 0 before the first solve); *passes, the
 * packed inner-CG launches that had work (the autotuner's included) since
 * creation; and, over the solves only, *node_passes, the sum over passes of
 * the grid nodes each covered (a pass moves 28 bytes per node), and
 * *pass_ms, the device time of the CUDA graphs that ran them (CUDA events).
 * Any output pointer may be NULL.
 */
eik_status eik_batch_info(const eik_batch *b, int *packed, int *variant, int *tile_rows,
                          int *tuned, int64_t *passes, int64_t *node_passes,
                          double *pass_ms);

/*
 * Componentwise residual of a given S without allocating any device memory
 * (the paper has no counterpart; this is a service for callers that cannot
 * allocate).  Code that runs inside a memory pool or arena that must not
 * grow, allocator hooks or plugins that may not call back into cudaMalloc,
 * and real-time loops that cannot afford cudaMalloc's implicit device
 * synchronisation can still check a solution with it.
 *
 * Computes max over non-source nodes of
 *   | (c / a_i) sum_{j~i} omega_ij exp((S_i - S_j)/hbar) - 1 |,  c = hbar^2/h^2,
 * which is |r_i| / (a_i phi_i) for phi = exp(-S/hbar) -- the quantity
 * eik_solve reports as eik_stats.res_cw -- and writes it to *res_max.
 *   ndim, dims, h, hbar, boundary   as for eik_create
 *   f, S        N = prod(dims) device values (forcing field, solution)
 *   src_idx     nsrc device indices of the source nodes (skipped); an index
 *               outside the grid makes the result NaN
 *   res_max     one device double (written asynchronously)
 *   stream      stream the work is queued on; the call does not synchronise
 * All pointers must be device pointers.  Returns EIK_ERR_ARG for invalid
 * arguments, including grids of more than 1048576 (2^20) nodes, which do not
 * fit the fixed working memory; EIK_ERR_CUDA on a CUDA error.
 *
 * Working memory: one file-scope device array of about 8.4 MB, held by every
 * GPU that loads the library until the process exits.  Nothing is allocated
 * or freed.  The first call on each device looks up that array's device
 * address (once per device, with the device current); make that first call
 * before any stream capture.  All calls share the array, so calls whose work
 * overlaps on the GPU (different streams, or host threads without ordering)
 * race and may return wrong results; order them on one stream.
 */
eik_status eik_residual_noalloc(int ndim, const int64_t *dims, double h, double hbar,
                                const double *f, const double *S, const int64_t *src_idx,
                                int64_t nsrc, int boundary, double *res_max,
                                eik_stream_t stream);

/*
 * Nodal gradient of S for path planning (path-planning section; the
 * gradient descent on S that Eq. PathPlanning-backTrackOnS integrates).
 * Component a of grad S at node i is (S[i+e_a] - S[i-e_a]) / (2h) inside the
 * grid and the one-sided difference on the two faces of axis a.
 *   dims   host array of ndim sizes (x first), each >= 2.
 *   S      device, N doubles (C order, x fastest), e.g. from eik_solve.
 *   gradS  device, ndim * N doubles, caller-owned; component a (x, y, z)
 *          at gradS + a * N.
 * Queued on `stream` and not awaited.  EIK_ERR_ARG for bad sizes, h <= 0 or
 * null pointers; EIK_ERR_CUDA if the launch fails.
 */
eik_status eik_grad_S(int ndim, const int64_t *dims, double h, const double *S, double *gradS,
                      eik_stream_t stream);

/*
 * Backtracking of optimal paths (path-planning section,
 * Eq. PathPlanning-backTrackOnS): from each start point, explicit Euler
 * steps of arc length `step` along -g/|g|, g the multilinear interpolation of
 * gradS in the cell holding the point; points are clamped to the grid box
 * [0, (n_a - 1) h].  Before every step a path stops if it lies within `eps`
 * of a source node (status 0) or if |g| is zero or not finite (status 2);
 * after max_steps steps it stops with status 1 (0 if then within eps).
 *   gradS    device, from eik_grad_S.
 *   starts   device, npaths * ndim doubles, world coordinates x = i h.
 *   src_idx  device, nsrc flat node indices of the sources.
 *   paths    device, npaths * (max_steps + 1) * ndim doubles, caller-owned:
 *            point k of path p at paths + (p * (max_steps + 1) + k) * ndim;
 *            points after the last are NaN.
 *   lengths  device, npaths ints: steps taken (points = lengths + 1).
 *   status   device, npaths ints (0 reached, 1 step limit, 2 flat gradient).
 * One GPU thread per path, queued on `stream` and not awaited.  EIK_ERR_ARG
 * for bad sizes, step <= 0, eps < 0, max_steps < 0 or null pointers.
 */
eik_status eik_backtrack(int ndim, const int64_t *dims, double h, const double *gradS,
                         const double *starts, int64_t npaths, double step, int max_steps,
                         const int64_t *src_idx, int64_t nsrc, double eps, double *paths,
                         int *lengths, int *status, eik_stream_t stream);

/*
 * Shape-from-shading forcing (shape-from-shading section, Eq.
 * SfS-forcingFunc): for a Lambertian image under vertical light,
 * P = 1/sqrt(|grad S|^2 + 1), the height field S solves the eikonal equation
 * with f = sqrt(1/P^2 - 1); seed eik_create with known heights as source
 * values U.  f is raised to f_min where the formula gives less (flat image
 * regions give 0, which eik_create rejects); P outside (0, 1] or not finite
 * yields NaN there (also rejected by eik_create).
 *   P, f   device, n doubles each (f caller-owned).
 * Queued on `stream`, not awaited.  EIK_ERR_ARG for n < 0, f_min < 0 or null
 * pointers with n > 0.
 */
eik_status eik_sfs_forcing(const double *P, int64_t n, double f_min, double *f,
                           eik_stream_t stream);

/*
 * FFT perturbation series (Sec. 5, Table 1) on a 2D grid: with a constant
 * f~, phi = phi_0 - phi_1 + ... + (-1)^T phi_T where phi_0 = G~ * delta_kron
 * (G~(x) = exp(-f~|x|/hbar), sources as Kronecker deltas: Sec. 3.2,
 * Eq. forcedPhiEquation) and phi_i = h^2 G * [(f^2 - f~^2) phi_{i-1}]
 * (Eqs. phiRecRelation, phi_i_Solution; G = K_0(f~|x|/hbar)/(2 pi hbar^2),
 * Eq. GreensFunction2D, averaged over the grid cell at the origin); then
 * S = -hbar log phi (Eq. SfromPhi).  Convolutions are linear over the grid,
 * by FP64 mixed-radix transforms of arrays zero-padded to the smallest
 * 2^a 3^b 5^c >= 2n - 1 per axis.  This is the paper's first solver, kept as
 * a second workload: the finite-difference solve above is the main path.
 *   dims        (nx, ny), each 2 .. 3600; node (x, y) is f[x + nx y].
 *   h, hbar     > 0.
 *   f           nx ny values, > 0 (host or device).
 *   src_idx     nsrc >= 1 flat node indices (host or device).
 *   terms       T, 0 .. 64.
 *   f_tilde     f~; 0 = sqrt((f_min^2 + f_max^2)/2) (Eq. fTildeValue), which
 *               makes the series converge (Sec. 5.1).
 *   S_out       nx ny values (host or device, caller-owned); NaN where the
 *               truncated series or the transforms' rounding (absolute errors
 *               near 1e-16 max phi, the paper's reason for MPFR) leave
 *               phi <= 0.
 *   phi_out     nx ny values or NULL.
 *   f_tilde_out the f~ used, or NULL.
 * Allocates its work arrays (about 48 bytes per padded node), runs on
 * `stream` and returns when the outputs are written.  EIK_ERR_ARG for bad
 * sizes, pointers, values or f not finite and positive; EIK_ERR_OOM.
 */
eik_status eik_fft_series(const int64_t *dims, double h, double hbar, const double *f,
                          const int64_t *src_idx, int64_t nsrc, int terms, double f_tilde,
                          double *S_out, double *phi_out, double *f_tilde_out,
                          eik_stream_t stream);

/* Per-kernel counters of a handle (diagnostics; the paper has no
 * counterpart).  launches counts every kernel launch the handle issued since
 * creation or the last eik_reset_kernel_stats (kernels inside captured graphs
 * count once per graph launch).  total_ms is the summed device time of those
 * launches measured with CUDA events on the library's stream; it is filled
 * only for launches made while profiling is enabled (eik_set_profiling),
 * which replaces graph launches by individually timed launches. */
typedef struct {
  char name[32];
  int64_t launches;
  int64_t timed_launches;
  double total_ms;
} eik_kernel_stat;

eik_status eik_set_profiling(eik_handle *h, int enable);
/* Writes up to max entries to out and the number of kernels to *count. */
eik_status eik_kernel_stats(eik_handle *h, eik_kernel_stat *out, int max, int *count);
eik_status eik_reset_kernel_stats(eik_handle *h);

/* Releases the handle and its device memory.  NULL is accepted. */
eik_status eik_destroy(eik_handle *h);

/* Thread-local description of the last error (never NULL). */
const char *eik_last_error(void);

/* Library version (EIK_ABI_VERSION) and the CUDA architecture compiled for
 * (e.g. 1030 for sm_103a). */
int eik_abi_version(void);
int eik_cuda_arch(void);

#ifdef __cplusplus
}
#endif

#endif /* EIK_H_ */
