// FP32 inner conjugate gradients of the mixed-precision solve (internal).
//
// The inner solve works on the correction equation of one refinement step in
// the Jacobi-scaled operator of eik_internal.cuh, with every vector stored
// in "kx units": the value of node i times 2^kx_i, kx a static power-of-two
// exponent per cell of B^d nodes taken from a distance estimate.  In these
// units the operator reads
//   (A v)_i = v_i - sig_i sum_{j~i} omega_ij sig_j v_j 2^(kx_i - kx_j),
// and the inner products of plain CG (unit diagonal, unweighted) become
// weighted sums  <u, v> = sum_i u_i v_i 2^(-2 kx_i).  Because phi decays
// like exp(-S/hbar) and kx follows S/(hbar ln 2), stored values stay within a
// few dozen powers of two of each other, which FP32 holds.
//
// The iteration is the single-reduction ("Chronopoulos-Gear") form of CG:
// one pass over the grid per iteration computes
//   p = r + beta p,  s = A p,  d += alpha p,  r -= alpha s,  w = A r,
// and the inner products <r, r>, <w, r> and <p, s>, from which the last block
// forms the next beta = <r,r>_new / <r,r>_old and
//   alpha = <r,r>_new / (<w,r>_new - beta^2 <p, s>),
// the denominator being <p', A p'> of the next direction.  (The textbook
// form carries <p, A p> as <r,r>_old / alpha_old instead; summing it in the
// pass keeps the FP32 recurrence from drifting on badly conditioned
// operators.)
// A pass recomputes s = A p instead of storing it, so it reads r and p with a
// two-node halo, sigma, d (and, in checking passes, the FP32 copy of the
// iterate) and writes r, p and d: 7 words per node.
//
// r and p share one global power-of-two "frame": stored = value * 2^-F.  Each
// pass writes them in frame F + dF, dF chosen from the previous pass's
// maximum, so they stay near 1 however far the residual falls.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "eik_internal.cuh"

namespace eik {

// Cells of the static exponents kx: cubes of B = 2^lgB nodes.
struct CellGrid {
  int B, lgB;        // cell edge in nodes (power of two >= 16) and its log2
  int cx, cy, cz;    // cells per axis
  int ncell;
};

// Device-resident control block of the mixed solve.  The FP64 residual
// kernel fills the first group and starts an inner solve; the inner passes
// advance the recurrence (only the last block of a pass writes).
struct MixCtl {
  // --- FP64 relative-form residual of the current iterate
  double rho_m;      // <rbar, rbar>_W = rho_m * 2^rho_s (rbar in kx units)
  int rho_s;
  double cw;         // max_i |r_i| / (a_i phi_i) over the active unknowns
  double r_inf;      // max_i |rbar_i| (kx units)
  double x_inf;      // max_i |xbar_i| (kx units)
  int band_lo, band_hi;   // level-set band: unknowns with band_lo <= kx < band_hi
  // --- inner CG recurrence (absolute values)
  double gam_m;      // <r, r>_W = gam_m * 2^gam_s of the current residual
  int gam_s;
  double alpha;      // step of the next pass
  double beta;       // direction update of the next pass
  int F;             // frame of the stored r, p
  int dF;            // the next pass writes r, p in frame F + dF
  int fd;            // the next pass sums dot terms as x * 2^(-2 kx - fd)
  int mode;          // 0: stop when max|r| (kx units) <= thresh;
                     // 1: stop when |r_i| <= theta |xref_i + d_i| for all i
  float thresh, theta;
  int iter;          // inner passes done in this solve
  int max_iter;
  int total_iter;
  int done;          // 1: further passes return at once
  int status;        // eik_status of the inner solve (EIK_OK also after a stall)
  int stalled;       // the recurrence lost positivity: the solve ended early
  int fault;         // a bounded device-side wait expired
  int withhold;      // test hook: one warp never gets its first copy
  // packed batches (the single-grid passes ignore these)
  int first;         // the next pass is the inner solve's first (w = A r only)
  int flip;          // the instance reads buffer set (launch set ^ flip)
  int seq;           // request number, echoed in the host record when done
  unsigned int counter[4];
};

// Host-side launch plan of the inner passes for one grid.
struct Cg32Plan {
  int ndim = 0;
  int variant = 0;       // 0 library choice; see cg32_plan
  // 2D: warp tiles of 128 columns x ty rows
  int tiles_x = 0, ty = 0, ntiles = 0, nblk = 0, wpb = 0, ns = 0;
  size_t smem = 0;
  // 3D: block tiles of 128 columns x ty rows x zc planes
  int tiles_y = 0, zc = 0;
  CUtensorMap tm_r[2], tm_p[2], tm_s;
};

struct Cg32Buffers {
  float *r[2], *p[2];    // two buffer sets: a pass reads one and writes the other
  float *s32;            // sigma (0 on sources and on nodes outside the band)
  float *d;              // correction (kx units), updated in place
  float *xref;           // FP32 copy of the iterate (kx units), checking passes
  const int *kx;         // cell exponents
  MixCtl *st;
  double *part;          // per-block partials
  int nblk_part;
  int px;                // row pitch (elements) of every FP32 array
};

// Picks the launch geometry and encodes the tensor maps.  Returns false (and
// leaves a message in *why) when the device cannot run the kernels.
bool cg32_plan(Cg32Plan *pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
               int num_sms, int variant, const char **why);
// Blocks whose partials the passes write (upper bound for part sizing).
int cg32_max_blocks(int ndim, int num_sms);
// First pass of an inner solve: w = A r on buffer set `set`, <r,r>, <w,r>,
// alpha, the frame; nothing is written but the control block.
void cg32_init(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
               int set, cudaStream_t s);
// One inner iteration: reads buffer set `set`, writes set 1 - set.
void cg32_iter(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
               int set, cudaStream_t s);

// ------------------------------------------------- packed 2D batches
// Many 2D instances share one set of FP32 arrays (the "atlas"): instance i
// occupies rows row0 .. row0 + ny - 1 of a pitched array of P columns (P >= every
// nx, a multiple of 4), with at least two zero rows between instances and zero
// columns right of each instance.  So a tile's two-row halo and its columns
// past nx read zeros, as they would from a single grid's out-of-bounds fill,
// and one set of tensor maps serves every instance.
struct BInst {
  int nx, ny;
  int wx;            // columns written per row: nx rounded up to 4
  int row0;          // atlas row of y = 0
  int tiles_x;       // 128-column tiles
  int boundary;      // EIK_BOUNDARY_*
  CellGrid cg;
  const int *kx;     // the instance's cell exponents
};

// Pass-level state of a packed batch.  act[0 .. m) lists the instances still
// iterating and pre[0 .. m] the prefix sums of their tile counts: list
// position t belongs to act[a] with pre[a] <= t < pre[a + 1].
struct BatchCtl {
  int m;               // active instances
  int ntiles;          // pre[m]
  int dirty;           // an instance finished during this pass
  int fault;           // a bounded device-side wait expired
  unsigned warps_done; // ticket of the pass's last warp
  int passes;          // passes that had work, since the list was set
  int req_head;        // requests admitted so far (see BatchRing)
  int pad;
  long long nodes;     // nodes of the instances in the list
  long long work;      // sum over passes of the nodes they covered
};

// Requests to join the tile list, in mapped host memory: the host writes
// ids[tail % cap] and then advances tail; the last warp of every pass admits
// ids[head .. tail) for the next pass.
struct BatchRing {
  volatile int tail;
  int pad[31];
  volatile int ids[1];   // cap entries (allocated with the ring)
};

// What the host learns when an instance's inner solve ends, in mapped host
// memory: the finisher writes the fields, then done_seq = the request number.
struct BatchDone {
  double alpha, beta;
  int iter, status, stalled, F;
  volatile int done_seq;
  int pad[7];
};

struct Cg32BatchBuffers {
  float *r[2], *p[2], *s32, *d, *xref;   // atlas arrays, pitch P
  int P, H;                              // pitch and rows of the atlas
  const BInst *bi;
  MixCtl *st;            // one control block per instance
  int *act, *pre;        // active list (device)
  unsigned *cnt;         // per-instance tile tickets of the current pass
  int *alive;            // 1 while an instance is in the list and iterating
  BatchCtl *bc;
  double *part;          // 6 x part_cap per-tile partials
  int part_cap;
  BatchRing *ring;       // device view of the mapped request ring
  int ring_cap;
  BatchDone *done;       // device view of the mapped completion records
};

struct Cg32BatchPlan {
  int variant = 0, ty = 0, nblk = 0, wpb = 0, ns = 0;
  size_t smem = 0;
  CUtensorMap tm_r[2], tm_p[2], tm_s;
};

// Launch geometry of the packed passes (variant as cg32_plan's 2D table, ty
// rows per tile) and the atlas tensor maps.
bool cg32_batch_plan(Cg32BatchPlan *pl, const Cg32BatchBuffers &b, int num_sms, int variant,
                     int ty, const char **why);
// One pass over every tile of the active instances (launch buffer set `set`;
// an instance whose MixCtl.first is set makes it its inner solve's first
// pass), then the admission of waiting requests for the next pass.
void cg32_batch_pass(const Cg32BatchPlan &pl, const Cg32BatchBuffers &b, int set,
                     cudaStream_t s);

}  // namespace eik
