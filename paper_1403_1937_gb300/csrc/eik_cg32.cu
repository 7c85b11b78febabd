// FP32 single-reduction inner CG passes for sm_103a (see eik_cg32.h for the
// arithmetic).  2D: every warp is an independent pipeline over its own tiles
// of 128 columns x ty rows; 3D: a block marches a tile of 128 columns x ty
// rows through z, one warp per row.
#include <math.h>

#include <algorithm>
#include <climits>
#include <cstdio>

#include "eik_cg32.h"
#include "eik_tma.cuh"

namespace eik {
namespace {

constexpr int kW = 128;        // output columns of a tile (4 per lane)
constexpr int kWin = kW + 8;   // staged columns of a row: x0 - 4 .. x0 + 131
// 2D: shared-memory slot of one staged row, rounded up to 128 bytes (every
// TMA destination in shared memory is 128-byte aligned)
constexpr int kSlot = 160;
static_assert(kSlot >= kWin && (kSlot * 4) % 128 == 0, "row slot");
// 3D: a staged plane is (TY + 4) rows of 136 floats, 544 (TY + 4) bytes, a
// multiple of 128 when TY + 4 is a multiple of 4

// 2^n as a float with n clamped to the normal range.
__device__ __forceinline__ float p2f(int n) {
  n = min(max(n, -126), 127);
  return __int_as_float((n + 127) << 23);
}

// Value m * 2^s with |m| in [0.5, 1) (m = 0 for zero).
struct Acc {
  double m;
  int s;
};
__device__ __forceinline__ Acc acc_of(double v, int s) {
  if (v == 0.0 || !isfinite(v)) return Acc{v, 0};
  int e;
  const double m = frexp(v, &e);
  return Acc{m, s + e};
}
__device__ __forceinline__ double acc_ratio(const Acc &a, const Acc &b) {
  return (a.m / b.m) * scalbn(1.0, a.s - b.s);
}

// --------------------------------------------------------------- pass tail
__device__ void cg_update(MixCtl *st, double G, double D, double R, double P, double Bd,
                          double PS, bool INIT);

// Per-block partials: <r,r>, <w,r> and <p,Ap> (units of 2^(2F + fd)), the
// largest |r| and |p| (frame units), and the componentwise-test flag.  The
// last block forms the next alpha, beta, frame and the stopping decision.
template <bool INIT>
__device__ void cg_tail(float gam, float dlt, float rmax, float pmax, int bad, float pap,
                        bool fault, MixCtl *st, double *part, int nblk_part) {
  __shared__ int flag;
  for (int o = 16; o > 0; o >>= 1) {
    gam += __shfl_down_sync(0xffffffffu, gam, o);
    dlt += __shfl_down_sync(0xffffffffu, dlt, o);
    pap += __shfl_down_sync(0xffffffffu, pap, o);
    rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
    pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  __shared__ float wg[32], wd[32], wr[32], wp[32], wq[32];
  __shared__ int wb[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (lane == 0) {
    wg[w] = gam;
    wd[w] = dlt;
    wr[w] = rmax;
    wp[w] = pmax;
    wb[w] = bad;
    wq[w] = pap;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double G = 0.0, D = 0.0, Q = 0.0;
    float R = 0.f, P = 0.f;
    int Bd = 0;
    for (int k = 0; k < nwarp; ++k) {
      G += (double)wg[k];
      D += (double)wd[k];
      Q += (double)wq[k];
      R = fmaxf(R, wr[k]);
      P = fmaxf(P, wp[k]);
      Bd |= wb[k];
    }
    part[0 * nblk_part + blockIdx.x] = G;
    part[1 * nblk_part + blockIdx.x] = D;
    part[2 * nblk_part + blockIdx.x] = (double)R;
    part[3 * nblk_part + blockIdx.x] = (double)P;
    part[4 * nblk_part + blockIdx.x] = (double)Bd;
    part[5 * nblk_part + blockIdx.x] = Q;
    if (fault) atomicExch(&st->fault, 1);
  }
  if (!last_block(&st->counter[1], &flag)) return;
  // the six partial arrays in one round: every load is issued before any is
  // used, then one shuffle tree and one shared-memory step per quantity
  double G = 0.0, D = 0.0, R = 0.0, P = 0.0, Bd = 0.0, Q = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double g0 = __ldcg(part + b), d0 = __ldcg(part + nblk_part + b);
    const double r0 = __ldcg(part + 2 * nblk_part + b), p0 = __ldcg(part + 3 * nblk_part + b);
    const double b0 = __ldcg(part + 4 * nblk_part + b), q0 = __ldcg(part + 5 * nblk_part + b);
    G += g0;
    D += d0;
    Q += q0;
    R = fmax(R, r0);
    P = fmax(P, p0);
    Bd = fmax(Bd, b0);
  }
  for (int o = 16; o > 0; o >>= 1) {
    G += __shfl_down_sync(0xffffffffu, G, o);
    D += __shfl_down_sync(0xffffffffu, D, o);
    Q += __shfl_down_sync(0xffffffffu, Q, o);
    R = fmax(R, __shfl_down_sync(0xffffffffu, R, o));
    P = fmax(P, __shfl_down_sync(0xffffffffu, P, o));
    Bd = fmax(Bd, __shfl_down_sync(0xffffffffu, Bd, o));
  }
  __shared__ double tg[32], td[32], tr[32], tp[32], tb[32], tq[32];
  if (lane == 0) {
    tg[w] = G;
    td[w] = D;
    tr[w] = R;
    tp[w] = P;
    tb[w] = Bd;
    tq[w] = Q;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  G = 0.0;
  D = 0.0;
  Q = 0.0;
  R = 0.0;
  P = 0.0;
  Bd = 0.0;
  for (int k = 0; k < nwarp; ++k) {   // fixed order: deterministic
    G += tg[k];
    D += td[k];
    Q += tq[k];
    R = fmax(R, tr[k]);
    P = fmax(P, tp[k]);
    Bd = fmax(Bd, tb[k]);
  }
  st->counter[1] = 0u;
  cg_update(st, G, D, R, P, Bd, Q, INIT);
}

// The recurrence step of one inner solve from the pass's totals: G = <r,r>,
// D = <w,r>, PS = <p,Ap> of this pass's direction (units 2^(2F + fd)),
// R = max|r|, P = max|p| (frame units), Bd the componentwise-test flag.
// INIT: the solve's first pass (w = A r).  Run by one thread.
__device__ void cg_update(MixCtl *st, double G, double D, double R, double P, double Bd,
                          double PS, bool INIT) {
  const int F = st->F, dF = st->dF, fd = st->fd;
  const Acc gam_new = acc_of(G, 2 * F + fd);
  const Acc dlt_new = acc_of(D, 2 * F + fd);
  const Acc gam_old{st->gam_m, st->gam_s};
  if (!INIT) {
    st->iter += 1;
    st->total_iter += 1;
  }
  if (st->fault) {
    st->done = 1;
    st->status = EIK_ERR_TIMEOUT;
    return;
  }
  if (!isfinite(G) || !isfinite(D) || !isfinite(R) || !isfinite(P) || !isfinite(PS)) {
    st->done = 1;
    st->status = EIK_ERR_BREAKDOWN;
    return;
  }
  // stopping tests on the new residual (frame F units, before this pass's
  // rescaling)
  bool conv = (G == 0.0);
  if (!INIT) {
    if (st->mode == 0)
      conv = conv || scalbn(R, F) <= (double)st->thresh;
    else if ((st->iter & 3) == 0)   // this pass was a checking pass
      conv = conv || Bd == 0.0;
  }
  if (conv) {
    st->done = 1;
    st->status = EIK_OK;
    return;
  }
  double alpha_new;
  if (INIT) {
    alpha_new = (D > 0.0) ? 1.0 / acc_ratio(dlt_new, gam_new) : -1.0;
    st->beta = 0.0;
  } else {
    const double beta_new = acc_ratio(gam_new, gam_old);
    // <p', A p'> of the next direction p' = r + beta p is <w, r> - beta^2
    // <p, A p> (CG's orthogonality), with <p, A p> of this pass's direction
    // summed in the pass itself: the single-reduction recurrence would carry
    // it as <r,r>_old / alpha_old instead, and in FP32 that chain loses the
    // positive definiteness on badly conditioned operators
    const double pap = D - beta_new * beta_new * PS;
    alpha_new = (PS > 0.0 && pap > 0.0 && isfinite(pap)) ? G / pap : -1.0;
    st->beta = beta_new;
  }
  if (!(alpha_new > 0.0) || !isfinite(alpha_new)) {
    // the recurrence lost positivity in FP32: end this inner solve (its
    // correction so far is kept; the refinement step restarts from the
    // true residual)
    st->done = 1;
    st->stalled = 1;
    st->status = INIT ? EIK_ERR_BREAKDOWN : EIK_OK;
    return;
  }
  st->alpha = alpha_new;
  st->gam_m = gam_new.m;
  st->gam_s = gam_new.s;
  // frames: values written by this pass are in F + dF; the next pass writes
  // in F + dF + dF', dF' bringing its largest stored value near 1
  const int Fn = INIT ? F : F + dF;
  const double M = INIT ? R : fmax(R, P) * scalbn(1.0, -dF);
  st->F = Fn;
  st->dF = (M > 0.0) ? ilogb(M) : 0;
  if (INIT) st->F = F;   // init writes nothing: the stored r keeps frame F
  // dot frame of the next pass: its partials then come out near 1
  st->fd = gam_new.s - 2 * st->F;
  if (!INIT && st->iter >= st->max_iter) {
    st->done = 1;
    st->status = EIK_ERR_NOT_CONVERGED;
  }
}

// ------------------------------------------------------------------ 2D pass
// One warp owns tiles of 128 columns x TY rows and runs them as its own
// pipeline: the tile's rows (with a two-row halo) arrive by one TMA row copy
// per array (r, p, sigma: 136 columns from x0 - 4) into a ring of NS stages,
// and d (and, in checking passes, the FP32 iterate) of the tile's rows come
// two steps ahead by plain vector loads.  At step j (input row y_j):
//   A, row y_j:      p = r + beta p, written back to the stage
//   B, row y_{j-1}:  u = sig p of rows y_{j-2} .. y_j, s = A p,
//                    r_new = r - alpha s, un = sig r_new into a four-row ring
//   C, row y_{j-2}:  w = A r_new, the dots, d += alpha p, stores
// Lane l computes columns x0 + 4l .. x0 + 4l + 3, and lanes 0 and 31 also the
// halo columns (A: x0 - 2, x0 - 1 / x0 + 128, x0 + 129; B: x0 - 1 / x0 + 128)
// that neighbouring columns read.  A stage is free once C has used it, two
// steps after A, so NS - 3 rows are in flight ahead of the one consumed.  Odd
// tile rows march upwards, so the halo rows that two neighbouring tiles share
// are read at about the same time.

// Cell factors of one row for one lane: 2^(kx_i - kx_j) for the neighbours j
// of the lane's columns i (and of its halo column), and the dot weight.
struct Fac2 {
  int cr;          // cell row of the row (INT_MIN: not computed)
  int brd;         // the row is next to another cell row
  float fL, fR;    // left neighbour of the first column, right of the last
  float fP, fN;    // rows y - dir and y + dir
  float fxh;       // halo column: its neighbour inside the tile
  float fPh, fNh;  // halo column: rows y - dir and y + dir
  float W;         // 2^(-2 kx - fd)
};

// Cell exponents of one tile's footprint, copied to shared memory at the
// start of the tile (kTab entries per warp); tiles whose footprint does not
// fit read kx from global memory instead.
constexpr int kTab = 64;
struct KTab {
  const int *t;    // shared table, or nullptr: use kx in global memory
  int cr0, cc0;    // first cell row and column of the table
  int ncol;
};

__device__ __forceinline__ int ktab_at(const KTab &k, const int *__restrict__ kx,
                                       const CellGrid &cg, int cr, int cc) {
  return k.t ? k.t[(cr - k.cr0) * k.ncol + (cc - k.cc0)] : __ldg(kx + cr * cg.cx + cc);
}

__device__ __forceinline__ void fac2_update(Fac2 &f, int y, int dir, const Grid &g,
                                            const CellGrid &cg, const int *__restrict__ kx,
                                            const KTab &kt, int cxo, int cxl, int cxr, int cxh,
                                            int fd) {
  const int cr = min(max(y, 0), g.ny - 1) >> cg.lgB;
  const int cp = min(max(y - dir, 0), g.ny - 1) >> cg.lgB;
  const int cn = min(max(y + dir, 0), g.ny - 1) >> cg.lgB;
  const int brd = (cp != cr) || (cn != cr);
  if (cr == f.cr && !brd && !f.brd) return;   // same cell row, interior rows
  const int kc = ktab_at(kt, kx, cg, cr, cxo), kh = ktab_at(kt, kx, cg, cr, cxh);
  f.fL = p2f(kc - ktab_at(kt, kx, cg, cr, cxl));
  f.fR = p2f(kc - ktab_at(kt, kx, cg, cr, cxr));
  f.fxh = p2f(kh - kc);
  if (brd) {
    f.fP = p2f(kc - ktab_at(kt, kx, cg, cp, cxo));
    f.fN = p2f(kc - ktab_at(kt, kx, cg, cn, cxo));
    f.fPh = p2f(kh - ktab_at(kt, kx, cg, cp, cxh));
    f.fNh = p2f(kh - ktab_at(kt, kx, cg, cn, cxh));
  } else {
    f.fP = f.fN = f.fPh = f.fNh = 1.f;
  }
  f.W = p2f(-2 * kc - fd);
  f.cr = cr;
  f.brd = brd;
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ float4 mul4(const float4 &a, const float4 &b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}

template <bool INIT, int NS, int WPB>
__global__ void __launch_bounds__(32 * WPB, WPB >= 7 ? 2 : 3)
k_cg2d(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_p,
       const __grid_constant__ CUtensorMap tm_s, Grid g, CellGrid cg,
       const int *__restrict__ kx, int tiles_x, int TY, int ntiles,
       float *__restrict__ r_out, float *__restrict__ p_out, float *__restrict__ d,
       const float *__restrict__ xref, MixCtl *st, double *part, int nblk_part, int px) {
  // stage: [r | p | sig] (kSlot floats each); ring row: [rn | un] (kWin each)
  constexpr int OR = 0, OP = kSlot, OS = 2 * kSlot;
  constexpr int STAGE = 3 * kSlot;
  constexpr int RING = 2 * kWin;
  constexpr int WARP_FLOATS = NS * STAGE + 4 * RING;
  static_assert((STAGE * 4) % 128 == 0 && (WARP_FLOATS * 4) % 128 == 0, "stage alignment");
  extern __shared__ __align__(128) unsigned char cg2_raw[];
  __shared__ __align__(8) uint64_t bars[WPB * NS];
  __shared__ int ktabs[WPB * kTab];
  if (st->done) return;
  float *cg2_smem = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(cg2_raw) + 127) & ~uintptr_t(127));
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * WPB + wib, nw = gridDim.x * WPB;
  const float beta = INIT ? 0.f : (float)st->beta;
  const float alpha = INIT ? 0.f : (float)st->alpha;
  const int F = st->F, dF = st->dF, fd = st->fd;
  const float gwr = p2f(-dF);
  const float alphaF = INIT ? 0.f : (float)scalbn(st->alpha, F);
  const bool check = !INIT && st->mode != 0 && ((st->iter & 3) == 3);
  const float thetaF = (float)scalbn((double)st->theta, -F);
  const bool half = g.boundary == EIK_BOUNDARY_HALF_CELL;
  const int withhold = (!INIT && st->withhold && st->iter == 0 && gw == 0) ? 1 : 0;
  const int steps = TY + 4;
  const int my_tiles = (gw < ntiles) ? (ntiles - 1 - gw) / nw + 1 : 0;
  const int nq = my_tiles * steps;
  float *sb = cg2_smem + (size_t)wib * WARP_FLOATS;
  float *ring = sb + NS * STAGE;
  uint64_t *bar = bars + wib * NS;

  // lane 0: the next row to copy, tracked incrementally (tile, step, origin)
  int nx_q = 0, nx_j = 0, nx_x0 = 0, nx_y0 = 0, nx_dir = 1, nx_t = gw;
  auto set_tile = [&](int t) {
    nx_t = t;
    const int cyk = t / tiles_x;
    nx_x0 = (t - cyk * tiles_x) * kW;
    nx_y0 = cyk * TY;
    nx_dir = (cyk & 1) ? -1 : 1;
  };
  auto issue_next = [&]() {
    const int y = (nx_dir > 0) ? nx_y0 - 2 + nx_j : nx_y0 + TY + 1 - nx_j;
    float *dst = sb + (nx_q % NS) * STAGE;
    uint64_t *b = bar + (nx_q % NS);
    if (!(nx_q == 0 && withhold)) {
      mbar_expect_tx(b, (INIT ? 2u : 3u) * kWin * 4u);
      tma_load_2d(dst + OR, &tm_r, nx_x0 - 4, y, b);
      if (!INIT) tma_load_2d(dst + OP, &tm_p, nx_x0 - 4, y, b);
      tma_load_2d(dst + OS, &tm_s, nx_x0 - 4, y, b);
    }
    ++nx_q;
    if (++nx_j == steps) {
      nx_j = 0;
      set_tile(nx_t + nw);
    }
  };
  if (lane == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    mbar_init_fence();
    set_tile(gw);
    while (nx_q < NS && nx_q < nq) issue_next();
  }
  __syncwarp();

  float gam = 0.f, dlt = 0.f, rmax = 0.f, pmax = 0.f, pap = 0.f;
  int bad = 0;
  bool fault = false;
  int q = 0;
  const int c = 4 + 4 * lane;              // staged column of the lane's first node
  const bool l0 = lane == 0, l31 = lane == 31;
  const int hA = l31 ? kW + 4 : 2;         // A's halo pair x0-2, x0-1 / x0+128, x0+129
  const int hB = l31 ? kW + 4 : 3;         // B's halo column x0-1 / x0+128
  const int hI = l31 ? hB - 1 : hB + 1;    // its neighbour inside the tile
  const int hO = l31 ? hB + 1 : hB - 1;    // and outside
  for (int k = 0; k < my_tiles && !fault; ++k) {
    const int t = gw + k * nw;
    const int cyk = t / tiles_x;
    const int x0 = (t - cyk * tiles_x) * kW;
    const int y0 = cyk * TY;
    const int dir = (cyk & 1) ? -1 : 1;
    const int ystart = (dir > 0) ? y0 - 2 : y0 + TY + 1;
    const int xl = x0 + 4 * lane;
    float hx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) hx[i] = (half && (xl + i == 0 || xl + i == g.nx - 1)) ? 0.5f : 1.f;
    const int xh = l31 ? x0 + kW : x0 - 1;
    const float hxh = (half && (xh == 0 || xh == g.nx - 1)) ? 0.5f : 1.f;
    const int cmax = cg.cx - 1;
    const int cxo = min(xl >> cg.lgB, cmax);
    const int cxl = (xl >= 1) ? min((xl - 1) >> cg.lgB, cmax) : cxo;
    const int cxr = (xl + 4 < g.nx) ? min((xl + 4) >> cg.lgB, cmax) : cxo;
    const int cxh = l31 ? cxr : cxl;
    const bool st_ok = xl < px;
    Fac2 fb{INT_MIN, 0}, fc{INT_MIN, 0};
    // the tile's cells (rows y0 - 3 .. y0 + TY + 2, columns x0 - 1 .. x0 + 128)
    KTab kt{nullptr, 0, 0, 1};
    {
      const int cr0 = max(y0 - 3, 0) >> cg.lgB, cr1 = min(y0 + TY + 2, g.ny - 1) >> cg.lgB;
      const int cc0 = max(x0 - 1, 0) >> cg.lgB, cc1 = min(min(x0 + kW, g.nx - 1) >> cg.lgB, cmax);
      const int nrow = cr1 - cr0 + 1, ncol = cc1 - cc0 + 1;
      __syncwarp();   // the previous tile's table is no longer read
      if (nrow * ncol <= kTab) {
        int *tab = ktabs + wib * kTab;
        for (int e = lane; e < nrow * ncol; e += 32)
          tab[e] = __ldg(kx + (cr0 + e / ncol) * cg.cx + cc0 + e % ncol);
        __syncwarp();
        kt = KTab{tab, cr0, cc0, ncol};
      }
    }
    float4 dq0 = make_float4(0, 0, 0, 0), dq1 = dq0, dq2 = dq0;   // d of rows j, j-1, j-2
    float4 xq0 = dq0, xq1 = dq0, xq2 = dq0;                       // xref likewise

    for (int j = 0; j < steps; ++j, ++q) {
      float *S0 = sb + (q % NS) * STAGE;
      // (a withheld first copy never lands: the bounded wait expires)
      bool ok = mbar_wait_bounded(&bar[q % NS], (uint32_t)(q / NS) & 1u);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        fault = true;
        break;
      }
      const int y = ystart + dir * j;
      // d (and xref) of an output row, used by stage C two steps on
      if (!INIT && j >= 2 && j < TY + 2 && y < g.ny && st_ok) {
        const int64_t o = (int64_t)y * px + xl;
        dq0 = ld4(d + o);
        if (check) xq0 = __ldg(reinterpret_cast<const float4 *>(xref + o));
      }
      // ---- A: row y_j, p in place
      if (!INIT) {
        const float4 r4 = ld4(S0 + OR + c), p4 = ld4(S0 + OP + c);
        st4(S0 + OP + c, fmaf(beta, p4.x, r4.x), fmaf(beta, p4.y, r4.y),
            fmaf(beta, p4.z, r4.z), fmaf(beta, p4.w, r4.w));
        if (l0 || l31) {
          const float2 r2 = *reinterpret_cast<const float2 *>(S0 + OR + hA);
          const float2 p2 = *reinterpret_cast<const float2 *>(S0 + OP + hA);
          *reinterpret_cast<float2 *>(S0 + OP + hA) =
              make_float2(fmaf(beta, p2.x, r2.x), fmaf(beta, p2.y, r2.y));
        }
      }
      __syncwarp();
      // ---- B: row y_{j-1}
      if (j >= 2) {
        const int y1 = y - dir;
        const float *S1 = sb + ((q - 1) % NS) * STAGE;    // centre row
        const float *S2 = sb + ((q - 2) % NS) * STAGE;    // row y1 - dir
        float *RB = ring + ((q - 1) & 3) * RING;
        const float hy1 = (half && (y1 == 0 || y1 == g.ny - 1)) ? 0.5f : 1.f;
        const float4 r4 = ld4(S1 + OR + c), s4 = ld4(S1 + OS + c);
        float rn[4];
        const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
        float ps = 0.f;   // sum of p (A p) over the lane's nodes of this row
        if (INIT) {
          rn[0] = r4.x; rn[1] = r4.y; rn[2] = r4.z; rn[3] = r4.w;
        } else {
          fac2_update(fb, y1, dir, g, cg, kx, kt, cxo, cxl, cxr, cxh, fd);
          const float4 p4 = ld4(S1 + OP + c);
          const float4 uc = mul4(s4, p4);
          const float4 up = mul4(ld4(S2 + OS + c), ld4(S2 + OP + c));
          const float4 un = mul4(ld4(S0 + OS + c), ld4(S0 + OP + c));
          const float uL = S1[OS + c - 1] * S1[OP + c - 1], uR = S1[OS + c + 4] * S1[OP + c + 4];
          const float xs[4] = {fmaf(uL, fb.fL, uc.y), uc.x + uc.z, uc.y + uc.w,
                               fmaf(uR, fb.fR, uc.z)};
          const float ysP[4] = {up.x, up.y, up.z, up.w}, ysN[4] = {un.x, un.y, un.z, un.w};
          const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ys = fmaf(ysP[i], fb.fP, ysN[i] * fb.fN);
            const float acc = fmaf(hy1, xs[i], hx[i] * ys);
            const float si = fmaf(-sv[i], acc, pv[i]);   // (A p)_i
            rn[i] = fmaf(-alpha, si, rv[i]);
            ps = fmaf(pv[i], si, ps);
          }
        }
        // <p, A p> over the tile's own rows (the halo rows belong to others)
        if (j >= 3 && j <= TY + 2 && y1 < g.ny) pap = fmaf(ps, fb.W, pap);
        st4(RB + c, rn[0], rn[1], rn[2], rn[3]);
        st4(RB + kWin + c, sv[0] * rn[0], sv[1] * rn[1], sv[2] * rn[2], sv[3] * rn[3]);
        if (l0 || l31) {
          // the halo column x0 - 1 / x0 + 128
          const float sh = S1[OS + hB];
          float rh = S1[OR + hB];
          if (!INIT) {
            const float uin = S1[OS + hI] * S1[OP + hI];
            const float uout = S1[OS + hO] * S1[OP + hO];
            const float upv = S2[OS + hB] * S2[OP + hB], unv = S0[OS + hB] * S0[OP + hB];
            const float acc = fmaf(hy1, fmaf(uin, fb.fxh, uout),
                                   hxh * fmaf(upv, fb.fPh, unv * fb.fNh));
            rh = fmaf(-alpha, fmaf(-sh, acc, S1[OP + hB]), rh);
          }
          RB[hB] = rh;
          RB[kWin + hB] = sh * rh;
        }
      }
      __syncwarp();
      // ---- C: row y_{j-2}
      if (j >= 4) {
        const int y2 = y - 2 * dir;
        if (y2 < g.ny) {
          fac2_update(fc, y2, dir, g, cg, kx, kt, cxo, cxl, cxr, cxh, fd);
          const float *S2 = sb + ((q - 2) % NS) * STAGE;
          const float *Rc = ring + ((q - 2) & 3) * RING;    // row y2
          const float *Rp = ring + ((q - 3) & 3) * RING;    // row y2 - dir
          const float *Rn = ring + ((q - 1) & 3) * RING;    // row y2 + dir
          const float hy2 = (half && (y2 == 0 || y2 == g.ny - 1)) ? 0.5f : 1.f;
          const float4 nc = ld4(Rc + kWin + c), np = ld4(Rp + kWin + c), nn = ld4(Rn + kWin + c);
          const float4 rn4 = ld4(Rc + c), s4 = ld4(S2 + OS + c);
          const float nL = Rc[kWin + c - 1], nR = Rc[kWin + c + 4];
          const float xs[4] = {fmaf(nL, fc.fL, nc.y), nc.x + nc.z, nc.y + nc.w,
                               fmaf(nR, fc.fR, nc.z)};
          const float ysP[4] = {np.x, np.y, np.z, np.w}, ysN[4] = {nn.x, nn.y, nn.z, nn.w};
          const float rv[4] = {rn4.x, rn4.y, rn4.z, rn4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
          float pv[4] = {0, 0, 0, 0};
          if (!INIT) {
            const float4 p4 = ld4(S2 + OP + c);
            pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
          }
          const float dv[4] = {dq2.x, dq2.y, dq2.z, dq2.w};
          const float xv[4] = {xq2.x, xq2.y, xq2.z, xq2.w};
          float dn[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ys = fmaf(ysP[i], fc.fP, ysN[i] * fc.fN);
            const float acc = fmaf(hy2, xs[i], hx[i] * ys);
            const float wv = fmaf(-sv[i], acc, rv[i]);
            const float tt = rv[i] * fc.W;
            gam = fmaf(tt, rv[i], gam);
            dlt = fmaf(tt, wv, dlt);
            rmax = fmaxf(rmax, fabsf(rv[i]));
            dn[i] = fmaf(alphaF, pv[i], dv[i]);
            pmax = fmaxf(pmax, fabsf(pv[i]));
            if (check && fabsf(rv[i]) > thetaF * fabsf(xv[i] + dn[i])) bad = 1;
          }
          if (!INIT && st_ok) {
            const int64_t o = (int64_t)y2 * px + xl;
            st4(d + o, dn[0], dn[1], dn[2], dn[3]);
            st4(r_out + o, rv[0] * gwr, rv[1] * gwr, rv[2] * gwr, rv[3] * gwr);
            st4(p_out + o, pv[0] * gwr, pv[1] * gwr, pv[2] * gwr, pv[3] * gwr);
          }
        }
      }
      dq2 = dq1;
      dq1 = dq0;
      xq2 = xq1;
      xq1 = xq0;
      // the stage of row q - 2 has been used for the last time: it takes
      // the next row of the warp's sequence
      __syncwarp();
      if (l0 && q >= 2 && nx_q < nq) {
        fence_proxy_async();
        issue_next();
      }
    }
  }
  if (fault && l0) {
    // leave no copy in flight: wait (bounded) for every row issued and not
    // yet waited for
    for (int qq = q; qq < nx_q; ++qq)
      if (!(qq == 0 && withhold)) mbar_wait_bounded(&bar[qq % NS], (uint32_t)(qq / NS) & 1u);
  }
  __syncwarp();
  cg_tail<INIT>(gam, dlt, rmax, pmax, bad, pap, fault, st, part, nblk_part);
}

// ------------------------------------------------------- packed 2D batch
// The 2D pass over a tile list spanning many instances of one atlas (BInst).
// List position t is a tile of act[a] (pre[a] <= t < pre[a + 1]); warp gw
// runs positions gw, gw + nw, ... as one pipeline, exactly as k_cg2d runs its
// tiles, with the tile's instance data and recurrence scalars read at the
// tile's start.  Instances join and leave the list between passes, each at
// its own pace:
//   * a tile's dots go to its own partial slot; the warp that completes an
//     instance's last tile of the pass combines that instance's slots in
//     list order and advances its recurrence (cg_update), and when the inner
//     solve has ended it writes the outcome to the instance's host record;
//   * the last warp of the pass drops the instances that ended and admits
//     the requests waiting in the host ring, for the next pass.
// An instance's first pass (MixCtl.first, with alpha = beta = 0 and p = 0)
// computes w = A r and the dots, and writes r as both r and p of the other
// buffer set, which is what its second pass expects (p = r + 0 p).  Each
// instance reads buffer set (launch set ^ flip), flip fixed on admission so
// that its first pass reads set 0, where the FP64 residual kernel put r.

__device__ __forceinline__ int ld_acquire_sys(const volatile int *p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int batch_find(const int *pre, int m, int t) {
  int lo = 0, hi = m;   // pre[lo] <= t < pre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= t)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// End of one tile: its six partials (as cg_tail's), and the instance's
// recurrence step when this was the instance's last tile of the pass.  Whole
// warp.
__device__ void batch_tile_done(float gam, float dlt, float rmax, float pmax, int bad,
                                float pap, int t, int inst, int a, const int *pre, MixCtl *st,
                                unsigned *cnt, int *alive, BatchCtl *bc, double *part, int cap,
                                BatchDone *done) {
  const int lane = threadIdx.x & 31;
  for (int o = 16; o > 0; o >>= 1) {
    gam += __shfl_down_sync(0xffffffffu, gam, o);
    dlt += __shfl_down_sync(0xffffffffu, dlt, o);
    pap += __shfl_down_sync(0xffffffffu, pap, o);
    rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
    pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  const int p0 = pre[a], p1 = pre[a + 1];
  int last = 0;
  if (lane == 0) {
    part[t] = (double)gam;
    part[cap + t] = (double)dlt;
    part[2 * cap + t] = (double)rmax;
    part[3 * cap + t] = (double)pmax;
    part[4 * cap + t] = (double)bad;
    part[5 * cap + t] = (double)pap;
    __threadfence();
    last = atomicAdd(&cnt[inst], 1u) == (unsigned)(p1 - p0 - 1);
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  double G = 0.0, D = 0.0, R = 0.0, P = 0.0, Bd = 0.0, Q = 0.0;
  for (int u = p0 + lane; u < p1; u += 32) {
    G += __ldcg(part + u);
    D += __ldcg(part + cap + u);
    R = fmax(R, __ldcg(part + 2 * cap + u));
    P = fmax(P, __ldcg(part + 3 * cap + u));
    Bd = fmax(Bd, __ldcg(part + 4 * cap + u));
    Q += __ldcg(part + 5 * cap + u);
  }
  for (int o = 16; o > 0; o >>= 1) {   // fixed tree: deterministic
    G += __shfl_down_sync(0xffffffffu, G, o);
    D += __shfl_down_sync(0xffffffffu, D, o);
    Q += __shfl_down_sync(0xffffffffu, Q, o);
    R = fmax(R, __shfl_down_sync(0xffffffffu, R, o));
    P = fmax(P, __shfl_down_sync(0xffffffffu, P, o));
    Bd = fmax(Bd, __shfl_down_sync(0xffffffffu, Bd, o));
  }
  if (lane == 0) {
    cnt[inst] = 0u;
    MixCtl *S = st + inst;
    const bool init = S->first != 0;
    S->first = 0;
    cg_update(S, G, D, R, P, Bd, Q, init);
    if (S->done) {
      alive[inst] = 0;
      BatchDone *h = done + inst;
      h->alpha = S->alpha;
      h->beta = S->beta;
      h->iter = S->iter;
      h->status = S->status;
      h->stalled = S->stalled;
      h->F = S->F;
      __threadfence_system();
      h->done_seq = S->seq;
      atomicExch(&bc->dirty, 1);
    }
  }
}

// The pass's last warp: keep the instances still iterating, in order, then
// append the requests waiting in the ring (they start with the next pass,
// launch set next_set).  The list is rewritten in place: a kept entry moves
// to a position no later than its own, and every chunk is read before it is
// written.
__device__ void batch_list_update(const BInst *__restrict__ bi, MixCtl *st, int *act, int *pre,
                                  unsigned *cnt, int *alive, BatchCtl *bc,
                                  const BatchRing *ring, int ring_cap, int m, int TY,
                                  int next_set) {
  const int lane = threadIdx.x & 31;
  int mnew = m, acc = __ldcg(&bc->ntiles);
  long long nodes = (lane == 0) ? __ldcg(&bc->nodes) : 0;   // summed over the warp below
  if (__ldcg(&bc->dirty)) {
    mnew = 0;
    acc = 0;
    nodes = 0;
    for (int base = 0; base < m; base += 32) {
      const int a = base + lane;
      const int inst = (a < m) ? act[a] : -1;
      const bool keep = inst >= 0 && __ldcg(&alive[inst]) != 0;
      const int T = keep ? bi[inst].tiles_x * ((bi[inst].ny + TY - 1) / TY) : 0;
      if (keep) nodes += (long long)bi[inst].nx * bi[inst].ny;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      int incl = T;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (keep) {
        const int pos = mnew + __popc(bal & ((1u << lane) - 1u));
        act[pos] = inst;
        pre[pos] = acc + incl - T;
      }
      mnew += __popc(bal);
      acc += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  const int head = __ldcg(&bc->req_head);
  const int tail = ld_acquire_sys(&ring->tail);   // every lane: orders its reads of ids
  for (int base = head; base < tail; base += 32) {
    const int k = base + lane;
    const int inst = (k < tail) ? ring->ids[k % ring_cap] : -1;
    const bool add = inst >= 0;
    const int T = add ? bi[inst].tiles_x * ((bi[inst].ny + TY - 1) / TY) : 0;
    if (add) nodes += (long long)bi[inst].nx * bi[inst].ny;
    const unsigned bal = __ballot_sync(0xffffffffu, add);
    int incl = T;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (add) {
      const int pos = mnew + __popc(bal & ((1u << lane) - 1u));
      act[pos] = inst;
      pre[pos] = acc + incl - T;
      st[inst].flip = next_set;
      cnt[inst] = 0u;
      alive[inst] = 1;
    }
    mnew += __popc(bal);
    acc += __shfl_sync(0xffffffffu, incl, 31);
  }
  for (int o = 16; o > 0; o >>= 1) nodes += __shfl_down_sync(0xffffffffu, nodes, o);
  if (lane == 0) {
    pre[mnew] = acc;
    bc->m = mnew;
    bc->ntiles = acc;
    bc->req_head = tail;
    bc->nodes = nodes;
  }
}

template <int NS, int WPB>
__global__ void __launch_bounds__(32 * WPB, WPB >= 7 ? 2 : 3)
k_cg2d_batch(const __grid_constant__ CUtensorMap tm_r0, const __grid_constant__ CUtensorMap tm_r1,
             const __grid_constant__ CUtensorMap tm_p0, const __grid_constant__ CUtensorMap tm_p1,
             const __grid_constant__ CUtensorMap tm_s, const BInst *__restrict__ bi, MixCtl *st,
             int *act, int *pre, unsigned *cnt, int *alive, BatchCtl *bc, int TY, int set,
             float *r0, float *r1, float *p0, float *p1, float *__restrict__ d,
             const float *__restrict__ xref, double *part, int part_cap, int P,
             const BatchRing *ring, int ring_cap, BatchDone *done) {
  constexpr int OR = 0, OP = kSlot, OS = 2 * kSlot;
  constexpr int STAGE = 3 * kSlot;
  constexpr int RING = 2 * kWin;
  constexpr int WARP_FLOATS = NS * STAGE + 4 * RING;
  static_assert((STAGE * 4) % 128 == 0 && (WARP_FLOATS * 4) % 128 == 0, "stage alignment");
  extern __shared__ __align__(128) unsigned char cgb_raw[];
  __shared__ __align__(8) uint64_t bars[WPB * NS];
  __shared__ int ktabs[WPB * kTab];
  // a pass that timed out abandons the solve: the passes left in the graph
  // return at once (the next solve resets the list and the flag)
  if (bc->fault) return;
  const int m = bc->m;
  const int ntot = bc->ntiles;
  float *cgb_smem = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(cgb_raw) + 127) & ~uintptr_t(127));
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * WPB + wib, nw = gridDim.x * WPB;
  const int steps = TY + 4;
  const int my_tiles = (gw < ntot) ? (ntot - 1 - gw) / nw + 1 : 0;
  const int nq = my_tiles * steps;
  float *sb = cgb_smem + (size_t)wib * WARP_FLOATS;
  float *ring_s = sb + NS * STAGE;
  uint64_t *bar = bars + wib * NS;

  // lane 0: the next row to copy (tile, step, atlas row of the tile's y0,
  // the buffer set its instance reads)
  int nx_q = 0, nx_j = 0, nx_x0 = 0, nx_row = 0, nx_dir = 1, nx_t = gw, nx_rs = 0;
  int withhold = 0;   // test hook (MixCtl.withhold): warp 0 never gets its first row
  auto set_tile = [&](int t) {
    nx_t = t;
    if (t >= ntot) return;
    const int a = batch_find(pre, m, t);
    const int inst = act[a];
    if (nx_q == 0 && gw == 0 && st[inst].withhold && st[inst].first) withhold = 1;
    const int local = t - pre[a];
    const int tx = bi[inst].tiles_x;
    const int cyk = local / tx;
    nx_x0 = (local - cyk * tx) * kW;
    nx_row = bi[inst].row0 + cyk * TY;
    nx_dir = (cyk & 1) ? -1 : 1;
    nx_rs = set ^ st[inst].flip;
  };
  auto issue_next = [&]() {
    const int y = (nx_dir > 0) ? nx_row - 2 + nx_j : nx_row + TY + 1 - nx_j;
    float *dst = sb + (nx_q % NS) * STAGE;
    uint64_t *b = bar + (nx_q % NS);
    if (!(nx_q == 0 && withhold)) {
      mbar_expect_tx(b, 3u * kWin * 4u);
      tma_load_2d(dst + OR, nx_rs ? &tm_r1 : &tm_r0, nx_x0 - 4, y, b);
      tma_load_2d(dst + OP, nx_rs ? &tm_p1 : &tm_p0, nx_x0 - 4, y, b);
      tma_load_2d(dst + OS, &tm_s, nx_x0 - 4, y, b);
    }
    ++nx_q;
    if (++nx_j == steps) {
      nx_j = 0;
      set_tile(nx_t + nw);
    }
  };
  if (lane == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    mbar_init_fence();
    set_tile(gw);
    while (nx_q < NS && nx_q < nq) issue_next();
  }
  __syncwarp();

  bool fault = false;
  int q = 0;
  const int c = 4 + 4 * lane;
  const bool l0 = lane == 0, l31 = lane == 31;
  const int hA = l31 ? kW + 4 : 2;
  const int hB = l31 ? kW + 4 : 3;
  const int hI = l31 ? hB - 1 : hB + 1;
  const int hO = l31 ? hB + 1 : hB - 1;
  for (int k = 0; k < my_tiles && !fault; ++k) {
    const int t = gw + k * nw;
    const int a = batch_find(pre, m, t);
    const int inst = act[a];
    const int local = t - pre[a];
    const BInst B = bi[inst];
    const MixCtl *S = st + inst;
    const float beta = (float)S->beta;
    const float alpha = (float)S->alpha;
    const int F = S->F, dF = S->dF, fd = S->fd;
    const float gwr = p2f(-dF);
    const float alphaF = (float)scalbn(S->alpha, F);
    const bool check = S->mode != 0 && ((S->iter & 3) == 3);
    const float thetaF = (float)scalbn((double)S->theta, -F);
    const bool half = B.boundary == EIK_BOUNDARY_HALF_CELL;
    const int wset = 1 - (set ^ S->flip);   // the other buffer set (written)
    Grid g{};
    g.nx = B.nx;
    g.ny = B.ny;
    g.nz = 1;
    g.boundary = B.boundary;
    const CellGrid cg = B.cg;
    const int *__restrict__ kx = B.kx;
    const int row0 = B.row0;
    const int cyk = local / B.tiles_x;
    const int x0 = (local - cyk * B.tiles_x) * kW;
    const int y0 = cyk * TY;
    const int dir = (cyk & 1) ? -1 : 1;
    const int ystart = (dir > 0) ? y0 - 2 : y0 + TY + 1;
    const int xl = x0 + 4 * lane;
    float hx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) hx[i] = (half && (xl + i == 0 || xl + i == g.nx - 1)) ? 0.5f : 1.f;
    const int xh = l31 ? x0 + kW : x0 - 1;
    const float hxh = (half && (xh == 0 || xh == g.nx - 1)) ? 0.5f : 1.f;
    const int cmax = cg.cx - 1;
    const int cxo = min(xl >> cg.lgB, cmax);
    const int cxl = (xl >= 1) ? min((xl - 1) >> cg.lgB, cmax) : cxo;
    const int cxr = (xl + 4 < g.nx) ? min((xl + 4) >> cg.lgB, cmax) : cxo;
    const int cxh = l31 ? cxr : cxl;
    const bool st_ok = xl < B.wx;
    Fac2 fb{INT_MIN, 0}, fc{INT_MIN, 0};
    KTab kt{nullptr, 0, 0, 1};
    {
      const int cr0 = max(y0 - 3, 0) >> cg.lgB, cr1 = min(y0 + TY + 2, g.ny - 1) >> cg.lgB;
      const int cc0 = max(x0 - 1, 0) >> cg.lgB, cc1 = min(min(x0 + kW, g.nx - 1) >> cg.lgB, cmax);
      const int nrow = cr1 - cr0 + 1, ncol = cc1 - cc0 + 1;
      __syncwarp();
      if (nrow * ncol <= kTab) {
        int *tab = ktabs + wib * kTab;
        for (int e = lane; e < nrow * ncol; e += 32)
          tab[e] = __ldg(kx + (cr0 + e / ncol) * cg.cx + cc0 + e % ncol);
        __syncwarp();
        kt = KTab{tab, cr0, cc0, ncol};
      }
    }
    float gam = 0.f, dlt = 0.f, rmax = 0.f, pmax = 0.f, pap = 0.f;
    int bad = 0;
    float4 dq0 = make_float4(0, 0, 0, 0), dq1 = dq0, dq2 = dq0;
    float4 xq0 = dq0, xq1 = dq0, xq2 = dq0;

    for (int j = 0; j < steps; ++j, ++q) {
      float *S0 = sb + (q % NS) * STAGE;
      bool ok = mbar_wait_bounded(&bar[q % NS], (uint32_t)(q / NS) & 1u);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        fault = true;
        break;
      }
      const int y = ystart + dir * j;
      if (j >= 2 && j < TY + 2 && y < g.ny && st_ok) {
        const int64_t o = (int64_t)(row0 + y) * P + xl;
        dq0 = ld4(d + o);
        if (check) xq0 = __ldg(reinterpret_cast<const float4 *>(xref + o));
      }
      // ---- A: row y_j, p in place
      {
        const float4 r4 = ld4(S0 + OR + c), p4 = ld4(S0 + OP + c);
        st4(S0 + OP + c, fmaf(beta, p4.x, r4.x), fmaf(beta, p4.y, r4.y),
            fmaf(beta, p4.z, r4.z), fmaf(beta, p4.w, r4.w));
        if (l0 || l31) {
          const float2 r2 = *reinterpret_cast<const float2 *>(S0 + OR + hA);
          const float2 p2 = *reinterpret_cast<const float2 *>(S0 + OP + hA);
          *reinterpret_cast<float2 *>(S0 + OP + hA) =
              make_float2(fmaf(beta, p2.x, r2.x), fmaf(beta, p2.y, r2.y));
        }
      }
      __syncwarp();
      // ---- B: row y_{j-1}
      if (j >= 2) {
        const int y1 = y - dir;
        const float *S1 = sb + ((q - 1) % NS) * STAGE;
        const float *S2 = sb + ((q - 2) % NS) * STAGE;
        float *RB = ring_s + ((q - 1) & 3) * RING;
        const float hy1 = (half && (y1 == 0 || y1 == g.ny - 1)) ? 0.5f : 1.f;
        const float4 r4 = ld4(S1 + OR + c), s4 = ld4(S1 + OS + c);
        float rn[4];
        const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
        float ps = 0.f;   // sum of p (A p) over the lane's nodes of this row
        {
          fac2_update(fb, y1, dir, g, cg, kx, kt, cxo, cxl, cxr, cxh, fd);
          const float4 p4 = ld4(S1 + OP + c);
          const float4 uc = mul4(s4, p4);
          const float4 up = mul4(ld4(S2 + OS + c), ld4(S2 + OP + c));
          const float4 un = mul4(ld4(S0 + OS + c), ld4(S0 + OP + c));
          const float uL = S1[OS + c - 1] * S1[OP + c - 1], uR = S1[OS + c + 4] * S1[OP + c + 4];
          const float xs[4] = {fmaf(uL, fb.fL, uc.y), uc.x + uc.z, uc.y + uc.w,
                               fmaf(uR, fb.fR, uc.z)};
          const float ysP[4] = {up.x, up.y, up.z, up.w}, ysN[4] = {un.x, un.y, un.z, un.w};
          const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ys = fmaf(ysP[i], fb.fP, ysN[i] * fb.fN);
            const float acc = fmaf(hy1, xs[i], hx[i] * ys);
            const float si = fmaf(-sv[i], acc, pv[i]);   // (A p)_i
            rn[i] = fmaf(-alpha, si, rv[i]);
            ps = fmaf(pv[i], si, ps);
          }
        }
        // <p, A p> over the tile's own rows (the halo rows belong to others)
        if (j >= 3 && j <= TY + 2 && y1 < g.ny) pap = fmaf(ps, fb.W, pap);
        st4(RB + c, rn[0], rn[1], rn[2], rn[3]);
        st4(RB + kWin + c, sv[0] * rn[0], sv[1] * rn[1], sv[2] * rn[2], sv[3] * rn[3]);
        if (l0 || l31) {
          const float sh = S1[OS + hB];
          float rh = S1[OR + hB];
          const float uin = S1[OS + hI] * S1[OP + hI];
          const float uout = S1[OS + hO] * S1[OP + hO];
          const float upv = S2[OS + hB] * S2[OP + hB], unv = S0[OS + hB] * S0[OP + hB];
          const float acc = fmaf(hy1, fmaf(uin, fb.fxh, uout),
                                 hxh * fmaf(upv, fb.fPh, unv * fb.fNh));
          rh = fmaf(-alpha, fmaf(-sh, acc, S1[OP + hB]), rh);
          RB[hB] = rh;
          RB[kWin + hB] = sh * rh;
        }
      }
      __syncwarp();
      // ---- C: row y_{j-2}
      if (j >= 4) {
        const int y2 = y - 2 * dir;
        if (y2 < g.ny) {
          fac2_update(fc, y2, dir, g, cg, kx, kt, cxo, cxl, cxr, cxh, fd);
          const float *S2 = sb + ((q - 2) % NS) * STAGE;
          const float *Rc = ring_s + ((q - 2) & 3) * RING;
          const float *Rp = ring_s + ((q - 3) & 3) * RING;
          const float *Rn = ring_s + ((q - 1) & 3) * RING;
          const float hy2 = (half && (y2 == 0 || y2 == g.ny - 1)) ? 0.5f : 1.f;
          const float4 nc = ld4(Rc + kWin + c), np = ld4(Rp + kWin + c), nn = ld4(Rn + kWin + c);
          const float4 rn4 = ld4(Rc + c), s4 = ld4(S2 + OS + c);
          const float nL = Rc[kWin + c - 1], nR = Rc[kWin + c + 4];
          const float xs[4] = {fmaf(nL, fc.fL, nc.y), nc.x + nc.z, nc.y + nc.w,
                               fmaf(nR, fc.fR, nc.z)};
          const float ysP[4] = {np.x, np.y, np.z, np.w}, ysN[4] = {nn.x, nn.y, nn.z, nn.w};
          const float rv[4] = {rn4.x, rn4.y, rn4.z, rn4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
          const float4 p4 = ld4(S2 + OP + c);
          const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
          const float dv[4] = {dq2.x, dq2.y, dq2.z, dq2.w};
          const float xv[4] = {xq2.x, xq2.y, xq2.z, xq2.w};
          float dn[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ys = fmaf(ysP[i], fc.fP, ysN[i] * fc.fN);
            const float acc = fmaf(hy2, xs[i], hx[i] * ys);
            const float wv = fmaf(-sv[i], acc, rv[i]);
            const float tt = rv[i] * fc.W;
            gam = fmaf(tt, rv[i], gam);
            dlt = fmaf(tt, wv, dlt);
            rmax = fmaxf(rmax, fabsf(rv[i]));
            dn[i] = fmaf(alphaF, pv[i], dv[i]);
            pmax = fmaxf(pmax, fabsf(pv[i]));
            if (check && fabsf(rv[i]) > thetaF * fabsf(xv[i] + dn[i])) bad = 1;
          }
          if (st_ok) {
            const int64_t o = (int64_t)(row0 + y2) * P + xl;
            st4(d + o, dn[0], dn[1], dn[2], dn[3]);
            st4((wset ? r1 : r0) + o, rv[0] * gwr, rv[1] * gwr, rv[2] * gwr, rv[3] * gwr);
            st4((wset ? p1 : p0) + o, pv[0] * gwr, pv[1] * gwr, pv[2] * gwr, pv[3] * gwr);
          }
        }
      }
      dq2 = dq1;
      dq1 = dq0;
      xq2 = xq1;
      xq1 = xq0;
      __syncwarp();
      if (l0 && q >= 2 && nx_q < nq) {
        fence_proxy_async();
        issue_next();
      }
    }
    if (fault) break;
    {
      // the tile's list entry again (not kept live through the tile)
      const int te = gw + k * nw;
      const int ae = batch_find(pre, m, te);
      batch_tile_done(gam, dlt, rmax, pmax, bad, pap, te, act[ae], ae, pre, st, cnt, alive, bc,
                      part, part_cap, done);
    }
  }
  if (fault && l0) {
    // leave no copy in flight: wait (bounded) for every row issued and not
    // yet waited for
    for (int qq = q; qq < nx_q; ++qq)
      if (!(qq == 0 && withhold)) mbar_wait_bounded(&bar[qq % NS], (uint32_t)(qq / NS) & 1u);
    atomicExch(&bc->fault, 1);
  }
  __syncwarp();
  // end of the pass for this warp; the last one updates the list
  int lastw = 0;
  if (l0) {
    __threadfence();
    lastw = atomicAdd(&bc->warps_done, 1u) == (unsigned)(nw - 1);
  }
  lastw = __shfl_sync(0xffffffffu, lastw, 0);
  if (!lastw) return;
  __threadfence();
  const long long nodes0 = __ldcg(&bc->nodes);   // this pass's (the update rewrites it)
  batch_list_update(bi, st, act, pre, cnt, alive, bc, ring, ring_cap, m, TY, set ^ 1);
  if (l0) {
    bc->warps_done = 0u;
    bc->dirty = 0;
    if (m > 0) {
      bc->passes += 1;
      bc->work += nodes0;
    }
  }
}

// ------------------------------------------------------------------ 3D pass
// A block owns tiles of 128 columns x TY rows x zc planes and marches them
// through z.  Each plane of r, p and sigma arrives by one TMA copy per array
// (box 136 x (TY + 4) x 1 from (x0 - 4, y0 - 2, z)) into a ring of NS
// stages, and stays there until consumed.  Warp w owns row y0 - 2 + w (TY + 4
// warps), lanes as in 2D.  At plane step j (plane z_j):
//   A, every warp, plane z_j:            p = r + beta p, in place
//   B, warps 1 .. TY + 2, plane z_{j-1}: u = sig p of the node and its six
//        neighbours, s = A p, r_new, un = sig r_new; r_new, sig, p of the
//        plane go to a two-plane ring and un to a three-plane ring
//   C, warps 2 .. TY + 1, plane z_{j-2}: w = A r_new, the dots,
//        d += alpha p, stores
// B takes the y and x neighbours from the stage of its plane (written by A
// one step earlier) and its own column's u of planes z_j and z_{j-2} from
// registers; C reads only the rings.  One block barrier per step orders the
// steps.  So a stage is free one step after A, and NS - 2 planes beyond the
// current one are in flight.  Measured, a step of the (12, 5) block costs
// about the same whatever NS: the pass is bound by the latency of one block
// step (the barrier and the shared-memory round trips of A, B, C), which is
// why taller tiles (fewer steps, more warps per barrier) do not help either.
// Odd z chunks march downwards, so the halo planes two neighbouring chunks
// share are read at about the same time.
__device__ __forceinline__ int cell_k(const CellGrid &cg, const int *__restrict__ kx, int cxi,
                                      int y, int z, const Grid &g) {
  const int cy = min(max(y, 0), g.ny - 1) >> cg.lgB;
  const int cz = min(max(z, 0), g.nz - 1) >> cg.lgB;
  return __ldg(kx + (cz * cg.cy + cy) * cg.cx + cxi);
}

template <bool INIT, int TY, int NS>
__global__ void __launch_bounds__(32 * (TY + 4), 1)
k_cg3d(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_p,
       const __grid_constant__ CUtensorMap tm_s, Grid g, CellGrid cg,
       const int *__restrict__ kx, int tiles_x, int tiles_y, int zc, int ntiles,
       float *__restrict__ r_out, float *__restrict__ p_out, float *__restrict__ d,
       const float *__restrict__ xref, MixCtl *st, double *part, int nblk_part, int px) {
  constexpr int NR = TY + 4;             // staged rows
  constexpr int PLANE = NR * kWin;       // floats per array and plane
  constexpr int STAGE = 3 * PLANE;       // r, p, sigma
  static_assert((PLANE * 4) % 128 == 0, "plane size");
  extern __shared__ __align__(128) unsigned char cg3_raw[];
  __shared__ __align__(8) uint64_t bars[NS];
  if (st->done) return;
  float *cg3_smem = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(cg3_raw) + 127) & ~uintptr_t(127));
  float *ring_n = cg3_smem + NS * STAGE;   // un: [3 planes][NR][kWin]
  float *ring_c = ring_n + 3 * PLANE;       // [2 planes][rn | sig | p][NR][kWin]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float beta = INIT ? 0.f : (float)st->beta;
  const float alpha = INIT ? 0.f : (float)st->alpha;
  const int F = st->F, dF = st->dF, fd = st->fd;
  const float gwr = p2f(-dF);
  const float alphaF = INIT ? 0.f : (float)scalbn(st->alpha, F);
  const bool check = !INIT && st->mode != 0 && ((st->iter & 3) == 3);
  const float thetaF = (float)scalbn((double)st->theta, -F);
  const bool half = g.boundary == EIK_BOUNDARY_HALF_CELL;
  const int withhold = (!INIT && st->withhold && st->iter == 0 && blockIdx.x == 0) ? 1 : 0;
  const int steps = zc + 4;
  const int my_tiles =
      ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nq = my_tiles * steps;
  const int plane_tiles = tiles_x * tiles_y;

  int next_issue = 0;   // thread 0
  auto issue = [&](int q) {
    const int k = q / steps, j = q - k * steps;
    const int t = blockIdx.x + k * gridDim.x;
    const int szc = t / plane_tiles, rem = t - szc * plane_tiles;
    const int sy = rem / tiles_x, sx = rem - sy * tiles_x;
    const int z = (szc & 1) ? (szc * zc + zc + 1 - j) : (szc * zc - 2 + j);
    float *dst = cg3_smem + (q % NS) * STAGE;
    uint64_t *b = &bars[q % NS];
    if (!(q == 0 && withhold)) {
      mbar_expect_tx(b, (INIT ? 2u : 3u) * PLANE * 4u);
      tma_load_3d(dst, &tm_r, sx * kW - 4, sy * TY - 2, z, b);
      if (!INIT) tma_load_3d(dst + PLANE, &tm_p, sx * kW - 4, sy * TY - 2, z, b);
      tma_load_3d(dst + 2 * PLANE, &tm_s, sx * kW - 4, sy * TY - 2, z, b);
    }
  };
  if (threadIdx.x == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (; next_issue < NS && next_issue < nq; ++next_issue) issue(next_issue);

  const bool doB = (w >= 1 && w <= TY + 2), doC = (w >= 2 && w <= TY + 1);
  const bool l0 = lane == 0, l31 = lane == 31;
  const int c = 4 + 4 * lane;                 // staged column of the lane's first node
  const int hA = l31 ? kW + 4 : 2;            // A's halo pair
  const int hB = l31 ? kW + 4 : 3;            // B's halo column
  const int hI = l31 ? hB - 1 : hB + 1;       // its neighbour inside the tile
  const int hO = l31 ? hB + 1 : hB - 1;       // and outside
  const int rw = w * kWin;                    // the warp's row in a plane
  float gam = 0.f, dlt = 0.f, rmax = 0.f, pmax = 0.f, pap = 0.f;
  float psb = 0.f, psc = 0.f;   // p (A p) of B's row this step / the step before
  int bad = 0;
  bool fault = false;
  int q = 0;
  for (int k = 0; k < my_tiles && !fault; ++k) {
    const int t = blockIdx.x + k * gridDim.x;
    const int szc = t / plane_tiles, rem = t - szc * plane_tiles;
    const int sy = rem / tiles_x, sx = rem - sy * tiles_x;
    const int x0 = sx * kW, y = sy * TY - 2 + w, z0 = szc * zc;
    const int dir = (szc & 1) ? -1 : 1;
    const int zstart = (dir > 0) ? z0 - 2 : z0 + zc + 1;
    const int xl = x0 + 4 * lane;
    float hx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) hx[i] = (half && (xl + i == 0 || xl + i == g.nx - 1)) ? 0.5f : 1.f;
    const int xh = l31 ? x0 + kW : x0 - 1;
    const float hxh = (half && (xh == 0 || xh == g.nx - 1)) ? 0.5f : 1.f;
    const float hy = (half && (y == 0 || y == g.ny - 1)) ? 0.5f : 1.f;
    const int cmax = cg.cx - 1;
    const int cxo = min(xl >> cg.lgB, cmax);
    const int cxl = (xl >= 1) ? min((xl - 1) >> cg.lgB, cmax) : cxo;
    const int cxr = (xl + 4 < g.nx) ? min((xl + 4) >> cg.lgB, cmax) : cxo;
    const int cxh = l31 ? cxr : cxl;
    const bool row_ok = y >= 0 && y < g.ny;
    const bool st_ok = xl < px && row_ok;
    // cell factors of stage B (plane z_{j-1}) and C (plane z_{j-2}), cached
    // per cell layer; z factors are 1 except next to another layer
    int layB = INT_MIN, layC = INT_MIN;
    float bL = 1, bR = 1, bS = 1, bN = 1, bP = 1, bNz = 1, bxh = 1, bhS = 1, bhN = 1, bhP = 1,
          bhNz = 1;
    float cL = 1, cR = 1, cS = 1, cN = 1, cP = 1, cNz = 1, cW = 0;
    float4 uA = make_float4(0, 0, 0, 0), uB = uA;     // own u of planes z_j, z_{j-1}
    float4 uBp = uA;                                  // own u of plane z_{j-2}
    float hA0 = 0.f, hB0 = 0.f, hBp = 0.f;            // the same for the halo column
    float4 dq0 = uA, dq1 = uA, dq2 = uA, xq0 = uA, xq1 = uA, xq2 = uA;
    for (int j = 0; j < zc + 4; ++j, ++q) {
      const int sidx = q % NS;
      const bool okw = mbar_wait_bounded(&bars[sidx], (uint32_t)(q / NS) & 1u);
      if (__syncthreads_or(!okw)) {
        fault = true;
        break;
      }
      const int z = zstart + dir * j;
      float *S0 = cg3_smem + sidx * STAGE;
      // ---- A: plane z_j, row y: p in place, own u kept
      uBp = uB;
      uB = uA;
      hBp = hB0;
      hB0 = hA0;
      if (!INIT) {
        const float4 r4 = ld4(S0 + rw + c), p4 = ld4(S0 + PLANE + rw + c);
        const float4 s4 = ld4(S0 + 2 * PLANE + rw + c);
        const float4 pn = make_float4(fmaf(beta, p4.x, r4.x), fmaf(beta, p4.y, r4.y),
                                      fmaf(beta, p4.z, r4.z), fmaf(beta, p4.w, r4.w));
        *reinterpret_cast<float4 *>(S0 + PLANE + rw + c) = pn;
        uA = mul4(s4, pn);
        if (l0 || l31) {
          const float2 r2 = *reinterpret_cast<const float2 *>(S0 + rw + hA);
          const float2 p2 = *reinterpret_cast<const float2 *>(S0 + PLANE + rw + hA);
          const float2 s2 = *reinterpret_cast<const float2 *>(S0 + 2 * PLANE + rw + hA);
          const float b0 = fmaf(beta, p2.x, r2.x), b1 = fmaf(beta, p2.y, r2.y);
          *reinterpret_cast<float2 *>(S0 + PLANE + rw + hA) = make_float2(b0, b1);
          hA0 = l31 ? s2.x * b0 : s2.y * b1;   // u of the column x0 + 128 / x0 - 1
        }
      }
      // d (and xref) of an output plane, for stage C two steps on
      if (!INIT && doC && row_ok && j >= 2 && j < zc + 2 && z < g.nz && xl < px) {
        const int64_t o = ((int64_t)z * g.ny + y) * px + xl;
        dq0 = ld4(d + o);
        if (check) xq0 = __ldg(reinterpret_cast<const float4 *>(xref + o));
      }
      // ---- B: plane z_{j-1}
      if (j >= 2 && doB) {
        const int z1 = z - dir;
        const float *S1 = cg3_smem + ((q - 1) % NS) * STAGE;   // plane z1
        float *RN = ring_n + ((q - 1) % 3) * PLANE;
        float *RC = ring_c + ((q - 1) & 1) * 3 * PLANE;
        const float4 r4 = ld4(S1 + rw + c), s4 = ld4(S1 + 2 * PLANE + rw + c);
        float rn[4];
        const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
        float ps = 0.f;   // sum of p (A p) over the lane's nodes of this row
        float hrn = S1[rw + hB];
        const float hs = S1[2 * PLANE + rw + hB];
        if (INIT) {
          rn[0] = r4.x; rn[1] = r4.y; rn[2] = r4.z; rn[3] = r4.w;
        } else {
          const int lay = min(max(z1, 0), g.nz - 1) >> cg.lgB;
          const int layp = min(max(z1 - dir, 0), g.nz - 1) >> cg.lgB;
          const int layn = min(max(z1 + dir, 0), g.nz - 1) >> cg.lgB;
          if (lay != layB || layp != lay || layn != lay) {
            // x / y factors change with the layer, z factors only next to
            // another layer (uniform across the block)
            layB = (layp != lay || layn != lay) ? INT_MIN : lay;
            const int kc = cell_k(cg, kx, cxo, y, z1, g), kh = cell_k(cg, kx, cxh, y, z1, g);
            bL = p2f(kc - cell_k(cg, kx, cxl, y, z1, g));
            bR = p2f(kc - cell_k(cg, kx, cxr, y, z1, g));
            bS = p2f(kc - cell_k(cg, kx, cxo, y - 1, z1, g));
            bN = p2f(kc - cell_k(cg, kx, cxo, y + 1, z1, g));
            bxh = p2f(kh - kc);
            bhS = p2f(kh - cell_k(cg, kx, cxh, y - 1, z1, g));
            bhN = p2f(kh - cell_k(cg, kx, cxh, y + 1, z1, g));
            bP = p2f(kc - cell_k(cg, kx, cxo, y, z1 - dir, g));
            bNz = p2f(kc - cell_k(cg, kx, cxo, y, z1 + dir, g));
            bhP = p2f(kh - cell_k(cg, kx, cxh, y, z1 - dir, g));
            bhNz = p2f(kh - cell_k(cg, kx, cxh, y, z1 + dir, g));
          }
          const float hz1 = (half && (z1 == 0 || z1 == g.nz - 1)) ? 0.5f : 1.f;
          const float wxe = hy * hz1;
          const float4 p4 = ld4(S1 + PLANE + rw + c);
          const float4 uc = uB;
          const float uL = S1[2 * PLANE + rw + c - 1] * S1[PLANE + rw + c - 1];
          const float uR = S1[2 * PLANE + rw + c + 4] * S1[PLANE + rw + c + 4];
          const float4 us = mul4(ld4(S1 + 2 * PLANE + rw - kWin + c), ld4(S1 + PLANE + rw - kWin + c));
          const float4 un = mul4(ld4(S1 + 2 * PLANE + rw + kWin + c), ld4(S1 + PLANE + rw + kWin + c));
          const float xs[4] = {fmaf(uL, bL, uc.y), uc.x + uc.z, uc.y + uc.w, fmaf(uR, bR, uc.z)};
          const float ysS[4] = {us.x, us.y, us.z, us.w}, ysN[4] = {un.x, un.y, un.z, un.w};
          const float zsP[4] = {uBp.x, uBp.y, uBp.z, uBp.w}, zsN[4] = {uA.x, uA.y, uA.z, uA.w};
          const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ys = fmaf(ysS[i], bS, ysN[i] * bN);
            const float zs = fmaf(zsP[i], bP, zsN[i] * bNz);
            const float acc = fmaf(wxe, xs[i], hx[i] * fmaf(hz1, ys, hy * zs));
            const float si = fmaf(-sv[i], acc, pv[i]);   // (A p)_i
            rn[i] = fmaf(-alpha, si, rv[i]);
            ps = fmaf(pv[i], si, ps);
          }
          if (l0 || l31) {
            const float uin = S1[2 * PLANE + rw + hI] * S1[PLANE + rw + hI];
            const float uout = S1[2 * PLANE + rw + hO] * S1[PLANE + rw + hO];
            const float uS = S1[2 * PLANE + rw - kWin + hB] * S1[PLANE + rw - kWin + hB];
            const float uN = S1[2 * PLANE + rw + kWin + hB] * S1[PLANE + rw + kWin + hB];
            const float acc =
                fmaf(wxe, fmaf(uin, bxh, uout),
                     hxh * fmaf(hz1, fmaf(uS, bhS, uN * bhN), hy * fmaf(hBp, bhP, hA0 * bhNz)));
            hrn = fmaf(-alpha, fmaf(-hs, acc, S1[PLANE + rw + hB]), hrn);
          }
        }
        st4(RN + rw + c, sv[0] * rn[0], sv[1] * rn[1], sv[2] * rn[2], sv[3] * rn[3]);
        if (l0 || l31) RN[rw + hB] = hs * hrn;
        if (doC) {   // C reads r_new, sig and p of this plane one step on
          st4(RC + rw + c, rn[0], rn[1], rn[2], rn[3]);
          *reinterpret_cast<float4 *>(RC + PLANE + rw + c) = s4;
          if (!INIT) *reinterpret_cast<float4 *>(RC + 2 * PLANE + rw + c) = ld4(S1 + PLANE + rw + c);
        }
        psb = ps;
      }
      // ---- C: plane z_{j-2} (B wrote its neighbours' un in earlier steps,
      // and this warp's own un of plane z_{j-1} just now)
      if (j >= 4 && doC) {
        const int z2 = z - 2 * dir;
        if (z2 < g.nz && row_ok) {
          const int lay = z2 >> cg.lgB;
          const int layp = min(max(z2 - dir, 0), g.nz - 1) >> cg.lgB;
          const int layn = min(max(z2 + dir, 0), g.nz - 1) >> cg.lgB;
          if (lay != layC || layp != lay || layn != lay) {
            layC = (layp != lay || layn != lay) ? INT_MIN : lay;
            const int kc = cell_k(cg, kx, cxo, y, z2, g);
            cL = p2f(kc - cell_k(cg, kx, cxl, y, z2, g));
            cR = p2f(kc - cell_k(cg, kx, cxr, y, z2, g));
            cS = p2f(kc - cell_k(cg, kx, cxo, y - 1, z2, g));
            cN = p2f(kc - cell_k(cg, kx, cxo, y + 1, z2, g));
            cP = p2f(kc - cell_k(cg, kx, cxo, y, z2 - dir, g));
            cNz = p2f(kc - cell_k(cg, kx, cxo, y, z2 + dir, g));
            cW = p2f(-2 * kc - fd);
          }
          const float hz2 = (half && (z2 == 0 || z2 == g.nz - 1)) ? 0.5f : 1.f;
          const float wxe = hy * hz2;
          const float *RC = ring_c + ((q - 2) & 1) * 3 * PLANE;   // plane z2: r_new, sig, p
          const float *Nc = ring_n + ((q - 2) % 3) * PLANE;       // un of plane z2
          const float *Np = ring_n + ((q - 3) % 3) * PLANE;       // plane z2 - dir
          const float *Nn = ring_n + ((q - 1) % 3) * PLANE;       // plane z2 + dir
          const float4 nc = ld4(Nc + rw + c);
          const float nL = Nc[rw + c - 1], nR = Nc[rw + c + 4];
          const float4 ns = ld4(Nc + rw - kWin + c), nn = ld4(Nc + rw + kWin + c);
          const float4 np = ld4(Np + rw + c), nz = ld4(Nn + rw + c);
          const float4 rn4 = ld4(RC + rw + c), s4 = ld4(RC + PLANE + rw + c);
          const float xs[4] = {fmaf(nL, cL, nc.y), nc.x + nc.z, nc.y + nc.w, fmaf(nR, cR, nc.z)};
          const float ysS[4] = {ns.x, ns.y, ns.z, ns.w}, ysN[4] = {nn.x, nn.y, nn.z, nn.w};
          const float zsP[4] = {np.x, np.y, np.z, np.w}, zsN[4] = {nz.x, nz.y, nz.z, nz.w};
          const float rv[4] = {rn4.x, rn4.y, rn4.z, rn4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
          float pv[4] = {0, 0, 0, 0};
          if (!INIT) {
            const float4 p4 = ld4(RC + 2 * PLANE + rw + c);
            pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
          }
          const float dv[4] = {dq2.x, dq2.y, dq2.z, dq2.w};
          const float xv[4] = {xq2.x, xq2.y, xq2.z, xq2.w};
          float dn[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float ys = fmaf(ysS[i], cS, ysN[i] * cN);
            const float zs = fmaf(zsP[i], cP, zsN[i] * cNz);
            const float acc = fmaf(wxe, xs[i], hx[i] * fmaf(hz2, ys, hy * zs));
            const float wv = fmaf(-sv[i], acc, rv[i]);
            const float tt = rv[i] * cW;
            gam = fmaf(tt, rv[i], gam);
            dlt = fmaf(tt, wv, dlt);
            rmax = fmaxf(rmax, fabsf(rv[i]));
            dn[i] = fmaf(alphaF, pv[i], dv[i]);
            pmax = fmaxf(pmax, fabsf(pv[i]));
            if (check && fabsf(rv[i]) > thetaF * fabsf(xv[i] + dn[i])) bad = 1;
          }
          pap = fmaf(psc, cW, pap);
          if (!INIT && st_ok) {
            const int64_t o = ((int64_t)z2 * g.ny + y) * px + xl;
            st4(d + o, dn[0], dn[1], dn[2], dn[3]);
            st4(r_out + o, rv[0] * gwr, rv[1] * gwr, rv[2] * gwr, rv[3] * gwr);
            st4(p_out + o, pv[0] * gwr, pv[1] * gwr, pv[2] * gwr, pv[3] * gwr);
          }
        }
      }
      psc = psb;
      dq2 = dq1;
      dq1 = dq0;
      xq2 = xq1;
      xq1 = xq0;
      // every warp is done with the stage of the plane of one step ago and
      // with the ring slots the next step overwrites
      __syncthreads();
      if (threadIdx.x == 0 && q >= 1 && next_issue < nq) {
        fence_proxy_async();
        issue(next_issue);
        ++next_issue;
      }
    }
  }
  if (fault) {
    if (threadIdx.x == 0)
      for (int qq = q; qq < next_issue; ++qq)
        if (!(qq == 0 && withhold)) mbar_wait_bounded(&bars[qq % NS], (uint32_t)(qq / NS) & 1u);
    __syncthreads();
  }
  cg_tail<INIT>(gam, dlt, rmax, pmax, bad, pap, fault, st, part, nblk_part);
}

// ------------------------------------------------------------------ host
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &qr) != cudaSuccess ||
        qr != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// FP32 tensor map over an nx x ny (x nz) array with row pitch px elements;
// box bw x bh (x bd); nz == 0 gives a 2D map.  Out-of-range elements read 0.
bool encode_f32(CUtensorMap *map, void *base, int nx, int px, int ny, int nz, int bw, int bh,
                int bd) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint32_t rank = nz > 0 ? 3 : 2;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)(nz > 0 ? nz : 1)};
  const cuuint64_t strides[2] = {(cuuint64_t)px * 4, (cuuint64_t)px * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, (cuuint32_t)bd};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// 2D variants: (warps per block, stages per warp)
template <int NS, int WPB>
size_t smem2d() {
  return (size_t)WPB * (NS * 3 * kSlot + 4 * 2 * kWin) * sizeof(float) + 128;
}

template <int NS, int WPB>
bool plan2d_t(Cg32Plan *pl, const Grid &g, int num_sms) {
  const size_t sm = smem2d<NS, WPB>();
  if (cudaFuncSetAttribute(k_cg2d<false, NS, WPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_cg2d<true, NS, WPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess)
    return false;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg2d<false, NS, WPB>, 32 * WPB, sm) !=
          cudaSuccess ||
      per < 1)
    return false;
  int per_i = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_i, k_cg2d<true, NS, WPB>, 32 * WPB, sm) !=
          cudaSuccess ||
      per_i < 1)
    return false;
  per = std::min(per, per_i);
  pl->wpb = WPB;
  pl->ns = NS;
  pl->smem = sm;
  pl->tiles_x = (g.nx + kW - 1) / kW;
  // rows per tile: one tile per resident warp where the grid is large enough,
  // at least 8 rows (the two-row halo costs (ty + 4) / ty in stage A)
  const int64_t warps = (int64_t)per * num_sms * WPB;
  const int64_t rows = (int64_t)pl->tiles_x * g.ny;
  int ty = (int)std::min<int64_t>(std::max<int64_t>((rows + warps - 1) / warps, 8), 1 << 20);
  ty = std::min(ty, g.ny);
  ty = std::max(ty, 1);
  pl->ty = ty;
  const int64_t chunks = (g.ny + ty - 1) / ty;
  const int64_t nt = (int64_t)pl->tiles_x * chunks;
  if (nt > INT_MAX / (ty + 4)) return false;
  pl->ntiles = (int)nt;
  const int64_t need_warps = std::min<int64_t>(nt, warps);
  pl->nblk = (int)std::max<int64_t>(1, (need_warps + WPB - 1) / WPB);
  return true;
}

template <bool INIT, int NS, int WPB>
void launch2d_t(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
                int set, cudaStream_t s) {
  const int a = set, o = 1 - set;
  k_cg2d<INIT, NS, WPB><<<pl.nblk, 32 * WPB, pl.smem, s>>>(
      pl.tm_r[a], pl.tm_p[a], pl.tm_s, g, cg, b.kx, pl.tiles_x, pl.ty, pl.ntiles, b.r[o],
      b.p[o], b.d, b.xref, b.st, b.part, b.nblk_part, b.px);
}

// 2D variant table (stages per warp, warps per block):
// 1 = (5, 5), 2 = (6, 4), 3 = (7, 4), 4 = (6, 7)
template <bool INIT>
void launch2d(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
              int set, cudaStream_t s) {
  switch (pl.variant) {
    case 2: launch2d_t<INIT, 6, 4>(pl, g, cg, b, set, s); break;
    case 3: launch2d_t<INIT, 7, 4>(pl, g, cg, b, set, s); break;
    case 4: launch2d_t<INIT, 6, 7>(pl, g, cg, b, set, s); break;
    default: launch2d_t<INIT, 5, 5>(pl, g, cg, b, set, s); break;
  }
}

bool plan2d(Cg32Plan *pl, const Grid &g, int num_sms) {
  switch (pl->variant) {
    case 2: return plan2d_t<6, 4>(pl, g, num_sms);
    case 3: return plan2d_t<7, 4>(pl, g, num_sms);
    case 4: return plan2d_t<6, 7>(pl, g, num_sms);
    default: pl->variant = 1; return plan2d_t<5, 5>(pl, g, num_sms);
  }
}

// 3D variants: (rows per tile TY, stages NS); shared memory: NS stages of
// three planes, a ring of three un planes and one of two (r_new, sig, p)
// planes, each (TY + 4) rows of 136 floats
template <int TY, int NS>
size_t smem3d() {
  return (size_t)(3 * NS + 3 + 6) * (TY + 4) * kWin * sizeof(float) + 128;
}

template <int TY, int NS>
bool plan3d_t(Cg32Plan *pl, const Grid &g, int num_sms) {
  const size_t sm = smem3d<TY, NS>();
  if (cudaFuncSetAttribute(k_cg3d<false, TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess ||
      cudaFuncSetAttribute(k_cg3d<true, TY, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess)
    return false;
  int per = 0, per_i = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg3d<false, TY, NS>, 32 * (TY + 4),
                                                    sm) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_i, k_cg3d<true, TY, NS>, 32 * (TY + 4),
                                                    sm) != cudaSuccess)
    return false;
  per = std::min(per, per_i);
  if (per < 1) return false;
  pl->ty = TY;
  pl->ns = NS;
  pl->wpb = TY + 4;
  pl->smem = sm;
  pl->tiles_x = (g.nx + kW - 1) / kW;
  pl->tiles_y = (g.ny + TY - 1) / TY;
  const int64_t plane_tiles = (int64_t)pl->tiles_x * pl->tiles_y;
  const int64_t slots = (int64_t)per * num_sms;
  // planes per tile: the fewest rounds over the resident blocks, each round
  // costing (zc + 4) plane steps; at least 8 planes
  int best_zc = std::max(8, g.nz);
  int64_t best_cost = INT64_MAX;
  for (int zc = 8; zc <= std::max(8, g.nz); ++zc) {
    const int64_t nt = plane_tiles * ((g.nz + zc - 1) / zc);
    const int64_t rounds = (nt + slots - 1) / slots;
    const int64_t cost = rounds * (zc + 4);
    if (cost < best_cost) {
      best_cost = cost;
      best_zc = zc;
    }
  }
  const int64_t nt = plane_tiles * ((g.nz + best_zc - 1) / best_zc);
  if (nt > INT_MAX / (best_zc + 4)) return false;
  pl->zc = best_zc;
  pl->ntiles = (int)nt;
  pl->nblk = (int)std::min<int64_t>(nt, slots);
  return true;
}

template <bool INIT, int TY, int NS>
void launch3d_t(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
                int set, cudaStream_t s) {
  const int a = set, o = 1 - set;
  k_cg3d<INIT, TY, NS><<<pl.nblk, 32 * (TY + 4), pl.smem, s>>>(
      pl.tm_r[a], pl.tm_p[a], pl.tm_s, g, cg, b.kx, pl.tiles_x, pl.tiles_y, pl.zc, pl.ntiles,
      b.r[o], b.p[o], b.d, b.xref, b.st, b.part, b.nblk_part, b.px);
}

// 3D variant table (TY, stages): 1 = (12, 5), 2 = (8, 6), 3 = (16, 4), 4 = (8, 8)
template <bool INIT>
void launch3d(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
              int set, cudaStream_t s) {
  switch (pl.variant) {
    case 2: launch3d_t<INIT, 8, 6>(pl, g, cg, b, set, s); break;
    case 3: launch3d_t<INIT, 16, 4>(pl, g, cg, b, set, s); break;
    case 4: launch3d_t<INIT, 8, 8>(pl, g, cg, b, set, s); break;
    default: launch3d_t<INIT, 12, 5>(pl, g, cg, b, set, s); break;
  }
}

bool plan3d(Cg32Plan *pl, const Grid &g, int num_sms) {
  switch (pl->variant) {
    case 2: return plan3d_t<8, 6>(pl, g, num_sms);
    case 3: return plan3d_t<16, 4>(pl, g, num_sms);
    case 4: return plan3d_t<8, 8>(pl, g, num_sms);
    default: pl->variant = 1; return plan3d_t<12, 5>(pl, g, num_sms);
  }
}

// packed batch: the 2D variants of the single-grid pass
template <int NS, int WPB>
bool plan2db_t(Cg32BatchPlan *pl, int num_sms) {
  const size_t sm = smem2d<NS, WPB>();
  if (cudaFuncSetAttribute(k_cg2d_batch<NS, WPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm) != cudaSuccess)
    return false;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cg2d_batch<NS, WPB>, 32 * WPB, sm) !=
          cudaSuccess ||
      per < 1)
    return false;
  pl->ns = NS;
  pl->wpb = WPB;
  pl->smem = sm;
  pl->nblk = per * num_sms;
  return true;
}

template <int NS, int WPB>
void launch2db_t(const Cg32BatchPlan &pl, const Cg32BatchBuffers &b, int set, cudaStream_t s) {
  k_cg2d_batch<NS, WPB><<<pl.nblk, 32 * WPB, pl.smem, s>>>(
      pl.tm_r[0], pl.tm_r[1], pl.tm_p[0], pl.tm_p[1], pl.tm_s, b.bi, b.st, b.act, b.pre, b.cnt,
      b.alive, b.bc, pl.ty, set, b.r[0], b.r[1], b.p[0], b.p[1], b.d, b.xref, b.part, b.part_cap,
      b.P, b.ring, b.ring_cap, b.done);
}

}  // namespace

int cg32_max_blocks(int ndim, int num_sms) { return 8 * num_sms; }

bool cg32_plan(Cg32Plan *pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
               int num_sms, int variant, const char **why) {
  pl->ndim = g.ndim;
  pl->variant = variant;
  *why = "";
  if (b.px % 4 != 0) {
    *why = "row pitch must be a multiple of 4";
    return false;
  }
  const bool planned = (g.ndim == 2) ? plan2d(pl, g, num_sms) : plan3d(pl, g, num_sms);
  if (!planned) {
    *why = "cannot configure the inner-CG kernels on this device";
    cudaGetLastError();
    return false;
  }
  if (pl->nblk > b.nblk_part) {
    *why = "partials buffer too small";
    return false;
  }
  bool ok = true;
  const int nz = (g.ndim == 3) ? g.nz : 0;
  const int bh = (g.ndim == 3) ? pl->ty + 4 : 1;
  for (int k = 0; k < 2; ++k) {
    ok = ok && encode_f32(&pl->tm_r[k], b.r[k], g.nx, b.px, g.ny, nz, kWin, bh, 1);
    ok = ok && encode_f32(&pl->tm_p[k], b.p[k], g.nx, b.px, g.ny, nz, kWin, bh, 1);
  }
  ok = ok && encode_f32(&pl->tm_s, b.s32, g.nx, b.px, g.ny, nz, kWin, bh, 1);
  if (!ok) *why = "cannot encode the TMA tensor maps";
  (void)cg;
  return ok;
}

void cg32_init(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
               int set, cudaStream_t s) {
  if (pl.ndim == 2)
    launch2d<true>(pl, g, cg, b, set, s);
  else
    launch3d<true>(pl, g, cg, b, set, s);
}

void cg32_iter(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
               int set, cudaStream_t s) {
  if (pl.ndim == 2)
    launch2d<false>(pl, g, cg, b, set, s);
  else
    launch3d<false>(pl, g, cg, b, set, s);
}

bool cg32_batch_plan(Cg32BatchPlan *pl, const Cg32BatchBuffers &b, int num_sms, int variant,
                     int ty, const char **why) {
  if (!encode_fn()) {
    *why = "cuTensorMapEncodeTiled is not available";
    return false;
  }
  if (ty < 1 || variant < 0 || variant > 4) {
    *why = "invalid batch tile shape";
    return false;
  }
  pl->variant = variant == 0 ? 1 : variant;
  pl->ty = ty;
  bool planned = false;
  switch (pl->variant) {
    case 2: planned = plan2db_t<6, 4>(pl, num_sms); break;
    case 3: planned = plan2db_t<7, 4>(pl, num_sms); break;
    case 4: planned = plan2db_t<6, 7>(pl, num_sms); break;
    default: planned = plan2db_t<5, 5>(pl, num_sms); break;
  }
  if (!planned) {
    *why = "cannot configure the packed inner-CG kernels on this device";
    cudaGetLastError();
    return false;
  }
  bool ok = true;
  for (int k = 0; k < 2; ++k) {
    ok = ok && encode_f32(&pl->tm_r[k], b.r[k], b.P, b.P, b.H, 0, kWin, 1, 1);
    ok = ok && encode_f32(&pl->tm_p[k], b.p[k], b.P, b.P, b.H, 0, kWin, 1, 1);
  }
  ok = ok && encode_f32(&pl->tm_s, b.s32, b.P, b.P, b.H, 0, kWin, 1, 1);
  if (!ok) *why = "cannot encode the atlas tensor maps";
  return ok;
}

void cg32_batch_pass(const Cg32BatchPlan &pl, const Cg32BatchBuffers &b, int set,
                     cudaStream_t s) {
  switch (pl.variant) {
    case 2: launch2db_t<6, 4>(pl, b, set, s); break;
    case 3: launch2db_t<7, 4>(pl, b, set, s); break;
    case 4: launch2db_t<6, 7>(pl, b, set, s); break;
    default: launch2db_t<5, 5>(pl, b, set, s); break;
  }
}

}  // namespace eik
