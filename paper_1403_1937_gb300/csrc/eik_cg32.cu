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
// Per-block partials: <r,r> and <w,r> (both in units of 2^(2F + fd)), the
// largest |r| and |p| (frame units), and the componentwise-test flag.  The
// last block forms the next alpha, beta, frame and the stopping decision.
template <bool INIT>
__device__ void cg_tail(float gam, float dlt, float rmax, float pmax, int bad, bool fault,
                        MixCtl *st, double *part, int nblk_part) {
  __shared__ double sh[32];
  __shared__ int flag;
  for (int o = 16; o > 0; o >>= 1) {
    gam += __shfl_down_sync(0xffffffffu, gam, o);
    dlt += __shfl_down_sync(0xffffffffu, dlt, o);
    rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
    pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  __shared__ float wg[32], wd[32], wr[32], wp[32];
  __shared__ int wb[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (lane == 0) {
    wg[w] = gam;
    wd[w] = dlt;
    wr[w] = rmax;
    wp[w] = pmax;
    wb[w] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double G = 0.0, D = 0.0;
    float R = 0.f, P = 0.f;
    int Bd = 0;
    for (int k = 0; k < nwarp; ++k) {
      G += (double)wg[k];
      D += (double)wd[k];
      R = fmaxf(R, wr[k]);
      P = fmaxf(P, wp[k]);
      Bd |= wb[k];
    }
    part[0 * nblk_part + blockIdx.x] = G;
    part[1 * nblk_part + blockIdx.x] = D;
    part[2 * nblk_part + blockIdx.x] = (double)R;
    part[3 * nblk_part + blockIdx.x] = (double)P;
    part[4 * nblk_part + blockIdx.x] = (double)Bd;
    if (fault) atomicExch(&st->fault, 1);
  }
  if (!last_block(&st->counter[1], &flag)) return;
  const double G = sum_partials(part, gridDim.x, sh);
  const double D = sum_partials(part + nblk_part, gridDim.x, sh);
  const double R = max_partials(part + 2 * nblk_part, gridDim.x, sh);
  const double P = max_partials(part + 3 * nblk_part, gridDim.x, sh);
  const double Bd = max_partials(part + 4 * nblk_part, gridDim.x, sh);
  if (threadIdx.x != 0) return;
  st->counter[1] = 0u;
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
  if (!isfinite(G) || !isfinite(D) || !isfinite(R) || !isfinite(P)) {
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
    const double den = acc_ratio(dlt_new, gam_new) - beta_new / st->alpha;
    alpha_new = (den > 0.0 && isfinite(den)) ? 1.0 / den : -1.0;
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
// One warp owns tiles of 128 columns x TY rows.  The tile's rows, with a
// two-row halo, stream through a ring of NS shared-memory stages, one TMA row
// copy (136 columns from x0 - 4) per array and stage.  Lane l holds columns
// x0 + 4l .. x0 + 4l + 3; lanes 0 and 31 also carry the halo columns
// x0 - 2, x0 - 1 and x0 + 128, x0 + 129.  At step j (input row y_j):
//   row y_j:       p = r + beta p, u = sig p            (stage A)
//   row y_{j-1}:   s = A p, r_new = r - alpha s, un = sig r_new   (stage B)
//   row y_{j-2}:   w = A r_new, the dots, d += alpha p, stores    (stage C)
// Odd tile rows march upwards, so the halo rows two neighbouring tiles share
// are read at the same time (and come from L2 the second time).
template <bool INIT, int NS, int WPB>
__global__ void __launch_bounds__(32 * WPB, 1)
k_cg2d(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_p,
       const __grid_constant__ CUtensorMap tm_s, Grid g, CellGrid cg,
       const int *__restrict__ kx, int tiles_x, int TY, int ntiles,
       float *__restrict__ r_out, float *__restrict__ p_out, float *__restrict__ d,
       const float *__restrict__ xref, MixCtl *st, double *part, int nblk_part, int px) {
  constexpr int STAGE = 3 * kSlot;   // floats per stage: r, p, sigma rows
  extern __shared__ __align__(128) unsigned char cg2_raw[];
  __shared__ __align__(8) uint64_t bars[WPB * NS];
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
  float *sb = cg2_smem + (size_t)wib * NS * STAGE;
  uint64_t *bar = bars + wib * NS;

  int next_issue = 0;   // lane 0: next row of the warp's sequence to copy
  auto issue = [&](int q) {
    const int k = q / steps, j = q - k * steps;
    const int t = gw + k * nw;
    const int cyk = t / tiles_x;
    const int x0 = (t - cyk * tiles_x) * kW;
    const int y = (cyk & 1) ? (cyk * TY + TY + 1 - j) : (cyk * TY - 2 + j);
    float *dst = sb + (q % NS) * STAGE;
    uint64_t *b = bar + (q % NS);
    mbar_expect_tx(b, (INIT ? 2u : 3u) * kWin * 4u);
    tma_load_2d(dst, &tm_r, x0 - 4, y, b);
    if (!INIT) tma_load_2d(dst + kSlot, &tm_p, x0 - 4, y, b);
    tma_load_2d(dst + 2 * kSlot, &tm_s, x0 - 4, y, b);
  };
  if (lane == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bar[k], 1);
    mbar_init_fence();
    for (; next_issue < NS && next_issue < nq; ++next_issue)
      if (!(next_issue == 0 && withhold)) issue(next_issue);
  }
  __syncwarp();

  float gam = 0.f, dlt = 0.f, rmax = 0.f, pmax = 0.f;
  int bad = 0;
  bool fault = false;
  int q = 0;
  for (int k = 0; k < my_tiles && !fault; ++k) {
    const int t = gw + k * nw;
    const int cyk = t / tiles_x;
    const int x0 = (t - cyk * tiles_x) * kW;
    const int y0 = cyk * TY;
    const int dir = (cyk & 1) ? -1 : 1;
    const int ystart = (dir > 0) ? y0 - 2 : y0 + TY + 1;
    const int xl = x0 + 4 * lane;
    const bool l31 = lane == 31;
    float hx[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) hx[c] = (half && (xl + c == 0 || xl + c == g.nx - 1)) ? 0.5f : 1.f;
    const int xh = l31 ? x0 + kW : x0 - 1;   // inner halo column of lanes 0 / 31
    const float hxh = (half && (xh == 0 || xh == g.nx - 1)) ? 0.5f : 1.f;
    const int hcol = l31 ? kW + 4 : 2;       // staged column of the halo pair
    // cell columns: own, of column xl - 1 and of column xl + 4 (clamped)
    const int cmax = cg.cx - 1;
    const int cxo = min(xl >> cg.lgB, cmax);
    const int cxl = (xl >= 1) ? min((xl - 1) >> cg.lgB, cmax) : cxo;
    const int cxr = (xl + 4 < g.nx) ? min((xl + 4) >> cg.lgB, cmax) : cxo;
    const bool st_ok = xl < px;              // the float4 lies inside the row pitch

    // ring registers (lag 0 = row y_j, 1 = y_{j-1}, ...)
    float r0[4], p0[4], s0[4], u0[4];
    float r1[4] = {0, 0, 0, 0}, p1[4] = {0, 0, 0, 0}, s1[4] = {0, 0, 0, 0},
          u1[4] = {0, 0, 0, 0};
    float p2[4] = {0, 0, 0, 0}, s2[4] = {0, 0, 0, 0}, u2[4] = {0, 0, 0, 0};
    float rn1[4] = {0, 0, 0, 0}, rn2[4] = {0, 0, 0, 0};
    float un1[4] = {0, 0, 0, 0}, un2[4] = {0, 0, 0, 0}, un3[4] = {0, 0, 0, 0};
    float4 dq0 = make_float4(0, 0, 0, 0), dq1 = dq0, dq2 = dq0;
    float4 xq0 = dq0, xq1 = dq0, xq2 = dq0;
    float hr0, hp0, hs0, hu0, hou0;
    float hr1 = 0, hp1 = 0, hs1 = 0, hu1 = 0, hou1 = 0, hu2 = 0;
    float hun1 = 0, hun2 = 0;
    int K0c = 0, K0l = 0, K0r = 0, K1c = 0, K1l = 0, K1r = 0, K2c = 0, K2l = 0, K2r = 0,
        K3c = 0;
    int cr_last = INT_MIN;
    int kc_cache = 0, kl_cache = 0, kr_cache = 0;

    for (int j = 0; j < steps; ++j, ++q) {
      // ---- row y_j from the stage
      const int sidx = q % NS;
      // (a withheld first copy never lands: the bounded wait expires)
      bool ok = mbar_wait_bounded(&bar[sidx], (uint32_t)(q / NS) & 1u);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        fault = true;
        break;
      }
      const float *S = sb + sidx * STAGE;
      {
        const float4 rv = *reinterpret_cast<const float4 *>(S + 4 + 4 * lane);
        const float4 sv = *reinterpret_cast<const float4 *>(S + 2 * kSlot + 4 + 4 * lane);
        const float2 rh = *reinterpret_cast<const float2 *>(S + hcol);
        const float2 sh2 = *reinterpret_cast<const float2 *>(S + 2 * kSlot + hcol);
        r0[0] = rv.x; r0[1] = rv.y; r0[2] = rv.z; r0[3] = rv.w;
        s0[0] = sv.x; s0[1] = sv.y; s0[2] = sv.z; s0[3] = sv.w;
        // lane 0: (.x, .y) = (outer x0-2, inner x0-1); lane 31: (inner, outer)
        hr0 = l31 ? rh.x : rh.y;
        hs0 = l31 ? sh2.x : sh2.y;
        const float ro = l31 ? rh.y : rh.x, so = l31 ? sh2.y : sh2.x;
        if (!INIT) {
          const float4 pv = *reinterpret_cast<const float4 *>(S + kSlot + 4 + 4 * lane);
          const float2 ph = *reinterpret_cast<const float2 *>(S + kSlot + hcol);
          p0[0] = fmaf(beta, pv.x, r0[0]);
          p0[1] = fmaf(beta, pv.y, r0[1]);
          p0[2] = fmaf(beta, pv.z, r0[2]);
          p0[3] = fmaf(beta, pv.w, r0[3]);
          hp0 = fmaf(beta, l31 ? ph.x : ph.y, hr0);
          hou0 = so * fmaf(beta, l31 ? ph.y : ph.x, ro);
        } else {
          p0[0] = p0[1] = p0[2] = p0[3] = 0.f;
          hp0 = 0.f;
          hou0 = 0.f;
        }
        hu0 = hs0 * hp0;
#pragma unroll
        for (int c = 0; c < 4; ++c) u0[c] = s0[c] * p0[c];
      }
      // every lane is done with the stage: it takes row q + NS
      __syncwarp();
      if (lane == 0 && next_issue < nq) {
        fence_proxy_async();
        issue(next_issue);
        ++next_issue;
      }
      const int y = ystart + dir * j;
      // cell row of y_j (rows outside the grid use the nearest grid row)
      {
        const int cr = min(max(y, 0), g.ny - 1) >> cg.lgB;
        if (cr != cr_last) {
          cr_last = cr;
          kc_cache = __ldg(kx + cr * cg.cx + cxo);
          kl_cache = __ldg(kx + cr * cg.cx + cxl);
          kr_cache = __ldg(kx + cr * cg.cx + cxr);
        }
        K0c = kc_cache;
        K0l = kl_cache;
        K0r = kr_cache;
      }
      // prefetch d (and xref) of an output row for stage C two steps on
      const bool out_row = (j >= 2) && (j < TY + 2) && (y < g.ny);
      if (!INIT && out_row && st_ok) {
        const int64_t o = (int64_t)y * px + xl;
        dq0 = *reinterpret_cast<const float4 *>(d + o);
        if (check) xq0 = __ldg(reinterpret_cast<const float4 *>(xref + o));
      }

      // ---- stage B: row y_{j-1}
      if (j >= 2) {
        const int y1 = y - dir;
        const float hy1 = (half && (y1 == 0 || y1 == g.ny - 1)) ? 0.5f : 1.f;
        const int K1h = l31 ? K1r : K1l, K0h = l31 ? K0r : K0l, K2h = l31 ? K2r : K2l;
        const float fL = p2f(K1c - K1l), fR = p2f(K1c - K1r);
        const float fP = p2f(K1c - K2c), fN = p2f(K1c - K0c);
        float uL = __shfl_up_sync(0xffffffffu, u1[3], 1);
        float uR = __shfl_down_sync(0xffffffffu, u1[0], 1);
        if (lane == 0) uL = hu1;
        if (l31) uR = hu1;
        const float xs[4] = {fmaf(uL, fL, u1[1]), u1[0] + u1[2], u1[1] + u1[3],
                             fmaf(uR, fR, u1[2])};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (INIT) {
            rn1[c] = r1[c];
          } else {
            const float ys = fmaf(u2[c], fP, u0[c] * fN);
            const float acc = fmaf(hy1, xs[c], hx[c] * ys);
            const float sv = fmaf(-s1[c], acc, p1[c]);
            rn1[c] = fmaf(-alpha, sv, r1[c]);
          }
          un1[c] = s1[c] * rn1[c];
        }
        // halo column (lanes 0 / 31; other lanes compute a value nobody uses)
        float hrn = hr1;
        if (!INIT) {
          const float uadj = l31 ? u1[3] : u1[0];
          const float fxh = p2f(K1h - K1c), fPh = p2f(K1h - K2h), fNh = p2f(K1h - K0h);
          const float acc = fmaf(hy1, fmaf(uadj, fxh, hou1), hxh * fmaf(hu2, fPh, hu0 * fNh));
          hrn = fmaf(-alpha, fmaf(-hs1, acc, hp1), hr1);
        }
        hun1 = hs1 * hrn;
      }

      // ---- stage C: row y_{j-2}
      if (j >= 4) {
        const int y2 = y - 2 * dir;
        if (y2 < g.ny) {
          const float hy2 = (half && (y2 == 0 || y2 == g.ny - 1)) ? 0.5f : 1.f;
          const float fL = p2f(K2c - K2l), fR = p2f(K2c - K2r);
          const float fP = p2f(K2c - K3c), fN = p2f(K2c - K1c);
          const float W = p2f(-2 * K2c - fd);
          float uL = __shfl_up_sync(0xffffffffu, un2[3], 1);
          float uR = __shfl_down_sync(0xffffffffu, un2[0], 1);
          if (lane == 0) uL = hun2;
          if (l31) uR = hun2;
          const float xs[4] = {fmaf(uL, fL, un2[1]), un2[0] + un2[2], un2[1] + un2[3],
                               fmaf(uR, fR, un2[2])};
          const float dv[4] = {dq2.x, dq2.y, dq2.z, dq2.w};
          const float xv[4] = {xq2.x, xq2.y, xq2.z, xq2.w};
          float dn[4], ro[4], po[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float ys = fmaf(un3[c], fP, un1[c] * fN);
            const float acc = fmaf(hy2, xs[c], hx[c] * ys);
            const float wv = fmaf(-s2[c], acc, rn2[c]);
            const float tt = rn2[c] * W;
            gam = fmaf(tt, rn2[c], gam);
            dlt = fmaf(tt, wv, dlt);
            rmax = fmaxf(rmax, fabsf(rn2[c]));
            if (!INIT) {
              dn[c] = fmaf(alphaF, p2[c], dv[c]);
              pmax = fmaxf(pmax, fabsf(p2[c]));
              ro[c] = rn2[c] * gwr;
              po[c] = p2[c] * gwr;
              if (check && fabsf(rn2[c]) > thetaF * fabsf(xv[c] + dn[c])) bad = 1;
            }
          }
          if (!INIT && st_ok) {
            const int64_t o = (int64_t)y2 * px + xl;
            *reinterpret_cast<float4 *>(d + o) = make_float4(dn[0], dn[1], dn[2], dn[3]);
            *reinterpret_cast<float4 *>(r_out + o) = make_float4(ro[0], ro[1], ro[2], ro[3]);
            *reinterpret_cast<float4 *>(p_out + o) = make_float4(po[0], po[1], po[2], po[3]);
          }
        }
      }

      // ---- rotate the ring
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        un3[c] = un2[c];
        un2[c] = un1[c];
        rn2[c] = rn1[c];
        p2[c] = p1[c];
        s2[c] = s1[c];
        u2[c] = u1[c];
        r1[c] = r0[c];
        p1[c] = p0[c];
        s1[c] = s0[c];
        u1[c] = u0[c];
      }
      dq2 = dq1;
      dq1 = dq0;
      xq2 = xq1;
      xq1 = xq0;
      hun2 = hun1;
      hu2 = hu1;
      hr1 = hr0;
      hp1 = hp0;
      hs1 = hs0;
      hu1 = hu0;
      hou1 = hou0;
      K3c = K2c;
      K2c = K1c;
      K2l = K1l;
      K2r = K1r;
      K1c = K0c;
      K1l = K0l;
      K1r = K0r;
    }
  }
  if (fault && lane == 0) {
    // leave no copy in flight: wait (bounded) for every row issued and not
    // yet waited for
    for (int qq = q; qq < next_issue; ++qq)
      if (!(qq == 0 && withhold)) mbar_wait_bounded(&bar[qq % NS], (uint32_t)(qq / NS) & 1u);
  }
  __syncwarp();
  cg_tail<INIT>(gam, dlt, rmax, pmax, bad, fault, st, part, nblk_part);
}

// ------------------------------------------------------------------ 3D pass
// A block owns tiles of 128 columns x TY rows x zc planes and marches them
// through z.  Each plane of r, p and sigma arrives by one TMA copy per array
// (box 136 x (TY + 4) x 1 from (x0 - 4, y0 - 2, z)) into a ring of NS
// stages.  Warp w owns row y0 - 2 + w (TY + 4 warps) with lanes as in 2D.  At
// plane step j (plane z_j):
//   every warp, plane z_j:               p = r + beta p, u = sig p      (A)
//   warps 1 .. TY + 2, plane z_{j-1}:    s = A p, r_new, un = sig r_new (B)
//   warps 2 .. TY + 1, plane z_{j-2}:    w = A r_new, dots, d, stores   (C)
// The z neighbours of a node are in its own thread's registers, the x
// neighbours come by warp shuffle, the y neighbours through two shared rings
// (u of the last plane, un of the last plane); one block barrier per step
// orders them.  Odd z chunks march downwards (shared halo planes are read by
// both neighbours at the same time).
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
  constexpr int STAGE = 3 * PLANE;
  static_assert((PLANE * 4) % 128 == 0, "plane size");
  extern __shared__ __align__(128) unsigned char cg3_raw[];
  __shared__ __align__(8) uint64_t bars[NS];
  if (st->done) return;
  float *cg3_smem = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(cg3_raw) + 127) & ~uintptr_t(127));
  float *ring_u = cg3_smem + NS * STAGE;   // [2][NR][kWin]
  float *ring_n = ring_u + 2 * PLANE;      // [2][NR][kWin]
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
    mbar_expect_tx(b, (INIT ? 2u : 3u) * PLANE * 4u);
    tma_load_3d(dst, &tm_r, sx * kW - 4, sy * TY - 2, z, b);
    if (!INIT) tma_load_3d(dst + PLANE, &tm_p, sx * kW - 4, sy * TY - 2, z, b);
    tma_load_3d(dst + 2 * PLANE, &tm_s, sx * kW - 4, sy * TY - 2, z, b);
  };
  if (threadIdx.x == 0) {
    for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (; next_issue < NS && next_issue < nq; ++next_issue)
      if (!(next_issue == 0 && withhold)) issue(next_issue);

  const bool doB = (w >= 1 && w <= TY + 2), doC = (w >= 2 && w <= TY + 1);
  const bool l31 = lane == 31;
  const int hcol = l31 ? kW + 4 : 2;
  float gam = 0.f, dlt = 0.f, rmax = 0.f, pmax = 0.f;
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
    for (int c = 0; c < 4; ++c) hx[c] = (half && (xl + c == 0 || xl + c == g.nx - 1)) ? 0.5f : 1.f;
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

    float r0[4], p0[4], s0[4], u0[4];
    float r1[4] = {0, 0, 0, 0}, p1[4] = {0, 0, 0, 0}, s1[4] = {0, 0, 0, 0},
          u1[4] = {0, 0, 0, 0};
    float p2[4] = {0, 0, 0, 0}, s2[4] = {0, 0, 0, 0}, u2[4] = {0, 0, 0, 0};
    float rn1[4] = {0, 0, 0, 0}, rn2[4] = {0, 0, 0, 0};
    float un1[4] = {0, 0, 0, 0}, un2[4] = {0, 0, 0, 0}, un3[4] = {0, 0, 0, 0};
    float4 dq0 = make_float4(0, 0, 0, 0), dq1 = dq0, dq2 = dq0;
    float4 xq0 = dq0, xq1 = dq0, xq2 = dq0;
    float hr0, hp0, hs0, hu0, hou0;
    float hr1 = 0, hp1 = 0, hs1 = 0, hu1 = 0, hou1 = 0, hu2 = 0, hun1 = 0, hun2 = 0;
    // cell exponents: own column (lags 0..3), halo column (lags 0..2)
    int K0 = 0, K1 = 0, K2 = 0, K3 = 0, H0 = 0, H1 = 0, H2 = 0;
    // x / y factors, recomputed when a stage's plane enters another cell layer
    int lay_B = INT_MIN, lay_C = INT_MIN, lay_A = INT_MIN;
    float bL = 1, bR = 1, bS = 1, bN = 1, bxh = 1, bhS = 1, bhN = 1;
    float cL = 1, cR = 1, cS = 1, cN = 1, cW = 0;
    int kA = 0, hA = 0;

    for (int j = 0; j < steps; ++j, ++q) {
      const int sidx = q % NS;
      const bool okw = mbar_wait_bounded(&bars[sidx], (uint32_t)(q / NS) & 1u);
      if (__syncthreads_or(!okw)) {
        fault = true;
        break;
      }
      const int z = zstart + dir * j;
      const float *S = cg3_smem + sidx * STAGE + w * kWin;
      // ---- A: plane z_j, row y
      {
        const float4 rv = *reinterpret_cast<const float4 *>(S + 4 + 4 * lane);
        const float4 sv = *reinterpret_cast<const float4 *>(S + 2 * PLANE + 4 + 4 * lane);
        const float2 rh = *reinterpret_cast<const float2 *>(S + hcol);
        const float2 sh2 = *reinterpret_cast<const float2 *>(S + 2 * PLANE + hcol);
        r0[0] = rv.x; r0[1] = rv.y; r0[2] = rv.z; r0[3] = rv.w;
        s0[0] = sv.x; s0[1] = sv.y; s0[2] = sv.z; s0[3] = sv.w;
        hr0 = l31 ? rh.x : rh.y;
        hs0 = l31 ? sh2.x : sh2.y;
        const float ro = l31 ? rh.y : rh.x, so = l31 ? sh2.y : sh2.x;
        if (!INIT) {
          const float4 pv = *reinterpret_cast<const float4 *>(S + PLANE + 4 + 4 * lane);
          const float2 ph = *reinterpret_cast<const float2 *>(S + PLANE + hcol);
          p0[0] = fmaf(beta, pv.x, r0[0]);
          p0[1] = fmaf(beta, pv.y, r0[1]);
          p0[2] = fmaf(beta, pv.z, r0[2]);
          p0[3] = fmaf(beta, pv.w, r0[3]);
          hp0 = fmaf(beta, l31 ? ph.x : ph.y, hr0);
          hou0 = so * fmaf(beta, l31 ? ph.y : ph.x, ro);
        } else {
          p0[0] = p0[1] = p0[2] = p0[3] = 0.f;
          hp0 = 0.f;
          hou0 = 0.f;
        }
        hu0 = hs0 * hp0;
#pragma unroll
        for (int c = 0; c < 4; ++c) u0[c] = s0[c] * p0[c];
        if (!INIT) {
          float *U = ring_u + (j & 1) * PLANE + w * kWin;
          *reinterpret_cast<float4 *>(U + 4 + 4 * lane) = make_float4(u0[0], u0[1], u0[2], u0[3]);
          if (lane == 0 || l31) U[l31 ? kW + 4 : 3] = hu0;
        }
        const int lay = min(max(z, 0), g.nz - 1) >> cg.lgB;
        if (lay != lay_A) {
          lay_A = lay;
          kA = cell_k(cg, kx, cxo, y, z, g);
          hA = cell_k(cg, kx, cxh, y, z, g);
        }
        K0 = kA;
        H0 = hA;
        if (!INIT && doC && row_ok && j >= 2 && j < zc + 2 && z < g.nz && xl < px) {
          const int64_t o = ((int64_t)z * g.ny + y) * px + xl;
          dq0 = *reinterpret_cast<const float4 *>(d + o);
          if (check) xq0 = __ldg(reinterpret_cast<const float4 *>(xref + o));
        }
      }
      // ---- B: plane z_{j-1}
      if (j >= 2 && doB) {
        const int z1 = z - dir;
        const int lay = min(max(z1, 0), g.nz - 1) >> cg.lgB;
        if (lay != lay_B) {
          lay_B = lay;
          const int kc = cell_k(cg, kx, cxo, y, z1, g), kh = cell_k(cg, kx, cxh, y, z1, g);
          bL = p2f(kc - cell_k(cg, kx, cxl, y, z1, g));
          bR = p2f(kc - cell_k(cg, kx, cxr, y, z1, g));
          bS = p2f(kc - cell_k(cg, kx, cxo, y - 1, z1, g));
          bN = p2f(kc - cell_k(cg, kx, cxo, y + 1, z1, g));
          bxh = p2f(kh - kc);
          bhS = p2f(kh - cell_k(cg, kx, cxh, y - 1, z1, g));
          bhN = p2f(kh - cell_k(cg, kx, cxh, y + 1, z1, g));
        }
        if (INIT) {
#pragma unroll
          for (int c = 0; c < 4; ++c) rn1[c] = r1[c];
          hun1 = hs1 * hr1;
        } else {
          const float hz1 = (half && (z1 == 0 || z1 == g.nz - 1)) ? 0.5f : 1.f;
          const float fP = p2f(K1 - K2), fN = p2f(K1 - K0);
          const float *Us = ring_u + ((j - 1) & 1) * PLANE + (w - 1) * kWin;
          const float *Un = Us + 2 * kWin;
          const float4 us = *reinterpret_cast<const float4 *>(Us + 4 + 4 * lane);
          const float4 un = *reinterpret_cast<const float4 *>(Un + 4 + 4 * lane);
          const float ysv[4] = {us.x, us.y, us.z, us.w}, ynv[4] = {un.x, un.y, un.z, un.w};
          float uL = __shfl_up_sync(0xffffffffu, u1[3], 1);
          float uR = __shfl_down_sync(0xffffffffu, u1[0], 1);
          if (lane == 0) uL = hu1;
          if (l31) uR = hu1;
          const float xs[4] = {fmaf(uL, bL, u1[1]), u1[0] + u1[2], u1[1] + u1[3],
                               fmaf(uR, bR, u1[2])};
          const float wxe = hy * hz1;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float ys = fmaf(ysv[c], bS, ynv[c] * bN);
            const float zs = fmaf(u2[c], fP, u0[c] * fN);
            const float acc = fmaf(wxe, xs[c], hx[c] * fmaf(hz1, ys, hy * zs));
            const float sv = fmaf(-s1[c], acc, p1[c]);
            rn1[c] = fmaf(-alpha, sv, r1[c]);
          }
          // halo column
          const float hyS = Us[l31 ? kW + 4 : 3], hyN = Un[l31 ? kW + 4 : 3];
          const float uadj = l31 ? u1[3] : u1[0];
          const float fPh = p2f(H1 - H2), fNh = p2f(H1 - H0);
          const float acc = fmaf(wxe, fmaf(uadj, bxh, hou1),
                                 hxh * fmaf(hz1, fmaf(hyS, bhS, hyN * bhN),
                                            hy * fmaf(hu2, fPh, hu0 * fNh)));
          hun1 = hs1 * fmaf(-alpha, fmaf(-hs1, acc, hp1), hr1);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) un1[c] = s1[c] * rn1[c];
        float *N = ring_n + ((j - 1) & 1) * PLANE + w * kWin;
        *reinterpret_cast<float4 *>(N + 4 + 4 * lane) = make_float4(un1[0], un1[1], un1[2], un1[3]);
        if (lane == 0 || l31) N[l31 ? kW + 4 : 3] = hun1;
      }
      // ---- C: plane z_{j-2}
      if (j >= 4 && doC) {
        const int z2 = z - 2 * dir;
        if (z2 < g.nz && row_ok) {
          const int lay = z2 >> cg.lgB;
          if (lay != lay_C) {
            lay_C = lay;
            const int kc = cell_k(cg, kx, cxo, y, z2, g);
            cL = p2f(kc - cell_k(cg, kx, cxl, y, z2, g));
            cR = p2f(kc - cell_k(cg, kx, cxr, y, z2, g));
            cS = p2f(kc - cell_k(cg, kx, cxo, y - 1, z2, g));
            cN = p2f(kc - cell_k(cg, kx, cxo, y + 1, z2, g));
            cW = p2f(-2 * kc - fd);
          }
          const float hz2 = (half && (z2 == 0 || z2 == g.nz - 1)) ? 0.5f : 1.f;
          const float fP = p2f(K2 - K3), fN = p2f(K2 - K1);
          const float *Ns = ring_n + ((j - 2) & 1) * PLANE + (w - 1) * kWin;
          const float *Nn = Ns + 2 * kWin;
          const float4 ns = *reinterpret_cast<const float4 *>(Ns + 4 + 4 * lane);
          const float4 nn = *reinterpret_cast<const float4 *>(Nn + 4 + 4 * lane);
          const float ysv[4] = {ns.x, ns.y, ns.z, ns.w}, ynv[4] = {nn.x, nn.y, nn.z, nn.w};
          float uL = __shfl_up_sync(0xffffffffu, un2[3], 1);
          float uR = __shfl_down_sync(0xffffffffu, un2[0], 1);
          if (lane == 0) uL = hun2;
          if (l31) uR = hun2;
          const float xs[4] = {fmaf(uL, cL, un2[1]), un2[0] + un2[2], un2[1] + un2[3],
                               fmaf(uR, cR, un2[2])};
          const float wxe = hy * hz2;
          const float dv[4] = {dq2.x, dq2.y, dq2.z, dq2.w};
          const float xv[4] = {xq2.x, xq2.y, xq2.z, xq2.w};
          float dn[4], ro[4], po[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const float ys = fmaf(ysv[c], cS, ynv[c] * cN);
            const float zs = fmaf(un3[c], fP, un1[c] * fN);
            const float acc = fmaf(wxe, xs[c], hx[c] * fmaf(hz2, ys, hy * zs));
            const float wv = fmaf(-s2[c], acc, rn2[c]);
            const float tt = rn2[c] * cW;
            gam = fmaf(tt, rn2[c], gam);
            dlt = fmaf(tt, wv, dlt);
            rmax = fmaxf(rmax, fabsf(rn2[c]));
            if (!INIT) {
              dn[c] = fmaf(alphaF, p2[c], dv[c]);
              pmax = fmaxf(pmax, fabsf(p2[c]));
              ro[c] = rn2[c] * gwr;
              po[c] = p2[c] * gwr;
              if (check && fabsf(rn2[c]) > thetaF * fabsf(xv[c] + dn[c])) bad = 1;
            }
          }
          if (!INIT && st_ok) {
            const int64_t o = ((int64_t)z2 * g.ny + y) * px + xl;
            *reinterpret_cast<float4 *>(d + o) = make_float4(dn[0], dn[1], dn[2], dn[3]);
            *reinterpret_cast<float4 *>(r_out + o) = make_float4(ro[0], ro[1], ro[2], ro[3]);
            *reinterpret_cast<float4 *>(p_out + o) = make_float4(po[0], po[1], po[2], po[3]);
          }
        }
      }
      // every warp is done with this plane's stage and with the ring slots
      // the next step overwrites
      __syncthreads();
      if (threadIdx.x == 0 && next_issue < nq) {
        fence_proxy_async();
        issue(next_issue);
        ++next_issue;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        un3[c] = un2[c];
        un2[c] = un1[c];
        rn2[c] = rn1[c];
        p2[c] = p1[c];
        s2[c] = s1[c];
        u2[c] = u1[c];
        r1[c] = r0[c];
        p1[c] = p0[c];
        s1[c] = s0[c];
        u1[c] = u0[c];
      }
      dq2 = dq1;
      dq1 = dq0;
      xq2 = xq1;
      xq1 = xq0;
      hun2 = hun1;
      hu2 = hu1;
      hr1 = hr0;
      hp1 = hp0;
      hs1 = hs0;
      hu1 = hu0;
      hou1 = hou0;
      K3 = K2;
      K2 = K1;
      K1 = K0;
      H2 = H1;
      H1 = H0;
    }
  }
  if (fault) {
    if (threadIdx.x == 0)
      for (int qq = q; qq < next_issue; ++qq)
        if (!(qq == 0 && withhold)) mbar_wait_bounded(&bars[qq % NS], (uint32_t)(qq / NS) & 1u);
    __syncthreads();
  }
  cg_tail<INIT>(gam, dlt, rmax, pmax, bad, fault, st, part, nblk_part);
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
  return (size_t)WPB * NS * 3 * kSlot * sizeof(float) + 128;
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
      pl.tm_r[a], pl.tm_p[a], pl.tm_s, g, cg, b.kx, pl.tiles_x, pl.ty, pl.ntiles, b.r[o], b.p[o],
      b.d, b.xref, b.st, b.part, b.nblk_part, b.px);
}

// 2D variant table: 1 = (8 stages, 8 warps), 2 = (6, 8), 3 = (8, 4), 4 = (12, 4)
template <bool INIT>
void launch2d(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
              int set, cudaStream_t s) {
  switch (pl.variant) {
    case 2: launch2d_t<INIT, 6, 8>(pl, g, cg, b, set, s); break;
    case 3: launch2d_t<INIT, 8, 4>(pl, g, cg, b, set, s); break;
    case 4: launch2d_t<INIT, 12, 4>(pl, g, cg, b, set, s); break;
    default: launch2d_t<INIT, 8, 8>(pl, g, cg, b, set, s); break;
  }
}

bool plan2d(Cg32Plan *pl, const Grid &g, int num_sms) {
  switch (pl->variant) {
    case 2: return plan2d_t<6, 8>(pl, g, num_sms);
    case 3: return plan2d_t<8, 4>(pl, g, num_sms);
    case 4: return plan2d_t<12, 4>(pl, g, num_sms);
    default: pl->variant = 1; return plan2d_t<8, 8>(pl, g, num_sms);
  }
}

// 3D variants: (rows per tile TY, stages NS); smem: NS stages of three
// arrays plus the two rings, each (TY + 4) rows of 136 floats
template <int TY, int NS>
size_t smem3d() {
  return (size_t)(3 * NS + 4) * (TY + 4) * kWin * sizeof(float) + 128;
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

// 3D variant table: 1 = (TY 8, 4 stages), 2 = (12, 4), 3 = (4, 4), 4 = (8, 3)
template <bool INIT>
void launch3d(const Cg32Plan &pl, const Grid &g, const CellGrid &cg, const Cg32Buffers &b,
              int set, cudaStream_t s) {
  switch (pl.variant) {
    case 2: launch3d_t<INIT, 12, 4>(pl, g, cg, b, set, s); break;
    case 3: launch3d_t<INIT, 4, 4>(pl, g, cg, b, set, s); break;
    case 4: launch3d_t<INIT, 8, 3>(pl, g, cg, b, set, s); break;
    default: launch3d_t<INIT, 8, 4>(pl, g, cg, b, set, s); break;
  }
}

bool plan3d(Cg32Plan *pl, const Grid &g, int num_sms) {
  switch (pl->variant) {
    case 2: return plan3d_t<12, 4>(pl, g, num_sms);
    case 3: return plan3d_t<4, 4>(pl, g, num_sms);
    case 4: return plan3d_t<8, 3>(pl, g, num_sms);
    default: pl->variant = 1; return plan3d_t<8, 4>(pl, g, num_sms);
  }
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

}  // namespace eik
