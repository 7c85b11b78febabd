// Mixed-precision solve (FP32 inner CG on the rescaled system, FP64
// iterative refinement): internal interface used by eik_api.cu.
#pragma once

#include "eik_internal.cuh"

namespace eik {

struct MixedState;
struct BatchExec;

struct MixedArgs {
  Grid g;
  TileCount tc;
  cudaStream_t stream;
  const double *f;
  double *sig;          // FP64 scaled coefficients (sources: 0)
  double *x;            // FP64 solution xh (sources: slots)
  double *r;            // FP64 scratch (true residual)
  double *aux;          // FP64 scratch
  double *part;
  int nblk_part;
  int nblk_stencil;
  CgState *st;
  CgState *h_st;
  const int64_t *src;
  const double *U;
  int64_t nsrc;
  eik_options opt;
};

// precond: EIK_PRECOND_* of the inner solve.
eik_status mixed_create(MixedState **out, const Grid &g, const TileCount &tc, int num_sms,
                        int tile_override, int precond, cudaStream_t s);
// A member of a packed 2D batch: its FP32 inner-CG arrays and control block
// are instance idx's in the batch's atlas, and its inner solves run through
// the batch (eik_batch.h).
eik_status mixed_create_member(MixedState **out, const Grid &g, const TileCount &tc,
                               int num_sms, BatchExec *batch, int idx, cudaStream_t s);
eik_status mixed_solve(MixedState *m, const MixedArgs &a, int *inner_iters, int *outer_iters,
                       double *res_cw, double *res_nw);
// Writes S (and phi if non-null) from the refined iterate; device pointers.
eik_status mixed_write_outputs(MixedState *m, const MixedArgs &a, double *S, double *phi);
// Writes the refined solution in hat-space FP64 (phi = s * xh) to xh.
eik_status mixed_export_hat(MixedState *m, const MixedArgs &a, double *xh);
void mixed_destroy(MixedState *m);
int64_t mixed_kernel_launches(const MixedState *m, int k);
void mixed_reset_launches(MixedState *m);
void mixed_set_profiling(MixedState *m, bool on);
void mixed_kernel_time(const MixedState *m, int k, int64_t *timed, double *ms);
const char *mixed_last_error();
// Name of mixed-mode kernel k (0-based), or NULL past the last one.
const char *mixed_kernel_name(int k);

}  // namespace eik
