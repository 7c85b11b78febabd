// Mixed-precision solve (FP32 inner CG on the rescaled system, FP64
// iterative refinement): internal interface used by eik_api.cu.
#pragma once

#include "eik_internal.cuh"

namespace eik {

struct MixedState;

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

eik_status mixed_create(MixedState **out, const Grid &g, const TileCount &tc, int num_sms,
                        cudaStream_t s);
eik_status mixed_solve(MixedState *m, const MixedArgs &a, int *inner_iters, int *outer_iters,
                       double *res_cw, double *res_nw);
void mixed_destroy(MixedState *m);
const char *mixed_last_error();

}  // namespace eik
