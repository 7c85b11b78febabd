// Multigrid-preconditioned FP32 inner solve of the mixed-precision path, 2D
// (internal).  Relative-form aggregation multigrid: see eik_mg.cu.
#pragma once

#include "eik_cg32.h"

namespace eik {

struct MgState;

// The mixed solver's level-0 arrays (pitched FP32 / cell exponents).
struct MgFine {
  float *r;            // residual of the correction equation (kx units); updated
  float *d;            // correction (kx units); updated
  const float *xref;   // FP32 copy of the iterate (kx units), componentwise test
  const float *s32;    // sigma (0 on the sources)
  const int *kx;       // cell exponents
  const float *St;     // cell distance estimate (S units)
};

eik_status mg_create(MgState **out, const Grid &g, const CellGrid &cg, int px, int num_sms,
                     cudaStream_t s);
// Per solve: the prolongation weights of level 0 and the Galerkin operators of
// every coarser level.  kmin = smallest cell exponent (reference of the
// inner-product weights).
eik_status mg_setup(MgState *mg, const MgFine &f, int kmin, cudaStream_t s);
// One inner solve of a refinement step.  Reads mode, thresh, theta and
// max_iter from *h_st and returns iter, status, stalled and done there.
eik_status mg_inner(MgState *mg, const MgFine &f, MixCtl *h_st, cudaStream_t s);
void mg_destroy(MgState *mg);
int mg_levels(const MgState *mg);
int64_t mg_launches(const MgState *mg);
// Profiling: CUDA events around every graph launch; mg_time returns the
// iterations so timed and their device milliseconds.
void mg_set_profiling(MgState *mg, bool on);
void mg_time(const MgState *mg, int64_t *iters, double *ms);
void mg_reset(MgState *mg);
const char *mg_last_error();

}  // namespace eik
