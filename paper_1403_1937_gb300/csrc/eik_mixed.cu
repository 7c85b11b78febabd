// Mixed-precision solve: placeholder until the FP32 kernels land.
#include "eik_mixed.h"

namespace eik {

struct MixedState {
  int dummy;
};

static const char *g_msg = "mixed precision is not available in this build";

eik_status mixed_create(MixedState **out, const Grid &, const TileCount &, int, cudaStream_t) {
  *out = nullptr;
  return EIK_ERR_ARG;
}
eik_status mixed_solve(MixedState *, const MixedArgs &, int *, int *, double *, double *) {
  return EIK_ERR_ARG;
}
void mixed_destroy(MixedState *m) { delete m; }
const char *mixed_last_error() { return g_msg; }

}  // namespace eik
