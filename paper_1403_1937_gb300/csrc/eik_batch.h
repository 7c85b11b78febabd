// Packed 2D mixed-precision batches (internal): the atlas of FP32 arrays that
// all instances share, the batched inner-CG passes over every instance's
// tiles, and the rendezvous that lets each instance keep its own refinement
// program (FP64 residual, correction update, level-set bands) while its inner
// solves run together with the other instances' in one launch per pass.
#pragma once

#include <stdint.h>

#include <string>

#include "eik_cg32.h"

namespace eik {

struct BatchExec;

// Instance i's FP32 arrays in the atlas (offset to its row y = 0; row pitch
// P) and its control block.
struct BatchMember {
  float *r0, *p0, *s32, *d, *xref;
  int P;
  MixCtl *st;
};

// Atlas and executor for `count` 2D instances of extents nx[i] x ny[i].
// variant (0..4) and ty (rows per tile) fix the packed pass's tile shape; 0
// for either lets the autotuner choose it at the first solve (measured on
// the batch and cached on disk, keyed by GPU and size class).
eik_status batch_exec_create(BatchExec **out, int count, const int *nx, const int *ny,
                             int boundary, int num_sms, int variant, int ty);
void batch_exec_destroy(BatchExec *e);
BatchMember batch_exec_member(BatchExec *e, int i);
// The cell grid and exponents of instance i (device pointer, owned by it).
void batch_exec_set_cells(BatchExec *e, int i, const CellGrid &cg, const int *kx);

// One solve of the whole batch: `live` instance programs then run
// concurrently (one host thread each); each calls batch_exec_inner for every
// inner solve and batch_exec_leave when it ends, and batch_exec_end follows
// once they have all returned.  Meanwhile an executor thread keeps launching
// graphs of packed passes while any instance iterates or waits to join:
// an inner solve joins the tile list at the next pass boundary and leaves it
// when it ends, independently of the other instances.
eik_status batch_exec_begin(BatchExec *e, int live);
// Request number for instance i's next inner solve (goes into MixCtl.seq,
// with MixCtl.first = 1, before the control block is copied to the device).
int batch_exec_ticket(BatchExec *e, int i);
// Instance i's inner solve, its control block (seq, first) and starting
// residual in place on the device: returns when it has ended, with the
// outcome in *out (iter, status, stalled, alpha, beta, F).
eik_status batch_exec_inner(BatchExec *e, int i, int seq, MixCtl *out);
void batch_exec_leave(BatchExec *e, int i);
eik_status batch_exec_end(BatchExec *e);

// Tile shape in use: variant, rows per tile, and how it was chosen (0 fixed
// by the caller, 1 measured, 2 read from the cache file).
void batch_exec_plan(const BatchExec *e, int *variant, int *ty, int *how);
// Packed passes that had work since the executor was created (the
// autotuner's included).
int64_t batch_exec_passes(const BatchExec *e);
// Solves only (not the autotuner): the sum over passes of the nodes each
// covered, and the device time of the graphs that ran them (CUDA events).
void batch_exec_work(const BatchExec *e, int64_t *node_passes, double *ms);
std::string batch_exec_error(const BatchExec *e);

}  // namespace eik
