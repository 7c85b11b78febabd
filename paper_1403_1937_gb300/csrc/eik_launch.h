// Host-side launch wrappers of the CUDA kernels (internal).
#pragma once

#include "eik_internal.cuh"

namespace eik {

TileCount tile_count(const Grid &g);
int stencil_grid_cap(int ndim, int num_sms);

void launch_setup64(const Grid &g, const double *f, double *sig, double *x, int *err,
                    cudaStream_t s, int cap);
void launch_sources64(const Grid &g, const int64_t *src, const double *U, int64_t nsrc,
                      double *sig, double *x, cudaStream_t s);
void launch_residual64(const Grid &g, const TileCount &tc, int nblk, const double *sig,
                       const double *x, const double *rhs, double *r, double *p,
                       CgState *st, double *part, int nblk_part, cudaStream_t s);
void launch_pass1_64(const Grid &g, const TileCount &tc, int nblk, const double *sig,
                     const double *r, const double *p, double *q, CgState *st,
                     double *part, int nblk_part, cudaStream_t s);
void launch_pass2_64(int64_t n, int nblk, double *x, double *r, double *p, const double *q,
                     const double *cw_weight, CgState *st, double *part, int nblk_part,
                     cudaStream_t s);
void launch_epilogue64(const Grid &g, const double *sig, const double *x, double *S,
                       double *phi, cudaStream_t s, int cap);
void launch_source_values(const int64_t *src, const double *U, int64_t nsrc, double *S,
                          cudaStream_t s);
void launch_adjoint_rhs64(const Grid &g, const double *sig, const double *x,
                          const double *dLdS, double *ghat, double *gmax_part, int nblk,
                          cudaStream_t s);
void launch_adjoint_grad64(const Grid &g, const double *f, const double *sig,
                           const double *x, const double *lam, double *dLdf,
                           cudaStream_t s, int cap);

}  // namespace eik
