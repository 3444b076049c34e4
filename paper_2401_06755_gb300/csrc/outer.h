// Launchers of the pointwise outer-loop kernels (outer.cu).
#pragma once

#include "internal.h"

namespace nn4 {

// x += e  (FP64 += inner type)
int launch_add_correction(nn4_dtype dt, double* x, const LevelGeom& g64, const void* e, const LevelGeom& gT,
                          cudaStream_t s);
// rT = (inner type) r
int launch_to_inner(nn4_dtype dt, const double* r, const LevelGeom& g64, void* rT, const LevelGeom& gT,
                    cudaStream_t s);
// invd = 1 / diag(A) for Eq. k-T from k and lk = L k (FP64)
int launch_inv_diag(const double* k, const double* lk, double* invd, const LevelGeom& g, double c0,
                    cudaStream_t s);
// out += sum of v^2 over free nodes
int launch_norm_masked(const double* v, const LevelGeom& g, double* out, cudaStream_t s);
// out += z . q
int launch_dot_zq(nn4_dtype dt, const void* z, const LevelGeom& gT, const double* q, const LevelGeom& g64,
                  double* out, cudaStream_t s);
// p = z - (zq / pq_old) p_old
int launch_new_direction(nn4_dtype dt, const void* z, const LevelGeom& gT, const double* p_old, double* p,
                         const LevelGeom& g64, const double* zq, const double* pq_old, cudaStream_t s);
// alpha = pr / pq; x += alpha p; r -= alpha q; rT = r (if rT); norm2 += r.r
int launch_fcg_update(nn4_dtype dt, double* x, double* r, const double* p, const double* q, const LevelGeom& g64,
                      void* rT, const LevelGeom& gT, const double* pr, const double* pq, double* norm2,
                      cudaStream_t s);

}  // namespace nn4
