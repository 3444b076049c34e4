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
// invd = 1 / diag(A) for Eq. k-T from k and lk = (1/2) L k (FP64)
int launch_inv_diag(const double* k, const double* lk, double* invd, const LevelGeom& g, double c0,
                    cudaStream_t s);
// Device scalars: p[a], p[b], p[c], p[d] = 0 (negative indices skipped), then p[dst] = p[src] if
// dst >= 0; one launch
int launch_scalars(double* p, int a, int b, int c, int d, int dst, int src, cudaStream_t s);
// r = b at free nodes, 0 at Dirichlet nodes
int launch_masked_copy(const double* b, double* r, const LevelGeom& g, cudaStream_t s);
// out += sum of v^2 over all nodes
int launch_sumsq(const double* v, const LevelGeom& g, double* out, cudaStream_t s);
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

// Generic-precision forms (vectors V in FP64 or FP32; z / rT in any storage type).
int launch_dot(nn4_dtype tz, const void* z, const LevelGeom& gz, nn4_dtype tv, const void* q, const LevelGeom& gv,
               double* out, cudaStream_t s);
int launch_direction(nn4_dtype tz, const void* z, const LevelGeom& gz, nn4_dtype tv, const void* p_old, void* p,
                     const LevelGeom& gv, const double* zq, const double* pq_old, cudaStream_t s);
int launch_update(nn4_dtype tv, void* x, void* r, const void* p, const void* q, const LevelGeom& gv, nn4_dtype tr,
                  void* rT, const LevelGeom& gT, const double* pr, const double* pq, double* norm2, cudaStream_t s);
int launch_convert(nn4_dtype ta, const void* a, const LevelGeom& ga, nn4_dtype tb, void* b, const LevelGeom& gb,
                   cudaStream_t s);

}  // namespace nn4
