// Host side of the C ABI for the single multigrid steps: argument validation, TMA tensor maps,
// error reporting, and the launch of the stencil / transfer kernels.
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nn4 {

namespace {
thread_local std::string t_last_error;
}

int set_error(int code, const std::string& msg) {
  if (code != NN4_OK) t_last_error = msg;
  return code;
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NN4_OK;
  return set_error(e == cudaErrorMemoryAllocation ? NN4_ENOMEM : NN4_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

size_t dtype_size(nn4_dtype dt) { return dt == NN4_F64 ? 8 : (dt == NN4_F32 ? 4 : 2); }

int sm_count() {
  static std::mutex mu;
  static int counts[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lock(mu);
  if (counts[dev] == 0) {
    int n = 0;
    counts[dev] = (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0) ? n : 152;
  }
  return counts[dev];
}

long long resident_grid(const void* kern, int threads, size_t smem, long long want) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void*, int>, int>> cache;  // (kernel, threads) -> blocks/SM
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : cache)
      if (e.first.first == kern && e.first.second == threads) per_sm = e.second;
    if (per_sm == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
      cache.push_back({{kern, threads}, per_sm});
    }
  }
  const long long cap = (long long)per_sm * sm_count();
  return want < 1 ? 1 : (want < cap ? want : cap);
}

Coef8 stencil_coef(const double h[3]) {
  // Interior Q1 stiffness = K(x)M(y)M(z) + M(x)K(y)M(z) + M(x)M(y)K(z) with the 1D stencils
  // K = [-1, 2, -1] / h and M = [1, 4, 1] h / 6 (element integrals of linear basis functions).
  const double F[2] = {2.0, -1.0}, G[2] = {4.0, 1.0};
  const double ax = h[1] * h[2] / (36.0 * h[0]);
  const double ay = h[0] * h[2] / (36.0 * h[1]);
  const double az = h[0] * h[1] / (36.0 * h[2]);
  Coef8 c;
  for (int t = 0; t < 8; ++t) {
    const int a = t & 1, b = (t >> 1) & 1, z = (t >> 2) & 1;
    c.c[t] = ax * F[a] * G[b] * G[z] + ay * G[a] * F[b] * G[z] + az * G[a] * G[b] * F[z];
  }
  return c;
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

bool make_tmap_3d(CUtensorMap* map, nn4_dtype dt, const void* base, int nx, int ny, int nz,
                  long long pitch, int box_x, int box_y) {
  auto enc = get_encode();
  if (!enc) return false;
  const size_t es = dtype_size(dt);
  CUtensorMapDataType ty = dt == NN4_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : dt == NN4_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * es), (cuuint64_t)(pitch * es * ny)};
  cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, ty, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_tmap_stack(CUtensorMap* map, nn4_dtype dt, const void* base, int nx, int ny, int nz, int nw,
                     long long pitch, int box_x, int box_y, int box_w) {
  auto enc = get_encode();
  if (!enc) return false;
  const size_t es = dtype_size(dt);
  CUtensorMapDataType ty = dt == NN4_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                           : dt == NN4_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)nw};
  cuuint64_t strides[3] = {(cuuint64_t)(pitch * es), (cuuint64_t)(pitch * es * ny),
                           (cuuint64_t)(pitch * es * ny * nz)};
  cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, (cuuint32_t)box_w};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(map, ty, 4, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------- validation
int validate_grid(const nn4_grid* g, nn4_dtype dt, int min_n) {
  if (!g) return set_error(NN4_EINVAL, "grid is NULL");
  if (dt != NN4_F64 && dt != NN4_F32 && dt != NN4_BF16) return set_error(NN4_EINVAL, "bad dtype");
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < min_n) return set_error(NN4_EINVAL, "grid needs at least " + std::to_string(min_n) + " nodes per axis");
    if (g->n[d] > (1 << 20)) return set_error(NN4_EINVAL, "grid axis too large");
    if (!(g->h[d] > 0.0)) return set_error(NN4_EINVAL, "grid spacing must be positive");
  }
  for (int f = 0; f < 6; ++f)
    if (g->bc[f] != NN4_BC_DIRICHLET && g->bc[f] != NN4_BC_NATURAL) return set_error(NN4_EINVAL, "bad face condition");
  if (g->pitch < g->n[0]) return set_error(NN4_EINVAL, "pitch smaller than nx");
  if ((g->pitch * (long long)dtype_size(dt)) % 16 != 0)
    return set_error(NN4_EINVAL, "pitch * element size must be a multiple of 16 bytes");
  return NN4_OK;
}

int validate_ptr(const void* p, const char* name) {
  if (!p) return set_error(NN4_EINVAL, std::string(name) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return set_error(NN4_EINVAL, std::string(name) + " is not 16-byte aligned");
  return NN4_OK;
}

LevelGeom geom_of(const nn4_grid* g) {
  LevelGeom G;
  G.nx = g->n[0];
  G.ny = g->n[1];
  G.nz = g->n[2];
  G.pitch = g->pitch;
  for (int f = 0; f < 6; ++f) G.dir[f] = g->bc[f] == NN4_BC_DIRICHLET ? 1 : 0;
  return G;
}

LevelGeom coarse_geom(const LevelGeom& f, nn4_dtype dt) {
  LevelGeom c = f;
  c.nx = (f.nx + 1) / 2;
  c.ny = (f.ny + 1) / 2;
  c.nz = (f.nz + 1) / 2;
  c.pitch = nn4_row_pitch(c.nx, dt);
  return c;
}

}  // namespace nn4

using namespace nn4;

extern "C" {

int64_t nn4_row_pitch(int32_t nx, nn4_dtype dt) {
  if (nx <= 0 || (dt != NN4_F64 && dt != NN4_F32 && dt != NN4_BF16)) return -1;
  const int64_t per = 128 / (int64_t)dtype_size(dt);
  return (nx + per - 1) / per * per;
}

const char* nn4_last_error(void) { return t_last_error.c_str(); }

const char* nn4_version(void) { return "nn4-gb300 0.1 (sm_103a)"; }

int nn4_device_error(void) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return check_cuda(e, "device synchronise");
  const unsigned int w = stencil_error_word() | flow_error_word() | tail_error_word() | restrict_error_word();
  if (w & 1u) return set_error(NN4_ETIMEOUT, "a bounded device wait gave up");
  if (w & 2u) return set_error(NN4_EBOUNDS, "a checked device index was out of range");
  return NN4_OK;
}

int nn4_stencil_apply(const nn4_grid* g, nn4_dtype dt, const void* x, const void* k, void* y,
                      void* stream) {
  int rc;
  if ((rc = validate_grid(g, dt, 2)) || (rc = validate_ptr(x, "x")) || (rc = validate_ptr(y, "y"))) return rc;
  if (k && (rc = validate_ptr(k, "k"))) return rc;
  if (y == x || y == k) return set_error(NN4_EINVAL, "y must not alias x or k");
  PassArgs a{};
  a.g = geom_of(g);
  a.L = stencil_coef(g->h);
  a.out = y;
  PassCfg cfg = default_pass_cfg(dt, k != nullptr, a.g);
  a.zchunk = cfg.zchunk;
  return launch_pass(dt, OP_APPLY, a, x, k, cfg, static_cast<cudaStream_t>(stream));
}

int nn4_residual(const nn4_grid* g, nn4_dtype dt, const void* b, const void* x, const void* k,
                 void* r, double* norm2, void* stream) {
  int rc;
  if ((rc = validate_grid(g, dt, 2)) || (rc = validate_ptr(b, "b")) || (rc = validate_ptr(x, "x")) ||
      (rc = validate_ptr(r, "r")))
    return rc;
  if (k && (rc = validate_ptr(k, "k"))) return rc;
  if (r == x || r == b || r == k) return set_error(NN4_EINVAL, "r must not alias b, x or k");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (norm2) {
    if ((rc = check_cuda(cudaMemsetAsync(norm2, 0, sizeof(double), s), "zero norm"))) return rc;
  }
  PassArgs a{};
  a.g = geom_of(g);
  a.L = stencil_coef(g->h);
  a.b = b;
  a.out = r;
  a.norm2 = norm2;
  PassCfg cfg = default_pass_cfg(dt, k != nullptr, a.g);
  a.zchunk = cfg.zchunk;
  return launch_pass(dt, OP_RESIDUAL, a, x, k, cfg, s);
}

int nn4_jacobi_smooth(const nn4_grid* g, nn4_dtype dt, const void* b, const void* k,
                      const void* x_in, void* x_out, double omega, void* stream) {
  int rc;
  if ((rc = validate_grid(g, dt, 2)) || (rc = validate_ptr(b, "b")) || (rc = validate_ptr(x_in, "x_in")) ||
      (rc = validate_ptr(x_out, "x_out")))
    return rc;
  if (k && (rc = validate_ptr(k, "k"))) return rc;
  if (x_out == x_in || x_out == b || x_out == k) return set_error(NN4_EINVAL, "x_out must not alias an input");
  if (!(omega > 0.0 && omega < 2.0)) return set_error(NN4_EINVAL, "omega must lie in (0, 2)");
  PassArgs a{};
  a.g = geom_of(g);
  a.L = stencil_coef(g->h);
  a.b = b;
  a.out = x_out;
  a.omega = omega;
  PassCfg cfg = default_pass_cfg(dt, k != nullptr, a.g);
  a.zchunk = cfg.zchunk;
  return launch_pass(dt, OP_JACOBI, a, x_in, k, cfg, static_cast<cudaStream_t>(stream));
}

int nn4_restrict(const nn4_grid* fine, nn4_dtype dt, const void* r_fine, void* r_coarse, void* stream) {
  int rc;
  if ((rc = validate_grid(fine, dt, 3)) || (rc = validate_ptr(r_fine, "r_fine")) ||
      (rc = validate_ptr(r_coarse, "r_coarse")))
    return rc;
  for (int d = 0; d < 3; ++d)
    if (fine->n[d] % 2 == 0) return set_error(NN4_EINVAL, "restriction needs an odd node count on every axis");
  LevelGeom gf = geom_of(fine);
  LevelGeom gc = coarse_geom(gf, dt);
  return launch_restrict(dt, r_fine, gf, r_coarse, gc, static_cast<cudaStream_t>(stream));
}

int nn4_residual_restrict(const nn4_grid* fine, nn4_dtype dt, const void* b, const void* x, const void* k,
                          void* r_coarse, double* norm2, void* stream) {
  int rc;
  if ((rc = validate_grid(fine, dt, 3)) || (rc = validate_ptr(b, "b")) || (rc = validate_ptr(x, "x")) ||
      (rc = validate_ptr(r_coarse, "r_coarse")))
    return rc;
  if (k && (rc = validate_ptr(k, "k"))) return rc;
  for (int d = 0; d < 3; ++d)
    if (fine->n[d] % 2 == 0) return set_error(NN4_EINVAL, "restriction needs an odd node count on every axis");
  if (r_coarse == x || r_coarse == b || r_coarse == k) return set_error(NN4_EINVAL, "r_coarse must not alias b, x or k");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (norm2) {
    if ((rc = check_cuda(cudaMemsetAsync(norm2, 0, sizeof(double), s), "zero norm"))) return rc;
  }
  PassArgs a{};
  a.g = geom_of(fine);
  a.L = stencil_coef(fine->h);
  a.b = b;
  a.out = r_coarse;
  a.norm2 = norm2;
  a.gc = coarse_geom(a.g, dt);
  a.zchunk = rr_default_zchunk(a.gc, 1216);
  return launch_residual_restrict(dt, a, x, k, s);
}

int nn4_prolong(const nn4_grid* fine, nn4_dtype dt, const void* e_coarse, void* e_fine, int accumulate,
                void* stream) {
  int rc;
  if ((rc = validate_grid(fine, dt, 3)) || (rc = validate_ptr(e_coarse, "e_coarse")) ||
      (rc = validate_ptr(e_fine, "e_fine")))
    return rc;
  for (int d = 0; d < 3; ++d)
    if (fine->n[d] % 2 == 0) return set_error(NN4_EINVAL, "prolongation needs an odd node count on every axis");
  LevelGeom gf = geom_of(fine);
  LevelGeom gc = coarse_geom(gf, dt);
  return launch_prolong(dt, e_coarse, gc, e_fine, gf, accumulate, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
