// Residual + restriction in one pass: r_1 = R (b - A x) with R = P^T (the stride-2 restriction of
// Section 2.4's sawtooth multigrid) and ||b - A x||^2, without storing the fine residual.  The
// tile machinery is the stencil passes' (pass_tile.cuh, OP_RESIDUAL_RESTRICT): a CTA computes the
// fine residual on 32 x 16 fine nodes shifted one node down from its 15 x 7 coarse nodes, so each
// coarse node's 3 x 3 x 3 fine neighbourhood is inside the tile, and it marches along z over
// `zchunk` coarse planes (2 zchunk + 1 fine planes).
#include <algorithm>

#include "pass_tile.cuh"

namespace nn4 {

NN4_DEFINE_ERROR_ACCESSOR(restrict_error_word)

namespace {

// One tile shape for every storage type: 32 x 16 fine nodes (128 threads, 4 rows each), three
// planes in flight.  It keeps the redundant fine rows and columns (one of every 15 and 7) and
// the coarse nodes per CTA (105 <= 128 threads) in balance.
constexpr int kWX = 1, kRY = 4, kTYT = 4, kS = 3;

template <typename T, int VC, bool ISO>
using RRLayout = PassLayout<T, OP_RESIDUAL_RESTRICT, VC, ISO, kWX, kRY, kTYT, kS>;

template <typename T, int VC, bool ISO>
int launch_rr_t(const PassArgs& a, const Maps& maps, cudaStream_t st) {
  using Lay = RRLayout<T, VC, ISO>;
  const size_t smem = Lay::SMEM;
  auto kern = k_pass<T, OP_RESIDUAL_RESTRICT, VC, ISO, kWX, kRY, kTYT, kS>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(residual + restriction)");
  }
  const LevelGeom& gc = a.gc;
  dim3 grid((gc.nx + Lay::CX - 1) / Lay::CX, (gc.ny + Lay::CY - 1) / Lay::CY, (gc.nz + a.zchunk - 1) / a.zchunk);
  kern<<<grid, dim3(32 * kWX, kTYT), smem, st>>>(maps, a);
  return check_cuda(cudaGetLastError(), "residual + restriction launch");
}

template <typename T, int VC>
int dispatch_rr_iso(bool iso, const PassArgs& a, const Maps& m, cudaStream_t st) {
  return iso ? launch_rr_t<T, VC, true>(a, m, st) : launch_rr_t<T, VC, false>(a, m, st);
}

template <typename T>
int dispatch_rr(int vc, const PassArgs& a, const Maps& m, cudaStream_t st) {
  const bool iso = a.L.c[1] == 0.0 && a.L.c[2] == 0.0 && a.L.c[4] == 0.0;
  if (vc == 0) return dispatch_rr_iso<T, 0>(iso, a, m, st);
  if (vc == 1) return dispatch_rr_iso<T, 1>(iso, a, m, st);
  return dispatch_rr_iso<T, 2>(iso, a, m, st);
}

template <typename T>
int launch_rr_batch_t(const BatchPass* items, int count, int total, const int* active, cudaStream_t st) {
  // batched instances have equal spacings per axis and a constant coefficient
  using Lay = RRLayout<T, 0, true>;
  auto kern = k_pass_batch<T, OP_RESIDUAL_RESTRICT, 0, true, kWX, kRY, kTYT, kS>;
  const size_t smem = Lay::SMEM;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(batched residual + restriction)");
  }
  const int grid = std::min(total, 152 * 8);
  kern<<<grid, dim3(32 * kWX, kTYT), smem, st>>>(items, count, total, active);
  return check_cuda(cudaGetLastError(), "batched residual + restriction launch");
}

bool valid_pair(const LevelGeom& g, const LevelGeom& gc) {
  return (g.nx & 1) && (g.ny & 1) && (g.nz & 1) && g.nx >= 3 && g.ny >= 3 && g.nz >= 3 &&
         gc.nx == (g.nx + 1) / 2 && gc.ny == (g.ny + 1) / 2 && gc.nz == (g.nz + 1) / 2;
}

}  // namespace

PassCfg rr_pass_cfg() {
  PassCfg c;
  c.wx = kWX;
  c.ry = kRY;
  c.tyt = kTYT;
  c.stages = kS;
  c.zchunk = 0;
  return c;
}

int rr_tiles_xy(const LevelGeom& gc, int* tx, int* ty) {
  constexpr int CX = 16 * kWX - 1, CY = kTYT * kRY / 2 - 1;
  *tx = (gc.nx + CX - 1) / CX;
  *ty = (gc.ny + CY - 1) / CY;
  return (*tx) * (*ty);
}

int rr_default_zchunk(const LevelGeom& gc, int min_ctas) {
  int tx, ty;
  const int tiles = rr_tiles_xy(gc, &tx, &ty);
  // halve the coarse planes per CTA until the grid fills the GPU, keeping at least 4 (9 fine
  // planes, one of them shared with the next chunk)
  int kc = gc.nz;
  while (kc > 4 && tiles * ((gc.nz + kc - 1) / kc) < min_ctas) kc = std::max(4, (kc + 1) / 2);
  return kc;
}

int rr_batch_tiles(BatchPass* bp) {
  int tx, ty;
  rr_tiles_xy(bp->args.gc, &tx, &ty);
  bp->tiles_x = tx;
  bp->tiles_y = ty;
  const int tz = (bp->args.gc.nz + bp->args.zchunk - 1) / bp->args.zchunk;
  return tx * ty * tz;
}

bool make_rr_maps(PassMaps* m, nn4_dtype dt, const PassArgs& a, const void* x, const void* k) {
  return make_pass_maps(m, dt, a, rr_pass_cfg(), x, k, /*wide_point=*/true);
}

int launch_residual_restrict(nn4_dtype dt, const PassArgs& a, const void* x, const void* k, cudaStream_t s,
                             const PassMaps* pm) {
  if (!a.b || !a.out) return set_error(NN4_EINVAL, "residual + restriction needs b and an output");
  if (a.zchunk < 1) return set_error(NN4_EINVAL, "residual + restriction needs zchunk >= 1");
  if (!valid_pair(a.g, a.gc))
    return set_error(NN4_EINVAL, "residual + restriction needs odd node counts and the grid of every second node");
  if (a.invd || a.dq || a.ec) return set_error(NN4_EINVAL, "residual + restriction takes no Jacobi-only field");
  PassMaps local;
  const bool vc = k != nullptr;
  if (!pm) {
    if (!make_rr_maps(&local, dt, a, x, k)) return set_error(NN4_ECUDA, "cuTensorMapEncodeTiled failed");
    pm = &local;
  }
  Maps m;
  m.x = pm->x;
  m.k = vc ? pm->k : pm->x;
  m.b = pm->b;
  m.lk = a.lk ? pm->lk : pm->x;
  m.invd = m.dq = m.ec = pm->x;
  const int vmode = vc ? (a.lk ? 2 : 1) : 0;
  switch (dt) {
    case NN4_F64: return dispatch_rr<double>(vmode, a, m, s);
    case NN4_F32: return dispatch_rr<float>(vmode, a, m, s);
    case NN4_BF16: return dispatch_rr<bf16>(vmode, a, m, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

int launch_rr_batch(nn4_dtype dt, const BatchPass* items, int count, int total, const int* active, cudaStream_t s) {
  if (total <= 0) return NN4_OK;
  switch (dt) {
    case NN4_F64: return launch_rr_batch_t<double>(items, count, total, active, s);
    case NN4_F32: return launch_rr_batch_t<float>(items, count, total, active, s);
    case NN4_BF16: return launch_rr_batch_t<bf16>(items, count, total, active, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

}  // namespace nn4
