// Q1 27-point stencil passes: apply, residual (+ FP64 norm), weighted Jacobi and the matrix-vector
// product, for the constant-coefficient operator and for the variable-coefficient identity of
// Eq. k-T (Section 2.2.4): launchers, tile-shape dispatch and the batched form.  The tile
// itself (TMA planes, sum factorisation, natural faces by mirroring) is in pass_tile.cuh.
#include <algorithm>

#include "pass_tile.cuh"

namespace nn4 {

NN4_DEFINE_ERROR_ACCESSOR(stencil_error_word)

namespace {

template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
int launch_t(const PassArgs& a, const Maps& maps, cudaStream_t st) {
  constexpr int TX = 32 * WX, TY = TYT * RY;
  const size_t smem = PassLayout<T, OP, VC, ISO, WX, RY, TYT, S>::SMEM;
  auto kern = k_pass<T, OP, VC, ISO, WX, RY, TYT, S>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(stencil pass)");
  }
  dim3 grid((a.g.nx + TX - 1) / TX, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zchunk - 1) / a.zchunk);
  kern<<<grid, dim3(TX, TYT), smem, st>>>(maps, a);
  return check_cuda(cudaGetLastError(), "stencil pass launch");
}

// The configurations the autotuner chooses from: {WX, RY, TYT, S}.
// The last ({1, 8, 2, 3}: eight rows a thread) is compiled for FP64 only, whose passes are bound by
// the FP64 pipe and gain from the fewer loads per output; for the other types it is refused and
// the autotuner skips it.
constexpr int kCfgs[][4] = {{1, 4, 4, 3}, {2, 2, 4, 4}, {1, 2, 8, 3}, {2, 4, 2, 4}, {1, 8, 2, 3}};
constexpr int kNumCfgs = 5;

template <typename T, int OP, int VC, bool ISO>
int dispatch_cfg(const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  for (int c = 0; c < kNumCfgs; ++c)
    if (cfg.wx == kCfgs[c][0] && cfg.ry == kCfgs[c][1] && cfg.tyt == kCfgs[c][2] && cfg.stages == kCfgs[c][3]) {
      switch (c) {
        case 0: return launch_t<T, OP, VC, ISO, 1, 4, 4, 3>(a, m, st);
        case 1: return launch_t<T, OP, VC, ISO, 2, 2, 4, 4>(a, m, st);
        case 2: return launch_t<T, OP, VC, ISO, 1, 2, 8, 3>(a, m, st);
        case 3: return launch_t<T, OP, VC, ISO, 2, 4, 2, 4>(a, m, st);
        case 4:
          if constexpr (sizeof(T) == 8) return launch_t<T, OP, VC, ISO, 1, 8, 2, 3>(a, m, st);
          break;
      }
    }
  return set_error(NN4_EINVAL, "unsupported stencil pass configuration");
}

template <typename T, int OP, int VC>
int dispatch_iso(bool iso, const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  return iso ? dispatch_cfg<T, OP, VC, true>(a, cfg, m, st) : dispatch_cfg<T, OP, VC, false>(a, cfg, m, st);
}

template <typename T, int OP>
int dispatch_vc(int vc, bool iso, const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  if (vc == 0) return dispatch_iso<T, OP, 0>(iso, a, cfg, m, st);
  if (vc == 1) return dispatch_iso<T, OP, 1>(iso, a, cfg, m, st);
  return dispatch_iso<T, OP, 2>(iso, a, cfg, m, st);
}

template <typename T>
int dispatch_op(int op, int vc, const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  const bool iso = a.L.c[1] == 0.0 && a.L.c[2] == 0.0 && a.L.c[4] == 0.0;
  switch (op) {
    case OP_APPLY: return dispatch_vc<T, OP_APPLY>(vc, iso, a, cfg, m, st);
    case OP_RESIDUAL: return dispatch_vc<T, OP_RESIDUAL>(vc, iso, a, cfg, m, st);
    case OP_JACOBI: return dispatch_vc<T, OP_JACOBI>(vc, iso, a, cfg, m, st);
    case OP_MATVEC: return dispatch_vc<T, OP_MATVEC>(vc, iso, a, cfg, m, st);
  }
  return set_error(NN4_EINVAL, "bad stencil op");
}

template <typename T, int OP, bool ISO, int WX, int RY, int TYT, int S>
int launch_batch_t(const BatchPass* items, int count, int total, const int* active, cudaStream_t st) {
  using Lay = PassLayout<T, OP, 0, ISO, WX, RY, TYT, S>;
  auto kern = k_pass_batch<T, OP, 0, ISO, WX, RY, TYT, S>;
  const size_t smem = Lay::SMEM;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(batched pass)");
  }
  // persistent CTAs: as many as are resident at once, striding over the items
  const int grid = (int)resident_grid((const void*)kern, 32 * WX * TYT, smem, total);
  kern<<<grid, dim3(32 * WX, TYT), smem, st>>>(items, count, total, active);
  return check_cuda(cudaGetLastError(), "batched stencil pass launch");
}

// the batched passes compile the first four tile shapes of kCfgs for every storage type
constexpr int kBatchShapes = 4;

template <typename T, int OP>
int launch_batch_shape(const PassCfg& c, const BatchPass* items, int count, int total, const int* active,
                       cudaStream_t st) {
  for (int i = 0; i < kBatchShapes; ++i)
    if (c.wx == kCfgs[i][0] && c.ry == kCfgs[i][1] && c.tyt == kCfgs[i][2] && c.stages == kCfgs[i][3]) {
      switch (i) {
        case 0: return launch_batch_t<T, OP, true, 1, 4, 4, 3>(items, count, total, active, st);
        case 1: return launch_batch_t<T, OP, true, 2, 2, 4, 4>(items, count, total, active, st);
        case 2: return launch_batch_t<T, OP, true, 1, 2, 8, 3>(items, count, total, active, st);
        case 3: return launch_batch_t<T, OP, true, 2, 4, 2, 4>(items, count, total, active, st);
      }
    }
  return set_error(NN4_EINVAL, "unsupported batched tile shape");
}

}  // namespace

PassCfg batch_pass_cfg(nn4_dtype dt) { return batch_shape_cfg(0); }

int num_batch_shapes() { return kBatchShapes; }

PassCfg batch_shape_cfg(int index) {
  PassCfg c;
  const int i = (index >= 0 && index < kBatchShapes) ? index : 0;
  c.wx = kCfgs[i][0];
  c.ry = kCfgs[i][1];
  c.tyt = kCfgs[i][2];
  c.stages = kCfgs[i][3];
  c.zchunk = 0;
  return c;
}

int batch_pass_tiles(nn4_dtype, BatchPass* bp, const PassCfg& cfg) {
  const LevelGeom& g = bp->args.g;
  const int tx = 32 * cfg.wx, ty = cfg.tyt * cfg.ry;
  bp->tiles_x = (g.nx + tx - 1) / tx;
  bp->tiles_y = (g.ny + ty - 1) / ty;
  const int tz = (g.nz + bp->args.zchunk - 1) / bp->args.zchunk;
  return bp->tiles_x * bp->tiles_y * tz;
}

int launch_pass_batch(nn4_dtype dt, int op, const PassCfg& cfg, const BatchPass* items, int count, int total,
                      const int* active, cudaStream_t s) {
  if (total <= 0) return NN4_OK;
  // every instance of a batch has equal spacing per axis (checked at batch creation)
  switch (dt * 4 + op) {
    case NN4_F64 * 4 + OP_RESIDUAL: return launch_batch_shape<double, OP_RESIDUAL>(cfg, items, count, total, active, s);
    case NN4_F64 * 4 + OP_JACOBI: return launch_batch_shape<double, OP_JACOBI>(cfg, items, count, total, active, s);
    case NN4_F32 * 4 + OP_RESIDUAL: return launch_batch_shape<float, OP_RESIDUAL>(cfg, items, count, total, active, s);
    case NN4_F32 * 4 + OP_JACOBI: return launch_batch_shape<float, OP_JACOBI>(cfg, items, count, total, active, s);
    case NN4_BF16 * 4 + OP_RESIDUAL: return launch_batch_shape<bf16, OP_RESIDUAL>(cfg, items, count, total, active, s);
    case NN4_BF16 * 4 + OP_JACOBI: return launch_batch_shape<bf16, OP_JACOBI>(cfg, items, count, total, active, s);
  }
  return set_error(NN4_EINVAL, "unsupported batched pass");
}

PassCfg default_pass_cfg(nn4_dtype dt, bool vc, const LevelGeom& g) {
  PassCfg c;
  c.wx = 1;
  c.ry = (dt == NN4_F64 && vc) ? 2 : 4;
  c.tyt = (dt == NN4_F64 && vc) ? 8 : 4;
  c.stages = 3;
  const int tiles = ((g.nx + 32 * c.wx - 1) / (32 * c.wx)) * ((g.ny + c.tyt * c.ry - 1) / (c.tyt * c.ry));
  // aim at >= ~1200 CTAs (8 per SM) but keep at least 8 output planes per CTA
  int zc = g.nz;
  while (zc > 8 && tiles * ((g.nz + zc - 1) / zc) < 1216) zc = (zc + 1) / 2;
  c.zchunk = zc;
  return c;
}

int num_pass_cfgs() { return kNumCfgs; }

PassCfg pass_cfg_candidate(int index, const LevelGeom& g, int zchunk) {
  PassCfg c;
  c.wx = kCfgs[index][0];
  c.ry = kCfgs[index][1];
  c.tyt = kCfgs[index][2];
  c.stages = kCfgs[index][3];
  c.zchunk = zchunk > 0 ? zchunk : g.nz;
  return c;
}

int pass_box(nn4_dtype dt, const PassCfg& cfg, int* box_x, int* box_y) {
  const int al = 16 / (int)dtype_size(dt);
  *box_x = 32 * cfg.wx + 2 * al;
  *box_y = cfg.tyt * cfg.ry + 2;
  return NN4_OK;
}

int pass_coarse_box(nn4_dtype dt, const PassCfg& cfg, int* box_x, int* box_y) {
  const int al = 16 / (int)dtype_size(dt);
  *box_x = 16 * cfg.wx + 2 * al;
  *box_y = cfg.tyt * cfg.ry / 2 + 2;
  return NN4_OK;
}

int pass_point_box(const PassCfg& cfg, int* box_x, int* box_y) {
  *box_x = 32 * cfg.wx;
  *box_y = cfg.tyt * cfg.ry;
  return NN4_OK;
}

bool make_pass_maps(PassMaps* m, nn4_dtype dt, const PassArgs& a, const PassCfg& cfg, const void* x, const void* k,
                    bool wide_point) {
  int bx, by, px, py;
  pass_box(dt, cfg, &bx, &by);
  pass_point_box(cfg, &px, &py);
  if (wide_point) px += 16 / (int)dtype_size(dt);
  const LevelGeom& g = a.g;
  bool ok = make_tmap_3d(&m->x, dt, x, g.nx, g.ny, g.nz, g.pitch, bx, by);
  if (k) ok = ok && make_tmap_3d(&m->k, dt, k, g.nx, g.ny, g.nz, g.pitch, bx, by);
  if (a.b) ok = ok && make_tmap_3d(&m->b, dt, a.b, g.nx, g.ny, g.nz, g.pitch, px, py);
  if (a.lk) ok = ok && make_tmap_3d(&m->lk, dt, a.lk, g.nx, g.ny, g.nz, g.pitch, px, py);
  if (a.invd) ok = ok && make_tmap_3d(&m->invd, dt, a.invd, g.nx, g.ny, g.nz, g.pitch, px, py);
  if (a.dq) ok = ok && make_tmap_3d(&m->dq, NN4_F32, a.dq, g.nx, g.ny, g.nz, a.dq_pitch, px, py);
  if (a.ec) {
    int cx, cy;
    pass_coarse_box(dt, cfg, &cx, &cy);
    ok = ok && make_tmap_3d(&m->ec, dt, a.ec, a.gc.nx, a.gc.ny, a.gc.nz, a.gc.pitch, cx, cy);
  }
  return ok;
}

int launch_pass(nn4_dtype dt, int op, const PassArgs& a, const void* x, const void* k,
                const PassCfg& cfg, cudaStream_t s, const PassMaps* pm) {
  PassMaps local;
  const bool vc = k != nullptr;
  if (!pm) {
    if (!make_pass_maps(&local, dt, a, cfg, x, k)) return set_error(NN4_ECUDA, "cuTensorMapEncodeTiled failed");
    pm = &local;
  }
  Maps m;
  m.x = pm->x;
  m.k = vc ? pm->k : pm->x;
  m.b = a.b ? pm->b : pm->x;
  m.lk = a.lk ? pm->lk : pm->x;
  m.invd = a.invd ? pm->invd : pm->x;
  m.dq = a.dq ? pm->dq : pm->x;
  m.ec = a.ec ? pm->ec : pm->x;
  if (a.ec && op != OP_JACOBI) return set_error(NN4_EINVAL, "the fused prolongation needs OP_JACOBI");
  // (every compiled tile shape has an even height, so a tile's first row y0 sits on a coarse row)
  if (a.ec && (a.gc.nx != (a.g.nx + 1) / 2 || a.gc.ny != (a.g.ny + 1) / 2 || a.gc.nz != (a.g.nz + 1) / 2 ||
               !(a.g.nx & 1) || !(a.g.ny & 1) || !(a.g.nz & 1)))
    return set_error(NN4_EINVAL, "the fused prolongation needs the grid of every second node");
  if (a.dq && (op != OP_JACOBI || !a.dq_out)) return set_error(NN4_EINVAL, "the fused dot needs OP_JACOBI and an output");
  if (op != OP_APPLY && !a.b) return set_error(NN4_EINVAL, "stencil pass needs b");
  const int vmode = vc ? (a.lk ? 2 : 1) : 0;
  switch (dt) {
    case NN4_F64: return dispatch_op<double>(op, vmode, a, cfg, m, s);
    case NN4_F32: return dispatch_op<float>(op, vmode, a, cfg, m, s);
    case NN4_BF16: return dispatch_op<bf16>(op, vmode, a, cfg, m, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

}  // namespace nn4
