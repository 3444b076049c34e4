// Host-side declarations shared between the library's translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/nn4.h"

namespace nn4 {

// Interior Q1 stencil on a mirror-extended field, by neighbour class: c[a + 2b + 4c] multiplies
// the sum over the 2^(a+b+c) neighbours offset by +-1 along the axes flagged a (x), b (y), c (z).
struct Coef8 {
  double c[8];
};

// Geometry of one level as the kernels see it.
struct LevelGeom {
  int nx, ny, nz;
  long long pitch;  // row pitch in elements of the array this geometry is used with
  int dir[6];       // 1 where the face is Dirichlet (x-, x+, y-, y+, z-, z+)
};

// OP_APPLY: out = A x.  OP_RESIDUAL: out = b - A x (0 at Dirichlet nodes), norm2 += out^2.
// OP_JACOBI: out = x + omega D^-1 (b - A x) (x at Dirichlet nodes).
// OP_MATVEC: out = A x (0 at Dirichlet nodes), norm2 += x.out, dot2 += x.b.
// OP_RESIDUAL_RESTRICT: out = R (b - A x) on the coarse grid gc (0 at coarse Dirichlet nodes),
// norm2 += sum over fine nodes of (b - A x)^2; zchunk counts coarse planes per block.
enum PassOp { OP_APPLY = 0, OP_RESIDUAL = 1, OP_JACOBI = 2, OP_MATVEC = 3, OP_RESIDUAL_RESTRICT = 4 };

struct PassArgs {
  LevelGeom g;
  Coef8 L;
  double omega;
  const void* b;     // right-hand side (OP_RESIDUAL, OP_JACOBI), pitch g.pitch
  void* out;         // y / r / x_out, pitch g.pitch
  double* norm2;     // optional: += sum out^2 (OP_RESIDUAL) or x.out (OP_MATVEC)
  double* dot2;      // OP_MATVEC: += x.b
  int zchunk;        // output planes per block
  // Eq. k-T with precomputed fields (optional): lk = (1/2) L k (assembled, pitch g.pitch) replaces the
  // on-the-fly stencil of k; invd = 1 / diag(A) replaces the division in Jacobi.
  const void* lk;
  const void* invd;
  // OP_JACOBI only (optional): dq_out += sum over nodes of (the new x rounded to the storage type)
  // times dq, an FP32 field read through its own tensor map (the flexible-CG dot z.q_old fused
  // into the sweep that produces z)
  const float* dq;
  long long dq_pitch;  // row pitch of dq (elements)
  double* dq_out;
  // OP_JACOBI only (optional): the input x is P ec, the trilinear prolongation of the coarse
  // field ec (geometry gc, the grid of every second node), formed in shared memory from coarse
  // tiles instead of read from memory (zero at Dirichlet nodes)
  const void* ec;
  LevelGeom gc;  // the coarse grid (fused prolongation; residual + restriction)
};

// Stencil pass launch configuration (chosen by the autotuner or by default).
struct PassCfg {
  int wx;      // warps along x (tile width 32 wx)
  int ry;      // outputs per thread along y
  int tyt;     // threads along y (x is always one warp of 32)
  int stages;  // TMA pipeline depth (planes in flight)
  int zchunk;  // output planes per block
};

// ---------------------------------------------------------------- helpers (api.cu)
Coef8 stencil_coef(const double h[3]);
int set_error(int code, const std::string& msg);
int check_cuda(cudaError_t e, const char* what);
bool make_tmap_3d(CUtensorMap* map, nn4_dtype dt, const void* base, int nx, int ny, int nz,
                  long long pitch, int box_x, int box_y);
// A stack of nw fields of one grid, field w starting pitch * ny * nz elements after field w - 1
// (4D map; box (box_x, box_y, 1, box_w)).
bool make_tmap_stack(CUtensorMap* map, nn4_dtype dt, const void* base, int nx, int ny, int nz, int nw,
                     long long pitch, int box_x, int box_y, int box_w);
size_t dtype_size(nn4_dtype dt);
// SMs of the current device (cached per device).
int sm_count();
// min(want, the blocks of `kern` that are resident at once with `threads` threads and `smem`
// dynamic shared memory): the grid of a grid-stride kernel, so no block waits for a second wave.
long long resident_grid(const void* kern, int threads, size_t smem, long long want);

// Per-unit device error words (read and cleared).
unsigned int stencil_error_word();
unsigned int flow_error_word();
unsigned int tail_error_word();
unsigned int restrict_error_word();

// ---------------------------------------------------------------- launchers
// Tensor maps of one stencil pass: haloed tiles of x and k, pointwise tiles of b, L k, 1/diag.
struct PassMaps {
  CUtensorMap x, k, b, lk, invd, dq, ec;
};

// One instance's part of a batched stencil pass (device table entry, 64-byte aligned maps).
struct alignas(64) BatchPass {
  PassMaps maps;
  PassArgs args;
  int inst;      // instance index (for the active flags)
  int first;     // index of this instance's first work item
  int tiles_x, tiles_y;
};

// Batched stencil pass over `count` instances (constant coefficient) with tile shape `cfg` (one of
// the num_batch_shapes() shapes; every entry of `items` was built for it); `items` is a device
// array; `active` (device, nullable) skips converged instances.
int launch_pass_batch(nn4_dtype dt, int op, const PassCfg& cfg, const BatchPass* items, int count, int total,
                      const int* active, cudaStream_t s);
// Fills the tiling fields of a batch entry for tile shape cfg (returns its item count).
int batch_pass_tiles(nn4_dtype dt, BatchPass* bp, const PassCfg& cfg);
PassCfg batch_pass_cfg(nn4_dtype dt);
int num_batch_shapes();
PassCfg batch_shape_cfg(int index);

// stencil.cu: constant coefficient (k == nullptr) or Eq. k-T (k given).  Every input is read with
// TMA; the maps are built here unless `maps` is given (built with make_pass_maps for this cfg).
int launch_pass(nn4_dtype dt, int op, const PassArgs& a, const void* x, const void* k,
                const PassCfg& cfg, cudaStream_t s, const PassMaps* maps = nullptr);
// wide_point: the pointwise boxes are 32 wx + 16/sizeof(T) wide (OP_RESIDUAL_RESTRICT's shifted tiles)
bool make_pass_maps(PassMaps* m, nn4_dtype dt, const PassArgs& a, const PassCfg& cfg, const void* x, const void* k,
                    bool wide_point = false);

// resrestrict.cu: out = R (b - A x) on the coarse grid a.gc and norm2 += ||b - A x||^2 in one pass
// (a.zchunk = coarse planes per CTA, see rr_default_zchunk); maps from make_rr_maps, or built here.
int launch_residual_restrict(nn4_dtype dt, const PassArgs& a, const void* x, const void* k, cudaStream_t s,
                             const PassMaps* maps = nullptr);
bool make_rr_maps(PassMaps* m, nn4_dtype dt, const PassArgs& a, const void* x, const void* k);
PassCfg rr_pass_cfg();
int rr_default_zchunk(const LevelGeom& gc, int min_ctas);
// Fills the tiling fields of a batch entry (args.gc and args.zchunk set) and returns its item count.
int rr_batch_tiles(BatchPass* bp);
int launch_rr_batch(nn4_dtype dt, const BatchPass* items, int count, int total, const int* active, cudaStream_t s);
PassCfg default_pass_cfg(nn4_dtype dt, bool vc, const LevelGeom& g);
int num_pass_cfgs();
PassCfg pass_cfg_candidate(int index, const LevelGeom& g, int zchunk);
int pass_box(nn4_dtype dt, const PassCfg& cfg, int* box_x, int* box_y);
int pass_point_box(const PassCfg& cfg, int* box_x, int* box_y);
// Box of the coarse tiles of the fused prolongation (Jacobi passes with PassArgs.ec).
int pass_coarse_box(nn4_dtype dt, const PassCfg& cfg, int* box_x, int* box_y);

// transfer.cu
int launch_restrict(nn4_dtype dt, const void* rf, const LevelGeom& gf, void* rc,
                    const LevelGeom& gc, cudaStream_t s);
int launch_prolong(nn4_dtype dt, const void* ec, const LevelGeom& gc, void* ef,
                   const LevelGeom& gf, int accumulate, cudaStream_t s);
// ef = base + P ec (base may be NULL for 0; may alias ef).  Fine Dirichlet nodes get base (or 0).
int launch_prolong_base(nn4_dtype dt, const void* ec, const LevelGeom& gc, void* ef, const void* base,
                        const LevelGeom& gf, cudaStream_t s);

// coarse.cu: e = Ainv r on the coarsest level (FP64 matrix over the free nodes, whose grid
// offsets are listed in `free_idx`).  Non-free nodes of e are set to 0; with `accumulate`,
// e += Ainv r at free nodes and other nodes are left alone.
int launch_coarse_solve(nn4_dtype dt, const double* ainv, const int* free_idx, int nfree,
                        const void* r, void* e, const LevelGeom& g, int accumulate, cudaStream_t s);

// tail.cu: the coarse levels of a V-cycle in one single-CTA launch.  Level 0 of the tail is the
// entry level (its r holds the restricted residual on entry, its e the correction on exit);
// the last level is the coarsest (dense solve with ainv over free_idx).
constexpr int kMaxTail = 12;
constexpr int kTailNodes = 800;  // levels at or below this many nodes join the tail (9^3)

struct TailLevel {
  LevelGeom g;
  Coef8 L;          // constant-coefficient stencil (used when a27 is NULL)
  void* r;
  void* e;
  void* t;
  const void* a27;  // Galerkin coefficients or NULL
};

struct TailArgs {
  int nlev;
  int dense_all;  // the last level is solved by ainv over all its nodes (free_idx: every node)
  TailLevel lv[kMaxTail];
  const double* ainv;
  const int* free_idx;
  int nfree;
  double omega;
};

int launch_tail(nn4_dtype dt, const TailArgs& a, cudaStream_t s);

// Cooperative launch over all SMs for levels lv[0 .. nlev-1] (the first with at most
// kCoarseNodes nodes down to the level solved by the dense map in ainv, dense_all = 1): the
// restrictions, the dense map, then a fused prolongation + Jacobi sweep per level back up, with
// grid barriers between the steps (`bar`: a zeroed GridBarrier in device memory owned by the
// caller).
struct GridBarrier {
  unsigned count;
  unsigned gen;
};
// Threads per block of the cooperative coarse-level launch: blocks of 256 spread the 33^3 level of a
// 257^3 hierarchy over 141 SMs (measured 32.8 us per cycle's coarse levels, against 40.2 us with 512
// and 34.9 us with 128).
constexpr int kCoarseThreads = 256;
constexpr long long kCoarseNodes = 40000;
int launch_coarse(nn4_dtype dt, const TailArgs& a, GridBarrier* bar, cudaStream_t s);
// One CTA per instance (tab: device array of `count` tails; `active` skips converged ones).
int launch_tail_batch(nn4_dtype dt, const TailArgs* tab, int count, const int* active, cudaStream_t s);

// Batched restriction (src = fine r, dst = coarse r) or prolongation (src = coarse e, dst = fine
// t, optional base) over instances; device table entries.
struct BatchXfer {
  LevelGeom gf, gc;
  const void* src;
  void* dst;
  const void* base;
  int inst, first, bx, by;
};
int batch_xfer_blocks(BatchXfer* X, bool prolong);
int launch_xfer_batch(nn4_dtype dt, bool prolong, const BatchXfer* tab, int count, int total, const int* active,
                      cudaStream_t s);

}  // namespace nn4
