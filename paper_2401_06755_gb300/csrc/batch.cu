// Batched pressure solves: many independent constant-coefficient solves of uneven grid sizes
// (ensembles of bubbles or columns) advanced together.  Every step of the V-cycle is ONE launch
// over the work items of all instances that have that level (stencil passes, transfers), the
// coarse tails run as one launch of one CTA per instance, and the FP64 outer loop (defect
// correction, Section 2.4's repeated cycles) is batched the same way.  Convergence is tracked
// per instance on the device: an instance whose relative residual reaches rtol stops (its work
// items are skipped) and stamps %globaltimer for its latency.  One outer iteration of the whole
// batch is one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nn4 {

LevelGeom geom_of(const nn4_grid* g);

namespace {

struct BLevel {
  LevelGeom g;
  double h[3];
  Coef8 L;
  void *r = nullptr, *e = nullptr, *t = nullptr;
};

struct BInst {
  nn4_grid grid;
  LevelGeom g64;
  Coef8 L64;
  double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;
  std::vector<BLevel> lv;
  int tail_start = 0;
  double* ainv = nullptr;
  int* free_idx = nullptr;
  int nfree = 0;
};

// Device-side per-instance record of the pointwise outer kernels.
struct BOuter {
  LevelGeom g64, gT;
  double* x64;
  const double* b64;
  double* r64;
  void* rT;  // level-0 right-hand side of the inner cycles
  void* eT;  // level-0 correction
  int first_row_block;
};

template <typename F>
__device__ __forceinline__ void for_rows(const BOuter* tab, int count, const int* active, F&& f) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].first_row_block <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  if (active && !active[lo]) return;
  const BOuter& O = tab[lo];
  const long long row = (long long)(blockIdx.x - O.first_row_block) * blockDim.y + threadIdx.y;
  if (row >= (long long)O.g64.ny * O.g64.nz) return;
  f(lo, O, row);
}

// mode 0: rT = (T) r64;  mode 1: x64 += eT
template <typename T>
__global__ void k_outer_batch(const BOuter* __restrict__ tab, int count, const int* __restrict__ active, int mode) {
  for_rows(tab, count, active, [&](int, const BOuter& O, long long row) {
    for (int i = threadIdx.x; i < O.g64.nx; i += blockDim.x) {
      const long long o64 = row * O.g64.pitch + i, oT = row * O.gT.pitch + i;
      if (mode == 0)
        static_cast<T*>(O.rT)[oT] = from_acc<T>(O.r64[o64]);
      else
        O.x64[o64] += (double)to_acc(static_cast<const T*>(O.eT)[oT]);
    }
  });
}

// ||b||^2 over free nodes per instance
__global__ void k_bnorm_batch(const BOuter* __restrict__ tab, int count, double* __restrict__ bn) {
  __shared__ double red[32];
  double s = 0.0;
  int inst = -1;
  for_rows(tab, count, nullptr, [&](int idx, const BOuter& O, long long row) {
    inst = idx;
    const int j = (int)(row % O.g64.ny), k = (int)(row / O.g64.ny);
    const LevelGeom& g = O.g64;
    for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
      const bool d = (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
                     (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
      const double v = O.b64[row * g.pitch + i];
      if (!d) s += v * v;
    }
  });
  // every row block belongs to one instance (row blocks never straddle instances)
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].first_row_block <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  (void)inst;
  block_sum_atomic(s, &bn[lo], red);
}

// Per-instance convergence check after an outer residual: deactivate converged (or non-finite)
// instances and stamp the time.  One thread per instance.
__global__ void k_check_batch(int count, const double* __restrict__ rn, const double* __restrict__ bn,
                              const double* __restrict__ rtol, int* __restrict__ active, int* __restrict__ iters,
                              unsigned long long* __restrict__ done_ns, double* __restrict__ rel, int* __restrict__ bad,
                              int count_iteration) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count || !active[i]) return;
  if (count_iteration) iters[i] += 1;
  const double r = sqrt(rn[i]) / (bn[i] > 0.0 ? sqrt(bn[i]) : 1.0);
  rel[i] = r;
  if (!isfinite(r)) {
    active[i] = 0;
    bad[i] = 1;
    done_ns[i] = globaltimer_ns();
  } else if (r <= *rtol) {
    active[i] = 0;
    done_ns[i] = globaltimer_ns();
  }
}

__global__ void k_stamp(unsigned long long* t) { *t = globaltimer_ns(); }

}  // namespace

struct BatchImpl {
  int count = 0;
  nn4_dtype T = NN4_F32;
  nn4_plan_opts o;
  std::vector<BInst> inst;
  int maxlev = 0;
  // device tables
  struct PassSet {
    BatchPass* d = nullptr;
    int count = 0, total = 0;
  };
  std::vector<PassSet> jac;       // Jacobi at slot l (l < tail_start of the instance)
  std::vector<PassCfg> jac_cfg;   // tile shape of slot l's Jacobi launch (autotuned)
  std::vector<int> jac_shape, jac_zmax;
  std::vector<float> jac_us;      // its measured time at creation (0: not timed)
  PassCfg res_cfg;                // tile shape of the FP64 outer residual
  PassSet rr0;                    // level-0 residual + restriction (inner, cycles >= 2)
  PassSet res64;                  // FP64 outer residual
  struct XferSet {
    BatchXfer* d = nullptr;
    int count = 0, total = 0;
  };
  std::vector<XferSet> restr;     // restriction slot l -> l+1
  std::vector<XferSet> prol;      // prolongation slot l+1 -> l
  XferSet prol0_base;             // finest prolongation with base e (cycles >= 2)
  TailArgs* tails = nullptr;
  BOuter* outer = nullptr;
  int outer_blocks = 0;
  // per-instance device state
  double *rn = nullptr, *bn = nullptr, *rtol = nullptr, *rel = nullptr;
  int *active = nullptr, *iters = nullptr, *bad = nullptr;
  unsigned long long *done_ns = nullptr, *start_ns = nullptr;
  int* host_active = nullptr;  // pinned
  cudaGraphExec_t graph = nullptr;
  cudaStream_t gstream = nullptr;
  std::vector<void*> allocs;
  int64_t graph_kernels = 0;
};

namespace {

int balloc(BatchImpl* B, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return check_cuda(e, "cudaMalloc (batch)");
  B->allocs.push_back(*p);
  return check_cuda(cudaMemset(*p, 0, bytes), "cudaMemset (batch)");
}

size_t fbytes(const LevelGeom& g, nn4_dtype dt) { return (size_t)g.pitch * g.ny * g.nz * dtype_size(dt); }

void bdestroy(BatchImpl* B) {
  if (!B) return;
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->gstream) cudaStreamDestroy(B->gstream);
  for (void* p : B->allocs) cudaFree(p);
  if (B->host_active) cudaFreeHost(B->host_active);
  delete B;
}

// Dense (pseudo-)inverse of one instance's coarsest constant-coefficient level (host).
int coarsest_inverse(BatchImpl* B, BInst& I) {
  const BLevel& C = I.lv.back();
  const int nx = C.g.nx, ny = C.g.ny, nz = C.g.nz, N = nx * ny * nz;
  auto m = [](int i, int n) { return i < 0 ? -i : (i >= n ? 2 * (n - 1) - i : i); };
  auto hc = [](int i, int n) { return 0.5 * ((i > 0) + (i < n - 1)); };
  auto isd = [&](int i, int j, int k) {
    return (C.g.dir[0] && i == 0) || (C.g.dir[1] && i == nx - 1) || (C.g.dir[2] && j == 0) ||
           (C.g.dir[3] && j == ny - 1) || (C.g.dir[4] && k == 0) || (C.g.dir[5] && k == nz - 1);
  };
  std::vector<int> lin, off;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        if (!isd(i, j, k)) {
          lin.push_back(i + nx * (j + ny * k));
          off.push_back((int)(i + C.g.pitch * (j + (long long)ny * k)));
        }
  const int n = (int)lin.size();
  if (n == 0 || n > 1024) return set_error(NN4_EUNSUPPORTED, "coarsest level size unsupported in a batch");
  std::vector<double> dense((size_t)N * N, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const double w = hc(i, nx) * hc(j, ny) * hc(k, nz);
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int cls = (dx != 0) + 2 * (dy != 0) + 4 * (dz != 0);
              dense[(size_t)(i + nx * (j + ny * k)) * N + (m(i + dx, nx) + nx * (m(j + dy, ny) + ny * m(k + dz, nz)))] +=
                  w * C.L.c[cls];
            }
      }
  std::vector<double> A((size_t)n * n), Iv((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) A[(size_t)a * n + b] = dense[(size_t)lin[a] * N + lin[b]];
  bool singular = true;
  for (int f = 0; f < 6; ++f) singular = singular && !C.g.dir[f];
  if (singular)
    for (auto& v : A) v += 1.0 / n;
  for (int i = 0; i < n; ++i) Iv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {  // Gauss-Jordan with partial pivoting
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (A[(size_t)piv * n + c] == 0.0) return set_error(NN4_EINVAL, "singular coarsest operator");
    if (piv != c)
      for (int t = 0; t < n; ++t) {
        std::swap(A[(size_t)c * n + t], A[(size_t)piv * n + t]);
        std::swap(Iv[(size_t)c * n + t], Iv[(size_t)piv * n + t]);
      }
    const double d = 1.0 / A[(size_t)c * n + c];
    for (int t = 0; t < n; ++t) {
      A[(size_t)c * n + t] *= d;
      Iv[(size_t)c * n + t] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int t = 0; t < n; ++t) {
        A[(size_t)r * n + t] -= f * A[(size_t)c * n + t];
        Iv[(size_t)r * n + t] -= f * Iv[(size_t)c * n + t];
      }
    }
  }
  if (singular)
    for (auto& v : Iv) v -= 1.0 / n;
  int rc;
  if ((rc = balloc(B, (void**)&I.ainv, sizeof(double) * n * n)) ||
      (rc = balloc(B, (void**)&I.free_idx, sizeof(int) * n)) ||
      (rc = check_cuda(cudaMemcpy(I.ainv, Iv.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice), "ainv")) ||
      (rc = check_cuda(cudaMemcpy(I.free_idx, off.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "idx")))
    return rc;
  I.nfree = n;
  return NN4_OK;
}

template <typename E>
int upload(BatchImpl* B, std::vector<E>& v, E** d) {
  if (v.empty()) return NN4_OK;
  int rc;
  if ((rc = balloc(B, (void**)d, sizeof(E) * v.size()))) return rc;
  return check_cuda(cudaMemcpy(*d, v.data(), sizeof(E) * v.size(), cudaMemcpyHostToDevice), "upload table");
}

int make_pass(BatchImpl* B, std::vector<BatchPass>& v, nn4_dtype dt, int inst, const LevelGeom& g, const Coef8& L,
              const void* x, const void* b, void* out, double omega, double* norm2, int* total, const PassCfg& shape,
              int zmax) {
  BatchPass bp;
  std::memset(&bp, 0, sizeof(bp));
  bp.args.g = g;
  bp.args.L = L;
  bp.args.omega = omega;
  bp.args.b = b;
  bp.args.out = out;
  bp.args.norm2 = norm2;
  PassCfg c = shape;
  // a few output planes per item keep the items many and short (latency across instances); zmax
  // caps the z-march depth
  int zc = g.nz;
  const int tx = 32 * shape.wx, ty = shape.tyt * shape.ry;
  const int tiles = ((g.nx + tx - 1) / tx) * ((g.ny + ty - 1) / ty);
  while (zc > 8 && tiles * ((g.nz + zc - 1) / zc) < 64) zc = (zc + 1) / 2;
  if (zc > zmax) zc = zmax;
  bp.args.zchunk = zc;
  c.zchunk = zc;
  if (!make_pass_maps(&bp.maps, dt, bp.args, c, x, nullptr)) return set_error(NN4_ECUDA, "tensor map encode failed");
  bp.inst = inst;
  bp.first = *total;
  *total += batch_pass_tiles(dt, &bp, c);
  v.push_back(bp);
  return NN4_OK;
}

// Level-0 residual + restriction of one instance: out (level 1's r) = R (b - A x).
int make_rr_pass(std::vector<BatchPass>& v, nn4_dtype dt, int inst, const LevelGeom& g, const Coef8& L,
                 const LevelGeom& gc, const void* x, const void* b, void* out, int* total) {
  if (!(g.nx & 1) || !(g.ny & 1) || !(g.nz & 1) || gc.nx != (g.nx + 1) / 2 || gc.ny != (g.ny + 1) / 2 ||
      gc.nz != (g.nz + 1) / 2)
    return set_error(NN4_EINVAL, "residual + restriction needs odd node counts and the grid of every second node");
  BatchPass bp;
  std::memset(&bp, 0, sizeof(bp));
  bp.args.g = g;
  bp.args.L = L;
  bp.args.b = b;
  bp.args.out = out;
  bp.args.gc = gc;
  // as for the other batched passes: enough short items per instance, at most 16 coarse planes
  bp.args.zchunk = std::min(rr_default_zchunk(gc, 64), 16);
  if (!make_rr_maps(&bp.maps, dt, bp.args, x, nullptr)) return set_error(NN4_ECUDA, "tensor map encode failed");
  bp.inst = inst;
  bp.first = *total;
  *total += rr_batch_tiles(&bp);
  v.push_back(bp);
  return NN4_OK;
}

void make_xfer(std::vector<BatchXfer>& v, int inst, bool prolong, const LevelGeom& gf, const LevelGeom& gc,
               const void* src, void* dst, const void* base, int* total) {
  BatchXfer X;
  std::memset(&X, 0, sizeof(X));
  X.gf = gf;
  X.gc = gc;
  X.src = src;
  X.dst = dst;
  X.base = base;
  X.inst = inst;
  X.first = *total;
  *total += batch_xfer_blocks(&X, prolong);
  v.push_back(X);
}

// ---------------------------------------------------------------- autotuner of the batched passes
// The Jacobi launch of level slot l (every instance that has that level in one launch) is timed
// at creation for each compiled tile shape and z-march depth cap, on the batch's own (zeroed)
// arrays with every instance active, and the fastest is kept.  plan option pass_shape >= 0 forces
// a shape (the cap stays at 32); autotune = 0 keeps shape 0 with the cap 32.
int build_jacobi(BatchImpl* B, int l, const PassCfg& shape, int zmax, std::vector<BatchPass>& v, int* total) {
  v.clear();
  *total = 0;
  int rc;
  for (int i = 0; i < B->count; ++i) {
    BInst& I = B->inst[i];
    if (l >= I.tail_start) continue;
    BLevel& L = I.lv[l];
    if ((rc = make_pass(B, v, B->T, i, L.g, L.L, L.t, L.r, L.e, B->o.omega, nullptr, total, shape, zmax))) return rc;
  }
  return NN4_OK;
}

int tune_jacobi(BatchImpl* B, int l, std::vector<BatchPass>& v, int* total) {
  B->jac_cfg.resize(B->maxlev, batch_pass_cfg(B->T));
  B->jac_shape.resize(B->maxlev, 0);
  B->jac_zmax.resize(B->maxlev, 32);
  B->jac_us.resize(B->maxlev, 0.0f);
  std::vector<std::pair<int, int>> cands;  // (shape, z cap)
  const int forced = B->o.pass_shape;
  if (forced >= 0 && forced < num_batch_shapes())
    cands.push_back({forced, 32});
  else if (B->o.autotune)
    for (int sh = 0; sh < num_batch_shapes(); ++sh)
      for (int zm : {16, 32, 64}) cands.push_back({sh, zm});
  else
    cands.push_back({0, 32});
  int rc;
  int best = 0;
  float best_us = 0.0f;
  if (cands.size() > 1) {
    cudaEvent_t e0, e1;
    if ((rc = check_cuda(cudaEventCreate(&e0), "event")) || (rc = check_cuda(cudaEventCreate(&e1), "event"))) return rc;
    for (size_t c = 0; c < cands.size(); ++c) {
      const PassCfg sh = batch_shape_cfg(cands[c].first);
      int tot = 0;
      if ((rc = build_jacobi(B, l, sh, cands[c].second, v, &tot))) break;
      if (v.empty()) break;
      BatchPass* d = nullptr;
      if ((rc = check_cuda(cudaMalloc(&d, sizeof(BatchPass) * v.size()), "tuning table"))) break;
      rc = check_cuda(cudaMemcpy(d, v.data(), sizeof(BatchPass) * v.size(), cudaMemcpyHostToDevice), "tuning table");
      const int reps = 5;
      float ms = 0.0f;
      for (int r = 0; !rc && r < 2; ++r) rc = launch_pass_batch(B->T, OP_JACOBI, sh, d, (int)v.size(), tot, nullptr, 0);
      if (!rc) rc = check_cuda(cudaEventRecord(e0, 0), "event");
      for (int r = 0; !rc && r < reps; ++r) rc = launch_pass_batch(B->T, OP_JACOBI, sh, d, (int)v.size(), tot, nullptr, 0);
      if (!rc) rc = check_cuda(cudaEventRecord(e1, 0), "event");
      if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "event");
      if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "event");
      cudaFree(d);
      if (rc) break;
      const float us = 1e3f * ms / reps;
      if (c == 0 || us < best_us) {
        best = (int)c;
        best_us = us;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
  }
  const PassCfg sh = batch_shape_cfg(cands[best].first);
  B->jac_cfg[l] = sh;
  B->jac_shape[l] = cands[best].first;
  B->jac_zmax[l] = cands[best].second;
  B->jac_us[l] = best_us;
  return build_jacobi(B, l, sh, cands[best].second, v, total);
}

// ---------------------------------------------------------------- the batched cycle
int bcycle(BatchImpl* B, bool first, cudaStream_t s, int64_t* kernels) {
  const nn4_dtype T = B->T;
  int rc;
  if (!first) {  // level 1's right-hand side R (r - A e) in one pass
    if ((rc = launch_rr_batch(T, B->rr0.d, B->rr0.count, B->rr0.total, B->active, s))) return rc;
    *kernels += 1;
  } else {
    if ((rc = launch_xfer_batch(T, false, B->restr[0].d, B->restr[0].count, B->restr[0].total, B->active, s)))
      return rc;
    *kernels += 1;
  }
  for (int l = 1; l < (int)B->restr.size(); ++l) {
    if (B->restr[l].count == 0) continue;
    if ((rc = launch_xfer_batch(T, false, B->restr[l].d, B->restr[l].count, B->restr[l].total, B->active, s))) return rc;
    *kernels += 1;
  }
  if ((rc = launch_tail_batch(T, B->tails, B->count, B->active, s))) return rc;
  *kernels += 1;
  for (int l = (int)B->jac.size() - 1; l >= 1; --l) {
    if (B->jac[l].count == 0) continue;
    if ((rc = launch_xfer_batch(T, true, B->prol[l].d, B->prol[l].count, B->prol[l].total, B->active, s))) return rc;
    if ((rc = launch_pass_batch(T, OP_JACOBI, B->jac_cfg[l], B->jac[l].d, B->jac[l].count, B->jac[l].total, B->active,
                                s)))
      return rc;
    *kernels += 2;
  }
  const auto& p0 = first ? B->prol[0] : B->prol0_base;
  if ((rc = launch_xfer_batch(T, true, p0.d, p0.count, p0.total, B->active, s))) return rc;
  if ((rc = launch_pass_batch(T, OP_JACOBI, B->jac_cfg[0], B->jac[0].d, B->jac[0].count, B->jac[0].total, B->active,
                              s)))
    return rc;
  *kernels += 2;
  return NN4_OK;
}

int outer_residual_batch(BatchImpl* B, cudaStream_t s, int64_t* kernels) {
  int rc;
  if ((rc = check_cuda(cudaMemsetAsync(B->rn, 0, sizeof(double) * B->count, s), "zero norms"))) return rc;
  *kernels += 1;
  return launch_pass_batch(NN4_F64, OP_RESIDUAL, B->res_cfg, B->res64.d, B->res64.count, B->res64.total, B->active, s);
}

int biteration(BatchImpl* B, cudaStream_t s, int64_t* kernels) {
  int rc;
  dim3 blk(32, 8);
  switch (B->T) {
    case NN4_F64: k_outer_batch<double><<<B->outer_blocks, blk, 0, s>>>(B->outer, B->count, B->active, 0); break;
    case NN4_F32: k_outer_batch<float><<<B->outer_blocks, blk, 0, s>>>(B->outer, B->count, B->active, 0); break;
    case NN4_BF16: k_outer_batch<bf16><<<B->outer_blocks, blk, 0, s>>>(B->outer, B->count, B->active, 0); break;
  }
  *kernels += 1;
  for (int c = 0; c < B->o.inner_cycles; ++c)
    if ((rc = bcycle(B, c == 0, s, kernels))) return rc;
  switch (B->T) {
    case NN4_F64: k_outer_batch<double><<<B->outer_blocks, blk, 0, s>>>(B->outer, B->count, B->active, 1); break;
    case NN4_F32: k_outer_batch<float><<<B->outer_blocks, blk, 0, s>>>(B->outer, B->count, B->active, 1); break;
    case NN4_BF16: k_outer_batch<bf16><<<B->outer_blocks, blk, 0, s>>>(B->outer, B->count, B->active, 1); break;
  }
  *kernels += 1;
  if ((rc = check_cuda(cudaGetLastError(), "batched outer kernels"))) return rc;
  if ((rc = outer_residual_batch(B, s, kernels))) return rc;
  k_check_batch<<<(B->count + 127) / 128, 128, 0, s>>>(B->count, B->rn, B->bn, B->rtol, B->active, B->iters,
                                                       B->done_ns, B->rel, B->bad, 1);
  *kernels += 1;
  return check_cuda(cudaGetLastError(), "batched check");
}

}  // namespace
}  // namespace nn4

using namespace nn4;

struct nn4_batch_s {
  BatchImpl* impl;
};

extern "C" {

int nn4_batch_create(const nn4_grid* grids, int32_t count, const nn4_plan_opts* opts, nn4_batch* out) {
  if (!out) return set_error(NN4_EINVAL, "out is NULL");
  *out = nullptr;
  if (!grids || count < 1 || count > 4096) return set_error(NN4_EINVAL, "bad instance count");
  nn4_plan_opts o;
  nn4_plan_opts_default(&o);
  if (opts) o = *opts;
  if (o.inner != NN4_F64 && o.inner != NN4_F32 && o.inner != NN4_BF16) return set_error(NN4_EINVAL, "bad inner dtype");
  if (o.inner_cycles < 1 || o.inner_cycles > 64) return set_error(NN4_EINVAL, "inner_cycles must be in 1..64");
  if (!(o.omega > 0.0 && o.omega < 2.0)) return set_error(NN4_EINVAL, "omega must lie in (0, 2)");
  for (int i = 0; i < count; ++i) {
    const nn4_grid& g = grids[i];
    for (int d = 0; d < 3; ++d)
      if (g.n[d] < 3 || !(g.h[d] > 0.0)) return set_error(NN4_EINVAL, "bad instance grid");
    if (!(g.h[0] == g.h[1] && g.h[1] == g.h[2]))
      return set_error(NN4_EUNSUPPORTED, "batched solves need equal spacing on the three axes");
    if (g.pitch < g.n[0] || (g.pitch * 8) % 16) return set_error(NN4_EINVAL, "bad FP64 pitch");
    for (int f = 0; f < 6; ++f)
      if (g.bc[f] != NN4_BC_DIRICHLET && g.bc[f] != NN4_BC_NATURAL) return set_error(NN4_EINVAL, "bad face condition");
  }
  BatchImpl* B = new BatchImpl();
  B->count = count;
  B->T = o.inner;
  B->o = o;
  B->inst.resize(count);
  int rc = NN4_OK;
  auto fail = [&](int code) {
    bdestroy(B);
    return code;
  };
  // per-instance hierarchies and FP64 outer buffers
  for (int i = 0; i < count; ++i) {
    BInst& I = B->inst[i];
    I.grid = grids[i];
    I.g64 = geom_of(&grids[i]);
    I.L64 = stencil_coef(grids[i].h);
    BLevel L;
    L.g = I.g64;
    L.g.pitch = nn4_row_pitch(L.g.nx, B->T);
    for (int d = 0; d < 3; ++d) L.h[d] = grids[i].h[d];
    I.lv.push_back(L);
    while (true) {
      const BLevel& f = I.lv.back();
      if (!(f.g.nx >= 5 && f.g.ny >= 5 && f.g.nz >= 5 && (f.g.nx & 1) && (f.g.ny & 1) && (f.g.nz & 1))) break;
      BLevel c;
      c.g = f.g;
      c.g.nx = (f.g.nx + 1) / 2;
      c.g.ny = (f.g.ny + 1) / 2;
      c.g.nz = (f.g.nz + 1) / 2;
      c.g.pitch = nn4_row_pitch(c.g.nx, B->T);
      for (int d = 0; d < 3; ++d) c.h[d] = 2.0 * f.h[d];
      I.lv.push_back(c);
    }
    const int nl = (int)I.lv.size();
    if (nl < 2) return fail(set_error(NN4_EUNSUPPORTED, "batched instances need at least two levels"));
    I.tail_start = -1;
    for (int l = 1; l < nl; ++l)
      if ((long long)I.lv[l].g.nx * I.lv[l].g.ny * I.lv[l].g.nz <= kTailNodes && nl - l <= kMaxTail) {
        I.tail_start = l;
        break;
      }
    if (I.tail_start < 0) return fail(set_error(NN4_EUNSUPPORTED, "no coarse tail for a batched instance"));
    for (auto& lv : I.lv) {
      lv.L = stencil_coef(lv.h);
      const size_t fb = fbytes(lv.g, B->T);
      if ((rc = balloc(B, &lv.r, fb)) || (rc = balloc(B, &lv.e, fb)) || (rc = balloc(B, &lv.t, fb))) return fail(rc);
    }
    const size_t fb64 = fbytes(I.g64, NN4_F64);
    if ((rc = balloc(B, (void**)&I.x64, fb64)) || (rc = balloc(B, (void**)&I.b64, fb64)) ||
        (rc = balloc(B, (void**)&I.r64, fb64)))
      return fail(rc);
    if ((rc = coarsest_inverse(B, I))) return fail(rc);
    B->maxlev = std::max(B->maxlev, nl);
  }
  // per-instance device state
  if ((rc = balloc(B, (void**)&B->rn, sizeof(double) * count)) || (rc = balloc(B, (void**)&B->bn, sizeof(double) * count)) ||
      (rc = balloc(B, (void**)&B->rel, sizeof(double) * count)) || (rc = balloc(B, (void**)&B->rtol, sizeof(double))) ||
      (rc = balloc(B, (void**)&B->active, sizeof(int) * count)) || (rc = balloc(B, (void**)&B->iters, sizeof(int) * count)) ||
      (rc = balloc(B, (void**)&B->bad, sizeof(int) * count)) ||
      (rc = balloc(B, (void**)&B->done_ns, sizeof(unsigned long long) * count)) ||
      (rc = balloc(B, (void**)&B->start_ns, sizeof(unsigned long long))))
    return fail(rc);
  if ((rc = check_cuda(cudaMallocHost(&B->host_active, sizeof(int) * count), "pinned flags"))) return fail(rc);
  // tables of every batched launch
  const nn4_dtype T = B->T;
  std::vector<std::vector<BatchPass>> jac(B->maxlev);
  std::vector<BatchPass> rr0, res64;
  std::vector<std::vector<BatchXfer>> restr(B->maxlev), prol(B->maxlev);
  std::vector<BatchXfer> prol0b;
  std::vector<TailArgs> tails(count);
  std::vector<BOuter> outer(count);
  B->res_cfg = batch_pass_cfg(NN4_F64);
  B->jac.resize(B->maxlev);
  B->restr.resize(B->maxlev);
  B->prol.resize(B->maxlev);
  int tot_rr0 = 0, tot_res64 = 0, tot_p0b = 0;
  std::vector<int> tot_jac(B->maxlev, 0), tot_restr(B->maxlev, 0), tot_prol(B->maxlev, 0);
  int rowblocks = 0;
  for (int i = 0; i < count; ++i) {
    BInst& I = B->inst[i];
    const int ts = I.tail_start;
    for (int l = 0; l < ts; ++l) {
      BLevel& L = I.lv[l];
      make_xfer(restr[l], i, false, L.g, I.lv[l + 1].g, l == 0 ? L.r : L.r, I.lv[l + 1].r, nullptr, &tot_restr[l]);
      make_xfer(prol[l], i, true, L.g, I.lv[l + 1].g, I.lv[l + 1].e, L.t, nullptr, &tot_prol[l]);
    }
    BLevel& L0 = I.lv[0];
    if ((rc = make_rr_pass(rr0, T, i, L0.g, L0.L, I.lv[1].g, L0.e, L0.r, I.lv[1].r, &tot_rr0))) return fail(rc);
    make_xfer(prol0b, i, true, L0.g, I.lv[1].g, I.lv[1].e, L0.t, L0.e, &tot_p0b);
    if ((rc = make_pass(B, res64, NN4_F64, i, I.g64, I.L64, I.x64, I.b64, I.r64, o.omega, B->rn + i, &tot_res64,
                        B->res_cfg, 32)))
      return fail(rc);
    TailArgs& ta = tails[i];
    std::memset(&ta, 0, sizeof(ta));
    ta.nlev = (int)I.lv.size() - ts;
    for (int l = ts; l < (int)I.lv.size(); ++l) {
      TailLevel& tl = ta.lv[l - ts];
      tl.g = I.lv[l].g;
      tl.L = I.lv[l].L;
      tl.r = I.lv[l].r;
      tl.e = I.lv[l].e;
      tl.t = I.lv[l].t;
      tl.a27 = nullptr;
    }
    ta.ainv = I.ainv;
    ta.free_idx = I.free_idx;
    ta.nfree = I.nfree;
    ta.omega = o.omega;
    BOuter& O = outer[i];
    O.g64 = I.g64;
    O.gT = L0.g;
    O.x64 = I.x64;
    O.b64 = I.b64;
    O.r64 = I.r64;
    O.rT = L0.r;
    O.eT = L0.e;
    O.first_row_block = rowblocks;
    rowblocks += (int)(((long long)I.g64.ny * I.g64.nz + 7) / 8);
  }
  for (int l = 0; l < B->maxlev; ++l) {
    if ((rc = tune_jacobi(B, l, jac[l], &tot_jac[l]))) return fail(rc);
    if ((rc = upload(B, jac[l], &B->jac[l].d)) || (rc = upload(B, restr[l], &B->restr[l].d)) ||
        (rc = upload(B, prol[l], &B->prol[l].d)))
      return fail(rc);
    B->jac[l].count = (int)jac[l].size();
    B->jac[l].total = tot_jac[l];
    B->restr[l].count = (int)restr[l].size();
    B->restr[l].total = tot_restr[l];
    B->prol[l].count = (int)prol[l].size();
    B->prol[l].total = tot_prol[l];
  }
  if ((rc = upload(B, rr0, &B->rr0.d)) || (rc = upload(B, res64, &B->res64.d)) ||
      (rc = upload(B, prol0b, &B->prol0_base.d)) ||
      (rc = upload(B, tails, &B->tails)) || (rc = upload(B, outer, &B->outer)))
    return fail(rc);
  B->rr0.count = count;
  B->rr0.total = tot_rr0;
  B->res64.count = count;
  B->res64.total = tot_res64;
  B->prol0_base.count = count;
  B->prol0_base.total = tot_p0b;
  B->outer_blocks = rowblocks;
  if ((rc = check_cuda(cudaDeviceSynchronize(), "batch build"))) return fail(rc);
  nn4_batch h = new nn4_batch_s;
  h->impl = B;
  *out = h;
  return NN4_OK;
}

int nn4_batch_query(nn4_batch b, nn4_batch_info* info) {
  if (!b || !info) return set_error(NN4_EINVAL, "NULL argument");
  BatchImpl* B = b->impl;
  std::memset(info, 0, sizeof(*info));
  info->levels = std::min<int>((int)B->jac.size(), 16);
  for (int l = 0; l < info->levels; ++l) {
    info->shape[l] = l < (int)B->jac_shape.size() ? B->jac_shape[l] : 0;
    info->zmax[l] = l < (int)B->jac_zmax.size() ? B->jac_zmax[l] : 32;
    info->jacobi_us[l] = l < (int)B->jac_us.size() ? B->jac_us[l] : 0.0f;
    info->items[l] = B->jac[l].total;
    long long nodes = 0;
    for (const auto& I : B->inst)
      if (l < I.tail_start) nodes += (long long)I.lv[l].g.nx * I.lv[l].g.ny * I.lv[l].g.nz;
    info->nodes[l] = nodes;
  }
  return NN4_OK;
}

int nn4_batch_destroy(nn4_batch b) {
  if (!b) return NN4_OK;
  bdestroy(b->impl);
  delete b;
  return NN4_OK;
}

int nn4_pressure_solve_batched(nn4_batch b, const double* const* bs, double* const* xs, double rtol,
                               int32_t max_iters, nn4_solve_info* infos, float* latency_ms, void* stream) {
  if (!b || !bs || !xs) return set_error(NN4_EINVAL, "NULL argument");
  if (max_iters < 0) return set_error(NN4_EINVAL, "max_iters must be >= 0");
  BatchImpl* B = b->impl;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = B->count;
  int rc;
  for (int i = 0; i < n; ++i) {
    if (!bs[i] || !xs[i]) return set_error(NN4_EINVAL, "NULL instance array");
    const size_t fb = fbytes(B->inst[i].g64, NN4_F64);
    if ((rc = check_cuda(cudaMemcpyAsync(B->inst[i].b64, bs[i], fb, cudaMemcpyDeviceToDevice, s), "copy b")) ||
        (rc = check_cuda(cudaMemcpyAsync(B->inst[i].x64, xs[i], fb, cudaMemcpyDeviceToDevice, s), "copy x")))
      return rc;
  }
  if (!B->graph) {  // capture one outer iteration of the whole batch
    if ((rc = check_cuda(cudaStreamCreateWithFlags(&B->gstream, cudaStreamNonBlocking), "graph stream"))) return rc;
    cudaGraph_t g;
    if ((rc = check_cuda(cudaStreamBeginCapture(B->gstream, cudaStreamCaptureModeThreadLocal), "capture"))) return rc;
    int64_t k = 0;
    rc = biteration(B, B->gstream, &k);
    cudaError_t e = cudaStreamEndCapture(B->gstream, &g);
    if (rc) return rc;
    if ((rc = check_cuda(e, "end capture"))) return rc;
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if ((rc = check_cuda(e, "instantiate"))) return rc;
    B->graph_kernels = k;
  }
  // start: all active, iteration counters 0, ||b||, initial residual and check
  std::vector<int> ones(n, 1);
  if ((rc = check_cuda(cudaMemcpyAsync(B->active, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s), "active")) ||
      (rc = check_cuda(cudaMemsetAsync(B->iters, 0, sizeof(int) * n, s), "iters")) ||
      (rc = check_cuda(cudaMemsetAsync(B->bad, 0, sizeof(int) * n, s), "bad")) ||
      (rc = check_cuda(cudaMemsetAsync(B->bn, 0, sizeof(double) * n, s), "bn")) ||
      (rc = check_cuda(cudaMemcpyAsync(B->rtol, &rtol, sizeof(double), cudaMemcpyHostToDevice, s), "rtol")))
    return rc;
  k_stamp<<<1, 1, 0, s>>>(B->start_ns);
  k_bnorm_batch<<<B->outer_blocks, dim3(32, 8), 0, s>>>(B->outer, n, B->bn);
  int64_t kernels = 2;
  if ((rc = outer_residual_batch(B, s, &kernels))) return rc;
  k_check_batch<<<(n + 127) / 128, 128, 0, s>>>(n, B->rn, B->bn, B->rtol, B->active, B->iters, B->done_ns, B->rel,
                                                B->bad, 0);
  kernels += 1;
  const int every = B->o.check_every > 0 ? B->o.check_every : 1;
  int it = 0;
  while (it < max_iters) {
    const int todo = std::min(every, max_iters - it);
    for (int t = 0; t < todo; ++t, ++it) {
      if ((rc = check_cuda(cudaGraphLaunch(B->graph, s), "graph launch"))) return rc;
      kernels += B->graph_kernels;
    }
    if ((rc = check_cuda(cudaMemcpyAsync(B->host_active, B->active, sizeof(int) * n, cudaMemcpyDeviceToHost, s), "flags")) ||
        (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
      return rc;
    int any = 0;
    for (int i = 0; i < n; ++i) any |= B->host_active[i];
    if (!any) break;
  }
  // results
  std::vector<int> iters(n), bad(n), act(n);
  std::vector<double> rel(n);
  std::vector<unsigned long long> done(n);
  unsigned long long t0 = 0;
  if ((rc = check_cuda(cudaMemcpyAsync(iters.data(), B->iters, sizeof(int) * n, cudaMemcpyDeviceToHost, s), "r")) ||
      (rc = check_cuda(cudaMemcpyAsync(bad.data(), B->bad, sizeof(int) * n, cudaMemcpyDeviceToHost, s), "r")) ||
      (rc = check_cuda(cudaMemcpyAsync(act.data(), B->active, sizeof(int) * n, cudaMemcpyDeviceToHost, s), "r")) ||
      (rc = check_cuda(cudaMemcpyAsync(rel.data(), B->rel, sizeof(double) * n, cudaMemcpyDeviceToHost, s), "r")) ||
      (rc = check_cuda(cudaMemcpyAsync(done.data(), B->done_ns, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s), "r")) ||
      (rc = check_cuda(cudaMemcpyAsync(&t0, B->start_ns, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s), "r")))
    return rc;
  for (int i = 0; i < n; ++i) {
    const size_t fb = fbytes(B->inst[i].g64, NN4_F64);
    if ((rc = check_cuda(cudaMemcpyAsync(xs[i], B->inst[i].x64, fb, cudaMemcpyDeviceToDevice, s), "copy x out"))) return rc;
  }
  if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
  int status = NN4_OK;
  for (int i = 0; i < n; ++i) {
    if (infos) {
      infos[i].iterations = iters[i];
      infos[i].cycles = iters[i] * B->o.inner_cycles;
      infos[i].rel_res = rel[i];
      infos[i].kernels = kernels;
    }
    if (latency_ms) latency_ms[i] = act[i] ? -1.0f : (float)((double)(done[i] - t0) * 1e-6);
    if (bad[i]) status = set_error(NN4_ENONFINITE, "non-finite residual in a batched instance");
    else if (act[i] && status == NN4_OK) status = set_error(NN4_ENOCONV, "iteration cap reached in a batched instance");
  }
  return status;
}

}  // extern "C"
