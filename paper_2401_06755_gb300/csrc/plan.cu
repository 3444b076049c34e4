// Multigrid plan: hierarchy, coarsest-level inverse, sawtooth V-cycle and pressure solves.
//
// The cycle follows the reading of the paper's U-Net multigrid (Section 2.4, multigrid figure):
// residual on the finest level, stride-2 restriction to the coarsest level, exact coarsest
// solve, then on every level on the way up prolongation followed by one weighted-Jacobi sweep.
// The solve wraps inner cycles (stored in FP64, FP32 or BF16) in an FP64 outer loop: plain
// defect correction (the paper's repeated cycles) or flexible CG.  Every outer iteration is one
// CUDA graph (captured at the first solve), so a solve is a few graph launches plus one
// residual-norm readback per `check_every` iterations.
#include <cmath>
#include <mutex>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "galerkin.h"
#include "internal.h"
#include "outer.h"

namespace nn4 {

LevelGeom geom_of(const nn4_grid* g);

namespace {

struct Level {
  LevelGeom g;      // inner-dtype pitch
  double h[3];
  Coef8 L;
  PassCfg cfg;
  void* r = nullptr;  // right-hand side of this level
  void* e = nullptr;  // correction (output of the Jacobi sweep)
  void* t = nullptr;  // prolongated correction / fine residual (input of the Jacobi sweep)
  PassMaps m_jac{}, m_res{};  // Jacobi (x = t, b = r) and residual (x = e, b = r) passes
  PassMaps m_rr{};            // level 0: residual + restriction (x = e, b = r, out = level 1's r)
  PassMaps m_jac_dq[2]{};     // level 0 with the inner Krylov loop: Jacobi + the fused dot with q[parity]
  void* a27 = nullptr;  // Galerkin coefficients (coefficient field, levels >= 1)
  void* k = nullptr;    // coefficient field in the inner type (level 0)
};

}  // namespace

struct PlanImpl {
  nn4_grid grid;
  nn4_plan_opts o;
  nn4_dtype T;
  bool vc = false;
  std::vector<Level> lv;
  // coarsest level
  double* ainv = nullptr;
  int* free_idx = nullptr;
  int nfree = 0;
  // FP64 outer loop (pitch grid.pitch)
  LevelGeom g64;
  Coef8 L64;
  PassCfg cfg64;
  double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr, *p64[2] = {nullptr, nullptr},
         *q64[2] = {nullptr, nullptr}, *k64 = nullptr;
  double *lk64 = nullptr, *invd64 = nullptr;  // (1/2) L k and 1/diag(A) for Eq. k-T (FP64)
  void* lkT = nullptr;      // (1/2) L k in the inner storage type at the level-0 pitch
  void* invdT = nullptr;    // 1/diag(A) in the inner storage type (the level-0 Jacobi sweep multiplies
                            // by it instead of dividing per node)
  float* lk32 = nullptr;    // (1/2) L k in FP32 for the inner Krylov mat-vec
  // inner flexible CG in FP32 vectors (opts.inner_krylov > 0): solution y, residual r, directions
  // p[2], q[2], coefficient k (FP32), all at the FP32 level-0 pitch
  LevelGeom g32;
  PassCfg cfg32;
  float *yi = nullptr, *ri = nullptr, *pi[2] = {nullptr, nullptr}, *qi[2] = {nullptr, nullptr}, *k32 = nullptr;
  PassMaps m_mat32[2]{};
  PassMaps m_res64{}, m_mat64[2]{};
  // device scalars: [0] ||r||^2 (current), [1] ||b||^2, [2] z.q, [3..4] p.q by parity,
  // [5..6] p.r by parity; inner loop: [8] z.q, [9..10] p.q, [11..12] p.r, [13] ||r||^2;
  // [15] the constant 1.0.  Then the per-iteration history of ||r||^2
  double* scal = nullptr;
  double* hist = nullptr;
  int hist_cap = 0;
  double* host_hist = nullptr;  // pinned
  // Coarse levels in one launch: levels >= tail_start run in the single-CTA tail or, with
  // coarse_coop, in the cooperative kernel; coarse_top (>= 1, or -1) is the level above them whose
  // restriction and prolongation the cooperative kernel also performs.
  int tail_start = -1;
  bool coarse_coop = false;
  int coarse_top = -1;
  GridBarrier* gbar = nullptr;
  // cooperative form: levels tail_start .. coarse_dense run in the kernel, and everything at and
  // below coarse_dense is applied as one dense FP64 map (tail_map, n x n over all its nodes at the
  // offsets tail_idx)
  int coarse_dense = -1;
  double* tail_map = nullptr;
  int* tail_idx = nullptr;
  int tail_n = 0;
  // host copies of the coarsest inverse (for the dense map)
  std::vector<double> ainv_host;
  std::vector<int> free_lin_host;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int64_t graph_kernels[2] = {0, 0};
  cudaStream_t graph_stream = nullptr;
  std::vector<void*> allocs;
  size_t device_bytes = 0;
  // launch accounting and optional per-kernel event timing
  int64_t kernels = 0;
  struct Rec {
    std::string name;
    cudaEvent_t e0, e1;
  };
  std::vector<Rec> recs;
};

namespace {

int alloc(PlanImpl* P, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) return check_cuda(e, "cudaMalloc (plan)");
  P->allocs.push_back(*p);
  P->device_bytes += bytes;
  return check_cuda(cudaMemset(*p, 0, bytes), "cudaMemset (plan)");
}

size_t field_bytes(const LevelGeom& g, nn4_dtype dt) {
  return (size_t)g.pitch * g.ny * g.nz * dtype_size(dt);
}

// Every kernel launch of the plan goes through K(): it counts the launch and, in profile mode,
// brackets it with CUDA events on the launching stream.
template <typename F>
int K(PlanImpl* P, const std::string& name, cudaStream_t s, F&& launch) {
  PlanImpl::Rec r;
  const bool prof = P->o.profile != 0;
  if (prof) {
    r.name = name;
    cudaEventCreate(&r.e0);
    cudaEventCreate(&r.e1);
    cudaEventRecord(r.e0, s);
  }
  const int rc = launch();
  P->kernels += 1;
  if (prof) {
    cudaEventRecord(r.e1, s);
    P->recs.push_back(r);
  }
  return rc;
}

std::string lvl(int l) { return l >= 3 ? std::string("L3+") : "L" + std::to_string(l); }
const char* opname(int op) {
  return op == OP_APPLY ? "apply" : op == OP_RESIDUAL ? "residual" : op == OP_JACOBI ? "jacobi" : "matvec";
}

// ---------------------------------------------------------------- host dense algebra
// Constant-coefficient operator on a level, applied on the host to a dense vector (mirror rule
// for natural faces as in the kernels), used only to assemble the coarsest matrix.
void host_apply_const(const Level& L, const std::vector<double>& x, std::vector<double>& y) {
  const int nx = L.g.nx, ny = L.g.ny, nz = L.g.nz;
  auto m = [](int i, int n) { return i < 0 ? -i : (i >= n ? 2 * (n - 1) - i : i); };
  auto hc = [](int i, int n) { return 0.5 * ((i > 0) + (i < n - 1)); };
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int cls = (dx != 0) + 2 * (dy != 0) + 4 * (dz != 0);
              s += L.L.c[cls] * x[m(i + dx, nx) + nx * (m(j + dy, ny) + ny * m(k + dz, nz))];
            }
        y[i + nx * (j + ny * k)] = hc(i, nx) * hc(j, ny) * hc(k, nz) * s;
      }
}

// In-place inverse of a dense n x n matrix by Gauss-Jordan elimination with partial pivoting.
bool invert(std::vector<double>& A, int n) {
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
    if (A[(size_t)piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int t = 0; t < n; ++t) {
        std::swap(A[(size_t)c * n + t], A[(size_t)piv * n + t]);
        std::swap(I[(size_t)c * n + t], I[(size_t)piv * n + t]);
      }
    const double d = 1.0 / A[(size_t)c * n + c];
    for (int t = 0; t < n; ++t) {
      A[(size_t)c * n + t] *= d;
      I[(size_t)c * n + t] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int t = 0; t < n; ++t) {
        A[(size_t)r * n + t] -= f * A[(size_t)c * n + t];
        I[(size_t)r * n + t] -= f * I[(size_t)c * n + t];
      }
    }
  }
  A.swap(I);
  return true;
}

// Operator of Eq. k-T on a level, applied on the host to a dense vector (mirror rule), for the
// coarsest matrix when the fine grid is already the coarsest level.
void host_apply_kt(const Level& L, const std::vector<double>& kf, const std::vector<double>& x,
                   std::vector<double>& y) {
  const int N = (int)x.size();
  std::vector<double> kx(N), Lx(N), Lkx(N), Lk(N);
  for (int t = 0; t < N; ++t) kx[t] = kf[t] * x[t];
  host_apply_const(L, x, Lx);
  host_apply_const(L, kx, Lkx);
  host_apply_const(L, kf, Lk);
  for (int t = 0; t < N; ++t) y[t] = 0.5 * (Lkx[t] + kf[t] * Lx[t] - x[t] * Lk[t]);
}

}  // namespace

int build_galerkin_hierarchy(PlanImpl* P, std::vector<double>& dense) {
  const nn4_dtype ct = P->T == NN4_F64 ? NN4_F64 : NN4_F32;
  const size_t cs = dtype_size(ct);
  int rc;
  void* prev = nullptr;
  LevelGeom gprev{};
  for (size_t l = 1; l < P->lv.size(); ++l) {
    Level& L = P->lv[l];
    const size_t n27 = (size_t)kA27 * L.g.pitch * L.g.ny * L.g.nz;
    void* tmp = nullptr;
    if ((rc = alloc(P, &tmp, n27 * cs))) return rc;
    if (l == 1)
      rc = launch_galerkin_from_k(ct, P->k64, P->g64, P->lv[0].h, tmp, L.g, 0);
    else
      rc = launch_galerkin_next(ct, prev, gprev, tmp, L.g, 0);
    if (rc || (rc = launch_symmetrize27(ct, tmp, L.g, 0))) return rc;
    if (P->T == ct) {
      L.a27 = tmp;
    } else {
      if ((rc = alloc(P, &L.a27, n27 * dtype_size(P->T)))) return rc;
      if ((rc = launch_convert27(ct, tmp, P->T, L.a27, L.g, 0))) return rc;
    }
    prev = tmp;
    gprev = L.g;
  }
  Level& C = P->lv.back();
  const int nx = C.g.nx, ny = C.g.ny, nz = C.g.nz, N = nx * ny * nz;
  dense.assign((size_t)N * N, 0.0);
  if (P->lv.size() == 1) {
    std::vector<double> kf(N), k64((size_t)P->g64.pitch * ny * nz);
    if ((rc = check_cuda(cudaMemcpy(k64.data(), P->k64, k64.size() * 8, cudaMemcpyDeviceToHost), "copy k")))
      return rc;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) kf[i + nx * (j + ny * k)] = k64[i + P->g64.pitch * (j + (size_t)ny * k)];
    std::vector<double> x(N, 0.0), y(N);
    for (int j = 0; j < N; ++j) {
      x[j] = 1.0;
      host_apply_kt(C, kf, x, y);
      for (int i = 0; i < N; ++i) dense[(size_t)i * N + j] = y[i];
      x[j] = 0.0;
    }
    return NN4_OK;
  }
  const size_t plane = (size_t)C.g.pitch * ny * nz;
  std::vector<char> host(kA27 * plane * cs);
  if ((rc = check_cuda(cudaMemcpy(host.data(), prev, host.size(), cudaMemcpyDeviceToHost), "copy coarsest")))
    return rc;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        for (int d = 0; d < kA27; ++d) {
          const int i2 = i + d % 3 - 1, j2 = j + (d / 3) % 3 - 1, k2 = k + d / 9 - 1;
          if (i2 < 0 || i2 >= nx || j2 < 0 || j2 >= ny || k2 < 0 || k2 >= nz) continue;
          const size_t o = d * plane + i + C.g.pitch * (j + (size_t)ny * k);
          const double v = ct == NN4_F64 ? reinterpret_cast<const double*>(host.data())[o]
                                         : (double)reinterpret_cast<const float*>(host.data())[o];
          dense[(size_t)(i + nx * (j + ny * k)) * N + (i2 + nx * (j2 + ny * k2))] = v;
        }
  return NN4_OK;
}

namespace {

bool is_dir(const LevelGeom& g, int i, int j, int k) {
  return (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
         (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
}

// Dense (pseudo-)inverse of the coarsest operator over its free nodes.
int build_coarsest(PlanImpl* P, const std::vector<double>& dense_all) {
  Level& C = P->lv.back();
  const int nx = C.g.nx, ny = C.g.ny, nz = C.g.nz, N = nx * ny * nz;
  std::vector<int> free_lin, free_off;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        if (!is_dir(C.g, i, j, k)) {
          free_lin.push_back(i + nx * (j + ny * k));
          free_off.push_back((int)(i + C.g.pitch * (j + (long long)ny * k)));
        }
  const int n = (int)free_lin.size();
  if (n > 1024) return set_error(NN4_EUNSUPPORTED, "coarsest level has more than 1024 free nodes");
  if (n == 0) return set_error(NN4_EINVAL, "coarsest level has no free node");
  std::vector<double> A((size_t)n * n);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) A[(size_t)a * n + b] = dense_all[(size_t)free_lin[a] * N + free_lin[b]];
  bool singular = true;
  for (int f = 0; f < 6; ++f) singular = singular && !C.g.dir[f];
  if (singular)  // null space = constants: pinv(A) = (A + J/n)^-1 - J/n
    for (auto& v : A) v += 1.0 / n;
  if (!invert(A, n)) return set_error(NN4_EINVAL, "coarsest operator is singular");
  if (singular)
    for (auto& v : A) v -= 1.0 / n;
  P->ainv_host = A;
  P->free_lin_host = free_lin;
  int rc;
  if ((rc = alloc(P, (void**)&P->ainv, sizeof(double) * n * n))) return rc;
  if ((rc = alloc(P, (void**)&P->free_idx, sizeof(int) * n))) return rc;
  if ((rc = check_cuda(cudaMemcpy(P->ainv, A.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice), "copy ainv")))
    return rc;
  if ((rc = check_cuda(cudaMemcpy(P->free_idx, free_off.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "copy idx")))
    return rc;
  P->nfree = n;
  return NN4_OK;
}

// ---------------------------------------------------------------- dense tail map
// With a zero initial guess, everything the cycle does at and below level T (restriction to the
// coarsest level, the coarsest solve, prolongation and one Jacobi sweep per level back up to T)
// is a linear map r_T -> e_T.  The cooperative form applies it as one dense mat-vec; it is built
// here column by column by running exactly those steps on the host in FP64 on unit vectors, with
// the coefficients the device holds (converted exactly to FP64).
struct HostLevel {
  LevelGeom g;
  Coef8 L;
  std::vector<double> a27;  // [27][nodes], empty for the constant operator
  int n = 0;
};

int host_level(PlanImpl* P, int l, HostLevel* H) {
  const Level& L = P->lv[l];
  H->g = L.g;
  H->L = L.L;
  H->n = L.g.nx * L.g.ny * L.g.nz;
  if (!(P->vc && L.a27)) return NN4_OK;
  const size_t plane = (size_t)L.g.pitch * L.g.ny * L.g.nz, es = dtype_size(P->T);
  std::vector<char> raw(kA27 * plane * es);
  int rc;
  if ((rc = check_cuda(cudaMemcpy(raw.data(), L.a27, raw.size(), cudaMemcpyDeviceToHost), "copy tail coefficients")))
    return rc;
  H->a27.assign((size_t)kA27 * H->n, 0.0);
  for (int d = 0; d < kA27; ++d)
    for (int k = 0; k < L.g.nz; ++k)
      for (int j = 0; j < L.g.ny; ++j)
        for (int i = 0; i < L.g.nx; ++i) {
          const size_t o = d * plane + i + L.g.pitch * (j + (size_t)L.g.ny * k);
          double v;
          if (P->T == NN4_F64) {
            v = reinterpret_cast<const double*>(raw.data())[o];
          } else if (P->T == NN4_F32) {
            v = reinterpret_cast<const float*>(raw.data())[o];
          } else {
            uint16_t h;
            std::memcpy(&h, raw.data() + o * 2, 2);
            const uint32_t w = (uint32_t)h << 16;
            float f;
            std::memcpy(&f, &w, 4);
            v = f;
          }
          H->a27[(size_t)d * H->n + i + L.g.nx * (j + (size_t)L.g.ny * k)] = v;
        }
  return NN4_OK;
}

int hmirror(int i, int n) { return i < 0 ? -i : (i >= n ? 2 * (n - 1) - i : i); }

void host_restrict(const HostLevel& F, const HostLevel& C, const std::vector<double>& rf, std::vector<double>& rc) {
  const LevelGeom &f = F.g, &c = C.g;
  rc.assign(C.n, 0.0);
  for (int K = 0; K < c.nz; ++K)
    for (int J = 0; J < c.ny; ++J)
      for (int I = 0; I < c.nx; ++I) {
        if (is_dir(c, I, J, K)) continue;
        double acc = 0.0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
              if (i < 0 || i >= f.nx || j < 0 || j >= f.ny || k < 0 || k >= f.nz) continue;
              acc += (dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0) * rf[i + f.nx * (j + f.ny * k)];
            }
        rc[I + c.nx * (J + c.ny * K)] = acc;
      }
}

void host_prolong(const HostLevel& C, const HostLevel& F, const std::vector<double>& ec, std::vector<double>& t) {
  const LevelGeom &f = F.g, &c = C.g;
  t.assign(F.n, 0.0);
  for (int k = 0; k < f.nz; ++k)
    for (int j = 0; j < f.ny; ++j)
      for (int i = 0; i < f.nx; ++i) {
        if (is_dir(f, i, j, k)) continue;
        double v = 0.0;
        for (int cz = 0; cz < 2; ++cz)
          for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx)
              v += ec[((i >> 1) + cx * (i & 1)) + c.nx * (((j >> 1) + cy * (j & 1)) + c.ny * ((k >> 1) + cz * (k & 1)))];
        t[i + f.nx * (j + f.ny * k)] = 0.125 * v;
      }
}

void host_jacobi(const HostLevel& L, double omega, const std::vector<double>& t, const std::vector<double>& r,
                 std::vector<double>& e) {
  const LevelGeom& g = L.g;
  e.assign(L.n, 0.0);
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) {
        const int o = i + g.nx * (j + g.ny * k);
        if (is_dir(g, i, j, k)) {
          e[o] = t[o];
          continue;
        }
        double s = 0.0, D;
        for (int d = 0; d < kA27; ++d) {
          const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
          const double xv = t[hmirror(i + dx, g.nx) + g.nx * (hmirror(j + dy, g.ny) + g.ny * hmirror(k + dz, g.nz))];
          if (!L.a27.empty())
            s += L.a27[(size_t)d * L.n + o] * xv;
          else
            s += L.L.c[(dx != 0) + 2 * (dy != 0) + 4 * (dz != 0)] * xv;
        }
        if (!L.a27.empty()) {
          D = L.a27[(size_t)13 * L.n + o];
        } else {
          const double w = 0.125 * ((i > 0) + (i < g.nx - 1)) * ((j > 0) + (j < g.ny - 1)) * ((k > 0) + (k < g.nz - 1));
          s *= w;
          D = w * L.L.c[0];
        }
        e[o] = t[o] + omega * (r[o] - s) / D;
      }
}

int build_tail_map(PlanImpl* P) {
  const int nl = (int)P->lv.size(), T = P->coarse_dense;
  std::vector<HostLevel> H(nl);
  int rc;
  for (int l = T; l < nl; ++l)
    if ((rc = host_level(P, l, &H[l]))) return rc;
  const int n = H[T].n, nf = P->nfree;
  std::vector<double> M((size_t)n * n, 0.0);
  std::vector<std::vector<double>> r(nl), e(nl);
  std::vector<double> t;
  for (int c = 0; c < n; ++c) {
    r[T].assign(n, 0.0);
    r[T][c] = 1.0;
    for (int l = T; l + 1 < nl; ++l) host_restrict(H[l], H[l + 1], r[l], r[l + 1]);
    e[nl - 1].assign(H[nl - 1].n, 0.0);
    for (int a = 0; a < nf; ++a) {
      double v = 0.0;
      for (int b = 0; b < nf; ++b) v += P->ainv_host[(size_t)a * nf + b] * r[nl - 1][P->free_lin_host[b]];
      e[nl - 1][P->free_lin_host[a]] = v;
    }
    for (int l = nl - 2; l >= T; --l) {
      host_prolong(H[l + 1], H[l], e[l + 1], t);
      host_jacobi(H[l], P->o.omega, t, r[l], e[l]);
    }
    for (int a = 0; a < n; ++a) M[(size_t)a * n + c] = e[T][a];
  }
  std::vector<int> idx(n);
  const LevelGeom& g = P->lv[T].g;
  for (int k = 0; k < g.nz; ++k)
    for (int j = 0; j < g.ny; ++j)
      for (int i = 0; i < g.nx; ++i) idx[i + g.nx * (j + g.ny * k)] = (int)(i + g.pitch * (j + (long long)g.ny * k));
  if ((rc = alloc(P, (void**)&P->tail_map, sizeof(double) * M.size())) ||
      (rc = alloc(P, (void**)&P->tail_idx, sizeof(int) * n)) ||
      (rc = check_cuda(cudaMemcpy(P->tail_map, M.data(), sizeof(double) * M.size(), cudaMemcpyHostToDevice), "copy tail map")) ||
      (rc = check_cuda(cudaMemcpy(P->tail_idx, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "copy tail index")))
    return rc;
  P->tail_n = n;
  return NN4_OK;
}

// ---------------------------------------------------------------- the cycle
// One V-cycle on A e = r at level 0.  `first`: e = 0 on entry (the fine residual is r itself).
// rhs/e/t pointers and maps of level 0 are taken from the level (inner solve) or given
// (standalone cycle on caller arrays).
struct Fine {
  const void* r;
  void* e;
  const PassMaps* res_maps;  // residual pass on (e, r); NULL: built per launch
  const PassMaps* jac_maps;  // level-0 Jacobi pass (t, r); NULL: built per launch
  const PassMaps* rr_maps = nullptr;  // residual + restriction on (e, r); NULL: built per launch
  const float* dq = nullptr;  // optional: the final level-0 sweep also adds e.dq to *dq_out
  double* dq_out = nullptr;
};

// Level-l residual / Jacobi pass.  Level 0 with a coefficient field uses k (and, for FP64
// hierarchies, the precomputed L k and inverse diagonal); Galerkin levels use their 27 arrays.
PassArgs level_args(PlanImpl* P, int l, const void* b, void* out) {
  Level& L = P->lv[l];
  PassArgs a{};
  a.g = L.g;
  a.L = L.L;
  a.omega = P->o.omega;
  a.b = b;
  a.out = out;
  a.zchunk = L.cfg.zchunk;
  if (P->vc && l == 0) {
    a.lk = P->lkT;
    a.invd = P->T == NN4_F64 ? P->invd64 : P->invdT;
  }
  return a;
}

int run_pass(PlanImpl* P, int l, int op, const void* x, const PassMaps* maps, const void* b, void* out,
             cudaStream_t s, double* norm2 = nullptr, const float* dq = nullptr, double* dq_out = nullptr,
             const void* ec = nullptr) {
  Level& L = P->lv[l];
  PassArgs a = level_args(P, l, b, out);
  a.norm2 = norm2;
  a.dq = dq;
  a.dq_pitch = P->g32.pitch;
  a.dq_out = dq_out;
  a.ec = ec;
  if (ec) a.gc = P->lv[l + 1].g;
  if (P->vc && l > 0)
    return K(P, std::string("pass27:") + opname(op) + ":" + lvl(l), s,
             [&] { return launch_pass27(P->T, op, a, x, L.a27, s); });
  const bool vc0 = P->vc && l == 0;
  return K(P, std::string("pass:") + opname(op) + ":" + lvl(l), s,
           [&] { return launch_pass(P->T, op, a, x, vc0 ? L.k : nullptr, L.cfg, s, maps); });
}

// Arguments of the level-0 residual + restriction pass (b = r, output level 1's right-hand side).
PassArgs rr_args(PlanImpl* P, const void* r) {
  PassArgs a = level_args(P, 0, r, P->lv[1].r);
  a.invd = nullptr;
  a.gc = P->lv[1].g;
  a.zchunk = rr_default_zchunk(a.gc, 1216);
  return a;
}

int vcycle_impl(PlanImpl* P, const Fine& F, bool first, cudaStream_t s) {
  const int nl = (int)P->lv.size();
  const nn4_dtype T = P->T;
  int rc;
  Level& L0 = P->lv[0];
  if (nl == 1) {  // the fine grid is the coarsest: e += A^-1 (r - A e)
    if (first)
      return K(P, "coarsest", s, [&] { return launch_coarse_solve(T, P->ainv, P->free_idx, P->nfree, F.r, F.e, L0.g, 0, s); });
    if ((rc = run_pass(P, 0, OP_RESIDUAL, F.e, F.res_maps, F.r, L0.t, s))) return rc;
    return K(P, "coarsest", s, [&] { return launch_coarse_solve(T, P->ainv, P->free_idx, P->nfree, L0.t, F.e, L0.g, 1, s); });
  }
  // down: level 1's right-hand side R (r - A e), then restriction to the coarsest level
  if (first) {  // e = 0: the fine residual is r itself
    if ((rc = K(P, "restrict:L0", s, [&] { return launch_restrict(T, F.r, L0.g, P->lv[1].r, P->lv[1].g, s); })))
      return rc;
  } else {  // one pass; the fine residual is not stored
    PassArgs a = rr_args(P, F.r);
    if ((rc = K(P, "residual_restrict:L0", s, [&] {
           return launch_residual_restrict(T, a, F.e, P->vc ? L0.k : nullptr, s, F.rr_maps);
         })))
      return rc;
  }
  const int ts = P->tail_start > 0 ? P->tail_start : nl;  // levels >= ts run in one launch
  const int top = P->coarse_coop ? P->coarse_top : -1;     // its transfers run there too
  const int host_down = top > 0 ? top : ts;                // host restrictions end at this level
  for (int l = 1; l + 1 < nl && l < host_down; ++l)
    if ((rc = K(P, "restrict:" + lvl(l), s,
                [&] { return launch_restrict(T, P->lv[l].r, P->lv[l].g, P->lv[l + 1].r, P->lv[l + 1].g, s); })))
      return rc;
  if (ts < nl) {
    TailArgs ta{};
    const int first = top > 0 ? top : ts;
    const int last = P->coarse_coop ? P->coarse_dense : nl - 1;
    ta.nlev = last - first + 1;
    for (int l = first; l <= last; ++l) {
      Level& L = P->lv[l];
      TailLevel& t = ta.lv[l - first];
      t.g = L.g;
      t.L = L.L;
      t.r = L.r;
      t.e = L.e;
      t.t = L.t;
      t.a27 = P->vc ? L.a27 : nullptr;
    }
    ta.ainv = P->coarse_coop ? P->tail_map : P->ainv;
    ta.free_idx = P->coarse_coop ? P->tail_idx : P->free_idx;
    ta.nfree = P->coarse_coop ? P->tail_n : P->nfree;
    ta.dense_all = P->coarse_coop ? 1 : 0;
    ta.omega = P->o.omega;
    if (P->coarse_coop) {
      if ((rc = K(P, "coarse_levels", s, [&] { return launch_coarse(T, ta, P->gbar, s); }))) return rc;
    } else if ((rc = K(P, "coarse_tail", s, [&] { return launch_tail(T, ta, s); }))) {
      return rc;
    }
  } else {
    Level& C = P->lv[nl - 1];
    if ((rc = K(P, "coarsest", s,
                [&] { return launch_coarse_solve(T, P->ainv, P->free_idx, P->nfree, C.r, C.e, C.g, 0, s); })))
      return rc;
  }
  // up: prolongation then one Jacobi sweep per level above the tail
  for (int l = std::min(ts, nl - 1) - 1; l >= 1; --l) {
    Level& L = P->lv[l];
    if (l != top && (rc = K(P, "prolong:" + lvl(l), s, [&] {
                       return launch_prolong_base(T, P->lv[l + 1].e, P->lv[l + 1].g, L.t, nullptr, L.g, s);
                     })))
      return rc;
    if ((rc = run_pass(P, l, OP_JACOBI, L.t, &L.m_jac, L.r, L.e, s))) return rc;
  }
  // a cycle from e = 0 with the plan's own maps: the level-0 sweep forms P e_1 itself
  const bool fuse = first && F.jac_maps != nullptr && P->o.fused_prolong;
  if (!fuse && (rc = K(P, "prolong:L0", s, [&] {
                  return launch_prolong_base(T, P->lv[1].e, P->lv[1].g, L0.t, first ? nullptr : F.e, L0.g, s);
                })))
    return rc;
  return run_pass(P, 0, OP_JACOBI, L0.t, F.jac_maps, F.r, F.e, s, nullptr, F.dq, F.dq_out,
                  fuse ? P->lv[1].e : nullptr);
}

// ---------------------------------------------------------------- outer iterations
// inner_cycles V-cycles on A e = r at level 0 from e = 0.  dq_par >= 0 (inner Krylov loop, more
// than one level): the last cycle's final sweep also accumulates e . q[dq_par] into scal[8].
int inner_solve(PlanImpl* P, cudaStream_t s, int dq_par = -1) {
  Level& L0 = P->lv[0];
  Fine F{L0.r, L0.e, &L0.m_res, &L0.m_jac};
  F.rr_maps = &L0.m_rr;
  int rc;
  for (int c = 0; c < P->o.inner_cycles; ++c) {
    Fine Fc = F;
    if (dq_par >= 0 && c + 1 == P->o.inner_cycles) {
      Fc.jac_maps = &L0.m_jac_dq[dq_par];
      Fc.dq = P->qi[dq_par];
      Fc.dq_out = P->scal + 8;
    }
    if ((rc = vcycle_impl(P, Fc, c == 0, s))) return rc;
  }
  return NN4_OK;
}

// The fused dot applies when the cycle ends in a level-0 Jacobi sweep (more than one level).
bool fused_dot(const PlanImpl* P) { return P->lv.size() > 1; }

int outer_residual(PlanImpl* P, cudaStream_t s, double* norm2) {
  // r64 = b - A x (FP64) and its squared norm
  PassArgs a{};
  a.g = P->g64;
  a.L = P->L64;
  a.b = P->b64;
  a.out = P->r64;
  a.norm2 = norm2;
  a.zchunk = P->cfg64.zchunk;
  a.lk = P->vc ? P->lk64 : nullptr;
  int rc;
  if ((rc = check_cuda(cudaMemsetAsync(norm2, 0, sizeof(double), s), "zero norm"))) return rc;
  return K(P, "pass64:residual", s, [&] {
    return launch_pass(NN4_F64, OP_RESIDUAL, a, P->x64, P->vc ? P->k64 : nullptr, P->cfg64, s, &P->m_res64);
  });
}

// The preconditioned vector z of the outer loop.
struct ZRef {
  nn4_dtype t;
  const void* p;
  LevelGeom g;
};

// Where the outer loop puts the residual for the preconditioner (rT) and its type.
void residual_sink(PlanImpl* P, nn4_dtype* t, void** p, LevelGeom* g) {
  if (P->o.inner_krylov > 0) {
    *t = NN4_F32;
    *p = P->ri;
    *g = P->g32;
  } else {
    *t = P->T;
    *p = P->T == NN4_F64 ? nullptr : P->lv[0].r;  // FP64: level 0 reads r64 directly
    *g = P->lv[0].g;
  }
}

// Inner flexible CG (FP32 vectors) on A y = ri from y = 0, `inner_krylov` iterations, each
// preconditioned by the V-cycles; ri holds the outer residual on entry.
int inner_krylov(PlanImpl* P, cudaStream_t s) {
  Level& L0 = P->lv[0];
  int rc;
  const size_t fb = field_bytes(P->g32, NN4_F32);
  if ((rc = check_cuda(cudaMemsetAsync(P->yi, 0, fb, s), "zero y")) ||
      (rc = check_cuda(cudaMemsetAsync(P->pi[1], 0, fb, s), "zero p")) ||
      (rc = check_cuda(cudaMemsetAsync(P->qi[1], 0, fb, s), "zero q")) ||
      (rc = K(P, "pointwise:scalars", s, [&] { return launch_scalars(P->scal, -1, -1, -1, -1, 10, 15, s); })))
    return rc;
  if (P->T == NN4_BF16 &&
      (rc = K(P, "pointwise:convert", s, [&] { return launch_convert(NN4_F32, P->ri, P->g32, NN4_BF16, L0.r, L0.g, s); })))
    return rc;
  const bool fuse = fused_dot(P);
  for (int j = 0; j < P->o.inner_krylov; ++j) {
    const int par = j & 1, old = 1 - par;
    // z.q_old, p.q, p.r of this iteration and |r|^2 of its update start at zero (one launch)
    if ((rc = K(P, "pointwise:scalars", s, [&] { return launch_scalars(P->scal, 8, 9 + par, 11 + par, 13, -1, 0, s); })))
      return rc;
    if ((rc = inner_solve(P, s, fuse ? old : -1))) return rc;
    if (!fuse && (rc = K(P, "inner:dot", s, [&] {
                    return launch_dot(P->T, L0.e, L0.g, NN4_F32, P->qi[old], P->g32, P->scal + 8, s);
                  })))
      return rc;
    if ((rc = K(P, "inner:direction", s, [&] {
           return launch_direction(P->T, L0.e, L0.g, NN4_F32, P->pi[old], P->pi[par], P->g32, P->scal + 8,
                                   P->scal + 9 + old, s);
         })))
      return rc;
    PassArgs a{};
    a.g = P->g32;
    a.L = L0.L;
    a.b = P->ri;
    a.lk = P->vc ? P->lk32 : nullptr;
    a.out = P->qi[par];
    a.norm2 = P->scal + 9 + par;
    a.dot2 = P->scal + 11 + par;
    a.zchunk = P->cfg32.zchunk;
    if ((rc = K(P, "inner:matvec", s, [&] {
           return launch_pass(NN4_F32, OP_MATVEC, a, P->pi[par], P->vc ? P->k32 : nullptr, P->cfg32, s,
                              &P->m_mat32[par]);
         })))
      return rc;
    if ((rc = K(P, "inner:update", s, [&] {
           return launch_update(NN4_F32, P->yi, P->ri, P->pi[par], P->qi[par], P->g32, P->T,
                                P->T == NN4_BF16 ? L0.r : nullptr, L0.g, P->scal + 11 + par, P->scal + 9 + par,
                                P->scal + 13, s);
         })))
      return rc;
  }
  return NN4_OK;
}

// Applies the preconditioner to the residual left by the outer loop in its sink.
int precondition(PlanImpl* P, cudaStream_t s, ZRef* z) {
  if (P->o.inner_krylov > 0) {
    *z = ZRef{NN4_F32, P->yi, P->g32};
    return inner_krylov(P, s);
  }
  *z = ZRef{P->T, P->lv[0].e, P->lv[0].g};
  return inner_solve(P, s);
}

// One defect-correction iteration: rT = r; e = B(rT); x += e; r = b - A x (norm -> scal[0]).
int iteration_cycles(PlanImpl* P, cudaStream_t s) {
  int rc;
  nn4_dtype tt;
  void* rt;
  LevelGeom gt;
  residual_sink(P, &tt, &rt, &gt);
  if (rt && (rc = K(P, "pointwise:to_inner", s, [&] { return launch_convert(NN4_F64, P->r64, P->g64, tt, rt, gt, s); })))
    return rc;
  ZRef z;
  if ((rc = precondition(P, s, &z))) return rc;
  if ((rc = K(P, "pointwise:add_correction", s, [&] { return launch_add_correction(z.t, P->x64, P->g64, z.p, z.g, s); })))
    return rc;
  return outer_residual(P, s, P->scal + 0);
}

// One flexible-CG iteration with parity `par` (p, q buffers and p.q, p.r slots alternate).
int iteration_fcg(PlanImpl* P, int par, cudaStream_t s) {
  const int old = 1 - par;
  int rc;
  ZRef z;
  // z.q_old, p.q, p.r and |r|^2 of this iteration start at zero (one launch)
  if ((rc = K(P, "pointwise:scalars", s, [&] { return launch_scalars(P->scal, 2, 3 + par, 5 + par, 0, -1, 0, s); })))
    return rc;
  if ((rc = precondition(P, s, &z))) return rc;
  if ((rc = K(P, "pointwise:dot", s,
              [&] { return launch_dot(z.t, z.p, z.g, NN4_F64, P->q64[old], P->g64, P->scal + 2, s); })))
    return rc;
  if ((rc = K(P, "pointwise:direction", s, [&] {
         return launch_direction(z.t, z.p, z.g, NN4_F64, P->p64[old], P->p64[par], P->g64, P->scal + 2,
                                 P->scal + 3 + old, s);
       })))
    return rc;
  PassArgs a{};
  a.g = P->g64;
  a.L = P->L64;
  a.b = P->r64;
  a.out = P->q64[par];
  a.norm2 = P->scal + 3 + par;
  a.dot2 = P->scal + 5 + par;
  a.zchunk = P->cfg64.zchunk;
  a.lk = P->vc ? P->lk64 : nullptr;
  if ((rc = K(P, "pass64:matvec", s, [&] {
         return launch_pass(NN4_F64, OP_MATVEC, a, P->p64[par], P->vc ? P->k64 : nullptr, P->cfg64, s,
                            &P->m_mat64[par]);
       })))
    return rc;
  nn4_dtype tt;
  void* rt;
  LevelGeom gt;
  residual_sink(P, &tt, &rt, &gt);
  return K(P, "pointwise:fcg_update", s, [&] {
    return launch_update(NN4_F64, P->x64, P->r64, P->p64[par], P->q64[par], P->g64, tt, rt, gt, P->scal + 5 + par,
                         P->scal + 3 + par, P->scal + 0, s);
  });
}

int iteration(PlanImpl* P, int it, cudaStream_t s) {
  return P->o.outer == NN4_OUTER_FCG ? iteration_fcg(P, it & 1, s) : iteration_cycles(P, s);
}

int ensure_graphs(PlanImpl* P) {
  if (!P->o.use_graph || P->o.profile || P->graph[0]) return NN4_OK;
  int rc;
  if (!P->graph_stream &&
      (rc = check_cuda(cudaStreamCreateWithFlags(&P->graph_stream, cudaStreamNonBlocking), "graph stream")))
    return rc;
  const int ng = P->o.outer == NN4_OUTER_FCG ? 2 : 1;
  for (int par = 0; par < ng; ++par) {
    cudaGraph_t g;
    if ((rc = check_cuda(cudaStreamBeginCapture(P->graph_stream, cudaStreamCaptureModeThreadLocal), "begin capture")))
      return rc;
    const int64_t k0 = P->kernels;
    rc = iteration(P, par, P->graph_stream);
    P->graph_kernels[par] = P->kernels - k0;
    P->kernels = k0;
    cudaError_t e = cudaStreamEndCapture(P->graph_stream, &g);
    if (rc) return rc;
    if ((rc = check_cuda(e, "end capture"))) return rc;
    e = cudaGraphInstantiate(&P->graph[par], g, 0);
    cudaGraphDestroy(g);
    if ((rc = check_cuda(e, "graph instantiate"))) return rc;
  }
  return NN4_OK;
}

int launch_iteration(PlanImpl* P, int it, cudaStream_t s) {
  if (P->o.use_graph && !P->o.profile) {
    const int par = P->o.outer == NN4_OUTER_FCG ? (it & 1) : 0;
    P->kernels += P->graph_kernels[par];
    return check_cuda(cudaGraphLaunch(P->graph[par], s), "graph launch");
  }
  return iteration(P, it, s);
}

int make_level_maps(PlanImpl* P, int l) {
  Level& L = P->lv[l];
  if (P->vc && l > 0) return NN4_OK;  // Galerkin levels use the 27-point kernel
  const void* k = (P->vc && l == 0) ? L.k : nullptr;
  PassArgs aj = level_args(P, l, L.r, L.e);
  PassArgs ar = level_args(P, l, L.r, L.t);
  if (l == 0 && P->lv.size() > 1 && P->o.fused_prolong) {  // coarse tiles of the fused prolongation
    aj.ec = P->lv[1].e;
    aj.gc = P->lv[1].g;
  }
  if (!make_pass_maps(&L.m_jac, P->T, aj, L.cfg, L.t, k) || !make_pass_maps(&L.m_res, P->T, ar, L.cfg, L.e, k))
    return set_error(NN4_ECUDA, "tensor map encode failed");
  if (l == 0 && P->lv.size() > 1 && !make_rr_maps(&L.m_rr, P->T, rr_args(P, L.r), L.e, k))
    return set_error(NN4_ECUDA, "tensor map encode failed");
  if (l == 0 && P->o.inner_krylov > 0)
    for (int t = 0; t < 2; ++t) {
      PassArgs ad = aj;
      ad.dq = P->qi[t];
      ad.dq_pitch = P->g32.pitch;
      if (!make_pass_maps(&L.m_jac_dq[t], P->T, ad, L.cfg, L.t, k)) return set_error(NN4_ECUDA, "tensor map encode failed");
    }
  return NN4_OK;
}

// Maps of the outer-loop passes (FP64) and of the inner Krylov mat-vec (FP32).
int make_outer_maps(PlanImpl* P) {
  PassArgs a{};
  a.g = P->g64;
  a.b = P->b64;
  a.lk = P->vc ? P->lk64 : nullptr;
  bool ok = make_pass_maps(&P->m_res64, NN4_F64, a, P->cfg64, P->x64, P->vc ? P->k64 : nullptr);
  if (P->o.outer == NN4_OUTER_FCG) {
    a.b = P->r64;
    for (int t = 0; t < 2; ++t)
      ok = ok && make_pass_maps(&P->m_mat64[t], NN4_F64, a, P->cfg64, P->p64[t], P->vc ? P->k64 : nullptr);
  }
  if (P->o.inner_krylov > 0) {
    PassArgs b{};
    b.g = P->g32;
    b.b = P->ri;
    b.lk = P->vc ? P->lk32 : nullptr;
    for (int t = 0; t < 2; ++t)
      ok = ok && make_pass_maps(&P->m_mat32[t], NN4_F32, b, P->cfg32, P->pi[t], P->vc ? P->k32 : nullptr);
  }
  return ok ? NN4_OK : set_error(NN4_ECUDA, "tensor map encode failed");
}

// ---------------------------------------------------------------- autotuner
// Picks, for every stencil pass of the plan, the fastest tile shape / pipeline depth / z-march
// depth among the compiled candidates by timing each on the plan's own arrays (outputs go to
// buffers that are scratch at plan creation).  Choices are cached per process by
// (dtype, operator kind, op, grid size).
struct TuneKey {
  int dt, vmode, op, nx, ny, nz, iso;
  bool operator==(const TuneKey& o) const {
    return dt == o.dt && vmode == o.vmode && op == o.op && nx == o.nx && ny == o.ny && nz == o.nz && iso == o.iso;
  }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, PassCfg>> g_tune_cache;

int tune_pass(nn4_dtype dt, int op, PassArgs a, const void* x, const void* k, PassCfg* cfg, cudaStream_t s) {
  const bool iso = a.L.c[1] == 0.0 && a.L.c[2] == 0.0 && a.L.c[4] == 0.0;
  const TuneKey key{(int)dt, k ? (a.lk ? 2 : 1) : 0, op, a.g.nx, a.g.ny, a.g.nz, iso ? 1 : 0};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& e : g_tune_cache)
      if (e.first == key) {
        *cfg = e.second;
        return NN4_OK;
      }
  }
  double* nrm = nullptr;
  int rc;
  if ((rc = check_cuda(cudaMalloc(&nrm, 2 * sizeof(double)), "tune scratch"))) return rc;
  a.norm2 = (op == OP_RESIDUAL || op == OP_MATVEC) ? nrm : nullptr;
  a.dot2 = op == OP_MATVEC ? nrm + 1 : nullptr;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const PassCfg base = default_pass_cfg(dt, k != nullptr, a.g);
  float best = 1e30f;
  PassCfg best_cfg = *cfg;
  for (int c = 0; c < num_pass_cfgs(); ++c) {
    for (int zf = 0; zf < 3; ++zf) {
      const int zc = std::max(4, std::min(a.g.nz, zf == 0 ? base.zchunk : zf == 1 ? base.zchunk * 2 : base.zchunk / 2));
      PassCfg cand = pass_cfg_candidate(c, a.g, zc);
      PassMaps m;
      if (!make_pass_maps(&m, dt, a, cand, x, k)) continue;
      a.zchunk = cand.zchunk;
      if (launch_pass(dt, op, a, x, k, cand, s, &m) != NN4_OK) {
        cudaGetLastError();
        continue;
      }
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) launch_pass(dt, op, a, x, k, cand, s, &m);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_cfg = cand;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(nrm);
  if ((rc = check_cuda(cudaGetLastError(), "autotune"))) return rc;
  *cfg = best_cfg;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.push_back({key, best_cfg});
  return NN4_OK;
}

// Every stencil pass of the plan on compiled shape `index` (z chunks as by default); shapes
// compiled for FP64 only are applied to the FP64 passes only.
void force_pass_shape(PlanImpl* P, int index) {
  const bool fp64_only = index == num_pass_cfgs() - 1;
  auto apply = [&](PassCfg* c, nn4_dtype dt, const LevelGeom& g) {
    if (fp64_only && dt != NN4_F64) return;
    *c = pass_cfg_candidate(index, g, c->zchunk);
  };
  for (auto& L : P->lv) apply(&L.cfg, P->T, L.g);
  apply(&P->cfg64, NN4_F64, P->g64);
  if (P->o.inner_krylov > 0) apply(&P->cfg32, NN4_F32, P->g32);
}

int autotune_plan(PlanImpl* P) {
  int rc;
  cudaStream_t s = 0;
  for (int l = 0; l < (int)P->lv.size(); ++l) {
    if (P->vc && l > 0) continue;
    if (P->tail_start > 0 && l >= P->tail_start) continue;
    Level& L = P->lv[l];
    PassArgs a = level_args(P, l, L.r, L.e);
    if ((rc = tune_pass(P->T, OP_JACOBI, a, L.t, (P->vc && l == 0) ? L.k : nullptr, &L.cfg, s))) return rc;
  }
  PassArgs a{};
  a.g = P->g64;
  a.L = P->L64;
  a.b = P->b64;
  a.out = P->r64;
  a.lk = P->vc ? P->lk64 : nullptr;
  if ((rc = tune_pass(NN4_F64, P->o.outer == NN4_OUTER_FCG ? OP_MATVEC : OP_RESIDUAL, a, P->x64,
                      P->vc ? P->k64 : nullptr, &P->cfg64, s)))
    return rc;
  if (P->o.inner_krylov > 0) {
    PassArgs b{};
    b.g = P->g32;
    b.L = P->lv[0].L;
    b.b = P->ri;
    b.lk = P->vc ? P->lk32 : nullptr;
    b.out = P->qi[0];
    if ((rc = tune_pass(NN4_F32, OP_MATVEC, b, P->pi[1], P->vc ? P->k32 : nullptr, &P->cfg32, s))) return rc;
  }
  return NN4_OK;
}

void destroy(PlanImpl* P) {
  if (!P) return;
  for (auto& g : P->graph)
    if (g) cudaGraphExecDestroy(g);
  if (P->graph_stream) cudaStreamDestroy(P->graph_stream);
  for (auto& r : P->recs) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (void* p : P->allocs) cudaFree(p);
  if (P->host_hist) cudaFreeHost(P->host_hist);
  delete P;
}

int validate_plan_grid(const nn4_grid* g) {
  if (!g) return set_error(NN4_EINVAL, "grid is NULL");
  for (int d = 0; d < 3; ++d) {
    if (g->n[d] < 3) return set_error(NN4_EINVAL, "plans need at least 3 nodes per axis");
    if (!(g->h[d] > 0.0)) return set_error(NN4_EINVAL, "grid spacing must be positive");
  }
  for (int f = 0; f < 6; ++f)
    if (g->bc[f] != NN4_BC_DIRICHLET && g->bc[f] != NN4_BC_NATURAL) return set_error(NN4_EINVAL, "bad face condition");
  if (g->pitch < g->n[0] || (g->pitch * 8) % 16 != 0) return set_error(NN4_EINVAL, "bad FP64 pitch");
  return NN4_OK;
}

// A grid barrier left half-counted by a wait that gave up (reported through the device error
// word) is re-armed before the next solve or cycle.
int reset_barrier(PlanImpl* P, cudaStream_t s) {
  if (!P->gbar) return NN4_OK;
  return check_cuda(cudaMemsetAsync(&P->gbar->count, 0, sizeof(unsigned), s), "reset grid barrier");
}

int solve_device(PlanImpl* P, double rtol, int32_t max_iters, nn4_solve_info* info, cudaStream_t s) {
  int rc;
  if (max_iters < 0) return set_error(NN4_EINVAL, "max_iters must be >= 0");
  if ((rc = reset_barrier(P, s))) return rc;
  if (max_iters + 1 > P->hist_cap) {
    // grow the history buffers (outside any capture)
    const int cap = max_iters + 64;
    double* h = nullptr;
    double* hh = nullptr;
    if ((rc = check_cuda(cudaMalloc(&h, sizeof(double) * cap), "history alloc"))) return rc;
    if ((rc = check_cuda(cudaMallocHost(&hh, sizeof(double) * cap), "history host alloc"))) {
      cudaFree(h);
      return rc;
    }
    P->allocs.push_back(h);
    if (P->host_hist) cudaFreeHost(P->host_hist);
    P->hist = h;
    P->host_hist = hh;
    P->hist_cap = cap;
  }
  if ((rc = ensure_graphs(P))) return rc;
  // ||b||^2 over free nodes and ||x0||^2; the initial residual of x0 = 0 is b itself (zero at
  // Dirichlet nodes), which saves the FP64 residual pass
  if ((rc = check_cuda(cudaMemsetAsync(P->scal + 1, 0, sizeof(double), s), "zero")) ||
      (rc = check_cuda(cudaMemsetAsync(P->scal + 7, 0, sizeof(double), s), "zero")))
    return rc;
  const int64_t kstart = P->kernels;
  if ((rc = K(P, "pointwise:norm", s, [&] { return launch_norm_masked(P->b64, P->g64, P->scal + 1, s); })) ||
      (rc = K(P, "pointwise:norm", s, [&] { return launch_sumsq(P->x64, P->g64, P->scal + 7, s); })))
    return rc;
  double xx = 1.0;
  if ((rc = check_cuda(cudaMemcpyAsync(P->host_hist, P->scal + 7, sizeof(double), cudaMemcpyDeviceToHost, s), "read")) ||
      (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
    return rc;
  xx = P->host_hist[0];
  if (xx == 0.0) {
    if ((rc = K(P, "pointwise:copy", s, [&] { return launch_masked_copy(P->b64, P->r64, P->g64, s); })) ||
        (rc = check_cuda(cudaMemcpyAsync(P->scal + 0, P->scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s), "r.r")))
      return rc;
  } else if ((rc = outer_residual(P, s, P->scal + 0))) {
    return rc;
  }
  if (P->o.outer == NN4_OUTER_FCG) {
    // r64 holds the residual; rT for the first inner solve; p_old = q_old = 0, p.q_old = 1
    nn4_dtype tt;
    void* rt;
    LevelGeom gt;
    residual_sink(P, &tt, &rt, &gt);
    if (rt && (rc = K(P, "pointwise:to_inner", s, [&] { return launch_convert(NN4_F64, P->r64, P->g64, tt, rt, gt, s); })))
      return rc;
    // the first iteration (parity 0) reads p and q of parity 1 as its old direction and writes
    // those of parity 0 before reading them: only parity 1 starts at zero
    const size_t fb = field_bytes(P->g64, NN4_F64);
    if ((rc = check_cuda(cudaMemsetAsync(P->p64[1], 0, fb, s), "zero p")) ||
        (rc = check_cuda(cudaMemsetAsync(P->q64[1], 0, fb, s), "zero q")))
      return rc;
    const double one[2] = {1.0, 1.0};
    if ((rc = check_cuda(cudaMemcpyAsync(P->scal + 3, one, sizeof(one), cudaMemcpyHostToDevice, s), "init pq")))
      return rc;
  }
  if ((rc = check_cuda(cudaMemcpyAsync(P->hist, P->scal + 0, sizeof(double), cudaMemcpyDeviceToDevice, s), "hist")))
    return rc;
  double bb = 0.0;
  if ((rc = check_cuda(cudaMemcpyAsync(P->host_hist, P->scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "read")))
    return rc;
  if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
  bb = P->host_hist[1];
  double rr = P->host_hist[0];
  const double bn = std::sqrt(bb) > 0 ? std::sqrt(bb) : 1.0;
  if (!std::isfinite(rr) || !std::isfinite(bb)) return set_error(NN4_ENONFINITE, "non-finite initial residual");
  int it = 0;
  double rel = std::sqrt(rr) / bn;
  const int every = P->o.check_every > 0 ? P->o.check_every : 1;
  int status = NN4_OK;
  bool fixed = rtol <= 0.0;  // rtol <= 0: run exactly max_iters iterations
  while (it < max_iters && (fixed || rel > rtol)) {
    const int todo = fixed ? max_iters - it : std::min(every, max_iters - it);
    for (int t = 0; t < todo; ++t, ++it) {
      if ((rc = launch_iteration(P, it, s))) return rc;
      if ((rc = check_cuda(cudaMemcpyAsync(P->hist + it + 1, P->scal + 0, sizeof(double), cudaMemcpyDeviceToDevice, s),
                           "hist")))
        return rc;
    }
    if ((rc = check_cuda(cudaMemcpyAsync(P->host_hist, P->hist + it, sizeof(double), cudaMemcpyDeviceToHost, s), "read")))
      return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
    if (!std::isfinite(P->host_hist[0])) {
      status = set_error(NN4_ENONFINITE, "non-finite residual norm");
      break;
    }
    rel = std::sqrt(P->host_hist[0]) / bn;
  }
  // final true residual (FCG keeps a recurrence)
  if (P->o.outer == NN4_OUTER_FCG) {
    if ((rc = outer_residual(P, s, P->scal + 0))) return rc;
  }
  std::vector<double> h(it + 1);
  if ((rc = check_cuda(cudaMemcpyAsync(P->host_hist, P->scal + 0, sizeof(double), cudaMemcpyDeviceToHost, s), "read")))
    return rc;
  if ((rc = check_cuda(cudaMemcpyAsync(h.data(), P->hist, sizeof(double) * (it + 1), cudaMemcpyDeviceToHost, s), "read")))
    return rc;
  if ((rc = check_cuda(cudaStreamSynchronize(s), "sync"))) return rc;
  const double final_rel = std::sqrt(P->host_hist[0]) / bn;
  if (info) {
    info->iterations = it;
    info->cycles = it * P->o.inner_cycles;
    info->rel_res = final_rel;
    info->kernels = P->kernels - kstart;
    if (info->history)
      for (int t = 0; t <= it && t < info->history_len; ++t) info->history[t] = std::sqrt(h[t]) / bn;
  }
  if (status != NN4_OK) return status;
  if (!std::isfinite(final_rel)) return set_error(NN4_ENONFINITE, "non-finite residual norm");
  if (!fixed && final_rel > rtol) return set_error(NN4_ENOCONV, "iteration cap reached before the tolerance");
  return NN4_OK;
}

}  // namespace
}  // namespace nn4

using namespace nn4;

struct nn4_plan_s {
  PlanImpl* impl;
};

extern "C" {

void nn4_plan_opts_default(nn4_plan_opts* o) {
  if (!o) return;
  o->inner = NN4_F64;
  o->inner_cycles = 1;
  o->outer = NN4_OUTER_CYCLES;
  o->omega = 2.0 / 3.0;
  o->use_graph = 1;
  o->check_every = 1;
  o->profile = 0;
  o->inner_krylov = 0;
  o->coarse_tail = 1;
  o->autotune = 1;
  o->coarse_entry_nodes = 0;
  o->pass_shape = -1;
  o->fused_prolong = 0;
}

int nn4_plan_create(const nn4_grid* g, const double* k, const nn4_plan_opts* opts, nn4_plan* out) {
  if (!out) return set_error(NN4_EINVAL, "out is NULL");
  *out = nullptr;
  int rc;
  if ((rc = validate_plan_grid(g))) return rc;
  nn4_plan_opts o;
  nn4_plan_opts_default(&o);
  if (opts) o = *opts;
  if (o.inner != NN4_F64 && o.inner != NN4_F32 && o.inner != NN4_BF16) return set_error(NN4_EINVAL, "bad inner dtype");
  if (o.inner_cycles < 1 || o.inner_cycles > 64) return set_error(NN4_EINVAL, "inner_cycles must be in 1..64");
  if (o.inner_krylov < 0 || o.inner_krylov > 64) return set_error(NN4_EINVAL, "inner_krylov must be in 0..64");
  if (o.outer != NN4_OUTER_CYCLES && o.outer != NN4_OUTER_FCG) return set_error(NN4_EINVAL, "bad outer method");
  if (!(o.omega > 0.0 && o.omega < 2.0)) return set_error(NN4_EINVAL, "omega must lie in (0, 2)");
  if (k && reinterpret_cast<uintptr_t>(k) % 16) return set_error(NN4_EINVAL, "k is not 16-byte aligned");

  PlanImpl* P = new PlanImpl();
  P->grid = *g;
  P->o = o;
  P->T = o.inner;
  P->vc = k != nullptr;
  P->g64 = geom_of(g);
  P->L64 = stencil_coef(g->h);
  P->cfg64 = default_pass_cfg(NN4_F64, P->vc, P->g64);

  // hierarchy: halve while every axis is odd and >= 5
  {
    Level L;
    L.g = P->g64;
    // FP64 hierarchies share the caller's pitch at level 0 so that the outer residual r64 is the
    // right-hand side of the inner cycles without a copy
    L.g.pitch = P->T == NN4_F64 ? g->pitch : nn4_row_pitch(g->n[0], P->T);
    for (int d = 0; d < 3; ++d) L.h[d] = g->h[d];
    P->lv.push_back(L);
    while (true) {
      const Level& f = P->lv.back();
      if (!(f.g.nx >= 5 && f.g.ny >= 5 && f.g.nz >= 5 && (f.g.nx & 1) && (f.g.ny & 1) && (f.g.nz & 1))) break;
      Level c;
      c.g = f.g;
      c.g.nx = (f.g.nx + 1) / 2;
      c.g.ny = (f.g.ny + 1) / 2;
      c.g.nz = (f.g.nz + 1) / 2;
      c.g.pitch = nn4_row_pitch(c.g.nx, P->T);
      for (int d = 0; d < 3; ++d) c.h[d] = 2.0 * f.h[d];
      P->lv.push_back(c);
    }
  }
  {
    const int nl = (int)P->lv.size();
    // entry: the first level below the finest with at most kCoarseNodes nodes.  At most
    // kTailNodes nodes: the single-CTA tail; more: the cooperative kernel over all SMs.
    auto nodes = [&](int l) { return (long long)P->lv[l].g.nx * P->lv[l].g.ny * P->lv[l].g.nz; };
    int E = -1;
    const long long entry = o.coarse_entry_nodes > 0 ? o.coarse_entry_nodes : kCoarseNodes;
    for (int l = 1; l < nl; ++l)
      if (nodes(l) <= entry) {
        E = l;
        break;
      }
    if (o.coarse_tail && E > 0) {
      if (nodes(E) <= kTailNodes) {
        if (nl - E <= kMaxTail) P->tail_start = E;
      } else {
        // the dense map covers the first level with at most kTailNodes nodes (or the coarsest)
        int T0 = nl - 1;
        for (int l = E + 1; l < nl; ++l)
          if (nodes(l) <= kTailNodes) {
            T0 = l;
            break;
          }
        if (T0 > E && nodes(T0) <= 1024 && T0 - E + 1 <= kMaxTail) {
          P->tail_start = E;
          P->coarse_coop = true;
          P->coarse_dense = T0;
        }
      }
    }
  }
  for (auto& L : P->lv) {
    L.L = stencil_coef(L.h);
    L.cfg = default_pass_cfg(P->T, P->vc && &L == &P->lv[0], L.g);
    const size_t fb = field_bytes(L.g, P->T);
    const bool alias_r = P->T == NN4_F64 && &L == &P->lv[0];
    if ((!alias_r && (rc = alloc(P, &L.r, fb))) || (rc = alloc(P, &L.e, fb)) || (rc = alloc(P, &L.t, fb))) {
      destroy(P);
      return rc;
    }
  }
  if (P->coarse_coop && (rc = alloc(P, (void**)&P->gbar, sizeof(GridBarrier)))) {
    destroy(P);
    return rc;
  }
  const size_t fb64 = field_bytes(P->g64, NN4_F64);
  if ((rc = alloc(P, (void**)&P->x64, fb64)) || (rc = alloc(P, (void**)&P->b64, fb64)) ||
      (rc = alloc(P, (void**)&P->r64, fb64)) || (rc = alloc(P, (void**)&P->scal, 16 * sizeof(double)))) {
    destroy(P);
    return rc;
  }
  if (P->T == NN4_F64) P->lv[0].r = P->r64;
  {
    const double one = 1.0;
    if ((rc = check_cuda(cudaMemcpy(P->scal + 15, &one, sizeof(one), cudaMemcpyHostToDevice), "init scalars"))) {
      destroy(P);
      return rc;
    }
  }
  if (o.outer == NN4_OUTER_FCG) {
    for (int t = 0; t < 2; ++t)
      if ((rc = alloc(P, (void**)&P->p64[t], fb64)) || (rc = alloc(P, (void**)&P->q64[t], fb64))) {
        destroy(P);
        return rc;
      }
  }
  if (o.inner_krylov > 0) {
    if (P->T == NN4_F64) {
      destroy(P);
      return set_error(NN4_EINVAL, "inner_krylov needs an FP32 or BF16 hierarchy");
    }
    P->g32 = P->g64;
    P->g32.pitch = nn4_row_pitch(g->n[0], NN4_F32);
    P->cfg32 = default_pass_cfg(NN4_F32, P->vc, P->g32);
    const size_t fb32 = field_bytes(P->g32, NN4_F32);
    if ((rc = alloc(P, (void**)&P->yi, fb32)) || (rc = alloc(P, (void**)&P->ri, fb32)) ||
        (rc = alloc(P, (void**)&P->pi[0], fb32)) || (rc = alloc(P, (void**)&P->pi[1], fb32)) ||
        (rc = alloc(P, (void**)&P->qi[0], fb32)) || (rc = alloc(P, (void**)&P->qi[1], fb32))) {
      destroy(P);
      return rc;
    }
    if (P->T == NN4_F32) P->lv[0].r = P->ri;  // the V-cycles read the inner residual directly
  }
  if (P->vc) {
    if ((rc = alloc(P, (void**)&P->k64, fb64)) ||
        (rc = check_cuda(cudaMemcpy(P->k64, k, fb64, cudaMemcpyDeviceToDevice), "copy k")) ||
        (rc = alloc(P, (void**)&P->lk64, fb64)) || (rc = alloc(P, (void**)&P->invd64, fb64))) {
      destroy(P);
      return rc;
    }
    // (1/2) L k (assembled, natural faces; the operator's coefficients halved, exactly) and the
    // inverse diagonal, once per plan
    PassArgs a{};
    a.g = P->g64;
    a.L = P->L64;
    for (int c = 0; c < 8; ++c) a.L.c[c] *= 0.5;
    a.out = P->lk64;
    PassCfg cfg0 = default_pass_cfg(NN4_F64, false, P->g64);
    a.zchunk = cfg0.zchunk;
    if ((rc = launch_pass(NN4_F64, OP_APPLY, a, P->k64, nullptr, cfg0, 0)) ||
        (rc = launch_inv_diag(P->k64, P->lk64, P->invd64, P->g64, P->L64.c[0], 0))) {
      destroy(P);
      return rc;
    }
    if (P->T == NN4_F64) {
      P->lv[0].k = P->k64;  // same pitch at level 0
    } else if ((rc = alloc(P, &P->lv[0].k, field_bytes(P->lv[0].g, P->T))) ||
               (rc = launch_to_inner(P->T, P->k64, P->g64, P->lv[0].k, P->lv[0].g, 0))) {
      destroy(P);
      return rc;
    }
    // L k in the inner type (level-0 passes) and in FP32 (inner Krylov mat-vec)
    if (P->T == NN4_F64) {
      P->lkT = P->lk64;
    } else if ((rc = alloc(P, &P->lkT, field_bytes(P->lv[0].g, P->T))) ||
               (rc = launch_convert(NN4_F64, P->lk64, P->g64, P->T, P->lkT, P->lv[0].g, 0)) ||
               (rc = alloc(P, &P->invdT, field_bytes(P->lv[0].g, P->T))) ||
               (rc = launch_convert(NN4_F64, P->invd64, P->g64, P->T, P->invdT, P->lv[0].g, 0))) {
      destroy(P);
      return rc;
    }
    if (o.inner_krylov > 0) {
      if (P->T == NN4_F32) {
        P->k32 = static_cast<float*>(P->lv[0].k);
        P->lk32 = static_cast<float*>(P->lkT);
      } else if ((rc = alloc(P, (void**)&P->k32, field_bytes(P->g32, NN4_F32))) ||
                 (rc = launch_convert(NN4_F64, P->k64, P->g64, NN4_F32, P->k32, P->g32, 0)) ||
                 (rc = alloc(P, (void**)&P->lk32, field_bytes(P->g32, NN4_F32))) ||
                 (rc = launch_convert(NN4_F64, P->lk64, P->g64, NN4_F32, P->lk32, P->g32, 0))) {
        destroy(P);
        return rc;
      }
    }
  }
  if (o.pass_shape >= num_pass_cfgs()) {
    destroy(P);
    return set_error(NN4_EINVAL, "pass_shape out of range");
  }
  if (o.pass_shape >= 0) {
    force_pass_shape(P, o.pass_shape);
  } else if (o.autotune && (rc = autotune_plan(P))) {
    destroy(P);
    return rc;
  }
  // tensor maps of every pass (all pointers and tile shapes are final now)
  if ((rc = make_outer_maps(P))) {
    destroy(P);
    return rc;
  }
  for (int l = 0; l < (int)P->lv.size(); ++l)
    if ((rc = make_level_maps(P, l))) {
      destroy(P);
      return rc;
    }
  // coarse operators and the coarsest inverse
  std::vector<double> dense;
  if (P->vc) {
    rc = build_galerkin_hierarchy(P, dense);
  } else {
    Level& C = P->lv.back();
    const int N = C.g.nx * C.g.ny * C.g.nz;
    dense.assign((size_t)N * N, 0.0);
    std::vector<double> x(N, 0.0), y(N);
    for (int j = 0; j < N; ++j) {
      x[j] = 1.0;
      host_apply_const(C, x, y);
      for (int i = 0; i < N; ++i) dense[(size_t)i * N + j] = y[i];
      x[j] = 0.0;
    }
    rc = NN4_OK;
  }
  if (rc || (rc = build_coarsest(P, dense)) || (P->coarse_coop && (rc = build_tail_map(P))) ||
      (rc = check_cuda(cudaDeviceSynchronize(), "plan build"))) {
    destroy(P);
    return rc;
  }
  nn4_plan h = new nn4_plan_s;
  h->impl = P;
  *out = h;
  return NN4_OK;
}

int32_t nn4_pass_shapes(void) { return num_pass_cfgs(); }

int nn4_plan_destroy(nn4_plan p) {
  if (!p) return NN4_OK;
  destroy(p->impl);
  delete p;
  return NN4_OK;
}

int nn4_vcycle(nn4_plan p, const void* b, void* x, void* stream) {
  if (!p || !b || !x) return set_error(NN4_EINVAL, "NULL argument");
  if (reinterpret_cast<uintptr_t>(b) % 16 || reinterpret_cast<uintptr_t>(x) % 16)
    return set_error(NN4_EINVAL, "arrays must be 16-byte aligned");
  PlanImpl* P = p->impl;
  Fine F{b, x, nullptr, nullptr};  // caller arrays: maps are built per launch
  const int rc = reset_barrier(P, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return vcycle_impl(P, F, false, static_cast<cudaStream_t>(stream));
}

int nn4_pressure_solve(nn4_plan p, const double* b, double* x, double rtol, int32_t max_iters,
                       nn4_solve_info* info, void* stream) {
  if (!p || !b || !x) return set_error(NN4_EINVAL, "NULL argument");
  PlanImpl* P = p->impl;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t fb = field_bytes(P->g64, NN4_F64);
  int rc;
  if ((rc = check_cuda(cudaMemcpyAsync(P->b64, b, fb, cudaMemcpyDeviceToDevice, s), "copy b")) ||
      (rc = check_cuda(cudaMemcpyAsync(P->x64, x, fb, cudaMemcpyDeviceToDevice, s), "copy x")))
    return rc;
  const int st = solve_device(P, rtol, max_iters, info, s);
  if (st != NN4_OK && st != NN4_ENOCONV) return st;
  if ((rc = check_cuda(cudaMemcpyAsync(x, P->x64, fb, cudaMemcpyDeviceToDevice, s), "copy x out")) ||
      (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
    return rc;
  return st;
}

int nn4_pressure_solve_host(nn4_plan p, const double* b_host, double* x_host, double rtol, int32_t max_iters,
                            nn4_solve_info* info, void* stream) {
  if (!p || !b_host || !x_host) return set_error(NN4_EINVAL, "NULL argument");
  PlanImpl* P = p->impl;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const LevelGeom& g = P->g64;
  const size_t dense = (size_t)g.nx * g.ny * g.nz * sizeof(double);
  int rc;
  // The host arrays are dense (row pitch nx).  Each goes over the link as one contiguous copy into
  // the FP64 residual field (free until the solve writes its first residual; as large as a pitched
  // field), and a device kernel moves it to the plan's row pitch: a pitched copy of rows of a few
  // kilobytes runs the host link far below its rate.
  LevelGeom gd = g;
  gd.pitch = g.nx;
  const bool same = g.pitch == g.nx;
  auto in = [&](const double* h, double* d, const char* what) {
    int r;
    if (same) return check_cuda(cudaMemcpyAsync(d, h, dense, cudaMemcpyHostToDevice, s), what);
    if ((r = check_cuda(cudaMemcpyAsync(P->r64, h, dense, cudaMemcpyHostToDevice, s), what))) return r;
    return launch_convert(NN4_F64, P->r64, gd, NN4_F64, d, g, s);
  };
  if ((rc = in(b_host, P->b64, "copy b in")) || (rc = in(x_host, P->x64, "copy x in"))) return rc;
  const int st = solve_device(P, rtol, max_iters, info, s);
  if (st != NN4_OK && st != NN4_ENOCONV) return st;
  const double* xs = P->x64;
  if (!same) {
    if ((rc = launch_convert(NN4_F64, P->x64, g, NN4_F64, P->r64, gd, s))) return rc;
    xs = P->r64;
  }
  if ((rc = check_cuda(cudaMemcpyAsync(x_host, xs, dense, cudaMemcpyDeviceToHost, s), "copy x out")) ||
      (rc = check_cuda(cudaStreamSynchronize(s), "sync")))
    return rc;
  return st;
}

int nn4_plan_profile(nn4_plan p, nn4_kernel_time* out, int32_t cap) {
  if (!p) return set_error(NN4_EINVAL, "NULL plan");
  PlanImpl* P = p->impl;
  int rc;
  if ((rc = check_cuda(cudaDeviceSynchronize(), "sync"))) return rc;
  std::vector<std::string> names;
  std::vector<int64_t> cnt;
  std::vector<double> tot;
  for (auto& r : P->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.e0, r.e1);
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
    size_t i = 0;
    while (i < names.size() && names[i] != r.name) ++i;
    if (i == names.size()) {
      names.push_back(r.name);
      cnt.push_back(0);
      tot.push_back(0.0);
    }
    cnt[i] += 1;
    tot[i] += ms;
  }
  P->recs.clear();
  for (size_t i = 0; i < names.size() && (int)i < cap; ++i) {
    std::strncpy(out[i].name, names[i].c_str(), sizeof(out[i].name) - 1);
    out[i].name[sizeof(out[i].name) - 1] = 0;
    out[i].launches = cnt[i];
    out[i].total_ms = tot[i];
  }
  return (int)names.size();
}

int nn4_plan_query(nn4_plan p, nn4_plan_info* out) {
  if (!p || !out) return set_error(NN4_EINVAL, "NULL argument");
  PlanImpl* P = p->impl;
  std::memset(out, 0, sizeof(*out));
  out->levels = (int)P->lv.size();
  for (size_t l = 0; l < P->lv.size() && l < 16; ++l) {
    out->n[l][0] = P->lv[l].g.nx;
    out->n[l][1] = P->lv[l].g.ny;
    out->n[l][2] = P->lv[l].g.nz;
  }
  out->coarsest_free = P->nfree;
  out->device_bytes = (int64_t)P->device_bytes;
  return NN4_OK;
}

}  // extern "C"
