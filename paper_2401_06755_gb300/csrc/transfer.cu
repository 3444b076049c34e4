// Inter-grid transfers of the sawtooth multigrid (Section 2.4): stride-2 restriction R = P^T and
// trilinear prolongation P between a fine vertex grid and the grid of its even-indexed nodes.
#include "common.cuh"
#include "internal.h"

namespace nn4 {
namespace {

__device__ __forceinline__ bool dir_node(const LevelGeom& g, int i, int j, int k) {
  return (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
         (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
}

// Pairs of consecutive nodes (an even first index on a row of even pitch: aligned) as one load.
__device__ __forceinline__ void ld2(const double* p, double& a, double& b) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  a = t.x, b = t.y;
}
__device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
  const float2 t = *reinterpret_cast<const float2*>(p);
  a = t.x, b = t.y;
}
__device__ __forceinline__ void ld2(const bf16* p, float& a, float& b) {
  const float2 t = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  a = t.x, b = t.y;
}
__device__ __forceinline__ void st2(double* p, double a, double b) { *reinterpret_cast<double2*>(p) = make_double2(a, b); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(bf16* p, float a, float b) {
  *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}

// Restriction r_c(I) = sum_{d in {-1,0,1}^3} prod_d (1/2)^|d| r_f(2I + d) over the fine nodes that
// exist; zero at coarse Dirichlet nodes.  A thread owns coarse column (I, J) over kRz coarse
// planes (unrolled, so all its loads are in flight together); lane I loads the fine pair
// (2I, 2I+1) of each row and the node 2I-1.  Consecutive coarse planes share a fine plane, read
// once.
constexpr int kRz = 2;

template <typename T>
__global__ void __launch_bounds__(128) k_restrict(const T* __restrict__ rf, T* __restrict__ rc, const LevelGeom gf,
                                                  const LevelGeom gc) {
  using A = typename Acc<T>::type;
  const int I = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * 4 + threadIdx.y;
  if (J >= gc.ny) return;
  // Neighbours that do not exist (past a boundary node) are read at a clamped position with weight
  // 0, so no load sits behind a branch.
  const int i0 = 2 * min(I, gc.nx - 1);
  const bool has_r = i0 + 1 < gf.nx;
  const int dl = i0 > 0 ? -1 : 0;
  const A wl = i0 > 0 ? A(0.5) : A(0), wr = A(0.5);
  const long long rs = gf.pitch, ps = gf.pitch * (long long)gf.ny;
  const int j0 = 2 * J;
  const long long om = J > 0 ? -rs : 0, op = j0 + 1 < gf.ny ? rs : 0;
  const A wm = J > 0 ? A(0.5) : A(0), wp = j0 + 1 < gf.ny ? A(0.5) : A(0);
  const int K0 = blockIdx.z * kRz;
  const T* P0 = rf + i0 + rs * j0 + ps * (2 * K0);  // fine plane 2 K0, row 2 J
  // Every raw value first (fine planes 2K0-1 .. 2K0+2kRz-1, clamped into the grid with weight 0
  // outside; rows 2J-1, 2J, 2J+1), then the arithmetic: all 2 (2 kRz + 1) 3 loads in flight.
  constexpr int NPL = 2 * kRz + 1;
  A c[NPL][3], r[NPL][3], l[NPL][3], wpl[NPL];
#pragma unroll
  for (int q = 0; q < NPL; ++q) {
    const int k = 2 * K0 - 1 + q;
    const int kc = min(max(k, 0), gf.nz - 1);
    wpl[q] = (k >= 0 && k < gf.nz) ? A(1) : A(0);
    const T* pq = P0 + ps * (kc - 2 * K0);
    const long long ro[3] = {om, 0, op};
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      ld2(pq + ro[w], c[q][w], r[q][w]);  // r lies past the row end for the last column: not used
      l[q][w] = to_acc(pq[ro[w] + dl]);
    }
  }
  A pl[NPL];
#pragma unroll
  for (int q = 0; q < NPL; ++q) {
    A row[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) row[w] = c[q][w] + wl * l[q][w] + (has_r ? wr * r[q][w] : A(0));
    pl[q] = row[1] + wm * row[0] + wp * row[2];
  }
  const bool dxy = (gc.dir[0] && I == 0) || (gc.dir[1] && I == gc.nx - 1) || (gc.dir[2] && J == 0) ||
                   (gc.dir[3] && J == gc.ny - 1);
  T* out = rc + I + gc.pitch * ((long long)J + (long long)gc.ny * K0);
  const long long cps = gc.pitch * (long long)gc.ny;
#pragma unroll
  for (int t = 0; t < kRz; ++t) {
    const int K = K0 + t;
    if (K >= gc.nz) break;
    const A v = pl[2 * t + 1] + A(0.5) * (wpl[2 * t] * pl[2 * t] + wpl[2 * t + 2] * pl[2 * t + 2]);
    const bool dn = dxy || (gc.dir[4] && K == 0) || (gc.dir[5] && K == gc.nz - 1);
    if (I < gc.nx) out[cps * t] = from_acc<T>(dn ? A(0) : v);
  }
}

// Prolongation e_f (+)= P e_c: each fine node takes the coarse nodes bracketing it, weight 1 at an
// even index and 1/2 for each of the two parents at an odd index, per axis.  A thread owns the
// fine pair (2I, 2I+1) of row j over kPz fine planes: x-even = e_c(I), x-odd = (e_c(I) + e_c(I+1))/2.
// Dirichlet fine nodes keep base (or 0).
constexpr int kPz = 8;

template <typename T>
__global__ void __launch_bounds__(128) k_prolong(const T* __restrict__ ec, T* ef, const T* base, const LevelGeom gc,
                                                 const LevelGeom gf) {
  using A = typename Acc<T>::type;
  const int lane = threadIdx.x;
  const int I = blockIdx.x * 32 + lane;
  const int j = blockIdx.y * 4 + threadIdx.y;
  if (j >= gf.ny) return;  // whole warps only
  const int Ic = min(I, gc.nx - 1);
  const bool has_next = Ic + 1 < gc.nx;
  const int J0 = j >> 1, J1 = J0 + (j & 1);
  // (x-even, x-odd) values of coarse plane K at fine row j
  // rows J0 and J1 (= J0 for an even j, weight 1/2 each then): the branch-free sum of both
  const int In = has_next ? Ic + 1 : Ic;
  const T* const c0 = ec + gc.pitch * (long long)J0;
  const long long d1 = gc.pitch * (long long)(J1 - J0), cps = gc.pitch * (long long)gc.ny;
  auto plane = [&](int K, A& ve, A& vo) {
    const T* r0 = c0 + cps * K;
    const T* r1 = r0 + d1;
    const A a = A(0.5) * (to_acc(r0[Ic]) + to_acc(r1[Ic]));
    const A an = A(0.5) * (to_acc(r0[In]) + to_acc(r1[In]));
    ve = a;
    vo = A(0.5) * (a + an);
  };
  const int k0 = blockIdx.z * kPz, k1 = min(gf.nz, k0 + kPz);
  const int K0 = k0 >> 1;
  A ce[kPz / 2 + 1], co[kPz / 2 + 1];
  // coarse planes past the grid are clamped (their values only feed fine planes past the grid,
  // which are not stored), so all coarse loads are issued without a branch
#pragma unroll
  for (int t = 0; t <= kPz / 2; ++t) plane(min(K0 + t, gc.nz - 1), ce[t], co[t]);
  const int i = 2 * I;
  const bool ok0 = I < gc.nx, ok1 = i + 1 < gf.nx;
  const bool dy = (gf.dir[2] && j == 0) || (gf.dir[3] && j == gf.ny - 1);
  const bool d0x = (gf.dir[0] && i == 0) || (gf.dir[1] && i == gf.nx - 1);
  const bool d1x = gf.dir[1] && i + 1 == gf.nx - 1;
  T* const out0 = ef + i + gf.pitch * ((long long)j + (long long)gf.ny * k0);
  const long long fps = gf.pitch * (long long)gf.ny;
#pragma unroll
  for (int t = 0; t < kPz; ++t) {
    const int k = k0 + t;
    if (k >= k1) break;
    A v0 = (t & 1) ? A(0.5) * (ce[t >> 1] + ce[(t >> 1) + 1]) : ce[t >> 1];
    A v1 = (t & 1) ? A(0.5) * (co[t >> 1] + co[(t >> 1) + 1]) : co[t >> 1];
    const bool dz = dy || (gf.dir[4] && k == 0) || (gf.dir[5] && k == gf.nz - 1);
    T* out = out0 + fps * t;
    A b0 = A(0), b1 = A(0);
    if (base) {
      const T* bp = base + (out - ef);
      if (ok1) {
        ld2(bp, b0, b1);
      } else if (ok0) {
        b0 = to_acc(bp[0]);
      }
    }
    v0 = (dz || d0x) ? b0 : v0 + b0;
    v1 = (dz || d1x) ? b1 : v1 + b1;
    if (ok1) {
      st2(out, v0, v1);
    } else if (ok0) {
      out[0] = from_acc<T>(v0);
    }
  }
}

// Batched transfers: CTA b handles block (b - first) of instance entry `lo` (a grid of 32 x 4
// thread blocks over (x, y) times z-blocks).
template <typename T>
__global__ void k_restrict_batch(const BatchXfer* __restrict__ tab, int count, int total, const int* __restrict__ active) {
  using A = typename Acc<T>::type;
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].first <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const BatchXfer& X = tab[lo];
  if (active && !active[X.inst]) return;
  const int b = blockIdx.x - X.first;
  const int I = (b % X.bx) * 32 + threadIdx.x;
  const int J = ((b / X.bx) % X.by) * 4 + threadIdx.y;
  const int K = b / (X.bx * X.by);
  const LevelGeom &gf = X.gf, &gc = X.gc;
  if (I >= gc.nx || J >= gc.ny) return;
  const T* rf = static_cast<const T*>(X.src);
  A acc = A(0);
  if (!dir_node(gc, I, J, K)) {
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      const int k = 2 * K + dz;
      if (k < 0 || k >= gf.nz) continue;
      A az = A(0);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int j = 2 * J + dy;
        if (j < 0 || j >= gf.ny) continue;
        const T* row = rf + gf.pitch * ((long long)j + (long long)gf.ny * k);
        const int i = 2 * I;
        A ax = to_acc(row[i]);
        if (i > 0) ax += A(0.5) * to_acc(row[i - 1]);
        if (i + 1 < gf.nx) ax += A(0.5) * to_acc(row[i + 1]);
        az += (dy == 0 ? A(1) : A(0.5)) * ax;
      }
      acc += (dz == 0 ? A(1) : A(0.5)) * az;
    }
  }
  static_cast<T*>(X.dst)[I + gc.pitch * ((long long)J + (long long)gc.ny * K)] = from_acc<T>(acc);
}

template <typename T>
__global__ void k_prolong_batch(const BatchXfer* __restrict__ tab, int count, int total, const int* __restrict__ active) {
  using A = typename Acc<T>::type;
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab[mid].first <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const BatchXfer& X = tab[lo];
  if (active && !active[X.inst]) return;
  const int b = blockIdx.x - X.first;
  const LevelGeom &gf = X.gf, &gc = X.gc;
  const int i = (b % X.bx) * 32 + threadIdx.x;
  const int j = ((b / X.bx) % X.by) * 4 + threadIdx.y;
  const int kb = b / (X.bx * X.by);
  if (i >= gf.nx || j >= gf.ny) return;
  const T* ec = static_cast<const T*>(X.src);
  T* ef = static_cast<T*>(X.dst);
  const T* base = static_cast<const T*>(X.base);
  const int I0 = i >> 1, J0 = j >> 1;
  const int I1 = I0 + (i & 1), J1 = J0 + (j & 1);
  const A wxy = ((i & 1) ? A(0.5) : A(1)) * ((j & 1) ? A(0.5) : A(1));
  const bool dxy = (gf.dir[0] && i == 0) || (gf.dir[1] && i == gf.nx - 1) || (gf.dir[2] && j == 0) ||
                   (gf.dir[3] && j == gf.ny - 1);
  auto plane = [&](int K) {
    const T* p = ec + gc.pitch * (long long)gc.ny * K;
    A v = to_acc(p[I0 + gc.pitch * (long long)J0]);
    if (i & 1) v += to_acc(p[I1 + gc.pitch * (long long)J0]);
    if (j & 1) {
      A t = to_acc(p[I0 + gc.pitch * (long long)J1]);
      if (i & 1) t += to_acc(p[I1 + gc.pitch * (long long)J1]);
      v += t;
    }
    return v * wxy;
  };
  const int k0 = kb * kPz, k1 = min(gf.nz, k0 + kPz);
  A cp[kPz / 2 + 1];
  const int K0 = k0 >> 1;
#pragma unroll
  for (int t = 0; t <= kPz / 2; ++t) cp[t] = (K0 + t < gc.nz) ? plane(K0 + t) : A(0);
#pragma unroll
  for (int t = 0; t < kPz; ++t) {
    const int k = k0 + t;
    if (k >= k1) break;
    const A v0 = (t & 1) ? A(0.5) * (cp[t >> 1] + cp[(t >> 1) + 1]) : cp[t >> 1];
    const long long idx = i + gf.pitch * ((long long)j + (long long)gf.ny * k);
    const bool dn = dxy || (gf.dir[4] && k == 0) || (gf.dir[5] && k == gf.nz - 1);
    if (dn) {
      ef[idx] = base ? base[idx] : from_acc<T>(A(0));
      continue;
    }
    ef[idx] = from_acc<T>(base ? v0 + to_acc(base[idx]) : v0);
  }
}

template <typename T>
int restrict_t(const void* rf, const LevelGeom& gf, void* rc, const LevelGeom& gc, cudaStream_t s) {
  if ((gf.pitch & 1) || (reinterpret_cast<uintptr_t>(rf) % (2 * sizeof(T))))
    return set_error(NN4_EINVAL, "restriction needs an even row pitch and an aligned fine field");
  dim3 blk(32, 4);
  dim3 grd((gc.nx + 31) / 32, (gc.ny + 3) / 4, (gc.nz + kRz - 1) / kRz);
  k_restrict<T><<<grd, blk, 0, s>>>(static_cast<const T*>(rf), static_cast<T*>(rc), gf, gc);
  return check_cuda(cudaGetLastError(), "restrict launch");
}

template <typename T>
int prolong_t(const void* ec, const LevelGeom& gc, void* ef, const void* base, const LevelGeom& gf,
              cudaStream_t s) {
  if ((gf.pitch & 1) || (reinterpret_cast<uintptr_t>(ef) % (2 * sizeof(T))) ||
      (base && reinterpret_cast<uintptr_t>(base) % (2 * sizeof(T))))
    return set_error(NN4_EINVAL, "prolongation needs an even row pitch and aligned fine fields");
  dim3 blk(32, 4);
  dim3 grd((gc.nx + 31) / 32, (gf.ny + 3) / 4, (gf.nz + kPz - 1) / kPz);
  k_prolong<T><<<grd, blk, 0, s>>>(static_cast<const T*>(ec), static_cast<T*>(ef), static_cast<const T*>(base), gc, gf);
  return check_cuda(cudaGetLastError(), "prolong launch");
}

}  // namespace

int launch_restrict(nn4_dtype dt, const void* rf, const LevelGeom& gf, void* rc,
                    const LevelGeom& gc, cudaStream_t s) {
  switch (dt) {
    case NN4_F64: return restrict_t<double>(rf, gf, rc, gc, s);
    case NN4_F32: return restrict_t<float>(rf, gf, rc, gc, s);
    case NN4_BF16: return restrict_t<bf16>(rf, gf, rc, gc, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

int launch_prolong_base(nn4_dtype dt, const void* ec, const LevelGeom& gc, void* ef, const void* base,
                        const LevelGeom& gf, cudaStream_t s) {
  switch (dt) {
    case NN4_F64: return prolong_t<double>(ec, gc, ef, base, gf, s);
    case NN4_F32: return prolong_t<float>(ec, gc, ef, base, gf, s);
    case NN4_BF16: return prolong_t<bf16>(ec, gc, ef, base, gf, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

int launch_prolong(nn4_dtype dt, const void* ec, const LevelGeom& gc, void* ef,
                   const LevelGeom& gf, int accumulate, cudaStream_t s) {
  return launch_prolong_base(dt, ec, gc, ef, accumulate ? ef : nullptr, gf, s);
}

int batch_xfer_blocks(BatchXfer* X, bool prolong) {
  const LevelGeom& g = prolong ? X->gf : X->gc;
  X->bx = (g.nx + 31) / 32;
  X->by = (g.ny + 3) / 4;
  const int bz = prolong ? (g.nz + kPz - 1) / kPz : g.nz;
  return X->bx * X->by * bz;
}

int launch_xfer_batch(nn4_dtype dt, bool prolong, const BatchXfer* tab, int count, int total, const int* active,
                      cudaStream_t s) {
  if (total <= 0) return NN4_OK;
  dim3 blk(32, 4);
  switch (dt) {
    case NN4_F64:
      if (prolong) k_prolong_batch<double><<<total, blk, 0, s>>>(tab, count, total, active);
      else k_restrict_batch<double><<<total, blk, 0, s>>>(tab, count, total, active);
      break;
    case NN4_F32:
      if (prolong) k_prolong_batch<float><<<total, blk, 0, s>>>(tab, count, total, active);
      else k_restrict_batch<float><<<total, blk, 0, s>>>(tab, count, total, active);
      break;
    case NN4_BF16:
      if (prolong) k_prolong_batch<bf16><<<total, blk, 0, s>>>(tab, count, total, active);
      else k_restrict_batch<bf16><<<total, blk, 0, s>>>(tab, count, total, active);
      break;
  }
  return check_cuda(cudaGetLastError(), "batched transfer launch");
}

}  // namespace nn4
