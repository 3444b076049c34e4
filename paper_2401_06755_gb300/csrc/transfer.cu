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

// One thread per coarse node: r_c(I) = sum_{d in {-1,0,1}^3} prod_d (1/2)^|d| r_f(2I + d) over
// the fine nodes that exist; zero at coarse Dirichlet nodes.  Separable: x, then y, then z.
template <typename T>
__global__ void k_restrict(const T* __restrict__ rf, T* __restrict__ rc, const LevelGeom gf,
                           const LevelGeom gc) {
  using A = typename Acc<T>::type;
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= gc.nx || J >= gc.ny) return;
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
  rc[I + gc.pitch * ((long long)J + (long long)gc.ny * K)] = from_acc<T>(acc);
}

// One thread per fine node: e_f(i) (+)= sum over the coarse nodes bracketing i of
// prod_d (1 at an even index, 1/2 for each of the two parents at an odd index) e_c.
// One thread per fine (i, j) column and a run of kPz fine planes: e_f (+)= sum over the coarse
// nodes bracketing each fine node of prod_d (1 at an even index, 1/2 for each of the two parents
// at an odd index) e_c.
constexpr int kPz = 8;

template <typename T>
__global__ void k_prolong(const T* __restrict__ ec, T* ef, const T* base, const LevelGeom gc,
                          const LevelGeom gf) {
  using A = typename Acc<T>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= gf.nx || j >= gf.ny) return;
  const int I0 = i >> 1, J0 = j >> 1;
  const int I1 = I0 + (i & 1), J1 = J0 + (j & 1);
  const A wxy = ((i & 1) ? A(0.5) : A(1)) * ((j & 1) ? A(0.5) : A(1));
  const bool dxy = (gf.dir[0] && i == 0) || (gf.dir[1] && i == gf.nx - 1) || (gf.dir[2] && j == 0) ||
                   (gf.dir[3] && j == gf.ny - 1);
  // in-plane interpolation of coarse plane K at (i, j)
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
  const int k0 = blockIdx.z * kPz, k1 = min(gf.nz, k0 + kPz);
  // coarse planes k0/2 .. k0/2 + kPz/2 interpolated in-plane first (independent loads)
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
    const A v = base ? v0 + to_acc(base[idx]) : v0;
    ef[idx] = from_acc<T>(v);
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
  dim3 blk(32, 4);
  dim3 grd((gc.nx + 31) / 32, (gc.ny + 3) / 4, gc.nz);
  k_restrict<T><<<grd, blk, 0, s>>>(static_cast<const T*>(rf), static_cast<T*>(rc), gf, gc);
  return check_cuda(cudaGetLastError(), "restrict launch");
}

template <typename T>
int prolong_t(const void* ec, const LevelGeom& gc, void* ef, const void* base, const LevelGeom& gf,
              cudaStream_t s) {
  dim3 blk(32, 4);
  dim3 grd((gf.nx + 31) / 32, (gf.ny + 3) / 4, (gf.nz + kPz - 1) / kPz);
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
