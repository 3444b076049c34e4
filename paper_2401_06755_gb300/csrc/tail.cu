// The coarse tail of the sawtooth V-cycle in one launch.  Levels with few nodes cannot fill the
// GPU and every separate launch costs several microseconds of latency, so all levels at or below
// a few hundred nodes run in a single CTA: restriction down to the coarsest level, the dense
// coarsest solve, then prolongation and one Jacobi sweep per level back up to the entry level
// (Section 2.4, multigrid figure: the same steps the per-level kernels perform).
#include "common.cuh"
#include "internal.h"

namespace nn4 {
namespace {

__device__ __forceinline__ bool tdir(const LevelGeom& g, int i, int j, int k) {
  return (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
         (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
}

__device__ __forceinline__ long long off(const LevelGeom& g, int i, int j, int k) {
  return i + g.pitch * ((long long)j + (long long)g.ny * k);
}

template <typename T>
__device__ void tail_restrict(const TailLevel& F, const TailLevel& C) {
  using A = typename Acc<T>::type;
  const T* rf = static_cast<const T*>(F.r);
  T* rc = static_cast<T*>(C.r);
  const int n = C.g.nx * C.g.ny * C.g.nz;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int I = t % C.g.nx, J = (t / C.g.nx) % C.g.ny, K = t / (C.g.nx * C.g.ny);
    A acc = A(0);
    if (!tdir(C.g, I, J, K)) {
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz) {
        const int k = 2 * K + dz;
        if (k < 0 || k >= F.g.nz) continue;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
          const int j = 2 * J + dy;
          if (j < 0 || j >= F.g.ny) continue;
          const A wyz = (dz ? A(0.5) : A(1)) * (dy ? A(0.5) : A(1));
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const int i = 2 * I + dx;
            if (i < 0 || i >= F.g.nx) continue;
            acc += wyz * (dx ? A(0.5) : A(1)) * to_acc(rf[off(F.g, i, j, k)]);
          }
        }
      }
    }
    rc[off(C.g, I, J, K)] = from_acc<T>(acc);
  }
}

template <typename T>
__device__ void tail_prolong(const TailLevel& C, const TailLevel& F) {
  using A = typename Acc<T>::type;
  const T* ec = static_cast<const T*>(C.e);
  T* tf = static_cast<T*>(F.t);
  const int n = F.g.nx * F.g.ny * F.g.nz;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % F.g.nx, j = (t / F.g.nx) % F.g.ny, k = t / (F.g.nx * F.g.ny);
    A v = A(0);
    if (!tdir(F.g, i, j, k)) {
      for (int cz = 0; cz <= (k & 1); ++cz)
        for (int cy = 0; cy <= (j & 1); ++cy)
          for (int cx = 0; cx <= (i & 1); ++cx)
            v += to_acc(ec[off(C.g, (i >> 1) + cx, (j >> 1) + cy, (k >> 1) + cz)]);
      v *= ((i & 1) ? A(0.5) : A(1)) * ((j & 1) ? A(0.5) : A(1)) * ((k & 1) ? A(0.5) : A(1));
    }
    tf[off(F.g, i, j, k)] = from_acc<T>(v);
  }
}

// e = t + omega D^-1 (r - A t), Dirichlet nodes copied.  A: 27 coefficients or the constant
// stencil on the mirrored field times prod_d s_d / 2.
template <typename T>
__device__ void tail_jacobi(const TailLevel& L, double omega) {
  using A = typename Acc<T>::type;
  const T* x = static_cast<const T*>(L.t);
  const T* b = static_cast<const T*>(L.r);
  const T* a27 = static_cast<const T*>(L.a27);
  T* out = static_cast<T*>(L.e);
  const LevelGeom& g = L.g;
  const long long plane = g.pitch * (long long)g.ny * g.nz;
  const int n = g.nx * g.ny * g.nz;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % g.nx, j = (t / g.nx) % g.ny, k = t / (g.nx * g.ny);
    const long long o = off(g, i, j, k);
    const A xc = to_acc(x[o]);
    if (tdir(g, i, j, k)) {
      out[o] = from_acc<T>(xc);
      continue;
    }
    A s = A(0), D;
    if (a27) {
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        const int i2 = mirror(i + d % 3 - 1, g.nx), j2 = mirror(j + (d / 3) % 3 - 1, g.ny),
                  k2 = mirror(k + d / 9 - 1, g.nz);
        s += to_acc(a27[d * plane + o]) * to_acc(x[off(g, i2, j2, k2)]);
      }
      D = to_acc(a27[13 * plane + o]);
    } else {
#pragma unroll
      for (int d = 0; d < 27; ++d) {
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int cls = (dx != 0) + 2 * (dy != 0) + 4 * (dz != 0);
        s += (A)L.L.c[cls] * to_acc(x[off(g, mirror(i + dx, g.nx), mirror(j + dy, g.ny), mirror(k + dz, g.nz))]);
      }
      const A w = A(0.125) * (A)(((i > 0) + (i < g.nx - 1)) * ((j > 0) + (j < g.ny - 1)) * ((k > 0) + (k < g.nz - 1)));
      s *= w;
      D = w * (A)L.L.c[0];
    }
    out[o] = from_acc<T>(xc + (A)omega * (to_acc(b[o]) - s) / D);
  }
}

template <typename T>
__device__ void tail_coarsest(const TailArgs& a) {
  const TailLevel& C = a.lv[a.nlev - 1];
  const T* r = static_cast<const T*>(C.r);
  T* e = static_cast<T*>(C.e);
  __shared__ double rs[1024];
  const int n = C.g.nx * C.g.ny * C.g.nz;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = t % C.g.nx, j = (t / C.g.nx) % C.g.ny, k = t / (C.g.nx * C.g.ny);
    e[off(C.g, i, j, k)] = from_acc<T>(0.0);
  }
  for (int t = threadIdx.x; t < a.nfree; t += blockDim.x) rs[t] = (double)to_acc(r[a.free_idx[t]]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = warp; row < a.nfree; row += nw) {
    double s = 0.0;
    for (int c = lane; c < a.nfree; c += 32) s += a.ainv[(long long)row * a.nfree + c] * rs[c];
    s = warp_sum(s);
    if (lane == 0) e[a.free_idx[row]] = from_acc<T>(s);
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_tail(const TailArgs a) {
  for (int l = 0; l + 1 < a.nlev; ++l) {
    tail_restrict<T>(a.lv[l], a.lv[l + 1]);
    __syncthreads();
  }
  tail_coarsest<T>(a);
  __syncthreads();
  for (int l = a.nlev - 2; l >= 0; --l) {
    tail_prolong<T>(a.lv[l + 1], a.lv[l]);
    __syncthreads();
    tail_jacobi<T>(a.lv[l], a.omega);
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_tail_batch(const TailArgs* __restrict__ tab, const int* __restrict__ active) {
  if (active && !active[blockIdx.x]) return;
  const TailArgs& a = tab[blockIdx.x];
  for (int l = 0; l + 1 < a.nlev; ++l) {
    tail_restrict<T>(a.lv[l], a.lv[l + 1]);
    __syncthreads();
  }
  tail_coarsest<T>(a);
  __syncthreads();
  for (int l = a.nlev - 2; l >= 0; --l) {
    tail_prolong<T>(a.lv[l + 1], a.lv[l]);
    __syncthreads();
    tail_jacobi<T>(a.lv[l], a.omega);
    __syncthreads();
  }
}

}  // namespace

int launch_tail_batch(nn4_dtype dt, const TailArgs* tab, int count, const int* active, cudaStream_t s) {
  if (count <= 0) return NN4_OK;
  switch (dt) {
    case NN4_F64: k_tail_batch<double><<<count, 1024, 0, s>>>(tab, active); break;
    case NN4_F32: k_tail_batch<float><<<count, 1024, 0, s>>>(tab, active); break;
    case NN4_BF16: k_tail_batch<bf16><<<count, 1024, 0, s>>>(tab, active); break;
  }
  return check_cuda(cudaGetLastError(), "batched coarse tail launch");
}

int launch_tail(nn4_dtype dt, const TailArgs& a, cudaStream_t s) {
  if (a.nlev < 1 || a.nlev > kMaxTail || a.nfree > 1024) return set_error(NN4_EINVAL, "bad coarse tail");
  switch (dt) {
    case NN4_F64: k_tail<double><<<1, 1024, 0, s>>>(a); break;
    case NN4_F32: k_tail<float><<<1, 1024, 0, s>>>(a); break;
    case NN4_BF16: k_tail<bf16><<<1, 1024, 0, s>>>(a); break;
  }
  return check_cuda(cudaGetLastError(), "coarse tail launch");
}

}  // namespace nn4
