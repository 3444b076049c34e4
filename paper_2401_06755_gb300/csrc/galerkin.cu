// Galerkin coarse operators P^T A P for a coefficient field, and the 27-point passes that apply
// them.  With a constant coefficient the coarse operators are the rediscretised ones and these
// kernels are not used; with a field k (Eq. k-T) an averaged-coefficient rediscretisation makes
// the sawtooth cycle diverge at large density ratios, while the Galerkin product keeps it
// convergent (the coarse-grid correction is then an A-orthogonal projection).
#include <vector>

#include "common.cuh"
#include "galerkin.h"
#include "internal.h"

namespace nn4 {
namespace {

__device__ __forceinline__ bool dnode(const LevelGeom& g, int i, int j, int k) {
  return (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
         (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
}

// Entries of the assembled 1D Q1 stiffness K and mass M at node i (n nodes, spacing h), offset d.
template <typename C>
__device__ __forceinline__ void k1m1(int i, int n, int d, C h, C& K, C& M) {
  const C eL = (C)(i > 0), eR = (C)(i < n - 1);
  if (d == 0) {
    K = (eL + eR) / h;
    M = (eL + eR) * h / (C)3;
  } else if (d < 0) {
    K = -eL / h;
    M = eL * h / (C)6;
  } else {
    K = -eR / h;
    M = eR * h / (C)6;
  }
}

// Assembled constant-coefficient entry L[(i,j,k), (i,j,k) + (dx,dy,dz)] (tensor-product form).
template <typename C>
__device__ __forceinline__ C l_entry(const LevelGeom& g, const C h[3], int i, int j, int k, int dx, int dy, int dz) {
  C Kx, Mx, Ky, My, Kz, Mz;
  k1m1<C>(i, g.nx, dx, h[0], Kx, Mx);
  k1m1<C>(j, g.ny, dy, h[1], Ky, My);
  k1m1<C>(k, g.nz, dz, h[2], Kz, Mz);
  return Kx * My * Mz + Mx * Ky * Mz + Mx * My * Kz;
}

// Fine-operator source for the triple product: row i of A_f as (offset -> value).
template <typename C>
struct FromK {  // Eq. k-T: off-diagonal 1/2 L_ij (k_i + k_j); diagonal L_ii k_i - 1/2 (L k)_i
  const double* k;
  LevelGeom g;
  C h[3];
  __device__ __forceinline__ void row(int i, int j, int kk, C* a) const {
    const C ki = (C)k[i + g.pitch * ((long long)j + (long long)g.ny * kk)];
    C lk = 0;
#pragma unroll
    for (int d = 0; d < 27; ++d) {
      const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
      const int i2 = i + dx, j2 = j + dy, k2 = kk + dz;
      if (i2 < 0 || i2 >= g.nx || j2 < 0 || j2 >= g.ny || k2 < 0 || k2 >= g.nz) {
        a[d] = 0;
        continue;
      }
      const C l = l_entry<C>(g, h, i, j, kk, dx, dy, dz);
      const C kj = (C)k[i2 + g.pitch * ((long long)j2 + (long long)g.ny * k2)];
      lk += l * kj;
      a[d] = (d == 13) ? l * ki : (C)0.5 * l * (ki + kj);
    }
    a[13] -= (C)0.5 * lk;
  }
};

template <typename C>
struct From27 {
  const C* a27;
  LevelGeom g;
  __device__ __forceinline__ void row(int i, int j, int kk, C* a) const {
    const long long plane = g.pitch * (long long)g.ny * g.nz;
    const long long o = i + g.pitch * ((long long)j + (long long)g.ny * kk);
#pragma unroll
    for (int d = 0; d < 27; ++d) a[d] = a27[d * plane + o];
  }
};

// One thread per coarse node I: A_c[I, I+D] = sum_{i child of I} P[i,I] sum_{j ~ i} A[i,j] P[j,I+D]
// over free fine nodes i, j and free coarse nodes; weights prod_d (1/2)^|offset_d| (exact).
template <typename C, typename Src>
__global__ void k_galerkin(const Src src, const LevelGeom gf, C* __restrict__ out, const LevelGeom gc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int K = blockIdx.z;
  if (I >= gc.nx || J >= gc.ny) return;
  C acc[27];
#pragma unroll
  for (int d = 0; d < 27; ++d) acc[d] = 0;
  const bool Idir = dnode(gc, I, J, K);
  if (!Idir) {
    for (int c = 0; c < 27; ++c) {
      const int cx = c % 3 - 1, cy = (c / 3) % 3 - 1, cz = c / 9 - 1;
      const int i = 2 * I + cx, j = 2 * J + cy, k = 2 * K + cz;
      if (i < 0 || i >= gf.nx || j < 0 || j >= gf.ny || k < 0 || k >= gf.nz) continue;
      if (dnode(gf, i, j, k)) continue;
      const C wi = (cx ? (C)0.5 : (C)1) * (cy ? (C)0.5 : (C)1) * (cz ? (C)0.5 : (C)1);
      C a[27];
      src.row(i, j, k, a);
      for (int d = 0; d < 27; ++d) {
        const C v = a[d];
        if (v == (C)0) continue;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int i2 = i + dx, j2 = j + dy, k2 = k + dz;
        if (dnode(gf, i2, j2, k2)) continue;
        // coarse parents of fine node (i2, j2, k2): one per axis at an even index, two at an odd one
        const int Ix0 = i2 >> 1, Ix1 = (i2 + 1) >> 1;
        const int Jy0 = j2 >> 1, Jy1 = (j2 + 1) >> 1;
        const int Kz0 = k2 >> 1, Kz1 = (k2 + 1) >> 1;
        const C px = (i2 & 1) ? (C)0.5 : (C)1, py = (j2 & 1) ? (C)0.5 : (C)1, pz = (k2 & 1) ? (C)0.5 : (C)1;
        const C base = wi * v * px * py * pz;
        for (int Zc = Kz0; Zc <= Kz1; ++Zc)
          for (int Yc = Jy0; Yc <= Jy1; ++Yc)
            for (int Xc = Ix0; Xc <= Ix1; ++Xc) {
              if (dnode(gc, Xc, Yc, Zc)) continue;
              const int D = (Xc - I + 1) + 3 * (Yc - J + 1) + 9 * (Zc - K + 1);
              acc[D] += base;
            }
      }
    }
  } else {
    acc[13] = 1;  // inert diagonal at Dirichlet nodes
  }
  const long long plane = gc.pitch * (long long)gc.ny * gc.nz;
  const long long o = I + gc.pitch * ((long long)J + (long long)gc.ny * K);
#pragma unroll
  for (int d = 0; d < 27; ++d) out[d * plane + o] = acc[d];
}

template <typename S, typename D>
__global__ void k_convert27(const S* __restrict__ src, D* __restrict__ dst, long long n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    dst[t] = from_acc<D>(to_acc(src[t]));
}

// 27-point residual / Jacobi with pointwise coefficients: one thread per node, neighbours via
// the read-only path (mirrored indices stay in bounds; their coefficients are zero).
template <typename T, int OP>
__global__ void k_pass27(const T* __restrict__ x, const T* __restrict__ a27, const PassArgs a) {
  using A = typename Acc<T>::type;
  const LevelGeom& g = a.g;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long long plane = g.pitch * (long long)g.ny * g.nz;
  const long long o = i + g.pitch * ((long long)j + (long long)g.ny * k);
  // the three mirrored x indices and nine row offsets once per node; coefficient d sits d planes
  // (of the 27-array block) after coefficient 0
  const int ix[3] = {mirror(i - 1, g.nx), i, mirror(i + 1, g.nx)};
  long long row[9];
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
      row[dy + 3 * dz] = g.pitch * ((long long)mirror(j + dy - 1, g.ny) + (long long)g.ny * mirror(k + dz - 1, g.nz));
  const T* ap = a27 + o;
  A s = 0;
#pragma unroll
  for (int d = 0; d < 27; ++d) s += to_acc(ap[d * plane]) * to_acc(x[row[d / 3] + ix[d % 3]]);
  const bool dn = dnode(g, i, j, k);
  const A bv = to_acc(reinterpret_cast<const T*>(a.b)[o]);
  T* out = reinterpret_cast<T*>(a.out);
  if (OP == OP_RESIDUAL) {
    out[o] = from_acc<T>(dn ? A(0) : bv - s);
  } else {
    const A xc = to_acc(x[o]);
    const A D = to_acc(ap[13 * plane]);
    const A omega = (A)a.omega;
    A corr;
    if constexpr (sizeof(A) == 4)
      corr = __fdividef(bv - s, D);
    else
      corr = (bv - s) / D;
    out[o] = from_acc<T>(dn ? xc : xc + omega * corr);
  }
}

template <typename C>
int galerkin_k_t(const double* k, const LevelGeom& gf, const double hf[3], void* out, const LevelGeom& gc,
                 cudaStream_t s) {
  FromK<C> src;
  src.k = k;
  src.g = gf;
  for (int d = 0; d < 3; ++d) src.h[d] = (C)hf[d];
  dim3 blk(32, 4), grd((gc.nx + 31) / 32, (gc.ny + 3) / 4, gc.nz);
  k_galerkin<C, FromK<C>><<<grd, blk, 0, s>>>(src, gf, static_cast<C*>(out), gc);
  return check_cuda(cudaGetLastError(), "galerkin (level 0)");
}

template <typename C>
int galerkin_next_t(const void* af, const LevelGeom& gf, void* out, const LevelGeom& gc, cudaStream_t s) {
  From27<C> src;
  src.a27 = static_cast<const C*>(af);
  src.g = gf;
  dim3 blk(32, 4), grd((gc.nx + 31) / 32, (gc.ny + 3) / 4, gc.nz);
  k_galerkin<C, From27<C>><<<grd, blk, 0, s>>>(src, gf, static_cast<C*>(out), gc);
  return check_cuda(cudaGetLastError(), "galerkin");
}

template <typename T>
int pass27_t(int op, const PassArgs& a, const void* x, const void* a27, cudaStream_t s) {
  dim3 blk(32, 4), grd((a.g.nx + 31) / 32, (a.g.ny + 3) / 4, a.g.nz);
  if (op == OP_RESIDUAL)
    k_pass27<T, OP_RESIDUAL><<<grd, blk, 0, s>>>(static_cast<const T*>(x), static_cast<const T*>(a27), a);
  else if (op == OP_JACOBI)
    k_pass27<T, OP_JACOBI><<<grd, blk, 0, s>>>(static_cast<const T*>(x), static_cast<const T*>(a27), a);
  else
    return set_error(NN4_EINVAL, "27-point pass supports residual and Jacobi only");
  return check_cuda(cudaGetLastError(), "27-point pass");
}

}  // namespace

int launch_galerkin_from_k(nn4_dtype ct, const double* k, const LevelGeom& gf, const double hf[3], void* out,
                           const LevelGeom& gc, cudaStream_t s) {
  return ct == NN4_F64 ? galerkin_k_t<double>(k, gf, hf, out, gc, s) : galerkin_k_t<float>(k, gf, hf, out, gc, s);
}

int launch_galerkin_next(nn4_dtype ct, const void* af, const LevelGeom& gf, void* out, const LevelGeom& gc,
                         cudaStream_t s) {
  return ct == NN4_F64 ? galerkin_next_t<double>(af, gf, out, gc, s) : galerkin_next_t<float>(af, gf, out, gc, s);
}

int launch_convert27(nn4_dtype ct, const void* src, nn4_dtype dt, void* dst, const LevelGeom& g, cudaStream_t s) {
  const long long n = 27LL * g.pitch * g.ny * g.nz;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152 * 32);
  if (ct == NN4_F64 && dt == NN4_F64)
    return check_cuda(cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, s), "copy27");
  if (ct == NN4_F32 && dt == NN4_F32)
    return check_cuda(cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, s), "copy27");
  if (ct == NN4_F32 && dt == NN4_BF16)
    k_convert27<float, bf16><<<blocks, 256, 0, s>>>(static_cast<const float*>(src), static_cast<bf16*>(dst), n);
  else if (ct == NN4_F64 && dt == NN4_F32)
    k_convert27<double, float><<<blocks, 256, 0, s>>>(static_cast<const double*>(src), static_cast<float*>(dst), n);
  else if (ct == NN4_F64 && dt == NN4_BF16)
    k_convert27<double, bf16><<<blocks, 256, 0, s>>>(static_cast<const double*>(src), static_cast<bf16*>(dst), n);
  else
    return set_error(NN4_EINVAL, "unsupported 27-array conversion");
  return check_cuda(cudaGetLastError(), "convert27");
}

int launch_pass27(nn4_dtype dt, int op, const PassArgs& a, const void* x, const void* a27, cudaStream_t s) {
  switch (dt) {
    case NN4_F64: return pass27_t<double>(op, a, x, a27, s);
    case NN4_F32: return pass27_t<float>(op, a, x, a27, s);
    case NN4_BF16: return pass27_t<bf16>(op, a, x, a27, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

}  // namespace nn4
