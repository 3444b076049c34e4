// Galerkin coarse operators P^T A P for a coefficient field, and the 27-point passes that apply
// them.  With a constant coefficient the coarse operators are the rediscretised ones and these
// kernels are not used; with a field k (Eq. k-T) an averaged-coefficient rediscretisation makes
// the sawtooth cycle diverge at large density ratios, while the Galerkin product keeps it
// convergent (the coarse-grid correction is then an A-orthogonal projection).
#include <algorithm>
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

// Lower entries from the upper ones: A[I, I+D] := A[I+D, I] for the 13 offsets before the centre
// (d < 13, mirror 26 - d), so the 27 arrays hold one exactly symmetric operator.  The triple
// product is symmetric in exact arithmetic; the two sums of one entry pair differ only by rounding.
template <typename C>
__global__ void k_symmetrize27(C* a27, const LevelGeom g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const long long plane = g.pitch * (long long)g.ny * g.nz;
  const long long o = i + g.pitch * ((long long)j + (long long)g.ny * k);
#pragma unroll
  for (int d = 0; d < 13; ++d) {
    const int i2 = i + d % 3 - 1, j2 = j + (d / 3) % 3 - 1, k2 = k + d / 9 - 1;
    C v = 0;
    if (i2 >= 0 && i2 < g.nx && j2 >= 0 && j2 < g.ny && k2 >= 0 && k2 < g.nz)
      v = a27[(26 - d) * plane + i2 + g.pitch * ((long long)j2 + (long long)g.ny * k2)];
    a27[d * plane + o] = v;
  }
}

// 27-point residual / Jacobi with a symmetric operator held as 27 arrays, of which only the 14
// upper ones (d = 13..26: the centre and every offset after it) are read:
//   (A x)_i = sum_{d >= 13} a_d(i) x_{i+D_d} + sum_{d < 13} a_{26-d}(i + D_d) x_{i+D_d}.
// A CTA owns a 32 x TY tile of columns and marches along z over `zchunk` output planes.  Each input
// plane p arrives by TMA in one ring stage: the 14 upper arrays as one 4D box with a one-node x/y
// halo, x with the same halo, and b (output planes only).  Output plane k reads the stages of
// planes k-1 (the neighbours' entries towards k), k and k+1 (x only), so each stored coefficient
// leaves HBM once per z chunk.  Nodes outside the grid arrive as zeros (TMA fill), and their
// coefficients are zero.  A thread keeps the 3 x 3 x 3 window of x around its node in registers.
// Rows of 32 m + 1 nodes: tiles cover columns 0 .. 32 m - 1 and the last tile's first lane also
// computes column 32 m (its box reaches that far).
constexpr int kUpper = 14;  // stored upper arrays read by the pass (13 .. 26)

template <typename T, int TY, int S>
struct Lay27 {
  static constexpr int AL = 16 / (int)sizeof(T);                   // TMA x alignment (elements)
  static constexpr int BX = (32 + AL + 2 + AL - 1) / AL * AL;      // columns x0-AL .. x0+33 at least
  static constexpr int BY = TY + 2;
  static constexpr int PL = BX * BY;                                // elements of one haloed box plane
  static constexpr int XBYTES = PL * (int)sizeof(T);
  static constexpr int ABYTES = kUpper * XBYTES;
  static constexpr int BBYTES = 32 * TY * (int)sizeof(T);
  static constexpr int XOFF = (ABYTES + 127) / 128 * 128;
  static constexpr int BOFF = XOFF + (XBYTES + 127) / 128 * 128;
  static constexpr int STAGE = BOFF + (BBYTES + 127) / 128 * 128;
  static constexpr size_t SMEM = (size_t)S * STAGE + S * 8;
};

struct Maps27 {
  CUtensorMap a, x, b;
};

// Sum of one row of the operator at box offset c, x read from the three planes' boxes.
template <typename T, typename A, int BX, int PL>
__device__ __forceinline__ A row27_smem(const T* am, const T* a0, const T* xm, const T* x0, const T* xp, int c) {
  A s = A(0);
#pragma unroll
  for (int d = 0; d < 27; ++d) {
    const int off = (d / 3) % 3 * BX - BX + d % 3 - 1;
    const T* xs = d < 9 ? xm : (d < 18 ? x0 : xp);
    const A av = d < 9 ? to_acc(am[(13 - d) * PL + c + off])
                       : (d < 13 ? to_acc(a0[(13 - d) * PL + c + off]) : to_acc(a0[(d - 13) * PL + c]));
    s = fma(av, to_acc(xs[c + off]), s);
  }
  return s;
}

template <typename T, int OP, int TY, int S>
__global__ void __launch_bounds__(32 * TY) k_pass27(const __grid_constant__ Maps27 maps, const PassArgs a) {
  using A = typename Acc<T>::type;
  using Lay = Lay27<T, TY, S>;
  constexpr int AL = Lay::AL, BX = Lay::BX, PL = Lay::PL;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * Lay::STAGE);
  const LevelGeom& g = a.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY;
  const int zs = blockIdx.z * a.zchunk, ze = min(nz, zs + a.zchunk);
  const int nplanes = ze - zs + 2;  // input planes zs-1 .. ze
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    prefetch_tmap(&maps.a);
    prefetch_tmap(&maps.x);
    prefetch_tmap(&maps.b);
  }
  __syncthreads();
  // stage of input plane zs-1+q: the upper arrays (not needed for plane ze), x, b (planes zs..ze-1)
  auto issue = [&](int q) {
    const int s = q % S;
    unsigned char* st = smem + s * Lay::STAGE;
    const int p = zs - 1 + q;
    const bool coef = p < ze, pt = p >= zs && p < ze;
    mbar_expect_tx(&bars[s], Lay::XBYTES + (coef ? Lay::ABYTES : 0) + (pt ? Lay::BBYTES : 0));
    if (coef) tma_load_4d(st, &maps.a, x0 - AL, y0 - 1, p, 13, &bars[s]);
    tma_load_3d(st + Lay::XOFF, &maps.x, x0 - AL, y0 - 1, p, &bars[s]);
    if (pt) tma_load_3d(st + Lay::BOFF, &maps.b, x0, y0, p, &bars[s]);
  };
  int issued = min(S, nplanes);
  if (tid == 0)
    for (int q = 0; q < issued; ++q) issue(q);

  const int c = (ty + 1) * BX + tx + AL;  // the thread's node in a haloed box
  const int i = x0 + tx, j = y0 + ty;
  const bool extra = tx == 0 && x0 + 32 == nx - 1;  // also column nx - 1 (last tile of a 32 m + 1 row)
  const A omega = (A)a.omega;
  T* out = reinterpret_cast<T*>(a.out);
  const T* bglob = reinterpret_cast<const T*>(a.b);
  A xw[3][9];  // x of planes k-1, k, k+1 at (dx, dy) = index (dx+1) + 3 (dy+1)
  bool failed = false;
  int q = 0;
  for (; q < nplanes; ++q) {
    const int s = q % S;
    if (!mbar_wait_bounded(&bars[s], (uint32_t)((q / S) & 1))) failed = true;
    const T* xs = reinterpret_cast<const T*>(smem + s * Lay::STAGE + Lay::XOFF);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      xw[0][t] = xw[1][t];
      xw[1][t] = xw[2][t];
      xw[2][t] = to_acc(xs[c + (t / 3 - 1) * BX + t % 3 - 1]);
    }
    if (q >= 2 && !failed) {
      const int k = zs + q - 2;
      const unsigned char* sm = smem + ((q - 2) % S) * Lay::STAGE;
      const unsigned char* s0 = smem + ((q - 1) % S) * Lay::STAGE;
      const T* am = reinterpret_cast<const T*>(sm);
      const T* a0 = reinterpret_cast<const T*>(s0);
      if (i < nx && j < ny) {
        A sum = A(0);
#pragma unroll
        for (int d = 0; d < 9; ++d)  // plane k-1: the neighbours' entries towards this node
          sum = fma(to_acc(am[(13 - d) * PL + c + (d / 3 - 1) * BX + d % 3 - 1]), xw[0][d], sum);
#pragma unroll
        for (int d = 9; d < 13; ++d)  // plane k, before the centre: likewise
          sum = fma(to_acc(a0[(13 - d) * PL + c + ((d / 3) % 3 - 1) * BX + d % 3 - 1]), xw[1][d - 9], sum);
#pragma unroll
        for (int d = 13; d < 27; ++d)  // the centre and after: the node's own entries
          sum = fma(to_acc(a0[(d - 13) * PL + c]), d < 18 ? xw[1][d - 9] : xw[2][d - 18], sum);
        const long long o = i + g.pitch * ((long long)j + (long long)ny * k);
        const bool dn = dnode(g, i, j, k);
        const A bv = to_acc(reinterpret_cast<const T*>(s0 + Lay::BOFF)[ty * 32 + tx]);
        if (OP == OP_RESIDUAL) {
          out[o] = from_acc<T>(dn ? A(0) : bv - sum);
        } else {
          const A xc = xw[1][4];
          const A D = to_acc(a0[c]);
          A corr;
          if constexpr (sizeof(A) == 4)
            corr = __fdividef(bv - sum, D);
          else
            corr = (bv - sum) / D;
          out[o] = from_acc<T>(dn ? xc : xc + omega * corr);
        }
      }
      if (extra && j < ny) {
        const T* xm = reinterpret_cast<const T*>(sm + Lay::XOFF);
        const T* x0s = reinterpret_cast<const T*>(s0 + Lay::XOFF);
        const int ce = c + 32, ie = x0 + 32;
        const A sum = row27_smem<T, A, BX, PL>(am, a0, xm, x0s, xs, ce);
        const long long o = ie + g.pitch * ((long long)j + (long long)ny * k);
        const bool dn = dnode(g, ie, j, k);
        const A bv = to_acc(bglob[o]);
        if (OP == OP_RESIDUAL) {
          out[o] = from_acc<T>(dn ? A(0) : bv - sum);
        } else {
          const A xc = to_acc(x0s[ce]);
          const A D = to_acc(a0[ce]);
          out[o] = from_acc<T>(dn ? xc : xc + omega * ((bv - sum) / D));
        }
      }
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    // the stage of plane q-2 is free: bring plane q-2+S into it
    if (q >= 2 && q - 2 + S < nplanes) {
      if (tid == 0) issue(q - 2 + S);
      ++issued;
    }
  }
  if (failed && tid == 0) {
    // drain every copy issued but not consumed before the CTA exits (bounded waits)
    for (int p = q; p < issued; ++p) mbar_wait_bounded(&bars[p % S], (uint32_t)((p / S) & 1));
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

template <typename T, int OP>
int pass27_op(const PassArgs& a, const Maps27& m, dim3 grd, size_t smem, cudaStream_t s) {
  k_pass27<T, OP, 8, 4><<<grd, dim3(32, 8), smem, s>>>(m, a);
  return check_cuda(cudaGetLastError(), "27-point pass");
}

// z planes per CTA: the fewest waves of resident CTAs times the planes each CTA reads.
int pass27_zchunk(int tiles, int nz, long long resident) {
  static const int cand[] = {32, 24, 16, 12, 8, 6, 4, 2};
  int best = nz, best_cost = 1 << 30;
  for (int zc : cand) {
    if (zc > nz && zc != cand[0]) continue;
    const long long blocks = (long long)tiles * ((nz + zc - 1) / zc);
    const long long waves = (blocks + resident - 1) / resident;
    const int cost = (int)(waves * (std::min(zc, nz) + 2));
    if (cost < best_cost) best_cost = cost, best = std::min(zc, nz);
  }
  return best;
}

template <typename T>
int pass27_t(int op, PassArgs a, const void* x, const void* a27, cudaStream_t s) {
  constexpr int TY = 8, S = 4;
  using Lay = Lay27<T, TY, S>;
  const LevelGeom& g = a.g;
  if (g.nx < 2 || g.ny < 2 || g.nz < 2) return set_error(NN4_EINVAL, "27-point pass needs two nodes per axis");
  const nn4_dtype dt = sizeof(T) == 8 ? NN4_F64 : (sizeof(T) == 4 ? NN4_F32 : NN4_BF16);
  Maps27 m;
  bool ok = make_tmap_stack(&m.a, dt, a27, g.nx, g.ny, g.nz, kA27, g.pitch, Lay::BX, Lay::BY, kUpper) &&
            make_tmap_3d(&m.x, dt, x, g.nx, g.ny, g.nz, g.pitch, Lay::BX, Lay::BY) &&
            make_tmap_3d(&m.b, dt, a.b, g.nx, g.ny, g.nz, g.pitch, 32, TY);
  if (!ok) return set_error(NN4_ECUDA, "tensor map encoding failed (27-point pass)");
  const int tiles_x = (g.nx - 1 + 31) / 32, tiles_y = (g.ny + TY - 1) / TY;
  if (op != OP_RESIDUAL && op != OP_JACOBI) return set_error(NN4_EINVAL, "27-point pass supports residual and Jacobi only");
  static int per_sm[2] = {0, 0};  // resident CTAs per SM of the two instantiations (set once)
  const int w = op == OP_JACOBI;
  if (!per_sm[w]) {
    auto kern = w ? k_pass27<T, OP_JACOBI, TY, S> : k_pass27<T, OP_RESIDUAL, TY, S>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[w], kern, 32 * TY, Lay::SMEM) != cudaSuccess)
      return check_cuda(cudaGetLastError(), "27-point pass occupancy");
    per_sm[w] = std::max(per_sm[w], 1);
  }
  a.zchunk = pass27_zchunk(tiles_x * tiles_y, g.nz, (long long)per_sm[w] * sm_count());
  dim3 grd(tiles_x, tiles_y, (g.nz + a.zchunk - 1) / a.zchunk);
  if (op == OP_RESIDUAL) return pass27_op<T, OP_RESIDUAL>(a, m, grd, Lay::SMEM, s);
  return pass27_op<T, OP_JACOBI>(a, m, grd, Lay::SMEM, s);
}

template <typename C>
int symmetrize27_t(void* a27, const LevelGeom& g, cudaStream_t s) {
  dim3 blk(32, 4), grd((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz);
  k_symmetrize27<C><<<grd, blk, 0, s>>>(static_cast<C*>(a27), g);
  return check_cuda(cudaGetLastError(), "symmetrize27");
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

int launch_symmetrize27(nn4_dtype ct, void* a27, const LevelGeom& g, cudaStream_t s) {
  return ct == NN4_F64 ? symmetrize27_t<double>(a27, g, s) : symmetrize27_t<float>(a27, g, s);
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
