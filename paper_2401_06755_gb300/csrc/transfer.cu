// Inter-grid transfers of the sawtooth multigrid (Section 2.4): stride-2 restriction R = P^T and
// trilinear prolongation P between a fine vertex grid and the grid of its even-indexed nodes.
#include <algorithm>

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
// exist; zero at coarse Dirichlet nodes.  A CTA owns 32 coarse columns x TYC coarse rows and marches
// along z over `kchunk` coarse planes: every fine plane 2K-1 .. 2K+1 of its region (fine columns
// 2 I0 - 1 .. 2 I0 + 63, rows 2 J0 - 1 .. 2 J0 + 2 TYC - 1) arrives as one TMA box in a ring of S
// stages (a power of two), each fine value leaves HBM once per chunk, and fine nodes outside the
// grid arrive as zeros (their weight).  A thread owns one coarse column and RPT consecutive coarse
// rows: it restricts the 2 RPT + 1 fine rows of a plane in x once (the fine pair as one load, the
// left neighbour from the previous lane), combines them in y per coarse row, and folds the z
// weights (1/2, 1, 1/2) into one running sum per coarse node.  Rows of 32 m + 1 coarse nodes: the
// last tile's first lane also computes coarse column 32 m.
template <typename T, int TYC, int S>
struct RLay {
  static constexpr int AL = 16 / (int)sizeof(T);
  static constexpr int BX = (64 + AL + 2 + AL - 1) / AL * AL;  // fine columns 2 I0 - AL .. 2 I0 + 65 at least
  static constexpr int BY = 2 * TYC + 1;
  static constexpr int BYTES = BX * BY * (int)sizeof(T);
  static constexpr int STAGE = (BYTES + 127) / 128 * 128;
  static constexpr size_t SMEM = (size_t)S * STAGE + S * 8;
  static_assert((S & (S - 1)) == 0, "ring depth is a power of two");
};
constexpr int kRTy = 8, kRpt = 2, kRStages = 8;

template <typename T, int TYC, int RPT, int S>
__global__ void __launch_bounds__(32 * TYC / RPT) k_restrict(const __grid_constant__ CUtensorMap fmap,
                                                             T* __restrict__ rc, const LevelGeom gc, int kchunk) {
  using A = typename Acc<T>::type;
  using Lay = RLay<T, TYC, S>;
  constexpr int AL = Lay::AL, BX = Lay::BX, NR = 2 * RPT + 1;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * Lay::STAGE);
  const int I0 = blockIdx.x * 32, J0 = blockIdx.y * TYC;
  const int Ks = blockIdx.z * kchunk, Ke = min(gc.nz, Ks + kchunk);
  const int f0 = 2 * Ks - 1;             // first fine plane (odd)
  const int nf = 2 * (Ke - Ks) + 1;      // fine planes 2 Ks - 1 .. 2 Ke - 1
  const int tid = threadIdx.x + 32 * threadIdx.y;
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
    prefetch_tmap(&fmap);
  }
  __syncthreads();
  auto issue = [&](int q) {
    const int s = q & (S - 1);
    mbar_expect_tx(&bars[s], Lay::BYTES);
    tma_load_3d(smem + s * Lay::STAGE, &fmap, 2 * I0 - AL, 2 * J0 - 1, f0 + q, &bars[s]);
  };
  int issued = min(S, nf);
  if (tid == 0)
    for (int q = 0; q < issued; ++q) issue(q);
  const int I = I0 + threadIdx.x, Jb = J0 + RPT * threadIdx.y;
  const bool extra = threadIdx.x == 0 && I0 + 32 == gc.nx - 1;
  const int cb = 2 * RPT * threadIdx.y * BX + 2 * threadIdx.x + AL;  // fine node (2I, 2Jb - 1) in a box
  const bool dx = (gc.dir[0] && I == 0) || (gc.dir[1] && I == gc.nx - 1);
  const bool dx2 = gc.dir[1];  // the extra column is the last one
  const long long cps = gc.pitch * (long long)gc.ny;
  T* const out = rc + I + gc.pitch * (long long)Jb;
  A acc[RPT], acc2[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) acc[r] = acc2[r] = A(0);
  bool failed = false;
  int q = 0;
  for (; q < nf; ++q) {
    const int s = q & (S - 1);
    if (!mbar_wait_bounded(&bars[s], (uint32_t)((q / S) & 1))) failed = true;
    const T* F = reinterpret_cast<const T*>(smem + s * Lay::STAGE);
    A xr[NR], xr2[NR];  // the fine rows restricted in x
#pragma unroll
    for (int w = 0; w < NR; ++w) {
      const int c = cb + w * BX;
      A a, b;
      ld2(F + c, a, b);
      A l = __shfl_up_sync(0xffffffffu, b, 1);
      if (threadIdx.x == 0) l = to_acc(F[c - 1]);
      xr[w] = a + A(0.5) * (l + b);
      xr2[w] = extra ? to_acc(F[c + 64]) + A(0.5) * (to_acc(F[c + 63]) + to_acc(F[c + 65])) : A(0);
    }
    const bool odd = (f0 + q) & 1;  // odd fine plane: closes coarse plane (f-1)/2, opens (f+1)/2
    const int K = (f0 + q - 1) >> 1;
    const bool dz = (gc.dir[4] && K == 0) || (gc.dir[5] && K == gc.nz - 1);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const A v = xr[2 * r + 1] + A(0.5) * (xr[2 * r] + xr[2 * r + 2]);
      const A v2 = xr2[2 * r + 1] + A(0.5) * (xr2[2 * r] + xr2[2 * r + 2]);
      if (odd) {
        const int J = Jb + r;
        if (q > 0 && !failed && J < gc.ny) {
          const bool dn = dz || (gc.dir[2] && J == 0) || (gc.dir[3] && J == gc.ny - 1);
          if (I < gc.nx) out[cps * K + gc.pitch * r] = from_acc<T>((dn || dx) ? A(0) : acc[r] + A(0.5) * v);
          if (extra) out[cps * K + gc.pitch * r + 32] = from_acc<T>((dn || dx2) ? A(0) : acc2[r] + A(0.5) * v2);
        }
        acc[r] = A(0.5) * v;
        acc2[r] = A(0.5) * v2;
      } else {
        acc[r] += v;
        acc2[r] += v2;
      }
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    if (q + S < nf) {  // every thread is done with stage s: bring fine plane q + S
      if (tid == 0) issue(q + S);
      ++issued;
    }
  }
  if (failed && tid == 0) {
    for (int p = q; p < issued; ++p) mbar_wait_bounded(&bars[p & (S - 1)], (uint32_t)((p / S) & 1));
  }
}

// Prolongation e_f (+)= P e_c: each fine node takes the coarse nodes bracketing it, weight 1 at an
// even index and 1/2 for each of the two parents at an odd index, per axis, applied in the order
// y, then x, then z.  A thread owns coarse columns I = 2L, 2L+1 and coarse row J: the fine columns
// 4L .. 4L+3 of fine rows 2J and 2J+1, over the fine planes of kPc coarse planes (2 kPc fine
// planes).  It loads the coarse values of columns 2L .. 2L+2, rows J and J+1, of its kPc + 1 coarse
// planes first, forms the plane values (row parity x 4 columns) per coarse plane and stores four
// fine values per fine row and plane as one vector; odd fine planes average two consecutive plane
// values.  For rows of 4 m + 1 fine nodes whose last lane ends at column 4 m - 1, that lane also
// stores fine column 4 m.  Dirichlet fine nodes keep base (or 0).
constexpr int kPc = 4;

template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void st(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
  static __device__ __forceinline__ void ld(const float* p, float v[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void st(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
  static __device__ __forceinline__ void ld(const double* p, double v[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
};
template <> struct Vec4<bf16> {
  static __device__ __forceinline__ void st(bf16* p, const float v[4]) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 u;
    u.x = *reinterpret_cast<unsigned*>(&a);
    u.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(p) = u;
  }
  static __device__ __forceinline__ void ld(const bf16* p, float v[4]) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
  }
};

template <typename T, bool BASE>
__global__ void __launch_bounds__(128) k_prolong(const T* __restrict__ ec, T* ef, const T* base, const LevelGeom gc,
                                                 const LevelGeom gf, int lanes_x) {
  using A = typename Acc<T>::type;
  const int L = blockIdx.x * 32 + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (J >= gc.ny) return;  // whole warps only (J is uniform across the warp)
  const int Ia = min(2 * L, gc.nx - 1), Ib = min(2 * L + 1, gc.nx - 1), In = min(2 * L + 2, gc.nx - 1);
  const int Jn = min(J + 1, gc.ny - 1);  // row J+1 (clamped: its values then feed no stored node)
  const long long cps = gc.pitch * (long long)gc.ny;
  const T* const r0 = ec + gc.pitch * (long long)J;
  const long long d1 = gc.pitch * (long long)(Jn - J);
  const int K0 = blockIdx.z * kPc;
  // raw values of coarse planes K0 .. K0 + kPc (clamped into the grid), rows J, J+1, columns
  // Ia, Ib, In: every load first
  A ca[kPc + 1][2], cb[kPc + 1][2], cn[kPc + 1][2];
#pragma unroll
  for (int t = 0; t <= kPc; ++t) {
    const T* p = r0 + cps * min(K0 + t, gc.nz - 1);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const T* pr = p + (r ? d1 : 0);
      ca[t][r] = to_acc(pr[Ia]);
      cb[t][r] = to_acc(pr[Ib]);
      cn[t][r] = to_acc(pr[In]);
    }
  }
  const int f = 4 * L, j = 2 * J;
  const bool full = f + 3 < gf.nx;                                // all four fine columns exist
  const bool extra = f + 4 == gf.nx - 1 && L + 1 == lanes_x;       // also the last fine column
  const bool okr = j + 1 < gf.ny;                                  // fine row 2J+1 exists
  bool dxe[5];                                                     // Dirichlet fine columns
#pragma unroll
  for (int e = 0; e < 5; ++e) dxe[e] = (gf.dir[0] && f + e == 0) || (gf.dir[1] && f + e == gf.nx - 1);
  const bool dy[2] = {(gf.dir[2] && j == 0) || (gf.dir[3] && j == gf.ny - 1), gf.dir[3] && j + 1 == gf.ny - 1};
  const long long fps = gf.pitch * (long long)gf.ny;
  T* const out0 = ef + f + gf.pitch * (long long)j;
  // plane values of coarse plane K0 + t at fine columns f .. f+4: y first, then x
  auto plane = [&](int t, A v[2][5]) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const A a = r ? A(0.5) * (ca[t][0] + ca[t][1]) : ca[t][0];
      const A b = r ? A(0.5) * (cb[t][0] + cb[t][1]) : cb[t][0];
      const A n = r ? A(0.5) * (cn[t][0] + cn[t][1]) : cn[t][0];
      v[r][0] = a;
      v[r][1] = A(0.5) * (a + b);
      v[r][2] = b;
      v[r][3] = A(0.5) * (b + n);
      v[r][4] = n;
    }
  };
  auto emit = [&](int k, const A v[2][5]) {
    const bool dz = (gf.dir[4] && k == 0) || (gf.dir[5] && k == gf.nz - 1);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      if (r == 1 && !okr) break;
      T* out = out0 + fps * k + (r ? gf.pitch : 0);
      A bv[4] = {A(0), A(0), A(0), A(0)};
      if (BASE && full) Vec4<T>::ld(base + (out - ef), bv);
      A w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (BASE && !full && f + e < gf.nx) bv[e] = to_acc(base[(out - ef) + e]);
        w[e] = (dz || dy[r] || dxe[e]) ? bv[e] : v[r][e] + bv[e];
      }
      if (full) {
        Vec4<T>::st(out, w);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (f + e < gf.nx) out[e] = from_acc<T>(w[e]);
      }
      if (extra) {
        const A b4 = BASE ? to_acc(base[(out - ef) + 4]) : A(0);
        out[4] = from_acc<T>((dz || dy[r] || dxe[4]) ? b4 : v[r][4] + b4);
      }
    }
  };
  A pv[2][5], cv[2][5];
  plane(0, pv);
#pragma unroll
  for (int t = 0; t < kPc; ++t) {
    const int K = K0 + t;
    if (K >= gc.nz) break;
    emit(2 * K, pv);
    if (2 * K + 1 >= gf.nz) break;
    plane(t + 1, cv);
    A mv[2][5];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int e = 0; e < 5; ++e) {
        mv[r][e] = A(0.5) * (pv[r][e] + cv[r][e]);
        pv[r][e] = cv[r][e];
      }
    emit(2 * K + 1, mv);
  }
}

// Fine planes per thread of the batched prolongation.
constexpr int kPz = 8;

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
  using Lay = RLay<T, kRTy, kRStages>;
  if (reinterpret_cast<uintptr_t>(rf) % 16 || (gf.pitch * (long long)sizeof(T)) % 16)
    return set_error(NN4_EINVAL, "restriction needs a 16-byte aligned fine field and row pitch");
  if (gc.nx < 2 || gc.ny < 1 || gc.nz < 1) return set_error(NN4_EINVAL, "restriction: empty coarse grid");
  const nn4_dtype dt = sizeof(T) == 8 ? NN4_F64 : (sizeof(T) == 4 ? NN4_F32 : NN4_BF16);
  CUtensorMap m;
  if (!make_tmap_3d(&m, dt, rf, gf.nx, gf.ny, gf.nz, gf.pitch, Lay::BX, Lay::BY))
    return set_error(NN4_ECUDA, "tensor map encoding failed (restriction)");
  auto kern = k_restrict<T, kRTy, kRpt, kRStages>;
  static int per_sm = 0;  // resident CTAs per SM (set once per instantiation)
  if (!per_sm) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kRTy / kRpt, Lay::SMEM) != cudaSuccess)
      return check_cuda(cudaGetLastError(), "restriction occupancy");
    per_sm = std::max(per_sm, 1);
  }
  const int tiles_x = (gc.nx - 1 + 31) / 32, tiles_y = (gc.ny + kRTy - 1) / kRTy;
  // coarse planes per CTA: the fewest waves of resident CTAs times the fine planes each CTA reads
  const long long resident = (long long)per_sm * sm_count();
  int kc = gc.nz;
  long long best = -1;
  for (int c : {16, 12, 8, 6, 4, 3, 2, 1}) {
    const int cc = std::min(c, gc.nz);
    const long long blocks = (long long)tiles_x * tiles_y * ((gc.nz + cc - 1) / cc);
    const long long cost = (blocks + resident - 1) / resident * (2 * cc + 1);
    if (best < 0 || cost < best) best = cost, kc = cc;
  }
  dim3 grd(tiles_x, tiles_y, (gc.nz + kc - 1) / kc);
  kern<<<grd, dim3(32, kRTy / kRpt), Lay::SMEM, s>>>(m, static_cast<T*>(rc), gc, kc);
  return check_cuda(cudaGetLastError(), "restrict launch");
}

template <typename T>
int prolong_t(const void* ec, const LevelGeom& gc, void* ef, const void* base, const LevelGeom& gf,
              cudaStream_t s) {
  // one vector access of four fine values: 16 bytes (8 for BF16); rows of a multiple of 16 bytes
  const size_t vb = std::min<size_t>(16, 4 * sizeof(T));
  if ((gf.pitch * (long long)sizeof(T)) % 16 || (reinterpret_cast<uintptr_t>(ef) % vb) ||
      (base && reinterpret_cast<uintptr_t>(base) % vb))
    return set_error(NN4_EINVAL, "prolongation needs 16-byte rows and aligned fine fields");
  // lanes of four fine columns: cover columns 0 .. 64 m - 1 of a 64 m + 1 row (the last lane also
  // takes the last column), else every column
  const int lanes = std::max(1, (gf.nx - 1 + 3) / 4);
  const int tiles_x = (lanes + 31) / 32;
  dim3 blk(32, 4);
  dim3 grd(tiles_x, (gc.ny + 3) / 4, (gc.nz + kPc - 1) / kPc);
  const int lanes_x = 32 * tiles_x;
  if (base)
    k_prolong<T, true><<<grd, blk, 0, s>>>(static_cast<const T*>(ec), static_cast<T*>(ef), static_cast<const T*>(base),
                                          gc, gf, lanes_x);
  else
    k_prolong<T, false><<<grd, blk, 0, s>>>(static_cast<const T*>(ec), static_cast<T*>(ef), nullptr, gc, gf, lanes_x);
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
