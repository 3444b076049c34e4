// Tiling helpers of the explicit multiphase kernels (volume fraction, momentum, sources, pressure
// right-hand sides and the velocity correction of Sections 2.3-2.4).
//
// Every Q1 filter of those terms is a tensor product a_x (x) a_y (x) a_z of 1D assembled factors
// (mass M, stiffness K, first derivative G and its transpose GT), truncated at the domain faces
// (natural boundaries: a missing element contributes nothing).  A kernel owns an x-y tile and marches
// along z: each plane of its inputs is staged once in shared memory (with a one-node x-y halo),
// every thread forms the x-then-y filtered values of that plane for its own column of RY nodes,
// and the z factor is applied by accumulation: the plane-s value contributes a_z[+1] to node s-1,
// a_z[0] to node s and a_z[-1] to node s+1, so a node is complete one plane after its own.
// State is FP64 in memory; the arithmetic runs in T (double, or float for the FP32-compute form).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace nn4 {
namespace ft {

// ---------------------------------------------------------------- geometry and 1D factors
template <typename T>
struct Geo {
  int nx, ny, nz;
  long long pitch, plane;  // elements
  T h[3], h6[3], h3[3], h2[3], ih[3];  // h, h/6, h/3, h/2, 1/h per axis (x, y, z)
};

template <typename T>
struct W3 {  // weights of the offsets -1, 0, +1
  T w[3];
};

// Assembled 1D factors at node i of n: M (mass), K (stiffness), G (int N_i dN_j/dx), GT (G
// transposed), and the lumped mass.  A missing element (i = 0 or i = n - 1) drops its half.
template <typename T>
struct Fac {
  W3<T> M, K, G, GT;
  T lump;
};

template <typename T>
__device__ __forceinline__ Fac<T> fac(int i, int n, T h6, T h3, T h2, T ih) {
  const T l = i > 0 ? T(1) : T(0), r = i < n - 1 ? T(1) : T(0);
  Fac<T> f;
  f.M.w[0] = l * h6;
  f.M.w[1] = (l + r) * h3;
  f.M.w[2] = r * h6;
  f.K.w[0] = -l * ih;
  f.K.w[1] = (l + r) * ih;
  f.K.w[2] = -r * ih;
  f.G.w[0] = T(-0.5) * l;
  f.G.w[1] = T(0.5) * (l - r);
  f.G.w[2] = T(0.5) * r;
  f.GT.w[0] = T(0.5) * l;
  f.GT.w[1] = T(0.5) * (l - r);
  f.GT.w[2] = T(-0.5) * r;
  f.lump = (l + r) * h2;
  return f;
}

template <typename T>
__device__ __forceinline__ Fac<T> facx(const Geo<T>& g, int i) {
  return fac<T>(i, g.nx, g.h6[0], g.h3[0], g.h2[0], g.ih[0]);
}
template <typename T>
__device__ __forceinline__ Fac<T> facy(const Geo<T>& g, int j) {
  return fac<T>(j, g.ny, g.h6[1], g.h3[1], g.h2[1], g.ih[1]);
}
template <typename T>
__device__ __forceinline__ Fac<T> facz(const Geo<T>& g, int k) {
  return fac<T>(k, g.nz, g.h6[2], g.h3[2], g.h2[2], g.ih[2]);
}

// a / b: IEEE division in FP64; in the FP32-compute form the fast approximate division (a few
// ulp), well inside that form's stated error
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }

template <typename T>
__device__ __forceinline__ T dot3(const W3<T>& a, T v0, T v1, T v2) {
  return fma(a.w[0], v0, fma(a.w[1], v1, a.w[2] * v2));
}

// ---------------------------------------------------------------- FP64 <-> FP32 conversions
// The FP64 pipe of this part is narrow (about 2 operations per clock per SM), and a hardware
// conversion between FP64 and FP32 issues on it.  Kernels bound by instruction issue use the
// hardware conversion (one instruction on an otherwise idle pipe); kernels bound by memory that
// convert every staged value use these integer-pipe conversions instead (conv_int).
// to_f32: IEEE round to nearest even; results below the FP32 normal range flush to signed zero,
// results beyond it become infinity; NaN stays NaN.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int hi = (unsigned int)(b >> 32), lo = (unsigned int)b;
  const unsigned int sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned int m23 = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned int rest = lo & 0x1FFFFFFFu;
  const int e32 = e - 1023 + 127;
  unsigned int out;
  if (e == 0x7FF) {
    out = sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u);
  } else if (e32 <= 0) {
    out = sign;
  } else if (e32 >= 255) {
    out = sign | 0x7F800000u;
  } else {
    const unsigned int up = (rest > 0x10000000u) || (rest == 0x10000000u && (m23 & 1u));
    out = ((unsigned int)e32 << 23) + m23 + up;  // a carry out of the mantissa bumps the exponent
    out = out >= 0x7F800000u ? 0x7F800000u : out;
    out |= sign;
  }
  return __uint_as_float(out);
}

// to_f64: exact for FP32 normals, zero and infinity (FP32 subnormals, which the FP32 arithmetic
// here flushes anyway, become zero); NaN stays NaN.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned int b = __float_as_uint(x);
  const unsigned int sign = b & 0x80000000u;
  const unsigned int e = (b >> 23) & 0xFFu;
  const unsigned int m = b & 0x7FFFFFu;
  unsigned int hi, lo;
  if (e == 0) {
    hi = sign;
    lo = 0;
  } else if (e == 0xFF) {
    hi = sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
    lo = 0;
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

template <typename T>
__device__ __forceinline__ T from64(double v);
template <>
__device__ __forceinline__ double from64<double>(double v) {
  return v;
}
template <>
__device__ __forceinline__ float from64<float>(double v) {
  return __double2float_rn(v);
}
__device__ __forceinline__ double to64(double v) { return v; }
__device__ __forceinline__ double to64(float v) { return (double)v; }

template <typename T>
__device__ __forceinline__ T conv(double v) {
  return from64<T>(v);
}
// conversion on the integer pipe (for kernels bound by memory, where the FP64 pipe that carries
// the hardware conversion would become the limit)
template <typename T>
__device__ __forceinline__ T conv_int(double v);
template <>
__device__ __forceinline__ double conv_int<double>(double v) {
  return v;
}
template <>
__device__ __forceinline__ float conv_int<float>(double v) {
  return f64_to_f32(v);
}
template <typename T>
__device__ __forceinline__ T conv_int(float v) {
  return (T)v;
}
template <typename T>
__device__ __forceinline__ T conv(float v);
template <>
__device__ __forceinline__ float conv<float>(float v) {
  return v;
}

template <typename T>
__device__ __forceinline__ T load_as(const double* p) {
  return from64<T>(__ldg(p));
}
template <typename T>
__device__ __forceinline__ T load_as(const float* p) {
  return (T)__ldg(p);
}

// store a computed value in the precision of the array
__device__ __forceinline__ void store_as(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_as(double* p, float v) { *p = to64(v); }
__device__ __forceinline__ void store_as(float* p, float v) { *p = v; }

// The 3 x (RY + 2) values around a thread's column of RY nodes: v[rr][c] = plane value at row
// r0 + rr, column c0 + c of the staged region (row stride SW).
template <typename T, int RY, int SW>
__device__ __forceinline__ void nb(const T* __restrict__ sh, int r0, int c0, T (&v)[RY + 2][3]) {
#pragma unroll
  for (int rr = 0; rr < RY + 2; ++rr)
#pragma unroll
    for (int c = 0; c < 3; ++c) v[rr][c] = sh[(r0 + rr) * SW + c0 + c];
}

// x pass with factor a, then y pass with the per-row factors ay[r]: out[r] = sum_dy ay[r][dy] sum_dx a[dx] v
template <typename T, int RY>
__device__ __forceinline__ void xy(const T (&v)[RY + 2][3], const W3<T>& ax, const W3<T> (&ay)[RY], T (&out)[RY]) {
  T xr[RY + 2];
#pragma unroll
  for (int rr = 0; rr < RY + 2; ++rr) xr[rr] = dot3(ax, v[rr][0], v[rr][1], v[rr][2]);
#pragma unroll
  for (int r = 0; r < RY; ++r) out[r] = dot3(ay[r], xr[r], xr[r + 1], xr[r + 2]);
}

// the same with the x pass already done: xr[rr] per row
template <typename T, int RY>
__device__ __forceinline__ void ypass(const T (&xr)[RY + 2], const W3<T> (&ay)[RY], T (&out)[RY]) {
#pragma unroll
  for (int r = 0; r < RY; ++r) out[r] = dot3(ay[r], xr[r], xr[r + 1], xr[r + 2]);
}

template <typename T, int RY>
__device__ __forceinline__ void xpass(const T (&v)[RY + 2][3], const W3<T>& ax, T (&xr)[RY + 2]) {
#pragma unroll
  for (int rr = 0; rr < RY + 2; ++rr) xr[rr] = dot3(ax, v[rr][0], v[rr][1], v[rr][2]);
}

// z accumulation of one filtered plane value P_s: node s-1 gets zp.w[2] P (complete after this
// step), node s gets zc.w[1] P, node s+1 gets zn.w[0] P.  acc[0]: node s-1, acc[1]: node s,
// acc[2]: node s+1 (zero after each zshift).
template <typename T>
__device__ __forceinline__ void zacc(T (&acc)[3], T P, const W3<T>& zp, const W3<T>& zc, const W3<T>& zn) {
  acc[0] = fma(zp.w[2], P, acc[0]);
  acc[1] = fma(zc.w[1], P, acc[1]);
  acc[2] = fma(zn.w[0], P, acc[2]);
}

template <typename T>
__device__ __forceinline__ void zshift(T (&acc)[3]) {
  acc[0] = acc[1];
  acc[1] = acc[2];
  acc[2] = T(0);
}

}  // namespace ft
}  // namespace nn4

namespace nn4 {
namespace ft {

// ---------------------------------------------------------------- TMA plane ring
// The staged planes of the flow kernels arrive by 3D TMA tile loads (cp.async.bulk.tensor) into a
// ring of NS raw slots in dynamic shared memory, NS - 1 planes ahead of the plane being computed;
// all boxes of one plane complete on that slot's mbarrier.  A box starts at an x coordinate
// rounded down to 16 bytes (CO elements before the first column the kernel needs) and is
// zero-filled outside the grid (every filter weight that reaches those nodes is zero).  After its
// barrier completes, a plane is converted once into the compute type (a compute slot of
// SW x SH values, row stride SW), which the x-y filters then read.
template <typename R, int BW_, int CO_, int BH_>
struct Box {
  using type = R;
  static constexpr int BW = BW_, CO = CO_, BH = BH_;
  static constexpr int TX = BW_ * BH_ * (int)sizeof(R);   // bytes the TMA load delivers
  static constexpr int BYTES = (TX + 127) / 128 * 128;     // its footprint in a slot
};

// Box of a field with a one-node halo around a 32-wide tile that starts at a multiple of 32:
// FP64 starts 2 columns early (16 bytes), FP32 4.
template <typename R, int SH>
using Halo1 = Box<R, sizeof(R) == 8 ? 36 : 40, sizeof(R) == 8 ? 1 : 3, SH>;
// Box of an FP64 field with a two-node halo around a 30-wide tile that starts at a multiple of
// 30 (the two-stage kernels): the first column needed is already 16-byte aligned.
template <int SH>
using Halo2 = Box<double, 34, 0, SH>;

// raw box (row stride BW, first needed column CO) -> compute slot (SW x SH, type T); IC: convert
// on the integer pipe
template <typename B, int SW, int SH, int NT, bool IC = false, typename T>
__device__ __forceinline__ void convert_box(T* __restrict__ dst, const unsigned char* __restrict__ raw, int tid) {
  const typename B::type* src = reinterpret_cast<const typename B::type*>(raw);
  for (int e = tid; e < SW * SH; e += NT) {
    const int r = e / SW, c = e - r * SW;
    const typename B::type v = src[r * B::BW + c + B::CO];
    dst[e] = IC ? conv_int<T>(v) : conv<T>(v);
  }
}

// the same, storing a + b * value (the density from C)
template <typename B, int SW, int SH, int NT, bool IC = false, typename T>
__device__ __forceinline__ void convert_box_affine(T* __restrict__ dst, const unsigned char* __restrict__ raw, int tid,
                                                   T a, T b) {
  const typename B::type* src = reinterpret_cast<const typename B::type*>(raw);
  for (int e = tid; e < SW * SH; e += NT) {
    const int r = e / SW, c = e - r * SW;
    const typename B::type v = src[r * B::BW + c + B::CO];
    dst[e] = fma(b, IC ? conv_int<T>(v) : conv<T>(v), a);
  }
}

// Plane bookkeeping of a block that stages planes j0, j0 + 1, ...: slot and barrier phase.
template <int NS>
struct Ring {
  uint64_t* bar;
  unsigned char* raw;
  int slot_bytes, j0;
  __device__ __forceinline__ int slot(int z) const { return (z - j0) % NS; }
  __device__ __forceinline__ uint32_t parity(int z) const { return (uint32_t)(((z - j0) / NS) & 1); }
  __device__ __forceinline__ unsigned char* at(int z) const { return raw + (size_t)slot(z) * slot_bytes; }
  __device__ __forceinline__ uint64_t* barrier(int z) const { return &bar[slot(z)]; }
  __device__ __forceinline__ bool wait(int z) const { return mbar_wait_bounded(barrier(z), parity(z)); }
  // thread 0: initialise the barriers (then the caller synchronises)
  __device__ __forceinline__ void init() const {
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    fence_barrier_init();
  }
  // after a failed wait: wait (bounded) for every plane issued and not yet consumed
  __device__ __forceinline__ void drain(int first_unconsumed, int last_issued) const {
    for (int z = first_unconsumed; z <= last_issued; ++z) mbar_wait_bounded(barrier(z), parity(z));
  }
};

// Up to four tensor maps of one kernel launch (64-byte aligned, passed as a grid constant).
struct alignas(64) FMaps {
  CUtensorMap m[4];
};

}  // namespace ft
}  // namespace nn4
