// Explicit multiphase terms: the compressive Petrov-Galerkin volume-fraction update of Section 2.3
// (Eqs. Petrov-C, Petrov-Cs, a_psi, efficient-kabs, Sx-lin, negativek, normalisation, positivek,
// alpha_min_and_max, transport-indicator-1), the momentum sources (Eqs. surface-tension-uvw and
// surface-tension-k with buoyancy), the Stage-1 and Stage-3 pressure right-hand sides (Eqs.
// ph_disc, ph_disc2), the velocity correction (Eq. vel-cor), the momentum predictor (Eqs.
// Petrov-u/v/w, k_Psi-n, k-abs, k-square, max-k, velocity-1) and the lumped-mass total of the mass
// diagnostic.
//
// Every kernel marches an x-y tile along z with its input planes staged in shared memory (see
// flow_tile.cuh).  The state (C, velocities, pressures and the results) is FP64 in memory; the
// arithmetic runs in T: FP64 (the plain path) or FP32 (the FP32-compute form, selected by
// `compute`; the per-node decisions that switch the scheme -- the 0.95 / 0.05 detector override
// -- are taken on the FP64 value, and the updates of FP64 state add an FP32 increment in FP64).
// Terms that need a field's filter at a node's neighbours (a_C needs g = u . grad C around the
// node; the curvature needs the normals around it) use two stages in one kernel: the inner
// quantity is formed for the tile plus a one-node halo, one plane behind the staging front, and
// filtered one plane later.
#include <algorithm>
#include <mutex>
#include <string>

#include "common.cuh"
#include "flow_tile.cuh"
#include "internal.h"

namespace nn4 {

NN4_DEFINE_ERROR_ACCESSOR(flow_error_word)

int validate_grid(const nn4_grid* g, nn4_dtype dt, int min_n);
int validate_ptr(const void* p, const char* name);

namespace {

using ft::Fac;
using ft::Geo;
using ft::W3;

template <typename T>
Geo<T> make_geo(const nn4_grid* g) {
  Geo<T> G;
  G.nx = g->n[0];
  G.ny = g->n[1];
  G.nz = g->n[2];
  G.pitch = g->pitch;
  G.plane = g->pitch * (long long)g->n[1];
  for (int d = 0; d < 3; ++d) {
    G.h[d] = (T)g->h[d];
    G.h6[d] = (T)(g->h[d] / 6.0);
    G.h3[d] = (T)(g->h[d] / 3.0);
    G.h2[d] = (T)(g->h[d] / 2.0);
    G.ih[d] = (T)(1.0 / g->h[d]);
  }
  return G;
}

struct Faces {
  int d[6];  // 1 where the face is Dirichlet (x-, x+, y-, y+, z-, z+)
};

__device__ __forceinline__ bool on_face(const Faces& f, int i, int j, int k, int nx, int ny, int nz) {
  return (f.d[0] && i == 0) || (f.d[1] && i == nx - 1) || (f.d[2] && j == 0) || (f.d[3] && j == ny - 1) ||
         (f.d[4] && k == 0) || (f.d[5] && k == nz - 1);
}

template <typename T>
__device__ __forceinline__ T zero() {
  return T(0);
}

// ---------------------------------------------------------------- volume fraction, stage A
// The directional diffusion coefficients k^x, k^y, k^z of the compressive scheme (Sections
// 2.3.5-2.3.6).  Threads cover the output tile plus a one-node halo (30 x (TY - 2) outputs); the
// staged C region adds one more node.  At step s: the x-y filters of C at plane s give the
// gradient of plane t = s - 1, hence g = u . grad C at t for the tile plus halo (shared); the
// mass filter of g then completes a_C of plane q = s - 2, which is emitted with the detectors.
template <typename T>
struct VofK {
  T alpha_a, alpha_kabs, eps_k, K_plus, K_minus, beta, eps_x, K_pos, kmin, kmax, third;
  T h[3], ih[3];
  double detect_hi, detect_lo;
};

template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_vof_coef(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                       const VofK<T> p, int zc, const double* __restrict__ C,
                                                       const double* __restrict__ u, const double* __restrict__ v,
                                                       const double* __restrict__ w, T* __restrict__ kx,
                                                       T* __restrict__ ky, T* __restrict__ kz) {
  constexpr int NT = 32 * TYT, TY = TYT * RY, SW = 34, SH = TY + 2;
  using BC = ft::Halo2<SH>;
  extern __shared__ __align__(128) unsigned char smem[];
  T* const cs = reinterpret_cast<T*>(smem + NS * BC::BYTES);  // compute slots [2][SH * SW]
  T* const sg = cs + 2 * SH * SW;                             // g of plane t, tile plus halo
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  const int X0 = blockIdx.x * 30, Y0 = blockIdx.y * (TY - 2);
  const int gx = X0 - 1 + tx, R0 = ty * RY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
  ft::Ring<NS> ring{reinterpret_cast<uint64_t*>(sg + SH * SW), smem, BC::BYTES, z0 - 2};
  const int last = z1 + 1;
  auto issue = [&](int z) {
    mbar_expect_tx(ring.barrier(z), BC::TX);
    tma_load_3d(ring.at(z), &maps.m[0], X0 - 2, Y0 - 2, z, ring.barrier(z));
  };
  if (tid == 0) ring.init();
  for (int i = tid; i < SH * SW; i += NT) sg[i] = T(0);
  __syncthreads();
  if (tid == 0)
    for (int z = ring.j0; z <= min(last, ring.j0 + NS - 2); ++z) issue(z);
  bool failed = !ring.wait(ring.j0);
  ft::convert_box<BC, SW, SH, NT, true>(cs, ring.at(ring.j0), tid);
  if (__syncthreads_or(failed)) {
    if (tid == 0) ring.drain(ring.j0, min(last, ring.j0 + NS - 2));
    return;
  }

  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yG[RY];
  T ly[RY];
  int gy[RY];
  bool in[RY], outp[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 - 1 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yG[r] = fy.G;
    ly[r] = fy.lump;
    in[r] = gx >= 0 && gx < g.nx && gy[r] >= 0 && gy[r] < g.ny;
    outp[r] = in[r] && tx >= 1 && tx <= 30 && R0 + r >= 1 && R0 + r <= TY - 2;
  }
  const bool wx0 = gx == 0, wx1 = gx == g.nx - 1;
  T gacc[3][RY][3], aacc[RY][3];
  T Cdq[3][RY], gq[RY], Uq[3][RY], Szq[RY];      // plane q = s - 2 (saved at step s - 1)
  T SxR[2][RY], SyR[2][RY], CnR[2][RY];          // detectors and node value of planes s - 2, s - 1
  double Ur[3][RY], cr[RY];                      // prefetched: u, v, w of plane s - 1; C of plane s - 2
#pragma unroll
  for (int r = 0; r < RY; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      gacc[0][r][c] = gacc[1][r][c] = gacc[2][r][c] = aacc[r][c] = T(0);
      Cdq[c][r] = Uq[c][r] = T(0);
      Ur[c][r] = 0.0;
    }
    gq[r] = Szq[r] = T(0);
    cr[r] = 0.0;
    SxR[0][r] = SxR[1][r] = SyR[0][r] = SyR[1][r] = CnR[0][r] = CnR[1][r] = T(0);
  }

  for (int s = ring.j0; s <= last; ++s) {
    if (tid == 0 && s + NS - 1 <= last) issue(s + NS - 1);
    const T* cur = cs + ((s - ring.j0) & 1) * SH * SW;
    const int t = s - 1, q = s - 2;
    const bool tin = t >= 0 && t < g.nz;
    const bool emit = q >= z0 && q < z1;
    T Ut[3][RY];
#pragma unroll
    for (int r = 0; r < RY; ++r)
#pragma unroll
      for (int d = 0; d < 3; ++d) Ut[d][r] = ft::from64<T>(Ur[d][r]);
    double c64[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) c64[r] = cr[r];
    // plane s: x-y filters of C, detectors along x and y, node value
    T SxN[RY], SyN[RY], CnN[RY];
    if (s >= 0 && s < g.nz) {
      T vv[RY + 2][3];
      ft::nb<T, RY, SW>(cur, R0, tx, vv);
      T xG[RY + 2], xM[RY + 2], GM[RY], MG[RY], MM[RY];
      ft::xpass<T, RY>(vv, FX.G, xG);
      ft::xpass<T, RY>(vv, FX.M, xM);
      ft::ypass<T, RY>(xG, yM, GM);
      ft::ypass<T, RY>(xM, yG, MG);
      ft::ypass<T, RY>(xM, yM, MM);
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        ft::zacc(gacc[0][r], GM[r], zp.M, zs.M, zn.M);
        ft::zacc(gacc[1][r], MG[r], zp.M, zs.M, zn.M);
        ft::zacc(gacc[2][r], MM[r], zp.G, zs.G, zn.G);
        const T c0 = vv[r + 1][1];
        // the copy-halo of the detector at walls: the missing neighbour takes the wall value
        const T xl = wx0 ? c0 : vv[r + 1][0], xr = wx1 ? c0 : vv[r + 1][2];
        const T yl = gy[r] == 0 ? c0 : vv[r][1], yr = gy[r] == g.ny - 1 ? c0 : vv[r + 2][1];
        SxN[r] = (c0 - xl) * (xr - c0);
        SyN[r] = (c0 - yl) * (yr - c0);
        CnN[r] = c0;
      }
    } else {
#pragma unroll
      for (int r = 0; r < RY; ++r) SxN[r] = SyN[r] = CnN[r] = T(0);
    }
    // plane t: pointwise gradient, g = u . grad C (to shared), detector along z
    T Cdt[3][RY], gt[RY], Szt[RY];
    {
      const T lz = ft::facz(g, t).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (tin && in[r]) {
          const T im = ft::qdiv(T(1), FX.lump * ly[r] * lz);
#pragma unroll
          for (int d = 0; d < 3; ++d) Cdt[d][r] = gacc[d][r][0] * im;
          gt[r] = Ut[0][r] * Cdt[0][r] + Ut[1][r] * Cdt[1][r] + Ut[2][r] * Cdt[2][r];
        } else {
          Cdt[0][r] = Cdt[1][r] = Cdt[2][r] = gt[r] = T(0);
        }
        sg[(R0 + r + 1) * SW + tx + 1] = gt[r];
        const T c0 = CnR[1][r];
        const T cm = t == 0 ? c0 : CnR[0][r];
        const T cp = t == g.nz - 1 ? c0 : CnN[r];
        Szt[r] = (c0 - cm) * (cp - c0);
#pragma unroll
        for (int d = 0; d < 3; ++d) ft::zshift(gacc[d][r]);
      }
    }
    // prefetch for the next step: u, v, w of plane s and C of plane s - 1
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const bool ok = in[r] && s >= 0 && s < g.nz;
      const long long o = (long long)s * g.plane + (long long)gy[r] * g.pitch + gx;
      Ur[0][r] = ok ? __ldg(u + o) : 0.0;
      Ur[1][r] = ok ? __ldg(v + o) : 0.0;
      Ur[2][r] = ok ? __ldg(w + o) : 0.0;
      cr[r] = (outp[r] && t >= z0 && t < z1) ? __ldg(C + o - g.plane) : 0.0;
    }
    __syncthreads();
    // mass filter of g at plane t: completes M g at plane q
    if (tin) {
      T vg[RY + 2][3], xr[RY + 2], P[RY];
      ft::nb<T, RY, SW>(sg, R0, tx, vg);
      ft::xpass<T, RY>(vg, FX.M, xr);
      ft::ypass<T, RY>(xr, yM, P);
      const Fac<T> zp = ft::facz(g, t - 1), zs = ft::facz(g, t), zn = ft::facz(g, t + 1);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(aacc[r], P[r], zp.M, zs.M, zn.M);
    }
    if (emit) {
      const T lz = ft::facz(g, q).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!outp[r]) continue;
        const T m = FX.lump * ly[r] * lz;
        const T a_C = p.alpha_a * (ft::qdiv(aacc[r][0], m) - gq[r]);  // Eq. a_psi
        const T cx = Cdq[0][r], cy = Cdq[1][r], cz = Cdq[2][r];
        const T ax = fabs(cx), ay = fabs(cy), az = fabs(cz), sabs = ax + ay + az;
        // Eq. efficient-kabs (general spacing)
        const T k_abs = ft::qdiv(p.alpha_kabs * fabs(a_C) * (p.h[0] * ax + p.h[1] * ay + p.h[2] * az),
                                 p.eps_k + sabs * sabs * p.third);
        // Eqs. normalisation and negativek
        const T gradsq = cx * cx + cy * cy + cz * cz;
        const T uu = Uq[0][r], vv_ = Uq[1][r], ww = Uq[2][r];
        const T proj = ft::qdiv(uu * cx + vv_ * cy + ww * cz, p.eps_x + gradsq);
        const T us = fabs(cx * proj) + fabs(cy * proj) + fabs(cz * proj);
        const T k_neg = ft::qdiv(-p.beta * (uu * uu + vv_ * vv_ + ww * ww), p.eps_x + gradsq * us * p.third);
        // detectors with the override (decided on the FP64 value), weights, combination, clamp
        const bool over = c64[r] > p.detect_hi || c64[r] < p.detect_lo;
        const T S[3] = {over ? T(-1) : SxR[0][r], over ? T(-1) : SyR[0][r], over ? T(-1) : Szq[r]};
        T kd[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T wp = -fmax(T(-1), fmin(T(0), p.K_plus * S[d]));
          const T wm = fmin(T(1), fmax(T(0), p.K_minus * S[d]));
          const T kk = wp * (p.K_pos * k_abs) + wm * (k_neg * p.ih[d]);
          kd[d] = fmax(-p.kmin, fmin(p.kmax, kk));
        }
        const long long o = (long long)q * g.plane + (long long)gy[r] * g.pitch + gx;
        kx[o] = kd[0];
        ky[o] = kd[1];
        kz[o] = kd[2];
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      ft::zshift(aacc[r]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Cdq[d][r] = Cdt[d][r];
        Uq[d][r] = Ut[d][r];
      }
      gq[r] = gt[r];
      Szq[r] = Szt[r];
      SxR[0][r] = SxR[1][r];
      SxR[1][r] = SxN[r];
      SyR[0][r] = SyR[1][r];
      SyR[1][r] = SyN[r];
      CnR[0][r] = CnR[1][r];
      CnR[1][r] = CnN[r];
    }
    if (s < last) {
      if (!ring.wait(s + 1)) failed = true;
      ft::convert_box<BC, SW, SH, NT, true>(cs + ((s + 1 - ring.j0) & 1) * SH * SW, ring.at(s + 1), tid);
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) ring.drain(s + 1, min(last, s + NS - 1));
      return;
    }
  }
}

template <typename T, int TY, int NS>
constexpr int vof_coef_smem() {
  return NS * ft::Halo2<TY + 2>::BYTES + 3 * (TY + 2) * 34 * (int)sizeof(T) + NS * 8;
}

// ---------------------------------------------------------------- volume fraction, stage B
// s_C = sum_d u_d f(C; w_d) + sum_d (1/2)[D_d(k^d C) + k^d D_d C - C D_d k^d] (Eq. Petrov-Cs with
// the directional filters D_x = K (x) M (x) M, ... in the form of Eq. k-Txx) and C_next = C - dt
// s_C / m (Eq. transport-indicator-1).
template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_vof_update(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                         double dt, T dtT, int zc, const double* __restrict__ C,
                                                         const double* __restrict__ u, const double* __restrict__ v,
                                                         const double* __restrict__ w, double* __restrict__ sC,
                                                         double* __restrict__ Cnext) {
  constexpr int NT = 32 * TYT, TY = TYT * RY, SW = 34, SH = TY + 2;
  using BC = ft::Halo1<double, SH>;
  using BK = ft::Halo1<T, SH>;
  constexpr int SLOT = BC::BYTES + 3 * BK::BYTES;
  extern __shared__ __align__(128) unsigned char smem[];
  T* const cs = reinterpret_cast<T*>(smem + NS * SLOT);  // compute slots [2][4][SH * SW]: C, k^x, k^y, k^z
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  const int X0 = blockIdx.x * 32, Y0 = blockIdx.y * TY;
  const int gx = X0 + tx, R0 = ty * RY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
  ft::Ring<NS> ring{reinterpret_cast<uint64_t*>(cs + 2 * 4 * SH * SW), smem, SLOT, z0 - 1};
  const int last = z1;
  auto issue = [&](int z) {
    unsigned char* d = ring.at(z);
    mbar_expect_tx(ring.barrier(z), BC::TX + 3 * BK::TX);
    tma_load_3d(d, &maps.m[0], X0 - 1 - BC::CO, Y0 - 1, z, ring.barrier(z));
#pragma unroll
    for (int f = 0; f < 3; ++f)
      tma_load_3d(d + BC::BYTES + f * BK::BYTES, &maps.m[1 + f], X0 - 1 - BK::CO, Y0 - 1, z, ring.barrier(z));
  };
  auto convert = [&](int z, T* dst) {
    const unsigned char* src = ring.at(z);
    ft::convert_box<BC, SW, SH, NT, true>(dst, src, tid);
#pragma unroll
    for (int f = 0; f < 3; ++f) ft::convert_box<BK, SW, SH, NT>(dst + (1 + f) * SH * SW, src + BC::BYTES + f * BK::BYTES, tid);
  };
  if (tid == 0) ring.init();
  __syncthreads();
  if (tid == 0)
    for (int z = ring.j0; z <= min(last, ring.j0 + NS - 2); ++z) issue(z);
  bool failed = !ring.wait(ring.j0);
  convert(ring.j0, cs);
  if (__syncthreads_or(failed)) {
    if (tid == 0) ring.drain(ring.j0, min(last, ring.j0 + NS - 2));
    return;
  }

  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yG[RY], yK[RY];
  T ly[RY];
  int gy[RY];
  bool in[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yG[r] = fy.G;
    yK[r] = fy.K;
    ly[r] = fy.lump;
    in[r] = gx < g.nx && gy[r] < g.ny;
  }
  // accumulators: f_x, f_y, f_z (raw gradient of C), D_x C, D_y C, D_z C, sum_d D_d(k^d C),
  // sum_d D_d k^d
  T A[8][RY][3];
  T Cq[RY], kq[3][RY];
  double Ur[3][RY], cr[RY];  // prefetched u, v, w and C of plane s - 1
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int r = 0; r < RY; ++r) A[a][r][0] = A[a][r][1] = A[a][r][2] = T(0);
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    Cq[r] = kq[0][r] = kq[1][r] = kq[2][r] = T(0);
    Ur[0][r] = Ur[1][r] = Ur[2][r] = cr[r] = 0.0;
  }

  for (int s = ring.j0; s <= last; ++s) {
    if (tid == 0 && s + NS - 1 <= last) issue(s + NS - 1);
    const T* cur = cs + ((s - ring.j0) & 1) * 4 * SH * SW;
    const int q = s - 1;
    const bool emit = q >= z0;
    T CnN[RY], kN[3][RY];
    if (s >= 0 && s < g.nz) {
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
      T vC[RY + 2][3];
      ft::nb<T, RY, SW>(cur, R0, tx, vC);
      {
        T xG[RY + 2], xM[RY + 2], xK[RY + 2], P[RY];
        ft::xpass<T, RY>(vC, FX.G, xG);
        ft::xpass<T, RY>(vC, FX.M, xM);
        ft::xpass<T, RY>(vC, FX.K, xK);
        ft::ypass<T, RY>(xG, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(A[0][r], P[r], zp.M, zs.M, zn.M);
        ft::ypass<T, RY>(xM, yG, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(A[1][r], P[r], zp.M, zs.M, zn.M);
        ft::ypass<T, RY>(xM, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          ft::zacc(A[2][r], P[r], zp.G, zs.G, zn.G);
          ft::zacc(A[5][r], P[r], zp.K, zs.K, zn.K);
        }
        ft::ypass<T, RY>(xK, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(A[3][r], P[r], zp.M, zs.M, zn.M);
        ft::ypass<T, RY>(xM, yK, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(A[4][r], P[r], zp.M, zs.M, zn.M);
#pragma unroll
        for (int r = 0; r < RY; ++r) CnN[r] = vC[r + 1][1];
      }
      // D_x(k^x C) + D_y(k^y C) + D_z(k^z C) and D_x k^x + D_y k^y + D_z k^z
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T vk[RY + 2][3], vkc[RY + 2][3];
        ft::nb<T, RY, SW>(cur + (1 + d) * SH * SW, R0, tx, vk);
#pragma unroll
        for (int rr = 0; rr < RY + 2; ++rr)
#pragma unroll
          for (int c = 0; c < 3; ++c) vkc[rr][c] = vk[rr][c] * vC[rr][c];
#pragma unroll
        for (int r = 0; r < RY; ++r) kN[d][r] = vk[r + 1][1];
        T xa[RY + 2], xb[RY + 2], Pa[RY], Pb[RY];
        const W3<T>& ax = d == 0 ? FX.K : FX.M;
        ft::xpass<T, RY>(vkc, ax, xa);
        ft::xpass<T, RY>(vk, ax, xb);
        if (d == 1) {
          ft::ypass<T, RY>(xa, yK, Pa);
          ft::ypass<T, RY>(xb, yK, Pb);
        } else {
          ft::ypass<T, RY>(xa, yM, Pa);
          ft::ypass<T, RY>(xb, yM, Pb);
        }
        const W3<T>& wp = d == 2 ? zp.K : zp.M;
        const W3<T>& ws = d == 2 ? zs.K : zs.M;
        const W3<T>& wn = d == 2 ? zn.K : zn.M;
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          ft::zacc(A[6][r], Pa[r], wp, ws, wn);
          ft::zacc(A[7][r], Pb[r], wp, ws, wn);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < RY; ++r) CnN[r] = kN[0][r] = kN[1][r] = kN[2][r] = T(0);
    }
    if (emit) {
      const T lz = ft::facz(g, q).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!in[r]) continue;
        const T sv = ft::from64<T>(Ur[0][r]) * A[0][r][0] + ft::from64<T>(Ur[1][r]) * A[1][r][0] +
                     ft::from64<T>(Ur[2][r]) * A[2][r][0] +
                     T(0.5) * (A[6][r][0] + kq[0][r] * A[3][r][0] + kq[1][r] * A[4][r][0] + kq[2][r] * A[5][r][0] -
                               Cq[r] * A[7][r][0]);
        const long long o = (long long)q * g.plane + (long long)gy[r] * g.pitch + gx;
        ft::store_as(sC + o, sv);
        if (Cnext) {
          const T m = FX.lump * ly[r] * lz;
          if constexpr (sizeof(T) == 8) {
            Cnext[o] = cr[r] - dt * (double)sv / (double)m;
          } else {
            Cnext[o] = cr[r] - ft::to64(dtT * sv / m);
          }
        }
      }
    }
    // prefetch for the next step: u, v, w, C of plane s (emitted then)
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const bool ok = in[r] && s >= z0 && s < z1;
      const long long o = (long long)s * g.plane + (long long)gy[r] * g.pitch + gx;
      Ur[0][r] = ok ? __ldg(u + o) : 0.0;
      Ur[1][r] = ok ? __ldg(v + o) : 0.0;
      Ur[2][r] = ok ? __ldg(w + o) : 0.0;
      cr[r] = ok ? __ldg(C + o) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
#pragma unroll
      for (int a = 0; a < 8; ++a) ft::zshift(A[a][r]);
      Cq[r] = CnN[r];
#pragma unroll
      for (int d = 0; d < 3; ++d) kq[d][r] = kN[d][r];
    }
    if (s < last) {
      if (!ring.wait(s + 1)) failed = true;
      convert(s + 1, cs + ((s + 1 - ring.j0) & 1) * 4 * SH * SW);
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) ring.drain(s + 1, min(last, s + NS - 1));
      return;
    }
  }
}

template <typename T, int TY, int NS>
constexpr int vof_update_smem() {
  return NS * (ft::Halo1<double, TY + 2>::BYTES + 3 * ft::Halo1<T, TY + 2>::BYTES) +
         2 * 4 * (TY + 2) * 34 * (int)sizeof(T) + NS * 8;
}

// ---------------------------------------------------------------- momentum sources
// s_d = sigma kappa C_d, s_z -= g rho, with C_d = m^-1 f(C; w_d), n = grad C / (eps_t + |grad C|)
// and kappa = m^-1 sum_d f(n_d; w_d) (Eqs. surface-tension-uvw, surface-tension-k).  Two stages as
// in k_vof_coef: the normals of plane t for the tile plus halo, then their divergence at plane q.
template <typename T>
struct SrcK {
  T eps_t, sigma, grho_g, grho_d;  // g rho = grho_g + grho_d C
};

template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_sources(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                      const SrcK<T> p, int zc, const double* __restrict__ C,
                                                      double* __restrict__ s0, double* __restrict__ s1,
                                                      double* __restrict__ s2, double* __restrict__ kappa) {
  constexpr int NT = 32 * TYT, TY = TYT * RY, SW = 34, SH = TY + 2;
  using BC = ft::Halo2<SH>;
  extern __shared__ __align__(128) unsigned char smem[];
  T* const cs = reinterpret_cast<T*>(smem + NS * BC::BYTES);  // compute slots [2][SH * SW]
  T* const sn = cs + 2 * SH * SW;                             // normals [3][SH * SW] of plane t
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  const int X0 = blockIdx.x * 30, Y0 = blockIdx.y * (TY - 2);
  const int gx = X0 - 1 + tx, R0 = ty * RY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
  ft::Ring<NS> ring{reinterpret_cast<uint64_t*>(sn + 3 * SH * SW), smem, BC::BYTES, z0 - 2};
  const int last = z1 + 1;
  auto issue = [&](int z) {
    mbar_expect_tx(ring.barrier(z), BC::TX);
    tma_load_3d(ring.at(z), &maps.m[0], X0 - 2, Y0 - 2, z, ring.barrier(z));
  };
  if (tid == 0) ring.init();
  for (int i = tid; i < 3 * SH * SW; i += NT) sn[i] = T(0);
  __syncthreads();
  if (tid == 0)
    for (int z = ring.j0; z <= min(last, ring.j0 + NS - 2); ++z) issue(z);
  bool failed = !ring.wait(ring.j0);
  ft::convert_box<BC, SW, SH, NT, true>(cs, ring.at(ring.j0), tid);
  if (__syncthreads_or(failed)) {
    if (tid == 0) ring.drain(ring.j0, min(last, ring.j0 + NS - 2));
    return;
  }
  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yG[RY];
  T ly[RY];
  int gy[RY];
  bool in[RY], outp[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 - 1 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yG[r] = fy.G;
    ly[r] = fy.lump;
    in[r] = gx >= 0 && gx < g.nx && gy[r] >= 0 && gy[r] < g.ny;
    outp[r] = in[r] && tx >= 1 && tx <= 30 && R0 + r >= 1 && R0 + r <= TY - 2;
  }
  T gacc[3][RY][3], kacc[RY][3], Cdq[3][RY];
  double cr[RY];  // prefetched C of plane s - 2
#pragma unroll
  for (int r = 0; r < RY; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) gacc[0][r][c] = gacc[1][r][c] = gacc[2][r][c] = kacc[r][c] = Cdq[c][r] = T(0);
    cr[r] = 0.0;
  }

  for (int s = ring.j0; s <= last; ++s) {
    if (tid == 0 && s + NS - 1 <= last) issue(s + NS - 1);
    const T* cur = cs + ((s - ring.j0) & 1) * SH * SW;
    const int t = s - 1, q = s - 2;
    const bool tin = t >= 0 && t < g.nz;
    const bool emit = q >= z0 && q < z1;
    double c64[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) c64[r] = cr[r];
    if (s >= 0 && s < g.nz) {
      T vv[RY + 2][3], xG[RY + 2], xM[RY + 2], GM[RY], MG[RY], MM[RY];
      ft::nb<T, RY, SW>(cur, R0, tx, vv);
      ft::xpass<T, RY>(vv, FX.G, xG);
      ft::xpass<T, RY>(vv, FX.M, xM);
      ft::ypass<T, RY>(xG, yM, GM);
      ft::ypass<T, RY>(xM, yG, MG);
      ft::ypass<T, RY>(xM, yM, MM);
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        ft::zacc(gacc[0][r], GM[r], zp.M, zs.M, zn.M);
        ft::zacc(gacc[1][r], MG[r], zp.M, zs.M, zn.M);
        ft::zacc(gacc[2][r], MM[r], zp.G, zs.G, zn.G);
      }
    }
    T Cdt[3][RY];
    {
      const T lz = ft::facz(g, t).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        T n[3] = {T(0), T(0), T(0)};
        if (tin && in[r]) {
          const T im = ft::qdiv(T(1), FX.lump * ly[r] * lz);
#pragma unroll
          for (int d = 0; d < 3; ++d) Cdt[d][r] = gacc[d][r][0] * im;
          const T inv = T(1) / (p.eps_t + sqrt(Cdt[0][r] * Cdt[0][r] + Cdt[1][r] * Cdt[1][r] + Cdt[2][r] * Cdt[2][r]));
#pragma unroll
          for (int d = 0; d < 3; ++d) n[d] = Cdt[d][r] * inv;
        } else {
          Cdt[0][r] = Cdt[1][r] = Cdt[2][r] = T(0);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          sn[d * SH * SW + (R0 + r + 1) * SW + tx + 1] = n[d];
          ft::zshift(gacc[d][r]);
        }
      }
    }
    // prefetch C of plane t (emitted at the next step)
#pragma unroll
    for (int r = 0; r < RY; ++r)
      cr[r] = (outp[r] && t >= z0 && t < z1) ? __ldg(C + (long long)t * g.plane + (long long)gy[r] * g.pitch + gx)
                                             : 0.0;
    __syncthreads();
    if (tin) {
      const Fac<T> zp = ft::facz(g, t - 1), zs = ft::facz(g, t), zn = ft::facz(g, t + 1);
      T vn[RY + 2][3], xr[RY + 2], P[RY], P2[RY];
      ft::nb<T, RY, SW>(sn, R0, tx, vn);
      ft::xpass<T, RY>(vn, FX.G, xr);
      ft::ypass<T, RY>(xr, yM, P);
      ft::nb<T, RY, SW>(sn + SH * SW, R0, tx, vn);
      ft::xpass<T, RY>(vn, FX.M, xr);
      ft::ypass<T, RY>(xr, yG, P2);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(kacc[r], P[r] + P2[r], zp.M, zs.M, zn.M);
      ft::nb<T, RY, SW>(sn + 2 * SH * SW, R0, tx, vn);
      ft::xpass<T, RY>(vn, FX.M, xr);
      ft::ypass<T, RY>(xr, yM, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(kacc[r], P[r], zp.G, zs.G, zn.G);
    }
    if (emit) {
      const T lz = ft::facz(g, q).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!outp[r]) continue;
        const T kap = kacc[r][0] / (FX.lump * ly[r] * lz);
        const T sk = p.sigma * kap;
        const T grho = p.grho_g + p.grho_d * ft::from64<T>(c64[r]);
        const long long o = (long long)q * g.plane + (long long)gy[r] * g.pitch + gx;
        ft::store_as(s0 + o, sk * Cdq[0][r]);
        ft::store_as(s1 + o, sk * Cdq[1][r]);
        ft::store_as(s2 + o, sk * Cdq[2][r] - grho);
        if (kappa) ft::store_as(kappa + o, kap);
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      ft::zshift(kacc[r]);
#pragma unroll
      for (int d = 0; d < 3; ++d) Cdq[d][r] = Cdt[d][r];
    }
    if (s < last) {
      if (!ring.wait(s + 1)) failed = true;
      ft::convert_box<BC, SW, SH, NT, true>(cs + ((s + 1 - ring.j0) & 1) * SH * SW, ring.at(s + 1), tid);
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) ring.drain(s + 1, min(last, s + NS - 1));
      return;
    }
  }
}

template <typename T, int TY, int NS>
constexpr int sources_smem() {
  return NS * ft::Halo2<TY + 2>::BYTES + 5 * (TY + 2) * 34 * (int)sizeof(T) + NS * 8;
}

// ---------------------------------------------------------------- single-stage passes
// Common frame of the passes whose filters reach only the node's neighbours: threads cover the
// output tile (32 x TY), each staged field carries a one-node halo.

// Frame of the single-stage passes (filters that reach only a node's neighbours): threads cover the
// output tile (32 x TY), and NF staged FP64 fields arrive per plane through the TMA ring with a
// one-node halo; IC: their conversion to T runs on the integer pipe (these passes are bound by
// memory, and the hardware conversion issues on the narrow FP64 pipe).  The macro opens the
// kernel body up to the z loop; NN4_PASS_STEP_END closes one step.
#define NN4_PASS_PROLOGUE(NF_, IC_)                                                                       \
  constexpr int NT = 32 * TYT, TY = TYT * RY, SW = 34, SH = TY + 2;                                       \
  using BF = ft::Halo1<double, SH>;                                                                       \
  constexpr int NF = NF_, SLOT = NF_ * BF::BYTES;                                                         \
  extern __shared__ __align__(128) unsigned char smem[];                                                  \
  T* const cs = reinterpret_cast<T*>(smem + NS * SLOT);                                                   \
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;                                       \
  const int X0 = blockIdx.x * 32, Y0 = blockIdx.y * TY;                                                   \
  const int gx = X0 + tx, R0 = ty * RY;                                                                   \
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);                                                \
  const ft::Ring<NS> ring{reinterpret_cast<uint64_t*>(cs + 2 * NF * SH * SW), smem, SLOT, z0 - 1};       \
  const int last = z1;                                                                                    \
  auto issue = [&](int z) {                                                                               \
    unsigned char* d = ring.at(z);                                                                        \
    mbar_expect_tx(ring.barrier(z), NF * BF::TX);                                                         \
    for (int f = 0; f < NF; ++f)                                                                          \
      tma_load_3d(d + f * BF::BYTES, &maps.m[f], X0 - 1 - BF::CO, Y0 - 1, z, ring.barrier(z));           \
  };                                                                                                      \
  auto convert = [&](int z, T* dst) {                                                                     \
    const unsigned char* src = ring.at(z);                                                                \
    for (int f = 0; f < NF; ++f) ft::convert_box<BF, SW, SH, NT, IC_>(dst + f * SH * SW, src + f * BF::BYTES, tid); \
  };                                                                                                      \
  if (tid == 0) ring.init();                                                                              \
  __syncthreads();                                                                                        \
  if (tid == 0)                                                                                           \
    for (int z = ring.j0; z <= min(last, ring.j0 + NS - 2); ++z) issue(z);                                \
  bool failed = !ring.wait(ring.j0);                                                                      \
  convert(ring.j0, cs);                                                                                   \
  if (__syncthreads_or(failed)) {                                                                         \
    if (tid == 0) ring.drain(ring.j0, min(last, ring.j0 + NS - 2));                                       \
    return;                                                                                               \
  }

#define NN4_PASS_STEP_BEGIN()                                                                             \
  if (tid == 0 && s + NS - 1 <= last) issue(s + NS - 1);                                                  \
  const T* cur = cs + ((s - ring.j0) & 1) * NF * SH * SW;

#define NN4_PASS_STEP_END()                                                                               \
  if (s < last) {                                                                                         \
    if (!ring.wait(s + 1)) failed = true;                                                                 \
    convert(s + 1, cs + ((s + 1 - ring.j0) & 1) * NF * SH * SW);                                          \
  }                                                                                                       \
  if (__syncthreads_or(failed)) {                                                                         \
    if (tid == 0) ring.drain(s + 1, min(last, s + NS - 1));                                               \
    return;                                                                                               \
  }

template <typename T, int TY, int NS, int NF>
constexpr int pass_smem() {
  return NS * NF * ft::Halo1<double, TY + 2>::BYTES + 2 * NF * (TY + 2) * 34 * (int)sizeof(T) + NS * 8;
}

// Stage-1 right-hand side b = sum_d G_d^T s_d (0 on the Dirichlet faces of the pressure grid);
// maps: s_x, s_y, s_z.
template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_rhs_hs(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                     const Faces pf, int zc, double* __restrict__ b) {
  NN4_PASS_PROLOGUE(3, true)
  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yGT[RY];
  int gy[RY];
  bool in[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yGT[r] = fy.GT;
    in[r] = gx < g.nx && gy[r] < g.ny;
  }
  T A[RY][3];
#pragma unroll
  for (int r = 0; r < RY; ++r) A[r][0] = A[r][1] = A[r][2] = T(0);
  for (int s = ring.j0; s <= last; ++s) {
    NN4_PASS_STEP_BEGIN()
    if (s >= 0 && s < g.nz) {
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
      T vv[RY + 2][3], xr[RY + 2], P[RY], P1[RY];
      ft::nb<T, RY, SW>(cur, R0, tx, vv);
      ft::xpass<T, RY>(vv, FX.GT, xr);
      ft::ypass<T, RY>(xr, yM, P);
      ft::nb<T, RY, SW>(cur + SH * SW, R0, tx, vv);
      ft::xpass<T, RY>(vv, FX.M, xr);
      ft::ypass<T, RY>(xr, yGT, P1);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(A[r], P[r] + P1[r], zp.M, zs.M, zn.M);
      ft::nb<T, RY, SW>(cur + 2 * SH * SW, R0, tx, vv);
      ft::xpass<T, RY>(vv, FX.M, xr);
      ft::ypass<T, RY>(xr, yM, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(A[r], P[r], zp.GT, zs.GT, zn.GT);
    }
    const int q = s - 1;
    if (q >= z0) {
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!in[r]) continue;
        const long long o = (long long)q * g.plane + (long long)gy[r] * g.pitch + gx;
        if (on_face(pf, gx, gy[r], q, g.nx, g.ny, g.nz))
          b[o] = 0.0;
        else
          ft::store_as(b + o, A[r][0]);
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) ft::zshift(A[r]);
    NN4_PASS_STEP_END()
  }
}

// Stage-3 right-hand side b = -(1/dt) sum_d [ f(rho u_d; w_d) - u_d f(rho; w_d) ] (Eq. ph_disc2),
// rho = rho_g + (rho_l - rho_g) C formed when C is converted; 0 on the Dirichlet faces.  maps:
// C, u, v, w.
template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_rhs_nh(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                     const Faces pf, int zc, T rho_g, T rho_d, T inv_dt,
                                                     double* __restrict__ b) {
  constexpr int NT = 32 * TYT, TY = TYT * RY, SW = 34, SH = TY + 2;
  using BF = ft::Halo1<double, SH>;
  constexpr int NF = 4, SLOT = 4 * BF::BYTES;
  extern __shared__ __align__(128) unsigned char smem[];
  T* const cs = reinterpret_cast<T*>(smem + NS * SLOT);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  const int X0 = blockIdx.x * 32, Y0 = blockIdx.y * TY;
  const int gx = X0 + tx, R0 = ty * RY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
  const ft::Ring<NS> ring{reinterpret_cast<uint64_t*>(cs + 2 * NF * SH * SW), smem, SLOT, z0 - 1};
  const int last = z1;
  auto issue = [&](int z) {
    unsigned char* d = ring.at(z);
    mbar_expect_tx(ring.barrier(z), NF * BF::TX);
    for (int f = 0; f < NF; ++f)
      tma_load_3d(d + f * BF::BYTES, &maps.m[f], X0 - 1 - BF::CO, Y0 - 1, z, ring.barrier(z));
  };
  auto convert = [&](int z, T* dst) {
    const unsigned char* src = ring.at(z);
    ft::convert_box_affine<BF, SW, SH, NT, true>(dst, src, tid, rho_g, rho_d);
    for (int f = 1; f < NF; ++f) ft::convert_box<BF, SW, SH, NT, true>(dst + f * SH * SW, src + f * BF::BYTES, tid);
  };
  if (tid == 0) ring.init();
  __syncthreads();
  if (tid == 0)
    for (int z = ring.j0; z <= min(last, ring.j0 + NS - 2); ++z) issue(z);
  bool failed = !ring.wait(ring.j0);
  convert(ring.j0, cs);
  if (__syncthreads_or(failed)) {
    if (tid == 0) ring.drain(ring.j0, min(last, ring.j0 + NS - 2));
    return;
  }
  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yG[RY];
  int gy[RY];
  bool in[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yG[r] = fy.G;
    in[r] = gx < g.nx && gy[r] < g.ny;
  }
  // A = sum_d f(rho u_d; w_d); B_d = f(rho; w_d); node velocities of plane q
  T A[RY][3], B[3][RY][3], Uq[3][RY];
#pragma unroll
  for (int r = 0; r < RY; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A[r][c] = B[0][r][c] = B[1][r][c] = B[2][r][c] = T(0);
      Uq[c][r] = T(0);
    }
  for (int s = ring.j0; s <= last; ++s) {
    NN4_PASS_STEP_BEGIN()
    T UN[3][RY];
    if (s >= 0 && s < g.nz) {
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
      T vr[RY + 2][3];
      ft::nb<T, RY, SW>(cur, R0, tx, vr);
      T xGr[RY + 2], xMr[RY + 2], P[RY];
      ft::xpass<T, RY>(vr, FX.G, xGr);
      ft::xpass<T, RY>(vr, FX.M, xMr);
      ft::ypass<T, RY>(xGr, yM, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(B[0][r], P[r], zp.M, zs.M, zn.M);
      ft::ypass<T, RY>(xMr, yG, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(B[1][r], P[r], zp.M, zs.M, zn.M);
      ft::ypass<T, RY>(xMr, yM, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(B[2][r], P[r], zp.G, zs.G, zn.G);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T vu[RY + 2][3];
        ft::nb<T, RY, SW>(cur + (1 + d) * SH * SW, R0, tx, vu);
#pragma unroll
        for (int r = 0; r < RY; ++r) UN[d][r] = vu[r + 1][1];
#pragma unroll
        for (int rr = 0; rr < RY + 2; ++rr)
#pragma unroll
          for (int c = 0; c < 3; ++c) vu[rr][c] *= vr[rr][c];
        T xr[RY + 2];
        ft::xpass<T, RY>(vu, d == 0 ? FX.G : FX.M, xr);
        ft::ypass<T, RY>(xr, d == 1 ? yG : yM, P);
        const W3<T>& wp = d == 2 ? zp.G : zp.M;
        const W3<T>& ws = d == 2 ? zs.G : zs.M;
        const W3<T>& wn = d == 2 ? zn.G : zn.M;
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(A[r], P[r], wp, ws, wn);
      }
    } else {
#pragma unroll
      for (int r = 0; r < RY; ++r) UN[0][r] = UN[1][r] = UN[2][r] = T(0);
    }
    const int q = s - 1;
    if (q >= z0) {
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!in[r]) continue;
        const long long o = (long long)q * g.plane + (long long)gy[r] * g.pitch + gx;
        if (on_face(pf, gx, gy[r], q, g.nx, g.ny, g.nz)) {
          b[o] = 0.0;
        } else {
          const T sum = A[r][0] - Uq[0][r] * B[0][r][0] - Uq[1][r] * B[1][r][0] - Uq[2][r] * B[2][r][0];
          ft::store_as(b + o, -sum * inv_dt);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      ft::zshift(A[r]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ft::zshift(B[d][r]);
        Uq[d][r] = UN[d][r];
      }
    }
    NN4_PASS_STEP_END()
  }
}

// Eq. vel-cor and the Stage-3 updates: u_d += -dt m^-1 f(dp; w_d) / rho (not on the no-slip faces),
// p += dp.  maps: dp.
template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_vel_correct(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                          const Faces vf, int zc, T rho_g, T rho_d, T dtT,
                                                          const double* __restrict__ C, const double* __restrict__ dp,
                                                          double* u0, double* u1, double* u2, double* p) {
  NN4_PASS_PROLOGUE(1, true)
  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yG[RY];
  T ly[RY];
  int gy[RY];
  bool in[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yG[r] = fy.G;
    ly[r] = fy.lump;
    in[r] = gx < g.nx && gy[r] < g.ny;
  }
  T A[3][RY][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int r = 0; r < RY; ++r) A[d][r][0] = A[d][r][1] = A[d][r][2] = T(0);
  double* uu[3] = {u0, u1, u2};
  double cr[RY], dr[RY], ur[3][RY];  // prefetched C, dp and u of plane s - 1
#pragma unroll
  for (int r = 0; r < RY; ++r) cr[r] = dr[r] = ur[0][r] = ur[1][r] = ur[2][r] = 0.0;
  for (int s = ring.j0; s <= last; ++s) {
    NN4_PASS_STEP_BEGIN()
    if (s >= 0 && s < g.nz) {
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
      T vv[RY + 2][3], xG[RY + 2], xM[RY + 2], P[RY];
      ft::nb<T, RY, SW>(cur, R0, tx, vv);
      ft::xpass<T, RY>(vv, FX.G, xG);
      ft::xpass<T, RY>(vv, FX.M, xM);
      ft::ypass<T, RY>(xG, yM, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(A[0][r], P[r], zp.M, zs.M, zn.M);
      ft::ypass<T, RY>(xM, yG, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(A[1][r], P[r], zp.M, zs.M, zn.M);
      ft::ypass<T, RY>(xM, yM, P);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(A[2][r], P[r], zp.G, zs.G, zn.G);
    }
    const int q = s - 1;
    if (q >= z0) {
      const T lz = ft::facz(g, q).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!in[r]) continue;
        const long long o = (long long)q * g.plane + (long long)gy[r] * g.pitch + gx;
        if (!on_face(vf, gx, gy[r], q, g.nx, g.ny, g.nz)) {
          if constexpr (sizeof(T) == 8) {
            const double rho = rho_g + rho_d * cr[r];
            const double f = -dtT / (FX.lump * ly[r] * lz * rho);
#pragma unroll
            for (int d = 0; d < 3; ++d) uu[d][o] = ur[d][r] + f * A[d][r][0];
          } else {
            const T rho = rho_g + rho_d * ft::from64<T>(cr[r]);
            const T f = -dtT / (FX.lump * ly[r] * lz * rho);
#pragma unroll
            for (int d = 0; d < 3; ++d) uu[d][o] = ur[d][r] + ft::to64(f * A[d][r][0]);
          }
        }
        if (p) p[o] += dr[r];
      }
    }
    // prefetch C, dp and u of plane s (emitted at the next step)
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const bool ok = in[r] && s >= z0 && s < z1;
      const long long o = (long long)s * g.plane + (long long)gy[r] * g.pitch + gx;
      cr[r] = ok ? __ldg(C + o) : 0.0;
      dr[r] = ok ? __ldg(dp + o) : 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) ur[d][r] = ok ? uu[d][o] : 0.0;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zshift(A[d][r]);
    NN4_PASS_STEP_END()
  }
}

// ---------------------------------------------------------------- momentum predictor
// Stage A for component c: k_c = rho min(k_max, k_abs, k_square) + mu from psi = u^{n+1/2}_c
// (Eqs. a_psi, efficient-kabs, h_Psi, k-square, max-k, k_Psi-n), two stages as in k_vof_coef with
// g = u^{n+1/2} . grad psi.
template <typename T>
struct MomK {
  T alpha_a, alpha_kabs, alpha_ksq, eps_k, third;
  T h[3];
  T rho_g, rho_d, mu_g, mu_d;  // rho = rho_g + rho_d C, mu = mu_g + mu_d C
};

template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_mom_coef(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                       const MomK<T> p, int zc, const double* __restrict__ C,
                                                       const double* __restrict__ uh0, const double* __restrict__ uh1,
                                                       const double* __restrict__ uh2, T* __restrict__ kout) {
  constexpr int NT = 32 * TYT, TY = TYT * RY, SW = 34, SH = TY + 2;
  using BC = ft::Halo2<SH>;
  extern __shared__ __align__(128) unsigned char smem[];
  T* const cs = reinterpret_cast<T*>(smem + NS * BC::BYTES);  // compute slots [2][SH * SW] of psi
  T* const sg = cs + 2 * SH * SW;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  const int X0 = blockIdx.x * 30, Y0 = blockIdx.y * (TY - 2);
  const int gx = X0 - 1 + tx, R0 = ty * RY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
  ft::Ring<NS> ring{reinterpret_cast<uint64_t*>(sg + SH * SW), smem, BC::BYTES, z0 - 2};
  const int last = z1 + 1;
  auto issue = [&](int z) {
    mbar_expect_tx(ring.barrier(z), BC::TX);
    tma_load_3d(ring.at(z), &maps.m[0], X0 - 2, Y0 - 2, z, ring.barrier(z));
  };
  if (tid == 0) ring.init();
  for (int i = tid; i < SH * SW; i += NT) sg[i] = T(0);
  __syncthreads();
  if (tid == 0)
    for (int z = ring.j0; z <= min(last, ring.j0 + NS - 2); ++z) issue(z);
  bool failed = !ring.wait(ring.j0);
  ft::convert_box<BC, SW, SH, NT, true>(cs, ring.at(ring.j0), tid);
  if (__syncthreads_or(failed)) {
    if (tid == 0) ring.drain(ring.j0, min(last, ring.j0 + NS - 2));
    return;
  }
  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yG[RY];
  T ly[RY];
  int gy[RY];
  bool in[RY], outp[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 - 1 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yG[r] = fy.G;
    ly[r] = fy.lump;
    in[r] = gx >= 0 && gx < g.nx && gy[r] >= 0 && gy[r] < g.ny;
    outp[r] = in[r] && tx >= 1 && tx <= 30 && R0 + r >= 1 && R0 + r <= TY - 2;
  }
  const double* uh[3] = {uh0, uh1, uh2};
  T gacc[3][RY][3], aacc[RY][3], Pdq[3][RY], gq[RY], Uq[3][RY];
  double Ur[3][RY], cr[RY];  // prefetched u^{n+1/2} of plane s - 1 and C of plane s - 2
#pragma unroll
  for (int r = 0; r < RY; ++r) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      gacc[0][r][c] = gacc[1][r][c] = gacc[2][r][c] = aacc[r][c] = T(0);
      Pdq[c][r] = Uq[c][r] = T(0);
      Ur[c][r] = 0.0;
    }
    gq[r] = T(0);
    cr[r] = 0.0;
  }
  for (int s = ring.j0; s <= last; ++s) {
    if (tid == 0 && s + NS - 1 <= last) issue(s + NS - 1);
    const T* cur = cs + ((s - ring.j0) & 1) * SH * SW;
    const int t = s - 1, q = s - 2;
    const bool tin = t >= 0 && t < g.nz;
    const bool emit = q >= z0 && q < z1;
    T Ut[3][RY];
    double c64[RY];
#pragma unroll
    for (int r = 0; r < RY; ++r) {
#pragma unroll
      for (int d = 0; d < 3; ++d) Ut[d][r] = ft::from64<T>(Ur[d][r]);
      c64[r] = cr[r];
    }
    if (s >= 0 && s < g.nz) {
      T vv[RY + 2][3], xG[RY + 2], xM[RY + 2], GM[RY], MG[RY], MM[RY];
      ft::nb<T, RY, SW>(cur, R0, tx, vv);
      ft::xpass<T, RY>(vv, FX.G, xG);
      ft::xpass<T, RY>(vv, FX.M, xM);
      ft::ypass<T, RY>(xG, yM, GM);
      ft::ypass<T, RY>(xM, yG, MG);
      ft::ypass<T, RY>(xM, yM, MM);
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        ft::zacc(gacc[0][r], GM[r], zp.M, zs.M, zn.M);
        ft::zacc(gacc[1][r], MG[r], zp.M, zs.M, zn.M);
        ft::zacc(gacc[2][r], MM[r], zp.G, zs.G, zn.G);
      }
    }
    T Pdt[3][RY], gt[RY];
    {
      const T lz = ft::facz(g, t).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (tin && in[r]) {
          const T im = ft::qdiv(T(1), FX.lump * ly[r] * lz);
#pragma unroll
          for (int d = 0; d < 3; ++d) Pdt[d][r] = gacc[d][r][0] * im;
          gt[r] = Ut[0][r] * Pdt[0][r] + Ut[1][r] * Pdt[1][r] + Ut[2][r] * Pdt[2][r];
        } else {
          Pdt[0][r] = Pdt[1][r] = Pdt[2][r] = gt[r] = T(0);
        }
        sg[(R0 + r + 1) * SW + tx + 1] = gt[r];
#pragma unroll
        for (int d = 0; d < 3; ++d) ft::zshift(gacc[d][r]);
      }
    }
    // prefetch u^{n+1/2} of plane s and C of plane t (used at the next step)
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const bool ok = in[r] && s >= 0 && s < g.nz;
      const long long o = (long long)s * g.plane + (long long)gy[r] * g.pitch + gx;
#pragma unroll
      for (int d = 0; d < 3; ++d) Ur[d][r] = ok ? __ldg(uh[d] + o) : 0.0;
      cr[r] = (outp[r] && t >= z0 && t < z1) ? __ldg(C + o - g.plane) : 0.0;
    }
    __syncthreads();
    if (tin) {
      T vg[RY + 2][3], xr[RY + 2], P[RY];
      ft::nb<T, RY, SW>(sg, R0, tx, vg);
      ft::xpass<T, RY>(vg, FX.M, xr);
      ft::ypass<T, RY>(xr, yM, P);
      const Fac<T> zp = ft::facz(g, t - 1), zs = ft::facz(g, t), zn = ft::facz(g, t + 1);
#pragma unroll
      for (int r = 0; r < RY; ++r) ft::zacc(aacc[r], P[r], zp.M, zs.M, zn.M);
    }
    if (emit) {
      const T lz = ft::facz(g, q).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!outp[r]) continue;
        const T m = FX.lump * ly[r] * lz;
        const T a = p.alpha_a * (ft::qdiv(aacc[r][0], m) - gq[r]);  // Eq. a_psi
        const T px = Pdq[0][r], py = Pdq[1][r], pz = Pdq[2][r];
        const T ax = fabs(px), ay = fabs(py), az = fabs(pz), sab = ax + ay + az;
        const T hsum = p.h[0] * ax + p.h[1] * ay + p.h[2] * az;
        const T k_abs = ft::qdiv(p.alpha_kabs * fabs(a) * hsum, p.eps_k + sab * sab * p.third);  // Eq. efficient-kabs
        const T h_psi = ft::qdiv(hsum, p.eps_k + sab);                                             // Eq. h_Psi
        const T u0 = Uq[0][r], u1 = Uq[1][r], u2 = Uq[2][r];
        const T k_sq = ft::qdiv(p.alpha_ksq * a * a * h_psi,
                                p.eps_k + (fabs(u0 * px) + fabs(u1 * py) + fabs(u2 * pz)) *
                                              (px * px + py * py + pz * pz) * p.third);  // Eq. k-square
        const T kmax = p.h[0] * fabs(u0) + p.h[1] * fabs(u1) + p.h[2] * fabs(u2);  // Eq. max-k
        const T c = ft::from64<T>(c64[r]);
        const T rho = p.rho_g + p.rho_d * c, mu = p.mu_g + p.mu_d * c;
        kout[(long long)q * g.plane + (long long)gy[r] * g.pitch + gx] = rho * fmin(kmax, fmin(k_abs, k_sq)) + mu;
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      ft::zshift(aacc[r]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Pdq[d][r] = Pdt[d][r];
        Uq[d][r] = Ut[d][r];
      }
      gq[r] = gt[r];
    }
    if (s < last) {
      if (!ring.wait(s + 1)) failed = true;
      ft::convert_box<BC, SW, SH, NT, true>(cs + ((s + 1 - ring.j0) & 1) * SH * SW, ring.at(s + 1), tid);
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) ring.drain(s + 1, min(last, s + NS - 1));
      return;
    }
  }
}

// Stage B for component c: s~ = rho (u^{n+1/2} . f_raw(psi)) + (1/2)[L(k psi) + k L psi - psi L k]
// + f(p; w_c) - f(s_c; w_m) (Eq. Petrov-u/v/w with the isotropic L = w_lap of Eq. k-T), then
// psi~ = psi^n - dt s~ / (m rho) (0 on the no-slip faces; Eq. velocity-1 with sigma = 0) and
// psi^{n+1/2} = (psi^n + psi~) / 2.
template <typename T, int RY, int TYT, int NS>
__global__ void __launch_bounds__(32 * TYT) k_mom_update(const __grid_constant__ ft::FMaps maps, const Geo<T> g,
                                                         const MomK<T> p, const Faces vf, int zc, int comp, double dt,
                                                         T dtT, const double* __restrict__ C,
                                                         const double* __restrict__ uh0, const double* __restrict__ uh1,
                                                         const double* __restrict__ uh2, const double* __restrict__ un,
                                                         double* __restrict__ ut, double* __restrict__ uh_next) {
  constexpr int NT = 32 * TYT, TY = TYT * RY, SW = 34, SH = TY + 2;
  using BD = ft::Halo1<double, SH>;
  using BK = ft::Halo1<T, SH>;
  // slot: psi, p, s (FP64), then k (type T)
  constexpr int NF = 4, SLOT = 3 * BD::BYTES + BK::BYTES;
  extern __shared__ __align__(128) unsigned char smem[];
  T* const cs = reinterpret_cast<T*>(smem + NS * SLOT);  // compute slots [2][4][SH * SW]: psi, k, p, s
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
  const int X0 = blockIdx.x * 32, Y0 = blockIdx.y * TY;
  const int gx = X0 + tx, R0 = ty * RY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nz);
  ft::Ring<NS> ring{reinterpret_cast<uint64_t*>(cs + 2 * NF * SH * SW), smem, SLOT, z0 - 1};
  const int last = z1;
  auto issue = [&](int z) {
    unsigned char* d = ring.at(z);
    mbar_expect_tx(ring.barrier(z), 3 * BD::TX + BK::TX);
    for (int f = 0; f < 3; ++f)
      tma_load_3d(d + f * BD::BYTES, &maps.m[f], X0 - 1 - BD::CO, Y0 - 1, z, ring.barrier(z));
    tma_load_3d(d + 3 * BD::BYTES, &maps.m[3], X0 - 1 - BK::CO, Y0 - 1, z, ring.barrier(z));
  };
  auto convert = [&](int z, T* dst) {
    const unsigned char* src = ring.at(z);
    ft::convert_box<BD, SW, SH, NT, true>(dst, src, tid);                                  // psi
    ft::convert_box<BK, SW, SH, NT>(dst + SH * SW, src + 3 * BD::BYTES, tid);             // k
    ft::convert_box<BD, SW, SH, NT, true>(dst + 2 * SH * SW, src + BD::BYTES, tid);       // p
    ft::convert_box<BD, SW, SH, NT, true>(dst + 3 * SH * SW, src + 2 * BD::BYTES, tid);   // s
  };
  if (tid == 0) ring.init();
  __syncthreads();
  if (tid == 0)
    for (int z = ring.j0; z <= min(last, ring.j0 + NS - 2); ++z) issue(z);
  bool failed = !ring.wait(ring.j0);
  convert(ring.j0, cs);
  if (__syncthreads_or(failed)) {
    if (tid == 0) ring.drain(ring.j0, min(last, ring.j0 + NS - 2));
    return;
  }
  const Fac<T> FX = ft::facx(g, gx);
  W3<T> yM[RY], yG[RY], yK[RY];
  T ly[RY];
  int gy[RY];
  bool in[RY];
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    gy[r] = Y0 + R0 + r;
    const Fac<T> fy = ft::facy(g, gy[r]);
    yM[r] = fy.M;
    yG[r] = fy.G;
    yK[r] = fy.K;
    ly[r] = fy.lump;
    in[r] = gx < g.nx && gy[r] < g.ny;
  }
  const double* uh[3] = {uh0, uh1, uh2};
  // accumulators: raw gradient of psi (3), A = (1/2) L(k psi) + f(p; w_c) - f(s; w_m), L psi, L k
  T Acc[6][RY][3], Pq[RY], Kq[RY];
  double Ur[3][RY], cr[RY], nr[RY];  // prefetched u^{n+1/2}, C and u^n_c of plane s - 1
#pragma unroll
  for (int a = 0; a < 6; ++a)
#pragma unroll
    for (int r = 0; r < RY; ++r) Acc[a][r][0] = Acc[a][r][1] = Acc[a][r][2] = T(0);
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    Pq[r] = Kq[r] = T(0);
    Ur[0][r] = Ur[1][r] = Ur[2][r] = cr[r] = nr[r] = 0.0;
  }

  for (int s = ring.j0; s <= last; ++s) {
    if (tid == 0 && s + NS - 1 <= last) issue(s + NS - 1);
    const T* cur = cs + ((s - ring.j0) & 1) * NF * SH * SW;
    const int q = s - 1;
    const bool emit = q >= z0;
    T PN[RY], KN[RY];
    if (s >= 0 && s < g.nz) {
      const Fac<T> zp = ft::facz(g, s - 1), zs = ft::facz(g, s), zn = ft::facz(g, s + 1);
      T P[RY], P2[RY];
      {
        // psi: raw gradient and L psi
        T v[RY + 2][3], xG[RY + 2], xM[RY + 2], xK[RY + 2];
        ft::nb<T, RY, SW>(cur, R0, tx, v);
#pragma unroll
        for (int r = 0; r < RY; ++r) PN[r] = v[r + 1][1];
        ft::xpass<T, RY>(v, FX.G, xG);
        ft::xpass<T, RY>(v, FX.M, xM);
        ft::xpass<T, RY>(v, FX.K, xK);
        ft::ypass<T, RY>(xG, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[0][r], P[r], zp.M, zs.M, zn.M);
        ft::ypass<T, RY>(xM, yG, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[1][r], P[r], zp.M, zs.M, zn.M);
        ft::ypass<T, RY>(xM, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) {
          ft::zacc(Acc[2][r], P[r], zp.G, zs.G, zn.G);
          ft::zacc(Acc[4][r], P[r], zp.K, zs.K, zn.K);
        }
        ft::ypass<T, RY>(xK, yM, P);
        ft::ypass<T, RY>(xM, yK, P2);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[4][r], P[r] + P2[r], zp.M, zs.M, zn.M);
        // k and k psi: L k and (1/2) L(k psi)
        T vk[RY + 2][3];
        ft::nb<T, RY, SW>(cur + SH * SW, R0, tx, vk);
#pragma unroll
        for (int r = 0; r < RY; ++r) KN[r] = vk[r + 1][1];
        ft::xpass<T, RY>(vk, FX.M, xM);
        ft::xpass<T, RY>(vk, FX.K, xK);
        ft::ypass<T, RY>(xK, yM, P);
        ft::ypass<T, RY>(xM, yK, P2);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[5][r], P[r] + P2[r], zp.M, zs.M, zn.M);
        ft::ypass<T, RY>(xM, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[5][r], P[r], zp.K, zs.K, zn.K);
#pragma unroll
        for (int rr = 0; rr < RY + 2; ++rr)
#pragma unroll
          for (int c = 0; c < 3; ++c) vk[rr][c] *= T(0.5) * v[rr][c];
        ft::xpass<T, RY>(vk, FX.M, xM);
        ft::xpass<T, RY>(vk, FX.K, xK);
        ft::ypass<T, RY>(xK, yM, P);
        ft::ypass<T, RY>(xM, yK, P2);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[3][r], P[r] + P2[r], zp.M, zs.M, zn.M);
        ft::ypass<T, RY>(xM, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[3][r], P[r], zp.K, zs.K, zn.K);
      }
      {
        // f(p; w_c) - f(s; w_m)
        T v[RY + 2][3], xr[RY + 2];
        ft::nb<T, RY, SW>(cur + 2 * SH * SW, R0, tx, v);
        ft::xpass<T, RY>(v, comp == 0 ? FX.G : FX.M, xr);
        ft::ypass<T, RY>(xr, comp == 1 ? yG : yM, P);
        const W3<T>& wp = comp == 2 ? zp.G : zp.M;
        const W3<T>& ws = comp == 2 ? zs.G : zs.M;
        const W3<T>& wn = comp == 2 ? zn.G : zn.M;
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[3][r], P[r], wp, ws, wn);
        ft::nb<T, RY, SW>(cur + 3 * SH * SW, R0, tx, v);
        ft::xpass<T, RY>(v, FX.M, xr);
        ft::ypass<T, RY>(xr, yM, P);
#pragma unroll
        for (int r = 0; r < RY; ++r) ft::zacc(Acc[3][r], -P[r], zp.M, zs.M, zn.M);
      }
    } else {
#pragma unroll
      for (int r = 0; r < RY; ++r) PN[r] = KN[r] = T(0);
    }
    if (emit) {
      const T lz = ft::facz(g, q).lump;
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        if (!in[r]) continue;
        const long long o = (long long)q * g.plane + (long long)gy[r] * g.pitch + gx;
        const T c = ft::from64<T>(cr[r]);
        const T rho = p.rho_g + p.rho_d * c;
        const T sv = rho * (ft::from64<T>(Ur[0][r]) * Acc[0][r][0] + ft::from64<T>(Ur[1][r]) * Acc[1][r][0] +
                            ft::from64<T>(Ur[2][r]) * Acc[2][r][0]) +
                     Acc[3][r][0] + T(0.5) * (Kq[r] * Acc[4][r][0] - Pq[r] * Acc[5][r][0]);
        const double un64 = nr[r];
        if (on_face(vf, gx, gy[r], q, g.nx, g.ny, g.nz)) {
          ut[o] = 0.0;
          if (uh_next) uh_next[o] = 0.5 * un64;
        } else {
          const T m = FX.lump * ly[r] * lz;
          if constexpr (sizeof(T) == 8) {
            const double v = un64 - dt * sv / (m * rho);
            ut[o] = v;
            if (uh_next) uh_next[o] = 0.5 * (un64 + v);
          } else {
            const T delta = -dtT * sv / (m * rho);
            ut[o] = un64 + ft::to64(delta);
            if (uh_next) uh_next[o] = un64 + ft::to64(T(0.5) * delta);
          }
        }
      }
    }
    // prefetch u^{n+1/2}, C and u^n_c of plane s (emitted at the next step)
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      const bool ok = in[r] && s >= z0 && s < z1;
      const long long o = (long long)s * g.plane + (long long)gy[r] * g.pitch + gx;
#pragma unroll
      for (int d = 0; d < 3; ++d) Ur[d][r] = ok ? __ldg(uh[d] + o) : 0.0;
      cr[r] = ok ? __ldg(C + o) : 0.0;
      nr[r] = ok ? __ldg(un + o) : 0.0;
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
#pragma unroll
      for (int a = 0; a < 6; ++a) ft::zshift(Acc[a][r]);
      Pq[r] = PN[r];
      Kq[r] = KN[r];
    }
    if (s < last) {
      if (!ring.wait(s + 1)) failed = true;
      convert(s + 1, cs + ((s + 1 - ring.j0) & 1) * NF * SH * SW);
    }
    if (__syncthreads_or(failed)) {
      if (tid == 0) ring.drain(s + 1, min(last, s + NS - 1));
      return;
    }
  }
}

template <typename T, int TY, int NS>
constexpr int mom_update_smem() {
  return NS * (3 * ft::Halo1<double, TY + 2>::BYTES + ft::Halo1<T, TY + 2>::BYTES) +
         2 * 4 * (TY + 2) * 34 * (int)sizeof(T) + NS * 8;
}

// ---------------------------------------------------------------- reductions
// sum_i m_i C_i = h_x h_y h_z sum over rows (j, k) of w_j w_k (sum_i C_i - (C_0 + C_{nx-1}) / 2),
// w = 1/2 on the first and last row and plane: one FP64 addition per node.  A warp takes a row;
// the grid holds the resident blocks and strides over rows; one atomic per block.
__global__ void __launch_bounds__(256) k_mass(int nx, int ny, int nz, long long pitch, double vol,
                                              const double* __restrict__ C, double* out) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long rows = (long long)ny * nz;
  double tot = 0.0;
  for (long long row = warp; row < rows; row += nwarps) {
    const int j = (int)(row % ny), k = (int)(row / ny);
    const double* p = C + row * pitch;
    double a = 0.0;
    for (int i = lane; i < nx; i += 32) a += __ldg(p + i);
    a = warp_sum(a);
    if (lane == 0) {
      a -= 0.5 * (__ldg(p) + __ldg(p + nx - 1));
      const double wy = (j == 0 || j == ny - 1) ? 0.5 : 1.0, wz = (k == 0 || k == nz - 1) ? 0.5 : 1.0;
      tot += wy * wz * a;
    }
  }
  block_sum_atomic(lane == 0 ? tot * vol : 0.0, out, red);
}

// min / max of a field (order-preserving integer image of doubles; out[0] = min, out[1] = max)
__device__ __forceinline__ unsigned long long ord(double v) {
  const unsigned long long b = __double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__global__ void __launch_bounds__(256) k_range(int nx, int ny, int nz, long long pitch, const double* __restrict__ C,
                                               unsigned long long* out) {
  unsigned long long lo = ~0ull, hi = 0ull;
  const long long n = (long long)nx * ny * nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / nx;
    const unsigned long long v = ord(__ldg(C + row * pitch + (e - row * nx)));
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&out[0], lo);
    atomicMax(&out[1], hi);
  }
}

// ---------------------------------------------------------------- launch shapes
// Launch shape of one kernel family: TYT threads along y (x is one warp), RY nodes per thread.
// 256 threads with two rows each (the register budget of the FP64 forms allows no more).
template <typename T>
struct Shape;
template <>
struct Shape<float> {
  static constexpr int RY = 2, TYT = 8;
};
template <>
struct Shape<double> {
  static constexpr int RY = 2, TYT = 8;
};

// z planes per block: enough blocks for two waves of 152 SMs, at most 64 planes per block
int zchunk_for(long long tiles_xy, int nz) {
  const long long want = 2LL * 152 * 2;
  long long chunks = (want + tiles_xy - 1) / tiles_xy;
  int zc = (int)((nz + chunks - 1) / chunks);
  zc = std::max(4, std::min(64, zc));
  return zc;
}

template <typename T>
dim3 grid_out(const nn4_grid* g, int tile_x, int tile_y, int* zc) {
  const int bx = (g->n[0] + tile_x - 1) / tile_x, by = (g->n[1] + tile_y - 1) / tile_y;
  *zc = zchunk_for((long long)bx * by, g->n[2]);
  return dim3(bx, by, (g->n[2] + *zc - 1) / *zc);
}

Faces faces_of(const nn4_grid* g) {
  Faces f;
  for (int i = 0; i < 6; ++i) f.d[i] = g->bc[i] == NN4_BC_DIRICHLET ? 1 : 0;
  return f;
}

template <typename T>
VofK<T> vof_k(const nn4_vof_params* p, const nn4_grid* g) {
  VofK<T> k;
  const double hmax = std::max(g->h[0], std::max(g->h[1], g->h[2]));
  const double hmin = std::min(g->h[0], std::min(g->h[1], g->h[2]));
  k.alpha_a = (T)p->alpha_a;
  k.alpha_kabs = (T)(1.0 / (8.0 * (double)(1 << p->p)));
  k.eps_k = (T)p->eps_k;
  k.K_plus = (T)p->K_plus;
  k.K_minus = (T)p->K_minus;
  k.beta = (T)p->beta;
  k.eps_x = (T)p->eps_x;
  k.K_pos = (T)p->K_pos;
  k.kmin = (T)(p->alpha_min * hmax * hmax / p->dt);
  k.kmax = (T)(p->alpha_max * hmin * hmin / p->dt);
  k.third = (T)(1.0 / 3.0);
  for (int d = 0; d < 3; ++d) {
    k.h[d] = (T)g->h[d];
    k.ih[d] = (T)(1.0 / g->h[d]);
  }
  k.detect_hi = p->detect_hi;
  k.detect_lo = p->detect_lo;
  return k;
}

template <typename T>
MomK<T> mom_k(const nn4_flow_params* fp, const nn4_grid* g) {
  MomK<T> k;
  k.alpha_a = (T)fp->alpha_a;
  k.alpha_kabs = (T)(1.0 / (8.0 * (double)(1 << fp->p)));
  k.alpha_ksq = (T)(8.0 / (double)(1 << fp->p));
  k.eps_k = (T)fp->eps_k;
  k.third = (T)(1.0 / 3.0);
  for (int d = 0; d < 3; ++d) k.h[d] = (T)g->h[d];
  k.rho_g = (T)fp->rho_g;
  k.rho_d = (T)(fp->rho_l - fp->rho_g);
  k.mu_g = (T)fp->mu_g;
  k.mu_d = (T)(fp->mu_l - fp->mu_g);
  return k;
}

// dynamic shared memory of a kernel above the default 48 KB
template <typename K>
int allow_smem(K kern, int bytes) {
  return check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes),
                    "cudaFuncSetAttribute(flow kernel)");
}

// tensor map of an FP64 or FP32 field on grid g (row pitch g->pitch elements) with box bw x bh
bool fmap(CUtensorMap* m, const nn4_grid* g, bool f64, const void* base, int bw, int bh) {
  return make_tmap_3d(m, f64 ? NN4_F64 : NN4_F32, base, g->n[0], g->n[1], g->n[2], g->pitch, bw, bh);
}

constexpr int kRing = 4;  // raw plane slots of the flow kernels (3 planes in flight)

// the VOF step on a scratch of three coefficient fields (elements f apart)
template <typename T>
int vof_launch(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u, const double* v,
               const double* w, double* s_C, double* C_next, void* scratch, size_t f, cudaStream_t s) {
  constexpr int RY = Shape<T>::RY, TYT = Shape<T>::TYT, TY = RY * TYT, SH = TY + 2;
  const Geo<T> G = make_geo<T>(g);
  T* k = static_cast<T*>(scratch);
  ft::FMaps ma{}, mb{};
  bool ok = fmap(&ma.m[0], g, true, C, ft::Halo2<SH>::BW, SH) && fmap(&mb.m[0], g, true, C, ft::Halo1<double, SH>::BW, SH);
  for (int d = 0; d < 3; ++d) ok = ok && fmap(&mb.m[1 + d], g, sizeof(T) == 8, k + d * f, ft::Halo1<T, SH>::BW, SH);
  if (!ok) return set_error(NN4_ECUDA, "tensor map encode failed (VOF)");
  auto ka = k_vof_coef<T, RY, TYT, kRing>;
  auto kb = k_vof_update<T, RY, TYT, kRing>;
  constexpr int sa = vof_coef_smem<T, TY, kRing>(), sb = vof_update_smem<T, TY, kRing>();
  int rc;
  if ((rc = allow_smem(ka, sa)) || (rc = allow_smem(kb, sb))) return rc;
  int zc = 0;
  dim3 ga = grid_out<T>(g, 30, TY - 2, &zc);
  ka<<<ga, dim3(32, TYT), sa, s>>>(ma, G, vof_k<T>(p, g), zc, C, u, v, w, k, k + f, k + 2 * f);
  dim3 gb = grid_out<T>(g, 32, TY, &zc);
  kb<<<gb, dim3(32, TYT), sb, s>>>(mb, G, p->dt, (T)p->dt, zc, C, u, v, w, s_C, C_next);
  return check_cuda(cudaGetLastError(), "VOF kernels");
}

int check_compute(int c) {
  if (c != NN4_F64 && c != NN4_F32) return set_error(NN4_EINVAL, "compute must be NN4_F64 or NN4_F32");
  return NN4_OK;
}

int check_vof_args(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u, const double* v,
                   const double* w, const double* s_C, const double* C_next) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = validate_ptr(C, "C")) || (rc = validate_ptr(u, "u")) ||
      (rc = validate_ptr(v, "v")) || (rc = validate_ptr(w, "w")) || (rc = validate_ptr(s_C, "s_C")))
    return rc;
  if (!p) return set_error(NN4_EINVAL, "params is NULL");
  if (!(p->dt > 0.0) || p->p < 1 || p->p > 3) return set_error(NN4_EINVAL, "bad VOF parameters");
  if ((rc = check_compute(p->compute))) return rc;
  if (C_next && (rc = validate_ptr(C_next, "C_next"))) return rc;
  if (s_C == C || C_next == C) return set_error(NN4_EINVAL, "outputs must not alias C");
  return NN4_OK;
}

template <typename T>
int sources_launch(const nn4_grid* g, const nn4_flow_params* fp, const double* C, double* s0, double* s1,
                          double* s2, double* kappa, cudaStream_t st) {
  constexpr int RY = Shape<T>::RY, TYT = Shape<T>::TYT, TY = RY * TYT;
  const double hmin = std::min(g->h[0], std::min(g->h[1], g->h[2]));
  SrcK<T> p;
  p.eps_t = (T)(1e-7 / hmin);
  p.sigma = (T)fp->sigma_t;
  p.grho_g = (T)(fp->g * fp->rho_g);
  p.grho_d = (T)(fp->g * (fp->rho_l - fp->rho_g));
  constexpr int SH = TY + 2;
  ft::FMaps m{};
  if (!fmap(&m.m[0], g, true, C, ft::Halo2<SH>::BW, SH)) return set_error(NN4_ECUDA, "tensor map encode failed (sources)");
  auto kern = k_sources<T, RY, TYT, kRing>;
  constexpr int sm = sources_smem<T, TY, kRing>();
  int rc;
  if ((rc = allow_smem(kern, sm))) return rc;
  int zc = 0;
  dim3 ga = grid_out<T>(g, 30, TY - 2, &zc);
  kern<<<ga, dim3(32, TYT), sm, st>>>(m, make_geo<T>(g), p, zc, C, s0, s1, s2, kappa);
  return check_cuda(cudaGetLastError(), "momentum sources");
}

template <typename T>
int rhs_hs_launch(const nn4_grid* g, const double* s0, const double* s1, const double* s2, double* b,
                         cudaStream_t st) {
  constexpr int RY = Shape<T>::RY, TYT = Shape<T>::TYT, TY = RY * TYT;
  constexpr int SH = TY + 2;
  ft::FMaps m{};
  const double* src[3] = {s0, s1, s2};
  for (int d = 0; d < 3; ++d)
    if (!fmap(&m.m[d], g, true, src[d], ft::Halo1<double, SH>::BW, SH))
      return set_error(NN4_ECUDA, "tensor map encode failed (stage-1 rhs)");
  auto kern = k_rhs_hs<T, RY, TYT, kRing>;
  constexpr int sm = pass_smem<T, TY, kRing, 3>();
  int rc;
  if ((rc = allow_smem(kern, sm))) return rc;
  int zc = 0;
  dim3 gb = grid_out<T>(g, 32, TY, &zc);
  kern<<<gb, dim3(32, TYT), sm, st>>>(m, make_geo<T>(g), faces_of(g), zc, b);
  return check_cuda(cudaGetLastError(), "stage-1 rhs");
}

template <typename T>
int rhs_nh_launch(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* u,
                         const double* v, const double* w, double* b, cudaStream_t st) {
  constexpr int RY = Shape<T>::RY, TYT = Shape<T>::TYT, TY = RY * TYT;
  constexpr int SH = TY + 2;
  ft::FMaps m{};
  const double* src[4] = {C, u, v, w};
  for (int d = 0; d < 4; ++d)
    if (!fmap(&m.m[d], g, true, src[d], ft::Halo1<double, SH>::BW, SH))
      return set_error(NN4_ECUDA, "tensor map encode failed (stage-3 rhs)");
  auto kern = k_rhs_nh<T, RY, TYT, kRing>;
  constexpr int sm = pass_smem<T, TY, kRing, 4>();
  int rc;
  if ((rc = allow_smem(kern, sm))) return rc;
  int zc = 0;
  dim3 gb = grid_out<T>(g, 32, TY, &zc);
  kern<<<gb, dim3(32, TYT), sm, st>>>(m, make_geo<T>(g), faces_of(g), zc, (T)fp->rho_g, (T)(fp->rho_l - fp->rho_g),
                                      (T)(1.0 / fp->dt), b);
  return check_cuda(cudaGetLastError(), "stage-3 rhs");
}

template <typename T>
int vel_launch(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* dp, double* u,
                      double* v, double* w, double* p_nh, cudaStream_t st) {
  constexpr int RY = Shape<T>::RY, TYT = Shape<T>::TYT, TY = RY * TYT;
  constexpr int SH = TY + 2;
  ft::FMaps m{};
  if (!fmap(&m.m[0], g, true, dp, ft::Halo1<double, SH>::BW, SH))
    return set_error(NN4_ECUDA, "tensor map encode failed (velocity correction)");
  auto kern = k_vel_correct<T, RY, TYT, kRing>;
  constexpr int sm = pass_smem<T, TY, kRing, 1>();
  int rc;
  if ((rc = allow_smem(kern, sm))) return rc;
  int zc = 0;
  dim3 gb = grid_out<T>(g, 32, TY, &zc);
  kern<<<gb, dim3(32, TYT), sm, st>>>(m, make_geo<T>(g), faces_of(g), zc, (T)fp->rho_g, (T)(fp->rho_l - fp->rho_g),
                                      (T)fp->dt, C, dp, u, v, w, p_nh);
  return check_cuda(cudaGetLastError(), "velocity correction");
}

template <typename T>
int predict_launch(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* const* un,
                          const double* const* uh, double* const* ut, double* const* uh_next, const double* p,
                          const double* const* src, void* workspace, cudaStream_t st) {
  constexpr int RY = Shape<T>::RY, TYT = Shape<T>::TYT, TY = RY * TYT;
  const Geo<T> G = make_geo<T>(g);
  const MomK<T> mk = mom_k<T>(fp, g);
  const size_t f = (size_t)g->pitch * g->n[1] * g->n[2];
  T* k = static_cast<T*>(workspace);
  constexpr int SH = TY + 2;
  auto ka = k_mom_coef<T, RY, TYT, kRing>;
  auto kb = k_mom_update<T, RY, TYT, kRing>;
  constexpr int sa = vof_coef_smem<T, TY, kRing>(), sb = mom_update_smem<T, TY, kRing>();
  int rc;
  if ((rc = allow_smem(ka, sa)) || (rc = allow_smem(kb, sb))) return rc;
  int zc = 0;
  dim3 ga = grid_out<T>(g, 30, TY - 2, &zc);
  for (int c = 0; c < 3; ++c) {
    ft::FMaps m{};
    if (!fmap(&m.m[0], g, true, uh[c], ft::Halo2<SH>::BW, SH))
      return set_error(NN4_ECUDA, "tensor map encode failed (predictor)");
    ka<<<ga, dim3(32, TYT), sa, st>>>(m, G, mk, zc, C, uh[0], uh[1], uh[2], k + c * f);
  }
  int zc2 = 0;
  dim3 gb = grid_out<T>(g, 32, TY, &zc2);
  const Faces vf = faces_of(g);
  for (int c = 0; c < 3; ++c) {
    ft::FMaps m{};
    const bool ok = fmap(&m.m[0], g, true, uh[c], ft::Halo1<double, SH>::BW, SH) &&
                    fmap(&m.m[1], g, true, p, ft::Halo1<double, SH>::BW, SH) &&
                    fmap(&m.m[2], g, true, src[c], ft::Halo1<double, SH>::BW, SH) &&
                    fmap(&m.m[3], g, sizeof(T) == 8, k + c * f, ft::Halo1<T, SH>::BW, SH);
    if (!ok) return set_error(NN4_ECUDA, "tensor map encode failed (predictor)");
    kb<<<gb, dim3(32, TYT), sb, st>>>(m, G, mk, vf, zc2, c, fp->dt, (T)fp->dt, C, uh[0], uh[1], uh[2], un[c], ut[c],
                                      uh_next ? uh_next[c] : nullptr);
  }
  return check_cuda(cudaGetLastError(), "momentum predictor");
}

}  // namespace

int launch_range(const nn4_grid* g, const double* C, unsigned long long* out, cudaStream_t s) {
  const long long n = (long long)g->n[0] * g->n[1] * g->n[2];
  const int blocks = (int)std::min<long long>((n + 255) / 256, (long long)sm_count() * 8);
  k_range<<<blocks, 256, 0, s>>>(g->n[0], g->n[1], g->n[2], g->pitch, C, out);
  return check_cuda(cudaGetLastError(), "range");
}

}  // namespace nn4

using namespace nn4;

extern "C" {

void nn4_vof_params_default(nn4_vof_params* p, double dt) {
  if (!p) return;
  p->dt = dt;
  p->alpha_a = 2.0;
  p->eps_k = 1e-7;
  p->K_plus = 300.0;
  p->K_minus = 300.0;
  p->beta = 0.1;
  p->eps_x = 1e-4;
  p->K_pos = 3.0;
  p->alpha_min = 1e-4;
  p->alpha_max = 0.05;
  p->detect_hi = 0.95;
  p->detect_lo = 0.05;
  p->p = 1;
  p->compute = NN4_F64;
}

int64_t nn4_vof_workspace_bytes(const nn4_grid* g) {
  if (!g || g->pitch <= 0) return -1;
  return 3LL * g->pitch * g->n[1] * g->n[2] * (int64_t)sizeof(double);
}

int nn4_vof_advect_residual(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u,
                            const double* v, const double* w, double* s_C, double* C_next, void* workspace,
                            void* stream) {
  int rc;
  if ((rc = check_vof_args(g, p, C, u, v, w, s_C, C_next)) || (rc = validate_ptr(workspace, "workspace"))) return rc;
  const size_t f = (size_t)g->pitch * g->n[1] * g->n[2];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->compute == NN4_F32) return vof_launch<float>(g, p, C, u, v, w, s_C, C_next, workspace, f, s);
  return vof_launch<double>(g, p, C, u, v, w, s_C, C_next, workspace, f, s);
}

// ---------------------------------------------------------------- allocation-free variant
// The same kernels with their scratch (the three coefficient fields) in a fixed device array
// instead of a caller buffer.  Every GPU that loads the library holds this array (18 MiB) until
// the process exits.
constexpr long long kVofStaticFieldElems = 786432;  // max pitch * ny * nz per scratch field
static __device__ __align__(256) double g_vof_scratch[3 * kVofStaticFieldElems];

namespace {
std::mutex g_vof_scratch_mu;
double* g_vof_scratch_ptr[128] = {nullptr};  // device address of g_vof_scratch, per device ordinal
}  // namespace

int nn4_vof_advect_residual_static(const nn4_grid* g, const nn4_vof_params* p, const double* C, const double* u,
                                   const double* v, const double* w, double* s_C, double* C_next, void* stream) {
  int rc;
  if ((rc = check_vof_args(g, p, C, u, v, w, s_C, C_next))) return rc;
  const long long f = (long long)g->pitch * g->n[1] * g->n[2];
  if (f > kVofStaticFieldElems)
    return set_error(NN4_EINVAL, "grid too large for the static scratch: pitch * ny * nz = " + std::to_string(f) +
                                     " > " + std::to_string(kVofStaticFieldElems));
  // set-up once per device, with that device current: the host-side name of the array is not a
  // device address, so take the address from the runtime
  int dev = 0;
  if ((rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
  if (dev < 0 || dev >= 128) return set_error(NN4_EUNSUPPORTED, "device ordinal out of range");
  double* ws = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_vof_scratch_mu);
    if (!g_vof_scratch_ptr[dev]) {
      void* ptr = nullptr;
      if ((rc = check_cuda(cudaGetSymbolAddress(&ptr, g_vof_scratch), "cudaGetSymbolAddress(scratch)"))) return rc;
      g_vof_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    ws = g_vof_scratch_ptr[dev];
  }
  // every scratch element the kernels read is written earlier in the same call (all nodes of the
  // three fields), so nothing needs clearing between calls
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->compute == NN4_F32) return vof_launch<float>(g, p, C, u, v, w, s_C, C_next, ws, (size_t)f, s);
  return vof_launch<double>(g, p, C, u, v, w, s_C, C_next, ws, (size_t)f, s);
}

void nn4_flow_params_default(nn4_flow_params* p, double dt) {
  if (!p) return;
  p->dt = dt;
  p->rho_l = 1000.0;
  p->rho_g = 1.0;
  p->mu_l = 1e-3;
  p->mu_g = 1.8e-5;
  p->sigma_t = 0.07;
  p->g = 9.81;
  p->alpha_a = 2.0;
  p->eps_k = 1e-7;
  p->p = 1;
  p->momentum_iters = 2;
  p->correction_iters = 2;
  p->pressure_cycles = 20;
  p->pressure_rtol = 0.0;
  p->compute = NN4_F64;
}

static int check_fp(const nn4_flow_params* fp) {
  if (!fp) return set_error(NN4_EINVAL, "flow params NULL");
  if (!(fp->dt > 0.0) || !(fp->rho_l > 0.0) || !(fp->rho_g > 0.0) || fp->p < 1 || fp->p > 3)
    return set_error(NN4_EINVAL, "bad flow parameters");
  return check_compute(fp->compute);
}


int nn4_momentum_sources(const nn4_grid* g, const nn4_flow_params* fp, const double* C, double* s0, double* s1,
                         double* s2, double* kappa, double* workspace, void* stream) {
  (void)workspace;
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(s0, "s0")) || (rc = validate_ptr(s1, "s1")) || (rc = validate_ptr(s2, "s2")))
    return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (fp->compute == NN4_F32) return sources_launch<float>(g, fp, C, s0, s1, s2, kappa, st);
  return sources_launch<double>(g, fp, C, s0, s1, s2, kappa, st);
}


int nn4_pressure_rhs_hs(const nn4_grid* g, const double* s0, const double* s1, const double* s2, double* b,
                        void* stream) {
  return nn4_pressure_rhs_hs_ex(g, NN4_F64, s0, s1, s2, b, stream);
}

int nn4_pressure_rhs_hs_ex(const nn4_grid* g, int compute, const double* s0, const double* s1, const double* s2,
                           double* b, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_compute(compute)) || (rc = validate_ptr(s0, "s0")) ||
      (rc = validate_ptr(s1, "s1")) || (rc = validate_ptr(s2, "s2")) || (rc = validate_ptr(b, "b")))
    return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (compute == NN4_F32) return rhs_hs_launch<float>(g, s0, s1, s2, b, st);
  return rhs_hs_launch<double>(g, s0, s1, s2, b, st);
}


int nn4_pressure_rhs_nh(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* u,
                        const double* v, const double* w, double* b, double* rho_ws, void* stream) {
  (void)rho_ws;
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(u, "u")) || (rc = validate_ptr(v, "v")) || (rc = validate_ptr(w, "w")) ||
      (rc = validate_ptr(b, "b")))
    return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (fp->compute == NN4_F32) return rhs_nh_launch<float>(g, fp, C, u, v, w, b, st);
  return rhs_nh_launch<double>(g, fp, C, u, v, w, b, st);
}


int nn4_velocity_correct(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* dp, double* u,
                         double* v, double* w, double* p_nh, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(dp, "dp")) || (rc = validate_ptr(u, "u")) || (rc = validate_ptr(v, "v")) ||
      (rc = validate_ptr(w, "w")))
    return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (fp->compute == NN4_F32) return vel_launch<float>(g, fp, C, dp, u, v, w, p_nh, st);
  return vel_launch<double>(g, fp, C, dp, u, v, w, p_nh, st);
}

int64_t nn4_momentum_workspace_bytes(const nn4_grid* g) {
  if (!g || g->pitch <= 0) return -1;
  return 3LL * g->pitch * g->n[1] * g->n[2] * (int64_t)sizeof(double);
}


int nn4_momentum_predict(const nn4_grid* g, const nn4_flow_params* fp, const double* C, const double* const* un,
                         const double* const* uh, double* const* ut, double* const* uh_next, const double* p,
                         const double* const* s, void* workspace, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = check_fp(fp)) || (rc = validate_ptr(C, "C")) ||
      (rc = validate_ptr(p, "p")) || (rc = validate_ptr(workspace, "workspace")))
    return rc;
  if (!un || !uh || !ut || !s) return set_error(NN4_EINVAL, "NULL component array");
  for (int c = 0; c < 3; ++c) {
    if ((rc = validate_ptr(un[c], "un")) || (rc = validate_ptr(uh[c], "uh")) || (rc = validate_ptr(ut[c], "ut")) ||
        (rc = validate_ptr(s[c], "s")))
      return rc;
    if (uh_next && (rc = validate_ptr(uh_next[c], "uh_next"))) return rc;
  }
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      if (ut[c] == uh[d] || ut[c] == un[d] || ut[c] == s[d] || ut[c] == p || ut[c] == C)
        return set_error(NN4_EINVAL, "ut must not alias an input");
      if (uh_next && (uh_next[c] == uh[d] || uh_next[c] == un[d] || uh_next[c] == ut[d] || uh_next[c] == s[d] ||
                      uh_next[c] == p || uh_next[c] == C))
        return set_error(NN4_EINVAL, "uh_next must not alias an input or ut");
    }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (fp->compute == NN4_F32) return predict_launch<float>(g, fp, C, un, uh, ut, uh_next, p, s, workspace, st);
  return predict_launch<double>(g, fp, C, un, uh, ut, uh_next, p, s, workspace, st);
}

int nn4_mass_sum(const nn4_grid* g, const double* C, double* out, void* stream) {
  int rc;
  if ((rc = validate_grid(g, NN4_F64, 2)) || (rc = validate_ptr(C, "C"))) return rc;
  if (!out) return set_error(NN4_EINVAL, "out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = check_cuda(cudaMemsetAsync(out, 0, sizeof(double), s), "zero mass"))) return rc;
  const long long rows = (long long)g->n[1] * g->n[2];
  const long long want = (rows + 7) / 8;  // 8 warps per block
  const int blocks = (int)resident_grid((const void*)k_mass, 256, 0, want);
  k_mass<<<blocks, 256, 0, s>>>(g->n[0], g->n[1], g->n[2], g->pitch, g->h[0] * g->h[1] * g->h[2], C, out);
  return check_cuda(cudaGetLastError(), "mass sum");
}

}  // extern "C"
