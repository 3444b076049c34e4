// Shared machinery of the Q1 27-point stencil passes (one tile of one pass): apply, residual
// (+ FP64 norm), weighted Jacobi, matrix-vector product, and residual + restriction, for the
// constant-coefficient operator and for the variable-coefficient identity of Eq. k-T
// (Section 2.2.4).  Included by the translation units that instantiate passes; everything is
// in an anonymous namespace, so each unit has its own copies (and its own device error word).
//
// Design (one kernel template for every pass):
//   * a CTA owns an x-y tile of 32 x (TYT*RY) output nodes and marches along z over `zchunk`
//     output planes; every input plane (with a one-node halo in x and y) is brought into shared
//     memory by a 3D TMA tile load, `stages` planes in flight, each stage guarded by an mbarrier;
//   * natural faces: the assembled boundary row equals the interior stencil on the field
//     mirrored about the boundary node, scaled by w = prod_d (s_d / 2), s_d the number of
//     elements next to the node along axis d.  Mirrored planes are fetched by mirrored TMA z
//     coordinates; in-plane neighbours by mirrored shared-memory indices;
//   * the interior stencil is sum-factorised by neighbour class: per input row the centre value
//     r0 and the sum of the two x-neighbours r1; per plane p00 = r0, p10 = r1 and the y-neighbour
//     sums p01, p11 of those; across planes the z-neighbour sums.  Output k then needs
//     u(k-1) + v(k) + u(k+1) with u = sum c_ab1 p_ab and v = sum c_ab0 p_ab, kept as two running
//     partial sums in registers (about 14 operations per node and field);
//   * residual + restriction (OP_RESIDUAL_RESTRICT): the tile is shifted one node down in x, y and
//     z and overlaps its neighbours, so that it holds the 2m+1 fine residuals around each of its
//     m coarse nodes per axis; each fine residual plane goes to shared memory, is restricted in
//     x and y there, and the z weights (1/2, 1, 1/2) fold into one running sum per coarse node as
//     the CTA marches along z.  Only the coarse residual and the norm leave the CTA.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace nn4 {
namespace {

template <typename T>
constexpr int kAlign = 16 / (int)sizeof(T);  // TMA x coordinates must be multiples of this

__device__ __forceinline__ float half_count(int i, int n) {
  return 0.5f * (float)((i > 0) + (i < n - 1));
}

__device__ __forceinline__ bool on_dirichlet(const LevelGeom& g, int i, int j, int k) {
  return (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
         (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
}

// Per-field running sums of one thread's RY outputs.
template <typename A, int RY>
struct Runner {
  A p1[RY];  // partial of the output at the previous plane (u(p-1) + v(p))
  A p2[RY];  // partial of the output at the current plane (u(p))
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < RY; ++r) p1[r] = p2[r] = A(0);
  }
};

// v is returned already added to `base` (the running partial of the same output), so the class
// sum and the running sum fold into FMAs.
template <typename T, typename A, int RY, bool PROD, bool ISO>
__device__ __forceinline__ void plane_uv(const T* __restrict__ sx, const T* __restrict__ sk,
                                         const int* rowoff, int cc, int cl, int cr, const A* c,
                                         const A* base, A* u, A* v, A* centre) {
  // Row sums r0 (centre) and r1 (x-neighbours) for the RY+2 rows the thread touches.
  A r0[RY + 2], r1[RY + 2];
#pragma unroll
  for (int q = 0; q < RY + 2; ++q) {
    const int o = rowoff[q];
    if (PROD) {
      r0[q] = to_acc(sx[o + cc]) * to_acc(sk[o + cc]);
      r1[q] = to_acc(sx[o + cl]) * to_acc(sk[o + cl]) + to_acc(sx[o + cr]) * to_acc(sk[o + cr]);
    } else {
      r0[q] = to_acc(sx[o + cc]);
      r1[q] = to_acc(sx[o + cl]) + to_acc(sx[o + cr]);
    }
  }
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const A p00 = r0[r + 1], p10 = r1[r + 1];
    const A p01 = r0[r] + r0[r + 2], p11 = r1[r] + r1[r + 2];
    if (ISO) {  // equal spacings: the face classes c[1], c[2], c[4] vanish
      v[r] = fma(c[0], p00, fma(c[3], p11, base[r]));
      u[r] = c[5] * p10 + c[6] * p01 + c[7] * p11;
    } else {
      v[r] = fma(c[0], p00, fma(c[1], p10, fma(c[2], p01, fma(c[3], p11, base[r]))));
      u[r] = c[4] * p00 + c[5] * p10 + c[6] * p01 + c[7] * p11;
    }
    if (centre) centre[r] = p00;
  }
}

// VC: 0 constant coefficient; 1 Eq. k-T with L k on the fly; 2 Eq. k-T with (1/2) L k (and
// optionally the inverse diagonal) read pointwise.  The CTA covers TX = 32 WX columns and TY = TYT RY rows.
// Every pipeline stage holds the haloed tiles of input plane p (x, and k for Eq. k-T) and the
// pointwise tiles (b, L k, 1/diag) of output plane p - 1, all brought by TMA onto one mbarrier,
// so no global load sits on the critical path of a plane.
struct Maps {
  CUtensorMap x, k, b, lk, invd, dq, ec;
};

template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
struct PassLayout {
  using A = typename Acc<T>::type;
  static constexpr int AL = kAlign<T>;
  static constexpr int TX = 32 * WX, TY = TYT * RY;
  static constexpr int NF = VC ? 2 : 1;
  static constexpr bool HAS_B = OP != OP_APPLY;
  static constexpr bool RR = OP == OP_RESIDUAL_RESTRICT;
  static constexpr int BX = TX + 2 * AL, BY = TY + 2;  // haloed tile (x from an aligned column)
  static constexpr int HALO_BYTES = BX * BY * (int)sizeof(T);
  static constexpr int HALO_PAD = (HALO_BYTES + 127) / 128 * 128;
  // pointwise tiles: the shifted tile of OP_RESIDUAL_RESTRICT starts at an odd column, so its
  // pointwise tiles start at the aligned column below and are AL wider
  static constexpr int PX = RR ? TX + AL : TX;
  static constexpr int PT_BYTES = PX * TY * (int)sizeof(T);
  static constexpr int PT_PAD = (PT_BYTES + 127) / 128 * 128;
  static constexpr int NP = (HAS_B ? 1 : 0) + (VC == 2 ? 2 : 0);
  static constexpr int DQ_BYTES = TX * TY * 4;
  static constexpr int DQ_PAD = OP == OP_JACOBI ? (DQ_BYTES + 127) / 128 * 128 : 0;  // FP32 dq tile
  // OP_JACOBI: two coarse tiles (the coarse planes bracketing the fine input plane) for the fused
  // prolongation, TX/2 + 2 AL columns from x0/2 - AL and TY/2 + 2 rows from y0/2 - 1
  static constexpr int BXC = TX / 2 + 2 * AL, BYC = TY / 2 + 2;
  static constexpr int CT_BYTES = BXC * BYC * (int)sizeof(T);
  static constexpr int CT_PAD = OP == OP_JACOBI ? (CT_BYTES + 127) / 128 * 128 : 0;
  static constexpr int CT_OFF = NF * HALO_PAD + NP * PT_PAD + DQ_PAD;  // first coarse tile in a stage
  static constexpr int STAGE = NF * HALO_PAD + NP * PT_PAD + DQ_PAD + 2 * CT_PAD;
  // OP_RESIDUAL_RESTRICT: coarse nodes per tile along x and y (the fine tile holds 2 CX + 1 of the
  // TX columns it computes), and the fine residual plane in the compute type
  static constexpr int CX = TX / 2 - 1, CY = TY / 2 - 1;
  static constexpr int RB_OFF = S * STAGE + S * 8 + 32 * 8;
  static constexpr int RB_BYTES = RR ? TX * TY * (int)sizeof(A) : 0;
  static constexpr size_t SMEM = (size_t)RB_OFF + RB_BYTES;
  static_assert(!RR || CX * CY <= TX * TYT, "one coarse node per thread at most");
};

// One output tile (tbx, tby) x z-chunk tbz of a stencil pass.  `qb` counts the planes this CTA has
// consumed before (stage = (qb + q) % S, phase parity from (qb + q) / S), so a CTA can run several
// tiles in a row on the same barriers.  Returns false if a bounded wait gave up.
template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
__device__ __forceinline__ bool pass_tile(const Maps* mp, const PassArgs& a, int tbx, int tby, int tbz,
                                          unsigned& qb) {
  const Maps& maps = *mp;
  using Lay = PassLayout<T, OP, VC, ISO, WX, RY, TYT, S>;
  using A = typename Lay::A;
  constexpr int AL = Lay::AL, TX = Lay::TX, TY = Lay::TY, BX = Lay::BX, BY = Lay::BY, NF = Lay::NF;
  constexpr int PX = Lay::PX, NP = Lay::NP, HALO_BYTES = Lay::HALO_BYTES, HALO_PAD = Lay::HALO_PAD;
  constexpr int PT_BYTES = Lay::PT_BYTES, PT_PAD = Lay::PT_PAD, DQ_BYTES = Lay::DQ_BYTES;
  constexpr int BXC = Lay::BXC, CT_BYTES = Lay::CT_BYTES, CT_PAD = Lay::CT_PAD, CT_OFF = Lay::CT_OFF;
  constexpr int STAGE = Lay::STAGE;
  constexpr bool HAS_B = Lay::HAS_B, RR = Lay::RR;
  constexpr bool KX_PLANE = VC == 2 && sizeof(T) == 8;  // k x formed once per plane (FP64 passes)
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * STAGE);
  double* red = reinterpret_cast<double*>(bars + S);
  const unsigned q0 = qb;

  const LevelGeom& g = a.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  // Output origin (x0, y0) and planes zs .. ze-1.  OP_RESIDUAL_RESTRICT: tile (tbx, tby, tbz) holds
  // coarse nodes I0 .. I0+CX-1 (J, K likewise, K over zchunk coarse planes) and computes the fine
  // residual from node 2 I0 - 1 on (one node below the first coarse node's fine position).
  const int x0 = RR ? 2 * tbx * Lay::CX - 1 : tbx * TX;
  const int y0 = RR ? 2 * tby * Lay::CY - 1 : tby * TY;
  const int K0 = tbz * a.zchunk;  // first coarse plane (OP_RESIDUAL_RESTRICT)
  const int zs = RR ? 2 * K0 - 1 : tbz * a.zchunk;
  const int ze = RR ? 2 * min(K0 + a.zchunk, (nz + 1) / 2) : min(nz, zs + a.zchunk);
  // first column of the haloed tile and of the pointwise tiles (TMA x coordinates: multiples of AL)
  const int xl = RR ? ((x0 - 1) & ~(AL - 1)) : x0 - AL;
  const int xp = RR ? (x0 & ~(AL - 1)) : x0;
  const int tid = threadIdx.x + TX * threadIdx.y;
  const int nplanes = ze - zs + 2;  // input planes zs-1 .. ze
  const bool use_invd = VC == 2 && OP == OP_JACOBI && a.invd != nullptr;
  const bool use_dq = OP == OP_JACOBI && a.dq != nullptr;
  const bool use_prol = OP == OP_JACOBI && a.ec != nullptr;  // x = P ec built in shared memory
  const int pt_loads = (HAS_B ? 1 : 0) + (VC == 2 ? 1 : 0) + (use_invd ? 1 : 0);

  if (tid == 0) {
    prefetch_tmap(&maps.x);
    if (VC) prefetch_tmap(&maps.k);
    if (HAS_B) prefetch_tmap(&maps.b);
  }

  auto issue = [&](int q) {
    const int s = (q0 + q) % S;
    unsigned char* st = smem + s * STAGE;
    const int zp = mirror(zs - 1 + q, nz);
    const int kout = zs + q - 2;
    const bool pt = q >= 2;
    mbar_expect_tx(&bars[s], (use_prol ? (NF - 1) * HALO_BYTES + 2 * CT_BYTES : NF * HALO_BYTES) +
                                 (pt ? pt_loads * PT_BYTES + (use_dq ? DQ_BYTES : 0) : 0));
    if (use_prol) {
      // coarse planes zp/2 and (zp+1)/2 (the same plane for an even zp)
      tma_load_3d(st + CT_OFF, &maps.ec, x0 / 2 - AL, y0 / 2 - 1, zp >> 1, &bars[s]);
      tma_load_3d(st + CT_OFF + CT_PAD, &maps.ec, x0 / 2 - AL, y0 / 2 - 1, (zp + 1) >> 1, &bars[s]);
    } else {
      tma_load_3d(st, &maps.x, xl, y0 - 1, zp, &bars[s]);
    }
    if (VC) tma_load_3d(st + HALO_PAD, &maps.k, xl, y0 - 1, zp, &bars[s]);
    if (pt) {
      unsigned char* pp = st + NF * HALO_PAD;
      if (HAS_B) {
        tma_load_3d(pp, &maps.b, xp, y0, kout, &bars[s]);
        pp += PT_PAD;
      }
      if (VC == 2) {
        tma_load_3d(pp, &maps.lk, xp, y0, kout, &bars[s]);
        if (use_invd) tma_load_3d(pp + PT_PAD, &maps.invd, xp, y0, kout, &bars[s]);
      }
      if (use_dq) tma_load_3d(st + NF * HALO_PAD + NP * PT_PAD, &maps.dq, x0, y0, kout, &bars[s]);
    }
  };
  if (tid == 0) {
    for (int q = 0; q < min(S, nplanes); ++q) issue(q);
  }

  // Column indices in the tile (clamped so that idle lanes read valid shared memory).
  const int i = x0 + threadIdx.x;
  const int ic = max(min(i, nx - 1), 0);
  const int cc = ic - xl;
  const int cl = mirror(ic - 1, nx) - xl;
  const int cr = mirror(ic + 1, nx) - xl;
  const int jb = y0 + threadIdx.y * RY;
  int rowoff[RY + 2];
#pragma unroll
  for (int q = 0; q < RY + 2; ++q) {
    int jm = mirror(jb - 1 + q, ny);
    jm = min(max(jm, y0 - 1), y0 + BY - 2);
    rowoff[q] = (jm - (y0 - 1)) * BX;
  }

  A c[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) c[t] = (A)a.L.c[t];
  const A wx = (A)half_count(ic, nx);
  A wy[RY], hwy[RY];  // boundary weight of each row (x and y factors) and half of it
  unsigned dmask = 0;  // bit r: output row r lies on a Dirichlet face of x or y
#pragma unroll
  for (int r = 0; r < RY; ++r) {
    const int j = min(jb + r, ny - 1);
    wy[r] = wx * (A)half_count(j, ny);
    hwy[r] = (A)0.5 * wy[r];
    const bool d = (g.dir[0] && i == 0) || (g.dir[1] && i == nx - 1) || (g.dir[2] && j == 0) || (g.dir[3] && j == ny - 1);
    dmask |= (d ? 1u : 0u) << r;
  }

  Runner<A, RY> sx, skx, sk;  // L~x, L~(kx), L~k
  sx.zero();
  if (VC) {
    skx.zero();
    sk.zero();
  }
  A xc1[RY], kc1[RY];  // centre values of the previous input plane (the pending output)
  // norm and dot partial sums in the compute type for the whole z-march (FP32 for FP32 and BF16
  // storage: the FP64 pipe of this part is narrow), FP64 across threads
  A nrm = A(0), dt2 = A(0), dqs = A(0);
  const A omega = opaque((A)a.omega);
  bool failed = false;
  T* out = reinterpret_cast<T*>(a.out);
  A* const rb = reinterpret_cast<A*>(smem + Lay::RB_OFF);  // OP_RESIDUAL_RESTRICT: fine residual plane
  A racc = A(0);  // OP_RESIDUAL_RESTRICT: running z sum of this thread's coarse node

  for (int q = 0; q < nplanes; ++q) {
    const int s = (q0 + q) % S;
    if (!mbar_wait_bounded(&bars[s], (uint32_t)(((q0 + q) / S) & 1))) failed = true;
    const unsigned char* st = smem + s * STAGE;
    const T* tx_ = reinterpret_cast<const T*>(st);
    const T* tk_ = reinterpret_cast<const T*>(st + HALO_PAD);
    const T* tb_ = reinterpret_cast<const T*>(st + NF * HALO_PAD);
    const T* tl_ = reinterpret_cast<const T*>(st + NF * HALO_PAD + (HAS_B ? PT_PAD : 0));
    const T* ti_ = tl_ + PT_PAD / sizeof(T);
    const float* tq_ = reinterpret_cast<const float*>(st + NF * HALO_PAD + NP * PT_PAD);
    if (use_prol) {
      // x tile = P ec on the fine columns x0-1 .. x0+TX and rows y0-1 .. y0+TY inside the grid (the
      // only ones read: mirrored indices stay in the grid), in the prolongation kernel's order of
      // operations (y, then x, then z) and rounded to the storage type as it stores; 0 at Dirichlet
      // nodes.  The x region of the stage is not a copy target in this mode.
      const int zp = mirror(zs - 1 + q, nz);
      const bool zodd = zp & 1;
      const bool dzf = (g.dir[4] && zp == 0) || (g.dir[5] && zp == nz - 1);
      const T* c0 = reinterpret_cast<const T*>(st + CT_OFF);
      const T* c1 = reinterpret_cast<const T*>(st + CT_OFF + CT_PAD);
      T* xt = reinterpret_cast<T*>(smem + s * STAGE);
      constexpr int FW = TX + 2, FH = TY + 2;
      for (int e = tid; e < FW * FH; e += TX * TYT) {
        const int fy = y0 - 1 + e / FW, fx = x0 - 1 + e % FW;
        if (fx < 0 || fx >= nx || fy < 0 || fy >= ny) continue;
        const int cx = (fx >> 1) - (x0 / 2 - AL), cy = (fy >> 1) - (y0 / 2 - 1);
        const int ox = fx & 1, oy = fy & 1;
        auto xy = [&](const T* cp) -> A {
          const T* r0 = cp + cy * BXC + cx;
          const T* r1 = r0 + oy * BXC;
          const A av = A(0.5) * (to_acc(r0[0]) + to_acc(r1[0]));
          if (!ox) return av;
          const A an = A(0.5) * (to_acc(r0[1]) + to_acc(r1[1]));
          return A(0.5) * (av + an);
        };
        A t = xy(c0);
        if (zodd) t = A(0.5) * (t + xy(c1));
        const bool dn = dzf || (g.dir[0] && fx == 0) || (g.dir[1] && fx == nx - 1) || (g.dir[2] && fy == 0) ||
                        (g.dir[3] && fy == ny - 1);
        xt[(fy - (y0 - 1)) * BX + (fx - (x0 - AL))] = from_acc<T>(dn ? A(0) : t);
      }
      __syncthreads();
    }
    A ux[RY], vx[RY], xcn[RY];
    plane_uv<T, A, RY, false, ISO>(tx_, tx_, rowoff, cc, cl, cr, c, sx.p2, ux, vx, xcn);
    A ukx[RY], vkx[RY], uk[RY], vk[RY], kcn[RY];
    if constexpr (KX_PLANE) {
      // FP64 with (1/2) L k stored: every k x product of the haloed plane is formed once (instead
      // of once per thread that reads it, about three times) into the k tile, which holds nothing
      // else this plane needs once each thread has its centre values of k
#pragma unroll
      for (int r = 0; r < RY; ++r) kcn[r] = to_acc(tk_[rowoff[r + 1] + cc]);
      __syncthreads();
      T* const kx_ = const_cast<T*>(tk_);
      for (int e = tid; e < BX * BY; e += TX * TYT) kx_[e] = tx_[e] * kx_[e];
      __syncthreads();
      plane_uv<T, A, RY, false, ISO>(tk_, tk_, rowoff, cc, cl, cr, c, skx.p2, ukx, vkx, nullptr);
    } else {
      if (VC) plane_uv<T, A, RY, true, ISO>(tx_, tk_, rowoff, cc, cl, cr, c, skx.p2, ukx, vkx, nullptr);
      if (VC == 1) plane_uv<T, A, RY, false, ISO>(tk_, tk_, rowoff, cc, cl, cr, c, sk.p2, uk, vk, kcn);
      if (VC == 2) {
#pragma unroll
        for (int r = 0; r < RY; ++r) kcn[r] = to_acc(tk_[rowoff[r + 1] + cc]);
      }
    }

    const int kout = zs + q - 2;  // output plane completed by this input plane
    if (q >= 2 && !failed) {
      A pn = A(0), pd = A(0);
      const A wz = (A)half_count(kout, nz);
      const bool dz = (g.dir[4] && kout == 0) || (g.dir[5] && kout == nz - 1);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const int j = jb + r;
        if (RR || (i < nx && j < ny)) {
          const A w = wy[r] * wz;
          const A Lx = sx.p1[r] + ux[r];
          const int po = (j - y0) * PX + (i - xp);  // pointwise tile offset
          A Ax, D;
          if (VC == 1) {
            const A Lkx = skx.p1[r] + ukx[r];
            const A Lk = sk.p1[r] + uk[r];
            Ax = (A)0.5 * w * (Lkx + kc1[r] * Lx - xc1[r] * Lk);
            D = w * (c[0] * kc1[r] - (A)0.5 * Lk);
          } else if (VC == 2) {
            const A Lkx = skx.p1[r] + ukx[r];
            const A hLk = to_acc(tl_[po]);  // (1/2) L k as stored, w included
            Ax = fma(hwy[r] * wz, fma(kc1[r], Lx, Lkx), -xc1[r] * hLk);
            D = w * c[0] * kc1[r] - hLk;
          } else {
            Ax = w * Lx;
            D = w * c[0];
          }
          const long long idx = (long long)i + g.pitch * ((long long)j + (long long)ny * kout);
          if (OP == OP_APPLY) {
            out[idx] = from_acc<T>(Ax);
          } else {
            const bool dirn = dz || ((dmask >> r) & 1u);
            const A bv = to_acc(tb_[po]);
            if constexpr (RR) {
              // every node of the tile gets a value: 0 outside the grid (the restriction weights
              // of nodes that do not exist) and at Dirichlet nodes
              const bool in = i >= 0 && i < nx && j >= 0 && j < ny && kout >= 0 && kout < nz;
              const A rv = (dirn || !in) ? A(0) : bv - Ax;
              rb[(j - y0) * TX + (i - x0)] = rv;
              // the norm counts the nodes this tile owns: its first TX-2 columns and TY-2 rows and
              // every plane but its last (the next z-chunk's first), which partitions the grid
              if (i - x0 < TX - 2 && j - y0 < TY - 2 && kout < ze - 1) pn += rv * rv;
            } else if (OP == OP_RESIDUAL) {
              const A rv = dirn ? A(0) : bv - Ax;
              out[idx] = from_acc<T>(rv);
              pn += rv * rv;
            } else if (OP == OP_MATVEC) {
              const A qv = dirn ? A(0) : Ax;
              out[idx] = from_acc<T>(qv);
              pn += xc1[r] * qv;
              pd += xc1[r] * bv;
            } else {
              A corr;
              if (use_invd)
                corr = (bv - Ax) * to_acc(ti_[po]);
              else if constexpr (sizeof(A) == 4)
                corr = __fdividef(bv - Ax, D);
              else
                corr = (bv - Ax) / D;
              const A xn = dirn ? xc1[r] : xc1[r] + omega * corr;
              const T xs = from_acc<T>(xn);
              out[idx] = xs;
              if (use_dq) dqs += to_acc(xs) * (A)tq_[po];
            }
          }
        }
      }
      if (OP == OP_RESIDUAL || OP == OP_MATVEC || RR) nrm += pn;
      if (OP == OP_MATVEC) dt2 += pd;
    }
    if constexpr (RR) {
      if (q >= 2) {
        __syncthreads();  // the fine residual plane kout is complete in shared memory
        if (!failed && tid < Lay::CX * Lay::CY) {
          // restriction in x and y (weights 1/2, 1, 1/2 per axis) at the fine node (2I, 2J) of
          // plane kout; in z, plane 2K adds with weight 1 and the odd planes 2K-1, 2K+1 with 1/2
          const int ci = tid % Lay::CX, cj = tid / Lay::CX;
          const A* rr = rb + (2 * cj + 1) * TX + 2 * ci + 1;
          auto row = [&](const A* p) { return p[0] + A(0.5) * (p[-1] + p[1]); };
          const A sp = row(rr) + A(0.5) * (row(rr - TX) + row(rr + TX));
          if (kout & 1) {
            if (kout > zs) {  // coarse plane (kout-1)/2 is complete
              const LevelGeom& gc = a.gc;
              const int I = tbx * Lay::CX + ci, J = tby * Lay::CY + cj, K = (kout - 1) >> 1;
              if (I < gc.nx && J < gc.ny) {
                const bool dn = (gc.dir[0] && I == 0) || (gc.dir[1] && I == gc.nx - 1) || (gc.dir[2] && J == 0) ||
                                (gc.dir[3] && J == gc.ny - 1) || (gc.dir[4] && K == 0) ||
                                (gc.dir[5] && K == gc.nz - 1);
                out[(long long)I + gc.pitch * ((long long)J + (long long)gc.ny * K)] =
                    from_acc<T>(dn ? A(0) : racc + A(0.5) * sp);
              }
            }
            racc = A(0.5) * sp;
          } else {
            racc += sp;
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < RY; ++r) {
      // shift the running sums: the output of this plane still needs u of the next plane
      sx.p1[r] = vx[r];
      sx.p2[r] = ux[r];
      xc1[r] = xcn[r];
      if (VC) {
        skx.p1[r] = vkx[r];
        skx.p2[r] = ukx[r];
        kc1[r] = kcn[r];
      }
      if (VC == 1) {
        sk.p1[r] = vk[r];
        sk.p2[r] = uk[r];
      }
    }
    // every thread is done with stage s: refill it with the plane S ahead
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    if (tid == 0 && q + S < nplanes) issue(q + S);
  }
  qb = q0 + nplanes;
  if (failed) {
    // drain copies that may still be in flight before the CTA exits
    if (tid == 0) {
      for (int q = 0; q < min(S, nplanes); ++q) mbar_wait_bounded(&bars[q], 0u);
    }
    __syncthreads();
    return false;
  }
  if ((OP == OP_RESIDUAL || OP == OP_MATVEC || RR) && a.norm2 != nullptr) block_sum_atomic((double)nrm, a.norm2, red);
  if (OP == OP_MATVEC && a.dot2 != nullptr) block_sum_atomic((double)dt2, a.dot2, red);
  if (use_dq) block_sum_atomic((double)dqs, a.dq_out, red);
  __syncthreads();  // stage buffers are free for the next tile
  return true;
}

template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
__device__ __forceinline__ void init_bars() {
  using Lay = PassLayout<T, OP, VC, ISO, WX, RY, TYT, S>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * Lay::STAGE);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
}

template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
__global__ void __launch_bounds__(32 * WX * TYT) k_pass(const __grid_constant__ Maps maps, const PassArgs a) {
  init_bars<T, OP, VC, ISO, WX, RY, TYT, S>();
  unsigned qb = 0;
  pass_tile<T, OP, VC, ISO, WX, RY, TYT, S>(&maps, a, blockIdx.x, blockIdx.y, blockIdx.z, qb);
}

// Batched form: one launch over the tiles of many independent instances.  Item t of instance i
// is tile (t % tiles_x, (t / tiles_x) % tiles_y, t / (tiles_x tiles_y)); CTAs stride over all
// items (persistent), skipping instances whose `active` flag is 0.
template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
__global__ void __launch_bounds__(32 * WX * TYT)
    k_pass_batch(const BatchPass* __restrict__ items, int count, int total, const int* __restrict__ active) {
  init_bars<T, OP, VC, ISO, WX, RY, TYT, S>();
  unsigned qb = 0;
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    int lo = 0, hi = count - 1;  // last instance whose first item is <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].first <= it) lo = mid;
      else hi = mid - 1;
    }
    const BatchPass& bp = items[lo];
    if (active && !active[bp.inst]) continue;
    const int t = it - bp.first;
    if (!pass_tile<T, OP, VC, ISO, WX, RY, TYT, S>(reinterpret_cast<const Maps*>(&bp.maps), bp.args,
                                                   t % bp.tiles_x, (t / bp.tiles_x) % bp.tiles_y,
                                                   t / (bp.tiles_x * bp.tiles_y), qb))
      return;
  }
}

}  // namespace
}  // namespace nn4
