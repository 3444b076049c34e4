// Q1 27-point stencil passes: apply, residual (+ FP64 norm) and weighted Jacobi, for the
// constant-coefficient operator and for the variable-coefficient identity of Eq. k-T
// (Section 2.2.4).
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
//     partial sums in registers (about 14 operations per node and field).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace nn4 {

NN4_DEFINE_ERROR_ACCESSOR(stencil_error_word)

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
  static constexpr int AL = kAlign<T>;
  static constexpr int TX = 32 * WX, TY = TYT * RY;
  static constexpr int NF = VC ? 2 : 1;
  static constexpr bool HAS_B = OP != OP_APPLY;
  static constexpr int HALO_PAD = ((TX + 2 * AL) * (TY + 2) * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int PT_PAD = (TX * TY * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int NP = (HAS_B ? 1 : 0) + (VC == 2 ? 2 : 0);
  static constexpr int DQ_PAD = OP == OP_JACOBI ? (TX * TY * 4 + 127) / 128 * 128 : 0;  // FP32 dq tile
  // OP_JACOBI: two coarse tiles (the coarse planes bracketing the fine input plane) for the fused
  // prolongation, TX/2 + 2 AL columns from x0/2 - AL and TY/2 + 2 rows from y0/2 - 1
  static constexpr int BXC = TX / 2 + 2 * AL, BYC = TY / 2 + 2;
  static constexpr int CT_PAD = OP == OP_JACOBI ? (BXC * BYC * (int)sizeof(T) + 127) / 128 * 128 : 0;
  static constexpr int STAGE = NF * HALO_PAD + NP * PT_PAD + DQ_PAD + 2 * CT_PAD;
  static constexpr size_t SMEM = (size_t)S * STAGE + S * 8 + 32 * 8;
};

// One output tile (tbx, tby) x z-chunk tbz of a stencil pass.  `qb` counts the planes this CTA has
// consumed before (stage = (qb + q) % S, phase parity from (qb + q) / S), so a CTA can run several
// tiles in a row on the same barriers.  Returns false if a bounded wait gave up.
template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
__device__ __forceinline__ bool pass_tile(const Maps* mp, const PassArgs& a, int tbx, int tby, int tbz,
                                          unsigned& qb) {
  const Maps& maps = *mp;
  using A = typename Acc<T>::type;
  constexpr int AL = kAlign<T>;
  constexpr int TX = 32 * WX, TY = TYT * RY;
  constexpr int BX = TX + 2 * AL;
  constexpr int BY = TY + 2;
  constexpr int NF = VC ? 2 : 1;
  constexpr bool HAS_B = OP != OP_APPLY;
  constexpr int HALO_BYTES = BX * BY * (int)sizeof(T);
  constexpr int HALO_PAD = (HALO_BYTES + 127) / 128 * 128;
  constexpr int PT_BYTES = TX * TY * (int)sizeof(T);
  constexpr int PT_PAD = (PT_BYTES + 127) / 128 * 128;
  constexpr int NP = (HAS_B ? 1 : 0) + (VC == 2 ? 2 : 0);  // pointwise slots per stage
  constexpr int DQ_BYTES = TX * TY * 4;
  constexpr int DQ_PAD = OP == OP_JACOBI ? (DQ_BYTES + 127) / 128 * 128 : 0;
  constexpr int BXC = TX / 2 + 2 * AL, BYC = TY / 2 + 2;
  constexpr int CT_BYTES = BXC * BYC * (int)sizeof(T);
  constexpr int CT_PAD = OP == OP_JACOBI ? (CT_BYTES + 127) / 128 * 128 : 0;
  constexpr int CT_OFF = NF * HALO_PAD + NP * PT_PAD + DQ_PAD;  // first coarse tile in a stage
  constexpr int STAGE = NF * HALO_PAD + NP * PT_PAD + DQ_PAD + 2 * CT_PAD;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * STAGE);
  double* red = reinterpret_cast<double*>(bars + S);
  const unsigned q0 = qb;

  const LevelGeom& g = a.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int x0 = tbx * TX, y0 = tby * TY;
  const int zs = tbz * a.zchunk;
  const int ze = min(nz, zs + a.zchunk);
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
      tma_load_3d(st, &maps.x, x0 - AL, y0 - 1, zp, &bars[s]);
    }
    if (VC) tma_load_3d(st + HALO_PAD, &maps.k, x0 - AL, y0 - 1, zp, &bars[s]);
    if (pt) {
      unsigned char* pp = st + NF * HALO_PAD;
      if (HAS_B) {
        tma_load_3d(pp, &maps.b, x0, y0, kout, &bars[s]);
        pp += PT_PAD;
      }
      if (VC == 2) {
        tma_load_3d(pp, &maps.lk, x0, y0, kout, &bars[s]);
        if (use_invd) tma_load_3d(pp + PT_PAD, &maps.invd, x0, y0, kout, &bars[s]);
      }
      if (use_dq) tma_load_3d(st + NF * HALO_PAD + NP * PT_PAD, &maps.dq, x0, y0, kout, &bars[s]);
    }
  };
  if (tid == 0) {
    for (int q = 0; q < min(S, nplanes); ++q) issue(q);
  }

  // Column indices in the tile (clamped so that idle lanes read valid shared memory).
  const int i = x0 + threadIdx.x;
  const int ic = min(i, nx - 1);
  const int cc = ic - (x0 - AL);
  const int cl = mirror(ic - 1, nx) - (x0 - AL);
  const int cr = mirror(ic + 1, nx) - (x0 - AL);
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
    if (VC) plane_uv<T, A, RY, true, ISO>(tx_, tk_, rowoff, cc, cl, cr, c, skx.p2, ukx, vkx, nullptr);
    if (VC == 1) plane_uv<T, A, RY, false, ISO>(tk_, tk_, rowoff, cc, cl, cr, c, sk.p2, uk, vk, kcn);
    if (VC == 2) {
#pragma unroll
      for (int r = 0; r < RY; ++r) kcn[r] = to_acc(tk_[rowoff[r + 1] + cc]);
    }

    const int kout = zs + q - 2;  // output plane completed by this input plane
    if (q >= 2 && !failed) {
      A pn = A(0), pd = A(0);
      const A wz = (A)half_count(kout, nz);
      const bool dz = (g.dir[4] && kout == 0) || (g.dir[5] && kout == nz - 1);
#pragma unroll
      for (int r = 0; r < RY; ++r) {
        const int j = jb + r;
        if (i < nx && j < ny) {
          const A w = wy[r] * wz;
          const A Lx = sx.p1[r] + ux[r];
          const int po = (j - y0) * TX + (i - x0);  // pointwise tile offset
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
            if (OP == OP_RESIDUAL) {
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
      if (OP == OP_RESIDUAL || OP == OP_MATVEC) nrm += pn;
      if (OP == OP_MATVEC) dt2 += pd;
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
  if ((OP == OP_RESIDUAL || OP == OP_MATVEC) && a.norm2 != nullptr) block_sum_atomic((double)nrm, a.norm2, red);
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

template <typename T, int OP, int VC, bool ISO, int WX, int RY, int TYT, int S>
int launch_t(const PassArgs& a, const Maps& maps, cudaStream_t st) {
  constexpr int TX = 32 * WX, TY = TYT * RY;
  const size_t smem = PassLayout<T, OP, VC, ISO, WX, RY, TYT, S>::SMEM;
  auto kern = k_pass<T, OP, VC, ISO, WX, RY, TYT, S>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(stencil pass)");
  }
  dim3 grid((a.g.nx + TX - 1) / TX, (a.g.ny + TY - 1) / TY, (a.g.nz + a.zchunk - 1) / a.zchunk);
  kern<<<grid, dim3(TX, TYT), smem, st>>>(maps, a);
  return check_cuda(cudaGetLastError(), "stencil pass launch");
}

// The configurations the autotuner chooses from: {WX, RY, TYT, S}.
// The last ({1, 8, 2, 3}: eight rows a thread) is compiled for FP64 only, whose passes are bound by
// the FP64 pipe and gain from the fewer loads per output; for the other types it is refused and
// the autotuner skips it.
constexpr int kCfgs[][4] = {{1, 4, 4, 3}, {2, 2, 4, 4}, {1, 2, 8, 3}, {2, 4, 2, 4}, {1, 8, 2, 3}};
constexpr int kNumCfgs = 5;

template <typename T, int OP, int VC, bool ISO>
int dispatch_cfg(const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  for (int c = 0; c < kNumCfgs; ++c)
    if (cfg.wx == kCfgs[c][0] && cfg.ry == kCfgs[c][1] && cfg.tyt == kCfgs[c][2] && cfg.stages == kCfgs[c][3]) {
      switch (c) {
        case 0: return launch_t<T, OP, VC, ISO, 1, 4, 4, 3>(a, m, st);
        case 1: return launch_t<T, OP, VC, ISO, 2, 2, 4, 4>(a, m, st);
        case 2: return launch_t<T, OP, VC, ISO, 1, 2, 8, 3>(a, m, st);
        case 3: return launch_t<T, OP, VC, ISO, 2, 4, 2, 4>(a, m, st);
        case 4:
          if constexpr (sizeof(T) == 8) return launch_t<T, OP, VC, ISO, 1, 8, 2, 3>(a, m, st);
          break;
      }
    }
  return set_error(NN4_EINVAL, "unsupported stencil pass configuration");
}

template <typename T, int OP, int VC>
int dispatch_iso(bool iso, const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  return iso ? dispatch_cfg<T, OP, VC, true>(a, cfg, m, st) : dispatch_cfg<T, OP, VC, false>(a, cfg, m, st);
}

template <typename T, int OP>
int dispatch_vc(int vc, bool iso, const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  if (vc == 0) return dispatch_iso<T, OP, 0>(iso, a, cfg, m, st);
  if (vc == 1) return dispatch_iso<T, OP, 1>(iso, a, cfg, m, st);
  return dispatch_iso<T, OP, 2>(iso, a, cfg, m, st);
}

template <typename T>
int dispatch_op(int op, int vc, const PassArgs& a, const PassCfg& cfg, const Maps& m, cudaStream_t st) {
  const bool iso = a.L.c[1] == 0.0 && a.L.c[2] == 0.0 && a.L.c[4] == 0.0;
  switch (op) {
    case OP_APPLY: return dispatch_vc<T, OP_APPLY>(vc, iso, a, cfg, m, st);
    case OP_RESIDUAL: return dispatch_vc<T, OP_RESIDUAL>(vc, iso, a, cfg, m, st);
    case OP_JACOBI: return dispatch_vc<T, OP_JACOBI>(vc, iso, a, cfg, m, st);
    case OP_MATVEC: return dispatch_vc<T, OP_MATVEC>(vc, iso, a, cfg, m, st);
  }
  return set_error(NN4_EINVAL, "bad stencil op");
}

template <typename T, int OP, bool ISO>
int launch_batch_t(const BatchPass* items, int count, int total, const int* active, cudaStream_t st) {
  using Lay = PassLayout<T, OP, 0, ISO, 1, 4, 4, 3>;
  auto kern = k_pass_batch<T, OP, 0, ISO, 1, 4, 4, 3>;
  const size_t smem = Lay::SMEM;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return check_cuda(e, "cudaFuncSetAttribute(batched pass)");
  }
  const int grid = std::min(total, 152 * 8);
  kern<<<grid, dim3(32, 4), smem, st>>>(items, count, total, active);
  return check_cuda(cudaGetLastError(), "batched stencil pass launch");
}

}  // namespace

PassCfg batch_pass_cfg(nn4_dtype dt) {
  PassCfg c;
  c.wx = 1;
  c.ry = 4;
  c.tyt = 4;
  c.stages = 3;
  c.zchunk = 0;
  return c;
}

int batch_pass_tiles(nn4_dtype, BatchPass* bp) {
  const LevelGeom& g = bp->args.g;
  bp->tiles_x = (g.nx + 31) / 32;
  bp->tiles_y = (g.ny + 15) / 16;
  const int tz = (g.nz + bp->args.zchunk - 1) / bp->args.zchunk;
  return bp->tiles_x * bp->tiles_y * tz;
}

int launch_pass_batch(nn4_dtype dt, int op, const BatchPass* items, int count, int total, const int* active,
                      cudaStream_t s) {
  if (total <= 0) return NN4_OK;
  // every instance of a batch has equal spacing per axis (checked at batch creation)
  switch (dt * 4 + op) {
    case NN4_F64 * 4 + OP_RESIDUAL: return launch_batch_t<double, OP_RESIDUAL, true>(items, count, total, active, s);
    case NN4_F64 * 4 + OP_JACOBI: return launch_batch_t<double, OP_JACOBI, true>(items, count, total, active, s);
    case NN4_F32 * 4 + OP_RESIDUAL: return launch_batch_t<float, OP_RESIDUAL, true>(items, count, total, active, s);
    case NN4_F32 * 4 + OP_JACOBI: return launch_batch_t<float, OP_JACOBI, true>(items, count, total, active, s);
    case NN4_BF16 * 4 + OP_RESIDUAL: return launch_batch_t<bf16, OP_RESIDUAL, true>(items, count, total, active, s);
    case NN4_BF16 * 4 + OP_JACOBI: return launch_batch_t<bf16, OP_JACOBI, true>(items, count, total, active, s);
  }
  return set_error(NN4_EINVAL, "unsupported batched pass");
}

PassCfg default_pass_cfg(nn4_dtype dt, bool vc, const LevelGeom& g) {
  PassCfg c;
  c.wx = 1;
  c.ry = (dt == NN4_F64 && vc) ? 2 : 4;
  c.tyt = (dt == NN4_F64 && vc) ? 8 : 4;
  c.stages = 3;
  const int tiles = ((g.nx + 32 * c.wx - 1) / (32 * c.wx)) * ((g.ny + c.tyt * c.ry - 1) / (c.tyt * c.ry));
  // aim at >= ~1200 CTAs (8 per SM) but keep at least 8 output planes per CTA
  int zc = g.nz;
  while (zc > 8 && tiles * ((g.nz + zc - 1) / zc) < 1216) zc = (zc + 1) / 2;
  c.zchunk = zc;
  return c;
}

int num_pass_cfgs() { return kNumCfgs; }

PassCfg pass_cfg_candidate(int index, const LevelGeom& g, int zchunk) {
  PassCfg c;
  c.wx = kCfgs[index][0];
  c.ry = kCfgs[index][1];
  c.tyt = kCfgs[index][2];
  c.stages = kCfgs[index][3];
  c.zchunk = zchunk > 0 ? zchunk : g.nz;
  return c;
}

int pass_box(nn4_dtype dt, const PassCfg& cfg, int* box_x, int* box_y) {
  const int al = 16 / (int)dtype_size(dt);
  *box_x = 32 * cfg.wx + 2 * al;
  *box_y = cfg.tyt * cfg.ry + 2;
  return NN4_OK;
}

int pass_coarse_box(nn4_dtype dt, const PassCfg& cfg, int* box_x, int* box_y) {
  const int al = 16 / (int)dtype_size(dt);
  *box_x = 16 * cfg.wx + 2 * al;
  *box_y = cfg.tyt * cfg.ry / 2 + 2;
  return NN4_OK;
}

int pass_point_box(const PassCfg& cfg, int* box_x, int* box_y) {
  *box_x = 32 * cfg.wx;
  *box_y = cfg.tyt * cfg.ry;
  return NN4_OK;
}

bool make_pass_maps(PassMaps* m, nn4_dtype dt, const PassArgs& a, const PassCfg& cfg, const void* x, const void* k) {
  int bx, by, px, py;
  pass_box(dt, cfg, &bx, &by);
  pass_point_box(cfg, &px, &py);
  const LevelGeom& g = a.g;
  bool ok = make_tmap_3d(&m->x, dt, x, g.nx, g.ny, g.nz, g.pitch, bx, by);
  if (k) ok = ok && make_tmap_3d(&m->k, dt, k, g.nx, g.ny, g.nz, g.pitch, bx, by);
  if (a.b) ok = ok && make_tmap_3d(&m->b, dt, a.b, g.nx, g.ny, g.nz, g.pitch, px, py);
  if (a.lk) ok = ok && make_tmap_3d(&m->lk, dt, a.lk, g.nx, g.ny, g.nz, g.pitch, px, py);
  if (a.invd) ok = ok && make_tmap_3d(&m->invd, dt, a.invd, g.nx, g.ny, g.nz, g.pitch, px, py);
  if (a.dq) ok = ok && make_tmap_3d(&m->dq, NN4_F32, a.dq, g.nx, g.ny, g.nz, a.dq_pitch, px, py);
  if (a.ec) {
    int cx, cy;
    pass_coarse_box(dt, cfg, &cx, &cy);
    ok = ok && make_tmap_3d(&m->ec, dt, a.ec, a.gc.nx, a.gc.ny, a.gc.nz, a.gc.pitch, cx, cy);
  }
  return ok;
}

int launch_pass(nn4_dtype dt, int op, const PassArgs& a, const void* x, const void* k,
                const PassCfg& cfg, cudaStream_t s, const PassMaps* pm) {
  PassMaps local;
  const bool vc = k != nullptr;
  if (!pm) {
    if (!make_pass_maps(&local, dt, a, cfg, x, k)) return set_error(NN4_ECUDA, "cuTensorMapEncodeTiled failed");
    pm = &local;
  }
  Maps m;
  m.x = pm->x;
  m.k = vc ? pm->k : pm->x;
  m.b = a.b ? pm->b : pm->x;
  m.lk = a.lk ? pm->lk : pm->x;
  m.invd = a.invd ? pm->invd : pm->x;
  m.dq = a.dq ? pm->dq : pm->x;
  m.ec = a.ec ? pm->ec : pm->x;
  if (a.ec && op != OP_JACOBI) return set_error(NN4_EINVAL, "the fused prolongation needs OP_JACOBI");
  // (every compiled tile shape has an even height, so a tile's first row y0 sits on a coarse row)
  if (a.ec && (a.gc.nx != (a.g.nx + 1) / 2 || a.gc.ny != (a.g.ny + 1) / 2 || a.gc.nz != (a.g.nz + 1) / 2 ||
               !(a.g.nx & 1) || !(a.g.ny & 1) || !(a.g.nz & 1)))
    return set_error(NN4_EINVAL, "the fused prolongation needs the grid of every second node");
  if (a.dq && (op != OP_JACOBI || !a.dq_out)) return set_error(NN4_EINVAL, "the fused dot needs OP_JACOBI and an output");
  if (op != OP_APPLY && !a.b) return set_error(NN4_EINVAL, "stencil pass needs b");
  const int vmode = vc ? (a.lk ? 2 : 1) : 0;
  switch (dt) {
    case NN4_F64: return dispatch_op<double>(op, vmode, a, cfg, m, s);
    case NN4_F32: return dispatch_op<float>(op, vmode, a, cfg, m, s);
    case NN4_BF16: return dispatch_op<bf16>(op, vmode, a, cfg, m, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

}  // namespace nn4
