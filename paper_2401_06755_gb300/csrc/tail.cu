// The coarse tail of the sawtooth V-cycle in one launch.  Levels with few nodes cannot fill the
// GPU and every separate launch costs several microseconds of latency, so all levels at or below
// a few hundred nodes run in a single CTA: restriction down to the coarsest level, the dense
// coarsest solve, then prolongation and one Jacobi sweep per level back up to the entry level
// (Section 2.4, multigrid figure: the same steps the per-level kernels perform).
#include "common.cuh"
#include "internal.h"

namespace nn4 {

NN4_DEFINE_ERROR_ACCESSOR(tail_error_word)

namespace {

__device__ __forceinline__ bool tdir(const LevelGeom& g, int i, int j, int k) {
  return (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
         (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
}

__device__ __forceinline__ long long off(const LevelGeom& g, int i, int j, int k) {
  return i + g.pitch * ((long long)j + (long long)g.ny * k);
}

// Every step below walks its nodes as t = t0, t0 + st, ...: (threadIdx.x, blockDim.x) inside one
// CTA, (global thread, grid threads) in the cooperative form.
// Out-of-range fine neighbours (only past a boundary node) get weight 0 and a clamped index, so
// the 27 loads carry no branch and are all in flight together.
template <typename T>
__device__ void tail_restrict(const TailLevel& F, const TailLevel& C, int t0, int st) {
  using A = typename Acc<T>::type;
  const T* rf = static_cast<const T*>(F.r);
  T* rc = static_cast<T*>(C.r);
  const int n = C.g.nx * C.g.ny * C.g.nz;
  for (int t = t0; t < n; t += st) {
    const int I = t % C.g.nx, J = (t / C.g.nx) % C.g.ny, K = t / (C.g.nx * C.g.ny);
    const int ix[3] = {max(2 * I - 1, 0), 2 * I, min(2 * I + 1, F.g.nx - 1)};
    const int jy[3] = {max(2 * J - 1, 0), 2 * J, min(2 * J + 1, F.g.ny - 1)};
    const int kz[3] = {max(2 * K - 1, 0), 2 * K, min(2 * K + 1, F.g.nz - 1)};
    const A wx[3] = {I > 0 ? A(0.5) : A(0), A(1), 2 * I + 1 < F.g.nx ? A(0.5) : A(0)};
    const A wy[3] = {J > 0 ? A(0.5) : A(0), A(1), 2 * J + 1 < F.g.ny ? A(0.5) : A(0)};
    const A wz[3] = {K > 0 ? A(0.5) : A(0), A(1), 2 * K + 1 < F.g.nz ? A(0.5) : A(0)};
    A acc = A(0);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const T* row = rf + F.g.pitch * ((long long)jy[b] + (long long)F.g.ny * kz[c]);
        acc += wz[c] * wy[b] * (wx[0] * to_acc(row[ix[0]]) + to_acc(row[ix[1]]) + wx[2] * to_acc(row[ix[2]]));
      }
    rc[off(C.g, I, J, K)] = from_acc<T>(tdir(C.g, I, J, K) ? A(0) : acc);
  }
}

// Trilinear interpolation as (1/8) * the sum over the 2 x 2 x 2 parent combinations, the two
// parents of an even index being the same node: eight independent loads, no branches.
template <typename T>
__device__ void tail_prolong(const TailLevel& C, const TailLevel& F, int t0, int st) {
  using A = typename Acc<T>::type;
  const T* ec = static_cast<const T*>(C.e);
  T* tf = static_cast<T*>(F.t);
  const int n = F.g.nx * F.g.ny * F.g.nz;
  for (int t = t0; t < n; t += st) {
    const int i = t % F.g.nx, j = (t / F.g.nx) % F.g.ny, k = t / (F.g.nx * F.g.ny);
    const int I0 = i >> 1, J0 = j >> 1, K0 = k >> 1;
    const int I1 = I0 + (i & 1), J1 = J0 + (j & 1), K1 = K0 + (k & 1);
    const long long r00 = C.g.pitch * ((long long)J0 + (long long)C.g.ny * K0);
    const long long r10 = C.g.pitch * ((long long)J1 + (long long)C.g.ny * K0);
    const long long r01 = C.g.pitch * ((long long)J0 + (long long)C.g.ny * K1);
    const long long r11 = C.g.pitch * ((long long)J1 + (long long)C.g.ny * K1);
    A v = to_acc(ec[r00 + I0]) + to_acc(ec[r00 + I1]) + to_acc(ec[r10 + I0]) + to_acc(ec[r10 + I1]) +
          to_acc(ec[r01 + I0]) + to_acc(ec[r01 + I1]) + to_acc(ec[r11 + I0]) + to_acc(ec[r11 + I1]);
    v *= A(0.125);
    tf[off(F.g, i, j, k)] = from_acc<T>(tdir(F.g, i, j, k) ? A(0) : v);
  }
}

// e = t + omega D^-1 (r - A t), Dirichlet nodes copied.  A: 27 coefficients or the constant
// stencil on the mirrored field times prod_d s_d / 2.
template <typename T>
__device__ void tail_jacobi(const TailLevel& L, double omega, int t0, int st) {
  using A = typename Acc<T>::type;
  const T* x = static_cast<const T*>(L.t);
  const T* b = static_cast<const T*>(L.r);
  const T* a27 = static_cast<const T*>(L.a27);
  T* out = static_cast<T*>(L.e);
  const LevelGeom& g = L.g;
  const long long plane = g.pitch * (long long)g.ny * g.nz;
  const int n = g.nx * g.ny * g.nz;
  for (int t = t0; t < n; t += st) {
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

// Coarsest level: e = A^+ r over the free nodes (dense FP64 inverse), e = 0 on Dirichlet nodes.
// rs: the block's shared copy of r at the free nodes (filled here; the caller syncs the block
// before the row loop via the returned flag protocol below).  Rows go to warps w0, w0 + wst, ...
template <typename T>
__device__ void tail_coarsest_load(const TailArgs& a, double* rs, int t0, int st) {
  const TailLevel& C = a.lv[a.nlev - 1];
  const T* r = static_cast<const T*>(C.r);
  T* e = static_cast<T*>(C.e);
  const int n = C.g.nx * C.g.ny * C.g.nz;
  if (!a.dense_all)
    for (int t = t0; t < n; t += st) {
      const int i = t % C.g.nx, j = (t / C.g.nx) % C.g.ny, k = t / (C.g.nx * C.g.ny);
      if (tdir(C.g, i, j, k)) e[off(C.g, i, j, k)] = from_acc<T>(0.0);
    }
  for (int t = threadIdx.x; t < a.nfree; t += blockDim.x) rs[t] = (double)to_acc(r[a.free_idx[t]]);
}

template <typename T>
__device__ void tail_coarsest_rows(const TailArgs& a, const double* rs, int w0, int wst) {
  const TailLevel& C = a.lv[a.nlev - 1];
  T* e = static_cast<T*>(C.e);
  const int lane = threadIdx.x & 31;
  for (int row = w0; row < a.nfree; row += wst) {
    double s = 0.0;
    for (int c = lane; c < a.nfree; c += 32) s += a.ainv[(long long)row * a.nfree + c] * rs[c];
    s = warp_sum(s);
    if (lane == 0) e[a.free_idx[row]] = from_acc<T>(s);
  }
}

// The whole tail inside one CTA, barriers = __syncthreads.
template <typename T>
__device__ void tail_block(const TailArgs& a) {
  __shared__ double rs[1024];
  const int t0 = threadIdx.x, st = blockDim.x;
  for (int l = 0; l + 1 < a.nlev; ++l) {
    tail_restrict<T>(a.lv[l], a.lv[l + 1], t0, st);
    __syncthreads();
  }
  tail_coarsest_load<T>(a, rs, t0, st);
  __syncthreads();
  tail_coarsest_rows<T>(a, rs, threadIdx.x >> 5, blockDim.x >> 5);
  __syncthreads();
  for (int l = a.nlev - 2; l >= 0; --l) {
    tail_prolong<T>(a.lv[l + 1], a.lv[l], t0, st);
    __syncthreads();
    tail_jacobi<T>(a.lv[l], a.omega, t0, st);
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_tail(const TailArgs a) {
  tail_block<T>(a);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_tail_batch(const TailArgs* __restrict__ tab, const int* __restrict__ active) {
  if (active && !active[blockIdx.x]) return;
  tail_block<T>(tab[blockIdx.x]);
}

// ---------------------------------------------------------------- cooperative coarse levels
// Grid barrier for a cooperative launch (all blocks resident): the last block to arrive resets
// the count and advances the generation; the others wait for the generation to change, at most
// 2 s, after which the barrier reports failure (error bit 0) and the kernel stops.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_barrier(GridBarrier* b, unsigned& gen) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const uint64_t t0 = globaltimer_ns();
      while (ld_acquire_gpu(&b->gen) == gen) {
        if (globaltimer_ns() - t0 > 2000000000ull) {
          raise_error(1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  gen += 1;
  return __syncthreads_and(ok) != 0;
}

// Prolongation fused into the Jacobi sweep of level L: t = P e_C is formed on the fly at the
// node's 27 (mirrored) neighbours from the 3 x 3 x 3 block of coarse values around them, each
// rounded to the storage type as a stored t would be, and zero at Dirichlet nodes; then
// e_L = t + omega D^-1 (r - A t) (Dirichlet nodes: e_L = t).  Per axis, fine index f takes coarse
// nodes f >> 1 and (f >> 1) + (f & 1) with weight 1/2 each (one node, weight 1, for an even f).
template <typename T>
__device__ void coarse_prolong_jacobi(const TailLevel& C, const TailLevel& L, double omega_d, int t0, int st) {
  using A = typename Acc<T>::type;
  const T* ec = static_cast<const T*>(C.e);
  const T* b = static_cast<const T*>(L.r);
  const T* a27 = static_cast<const T*>(L.a27);
  T* out = static_cast<T*>(L.e);
  const LevelGeom& g = L.g;
  const LevelGeom& gc = C.g;
  const long long plane = g.pitch * (long long)g.ny * g.nz;
  const A omega = (A)omega_d;
  const int nf[3] = {g.nx, g.ny, g.nz}, ncs[3] = {gc.nx, gc.ny, gc.nz};
  const int n = g.nx * g.ny * g.nz;
  for (int t = t0; t < n; t += st) {
    const int idx[3] = {t % g.nx, (t / g.nx) % g.ny, t / (g.nx * g.ny)};
    int cb[3], cc[3][3];
    A W[3][3][3];  // [axis][fine neighbour a][coarse c]
    bool dfn[3][3];  // fine neighbour a of this axis lies on a Dirichlet face of the axis
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      int f[3], lo[3], hi[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        f[q] = mirror(idx[ax] + q - 1, nf[ax]);
        lo[q] = f[q] >> 1;
        hi[q] = lo[q] + (f[q] & 1);
        dfn[ax][q] = (g.dir[2 * ax] && f[q] == 0) || (g.dir[2 * ax + 1] && f[q] == nf[ax] - 1);
      }
      cb[ax] = min(lo[0], min(lo[1], lo[2]));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cc[ax][c] = min(cb[ax] + c, ncs[ax] - 1);
#pragma unroll
        for (int q = 0; q < 3; ++q)
          W[ax][q][c] = (lo[q] == cb[ax] + c ? A(0.5) : A(0)) + (hi[q] == cb[ax] + c ? A(0.5) : A(0));
      }
    }
    A E[3][3][3];  // coarse block [x][y][z]
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
      for (int y = 0; y < 3; ++y) {
        const T* row = ec + gc.pitch * ((long long)cc[1][y] + (long long)gc.ny * cc[2][z]);
#pragma unroll
        for (int x = 0; x < 3; ++x) E[x][y][z] = to_acc(row[cc[0][x]]);
      }
    const long long o = idx[0] + g.pitch * ((long long)idx[1] + (long long)g.ny * idx[2]);
    const bool dnode = dfn[0][1] || dfn[1][1] || dfn[2][1];
    A s = A(0), xc = A(0);
    const A cw = A(0.125) * (A)(((idx[0] > 0) + (idx[0] < g.nx - 1)) * ((idx[1] > 0) + (idx[1] < g.ny - 1)) *
                                ((idx[2] > 0) + (idx[2] < g.nz - 1)));
#pragma unroll
    for (int c = 0; c < 3; ++c) {  // fine neighbour plane dz = c - 1
      A Fz[3][3];
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int y = 0; y < 3; ++y) Fz[x][y] = W[2][c][0] * E[x][y][0] + W[2][c][1] * E[x][y][1] + W[2][c][2] * E[x][y][2];
#pragma unroll
      for (int bq = 0; bq < 3; ++bq) {
        A G[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) G[x] = W[1][bq][0] * Fz[x][0] + W[1][bq][1] * Fz[x][1] + W[1][bq][2] * Fz[x][2];
#pragma unroll
        for (int aq = 0; aq < 3; ++aq) {
          A tv = W[0][aq][0] * G[0] + W[0][aq][1] * G[1] + W[0][aq][2] * G[2];
          tv = (dfn[0][aq] || dfn[1][bq] || dfn[2][c]) ? A(0) : to_acc(from_acc<T>(tv));
          const int d = aq + 3 * bq + 9 * c;
          if (d == 13) xc = tv;
          if (a27)
            s += to_acc(a27[d * plane + o]) * tv;
          else
            s += (A)L.L.c[(aq != 1) + 2 * (bq != 1) + 4 * (c != 1)] * tv;
        }
      }
    }
    if (dnode) {
      out[o] = from_acc<T>(xc);
      continue;
    }
    A D;
    if (a27) {
      D = to_acc(a27[13 * plane + o]);
    } else {
      s *= cw;
      D = cw * (A)L.L.c[0];
    }
    out[o] = from_acc<T>(xc + omega * (to_acc(b[o]) - s) / D);
  }
}

// Levels lv[0 .. nlev-1]: restrictions down to lv[nlev-1], its dense map e = ainv r (over the
// nodes in free_idx), then a fused prolongation + Jacobi sweep per level back up to lv[0].
template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse(const TailArgs a, GridBarrier* bar) {
  __shared__ double rs[1024];
  unsigned gen = ld_acquire_gpu(&bar->gen);
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, st = gridDim.x * blockDim.x;
  for (int l = 0; l + 1 < a.nlev; ++l) {
    tail_restrict<T>(a.lv[l], a.lv[l + 1], t0, st);
    if (!grid_barrier(bar, gen)) return;
  }
  tail_coarsest_load<T>(a, rs, t0, st);
  __syncthreads();
  tail_coarsest_rows<T>(a, rs, t0 >> 5, st >> 5);
  if (a.nlev > 1 && !grid_barrier(bar, gen)) return;
  for (int l = a.nlev - 2; l >= 0; --l) {
    coarse_prolong_jacobi<T>(a.lv[l + 1], a.lv[l], a.omega, t0, st);
    if (l > 0 && !grid_barrier(bar, gen)) return;
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

template <typename T>
int coarse_t(const TailArgs& a, GridBarrier* bar, cudaStream_t s) {
  auto kern = k_coarse<T>;
  const long long most = (long long)a.lv[0].g.nx * a.lv[0].g.ny * a.lv[0].g.nz;
  const int grid = (int)resident_grid(reinterpret_cast<const void*>(kern), kCoarseThreads, 0,
                                      (most + kCoarseThreads - 1) / kCoarseThreads);
  TailArgs args = a;
  GridBarrier* b = bar;
  void* params[] = {&args, &b};
  return check_cuda(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(kCoarseThreads),
                                                params, 0, s),
                    "cooperative coarse-level launch");
}

int launch_coarse(nn4_dtype dt, const TailArgs& a, GridBarrier* bar, cudaStream_t s) {
  if (a.nlev < 2 || a.nlev > kMaxTail || a.nfree > 1024 || !a.dense_all || !bar)
    return set_error(NN4_EINVAL, "bad coarse levels");
  switch (dt) {
    case NN4_F64: return coarse_t<double>(a, bar, s);
    case NN4_F32: return coarse_t<float>(a, bar, s);
    case NN4_BF16: return coarse_t<bf16>(a, bar, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
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
