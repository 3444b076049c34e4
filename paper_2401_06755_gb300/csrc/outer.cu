// Pointwise FP64 kernels of the outer loop of the pressure solve: defect-correction update,
// conversion of the FP64 residual to the inner storage type, and the flexible-CG recurrences
// (Notay 2000) with their dot products.  All sums are accumulated in FP64.
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "outer.h"

namespace nn4 {
namespace {

// Grid-stride loop over the nodes of a pitched field: one thread per x, rows spread over the grid.
#define NN4_FOR_NODES(G)                                                                    \
  for (long long row = blockIdx.x * (long long)blockDim.y + threadIdx.y;                     \
       row < (long long)(G).ny * (G).nz; row += (long long)gridDim.x * blockDim.y)           \
    _Pragma("unroll 4") for (int i = threadIdx.x; i < (G).nx; i += blockDim.x)

__device__ __forceinline__ bool dirichlet_row(const LevelGeom& g, long long row, int i) {
  const int j = (int)(row % g.ny), k = (int)(row / g.ny);
  return (g.dir[0] && i == 0) || (g.dir[1] && i == g.nx - 1) || (g.dir[2] && j == 0) ||
         (g.dir[3] && j == g.ny - 1) || (g.dir[4] && k == 0) || (g.dir[5] && k == g.nz - 1);
}

// ---------------------------------------------------------------- 4-node chunks
// The pointwise kernels walk each row in chunks of 4 nodes, one chunk per thread.  A chunk that
// is full and whose addresses are all 4-element aligned moves as vectors (the rows of the
// library's own fields start on 128-byte boundaries); any other chunk moves element by element,
// so caller-provided fields of any pitch stay correct.
template <typename T>
__device__ __forceinline__ bool al4(const T* p) {
  return (reinterpret_cast<uintptr_t>(p) & (4 * sizeof(T) - 1)) == 0;
}
__device__ __forceinline__ void ld4v(const float* p, float* v) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
}
__device__ __forceinline__ void ld4v(const double* p, double* v) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
}
__device__ __forceinline__ void ld4v(const bf16* p, bf16* v) {
  const uint2 t = *reinterpret_cast<const uint2*>(p);
  const bf16* e = reinterpret_cast<const bf16*>(&t);
  v[0] = e[0], v[1] = e[1], v[2] = e[2], v[3] = e[3];
}
__device__ __forceinline__ void st4v(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4v(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4v(bf16* p, const bf16* v) {
  uint2 t;
  bf16* e = reinterpret_cast<bf16*>(&t);
  e[0] = v[0], e[1] = v[1], e[2] = v[2], e[3] = v[3];
  *reinterpret_cast<uint2*>(p) = t;
}
// Loads acc-type values of a chunk (0 past its n valid nodes) / stores its n valid nodes.
template <typename T, typename A>
__device__ __forceinline__ void ld4(const T* p, bool vec, int n, A* v) {
  if (vec) {
    T t[4];
    ld4v(p, t);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (A)to_acc(t[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = k < n ? (A)to_acc(p[k]) : A(0);
  }
}
template <typename T, typename A>
__device__ __forceinline__ void st4(T* p, bool vec, int n, const A* v) {
  T t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) t[k] = from_acc<T>(v[k]);
  if (vec) {
    st4v(p, t);
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < n) p[k] = t[k];
  }
}

// Grid-stride loop over the 4-node chunks of a pitched field; defines row, i0 (first x of the
// chunk) and n (valid nodes in it).  Chunk counts fit 32 bits (checked by the launchers).
#define NN4_FOR_CHUNKS(G)                                                                      \
  for (unsigned c_ = blockIdx.x * blockDim.x + threadIdx.x, cpr_ = ((unsigned)(G).nx + 3u) >> 2, \
                tot_ = (unsigned)(G).ny * (unsigned)(G).nz * cpr_;                            \
       c_ < tot_; c_ += gridDim.x * blockDim.x)                                                \
    for (long long row = c_ / cpr_, i0 = (long long)(c_ - (unsigned)row * cpr_) * 4, n = min(4LL, (G).nx - i0), \
                   once_ = 1;                                                                  \
         once_; once_ = 0)

template <typename T>
__global__ void k_add_correction(double* __restrict__ x, LevelGeom g64, const T* __restrict__ e, LevelGeom gT) {
  NN4_FOR_CHUNKS(g64) {
    double* xp = x + row * g64.pitch + i0;
    const T* ep = e + row * gT.pitch + i0;
    const bool vec = n == 4 && al4(xp) && al4(ep);
    double xv[4], ev[4];
    ld4(xp, vec, (int)n, xv);
    ld4(ep, vec, (int)n, ev);
#pragma unroll
    for (int k = 0; k < 4; ++k) xv[k] += ev[k];
    st4(xp, vec, (int)n, xv);
  }
}

template <typename T>
__global__ void k_to_inner(const double* __restrict__ r, LevelGeom g64, T* __restrict__ rT, LevelGeom gT) {
  NN4_FOR_CHUNKS(g64) {
    const double* rp = r + row * g64.pitch + i0;
    T* tp = rT + row * gT.pitch + i0;
    const bool vec = n == 4 && al4(rp) && al4(tp);
    double v[4];
    ld4(rp, vec, (int)n, v);
    st4(tp, vec, (int)n, v);
  }
}

// r = b at free nodes, 0 at Dirichlet nodes (the residual of a zero initial guess)
__global__ void k_masked_copy(const double* __restrict__ b, double* __restrict__ r, LevelGeom g) {
  NN4_FOR_NODES(g) {
    const long long o = row * g.pitch + i;
    r[o] = dirichlet_row(g, row, i) ? 0.0 : b[o];
  }
}

// out += sum of v^2 over every node
__global__ void k_sumsq(const double* __restrict__ v, LevelGeom g, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  NN4_FOR_NODES(g) {
    const double t = v[row * g.pitch + i];
    s += t * t;
  }
  block_sum_atomic(s, out, red);
}

__global__ void k_norm_masked(const double* __restrict__ v, LevelGeom g, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  NN4_FOR_NODES(g) {
    if (!dirichlet_row(g, row, i)) {
      const double t = v[row * g.pitch + i];
      s += t * t;
    }
  }
  block_sum_atomic(s, out, red);
}

// out += sum z_i * q_i (z of type TZ, q of type V).  With a low-precision z the products and the
// per-thread partial sums are FP32 (they only set the conjugation coefficient of flexible CG);
// the sum across threads is FP64.
template <typename TZ, typename V>
__global__ void k_dot_zq(const TZ* __restrict__ z, LevelGeom gz, const V* __restrict__ q, LevelGeom gv,
                         double* out) {
  __shared__ double red[32];
  using P = typename std::conditional<sizeof(TZ) == 8, double, float>::type;  // FP64 z: FP64 products
  P s = 0;
  NN4_FOR_CHUNKS(gv) {
    const TZ* zp = z + row * gz.pitch + i0;
    const V* qp = q + row * gv.pitch + i0;
    const bool vec = n == 4 && al4(zp) && al4(qp);
    P zv[4], qv[4];
    ld4(zp, vec, (int)n, zv);
    ld4(qp, vec, (int)n, qv);
#pragma unroll
    for (int k = 0; k < 4; ++k) s += zv[k] * qv[k];
  }
  block_sum_atomic((double)s, out, red);
}

// p = z - beta p_old with beta = zq / pq_old
template <typename TZ, typename V>
__global__ void k_new_direction(const TZ* __restrict__ z, LevelGeom gz, const V* __restrict__ p_old,
                                V* __restrict__ p, LevelGeom gv, const double* zq, const double* pq_old) {
  __shared__ V beta_s;
  if (threadIdx.x == 0 && threadIdx.y == 0) beta_s = (V)(*zq / *pq_old);  // one FP64 division per block
  __syncthreads();
  const V beta = beta_s;
  NN4_FOR_CHUNKS(gv) {
    const TZ* zp = z + row * gz.pitch + i0;
    const long long o = row * gv.pitch + i0;
    const bool vec = n == 4 && al4(zp) && al4(p_old + o) && al4(p + o);
    V zv[4], pv[4];
    ld4(zp, vec, (int)n, zv);
    ld4(p_old + o, vec, (int)n, pv);
#pragma unroll
    for (int k = 0; k < 4; ++k) pv[k] = zv[k] - beta * pv[k];
    st4(p + o, vec, (int)n, pv);
  }
}

// alpha = pr / pq; x += alpha p; r -= alpha q; rT = r (if rT); norm += r^2 (partial sums in V)
template <typename V, typename TR>
__global__ void k_fcg_update(V* __restrict__ x, V* __restrict__ r, const V* __restrict__ p,
                             const V* __restrict__ q, LevelGeom gv, TR* __restrict__ rT, LevelGeom gT,
                             const double* pr, const double* pq, double* norm2) {
  __shared__ double red[32];
  __shared__ V alpha_s;
  if (threadIdx.x == 0 && threadIdx.y == 0) alpha_s = (V)(*pr / *pq);  // one FP64 division per block
  __syncthreads();
  const V alpha = alpha_s;
  V s = 0;
  NN4_FOR_CHUNKS(gv) {
    const long long o = row * gv.pitch + i0;
    TR* tp = rT ? rT + row * gT.pitch + i0 : nullptr;
    const bool vec = n == 4 && al4(x + o) && al4(r + o) && al4(p + o) && al4(q + o) && (!tp || al4(tp));
    V xv[4], rv[4], pv[4], qv[4];
    ld4(x + o, vec, (int)n, xv);
    ld4(r + o, vec, (int)n, rv);
    ld4(p + o, vec, (int)n, pv);
    ld4(q + o, vec, (int)n, qv);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      xv[k] += alpha * pv[k];
      rv[k] -= alpha * qv[k];
      s += rv[k] * rv[k];
    }
    st4(x + o, vec, (int)n, xv);
    st4(r + o, vec, (int)n, rv);
    if (tp) st4(tp, vec, (int)n, rv);
  }
  block_sum_atomic((double)s, norm2, red);
}

// invd = 1 / (w c0 k - hlk) with hlk = (1/2) L k: the diagonal of Eq. k-T (w = prod_d s_d / 2, c0 the interior
// centre weight of the stencil).
__global__ void k_inv_diag(const double* __restrict__ k, const double* __restrict__ hlk, double* __restrict__ invd,
                           LevelGeom g, double c0) {
  NN4_FOR_NODES(g) {
    const int j = (int)(row % g.ny), kk = (int)(row / g.ny);
    const double w = 0.125 * ((i > 0) + (i < g.nx - 1)) * ((j > 0) + (j < g.ny - 1)) * ((kk > 0) + (kk < g.nz - 1));
    const long long o = row * g.pitch + i;
    invd[o] = 1.0 / (w * c0 * k[o] - hlk[o]);
  }
}

dim3 pw_grid(const LevelGeom& g) {
  long long rows = (long long)g.ny * g.nz;
  long long blocks = (rows + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return dim3((unsigned)blocks);
}
const dim3 kPwBlock(32, 8);
// Grid of a chunked kernel: 256 threads a block, as many blocks as are resident at once.
template <typename Kern>
dim3 cw_grid(Kern kern, const LevelGeom& g) {
  const long long chunks = (long long)g.ny * g.nz * ((g.nx + 3) / 4);
  return dim3((unsigned)resident_grid(reinterpret_cast<const void*>(kern), 256, 0, (chunks + 255) / 256));
}
const dim3 kCwBlock(256);
// The chunk index is 32-bit: fields beyond 2^31 chunks (8.6e9 nodes) are refused.
bool chunks_fit(const LevelGeom& g) { return (unsigned long long)g.ny * g.nz * ((g.nx + 3) / 4) < (1ull << 31); }
#define NN4_CHECK_CHUNKS(g) \
  if (!chunks_fit(g)) return set_error(NN4_EINVAL, "field too large for the pointwise kernels")

template <typename T>
int add_correction_t(double* x, const LevelGeom& g64, const void* e, const LevelGeom& gT, cudaStream_t s) {
  NN4_CHECK_CHUNKS(g64);
  k_add_correction<T><<<cw_grid(k_add_correction<T>, g64), kCwBlock, 0, s>>>(x, g64, static_cast<const T*>(e), gT);
  return check_cuda(cudaGetLastError(), "add correction");
}
template <typename T>
int to_inner_t(const double* r, const LevelGeom& g64, void* rT, const LevelGeom& gT, cudaStream_t s) {
  NN4_CHECK_CHUNKS(g64);
  k_to_inner<T><<<cw_grid(k_to_inner<T>, g64), kCwBlock, 0, s>>>(r, g64, static_cast<T*>(rT), gT);
  return check_cuda(cudaGetLastError(), "to inner");
}
template <typename TZ, typename V>
int dot_zq_t(const void* z, const LevelGeom& gz, const void* q, const LevelGeom& gv, double* out, cudaStream_t s) {
  NN4_CHECK_CHUNKS(gv);
  k_dot_zq<TZ, V><<<cw_grid(k_dot_zq<TZ, V>, gv), kCwBlock, 0, s>>>(static_cast<const TZ*>(z), gz, static_cast<const V*>(q), gv, out);
  return check_cuda(cudaGetLastError(), "dot");
}
template <typename TZ, typename V>
int new_direction_t(const void* z, const LevelGeom& gz, const void* p_old, void* p, const LevelGeom& gv,
                    const double* zq, const double* pq_old, cudaStream_t s) {
  NN4_CHECK_CHUNKS(gv);
  k_new_direction<TZ, V><<<cw_grid(k_new_direction<TZ, V>, gv), kCwBlock, 0, s>>>(static_cast<const TZ*>(z), gz, static_cast<const V*>(p_old),
                                                           static_cast<V*>(p), gv, zq, pq_old);
  return check_cuda(cudaGetLastError(), "new direction");
}
template <typename V, typename TR>
int fcg_update_t(void* x, void* r, const void* p, const void* q, const LevelGeom& gv, void* rT,
                 const LevelGeom& gT, const double* pr, const double* pq, double* norm2, cudaStream_t s) {
  NN4_CHECK_CHUNKS(gv);
  k_fcg_update<V, TR><<<cw_grid(k_fcg_update<V, TR>, gv), kCwBlock, 0, s>>>(static_cast<V*>(x), static_cast<V*>(r), static_cast<const V*>(p),
                                                        static_cast<const V*>(q), gv, static_cast<TR*>(rT), gT, pr, pq,
                                                        norm2);
  return check_cuda(cudaGetLastError(), "fcg update");
}
template <typename TS, typename TD>
__global__ void k_convert(const TS* __restrict__ a, LevelGeom ga, TD* __restrict__ b, LevelGeom gb) {
  using A = typename Acc<TS>::type;
  NN4_FOR_CHUNKS(ga) {
    const TS* ap = a + row * ga.pitch + i0;
    TD* bp = b + row * gb.pitch + i0;
    const bool vec = n == 4 && al4(ap) && al4(bp);
    A v[4];
    ld4(ap, vec, (int)n, v);
    st4(bp, vec, (int)n, v);
  }
}

// The per-iteration device scalars in one launch: p[a], p[b], p[c], p[d] = 0 (negative indices
// skipped), then p[dst] = p[src] when dst >= 0.  One small kernel instead of separate memset and
// copy nodes in the captured iterations, each of which costs a few microseconds of the graph.
__global__ void k_scalars(double* p, int a, int b, int c, int d, int dst, int src) {
  if (threadIdx.x != 0) return;
  if (a >= 0) p[a] = 0.0;
  if (b >= 0) p[b] = 0.0;
  if (c >= 0) p[c] = 0.0;
  if (d >= 0) p[d] = 0.0;
  if (dst >= 0) p[dst] = p[src];
}

}  // namespace

#define NN4_DISPATCH(dt, call)                         \
  switch (dt) {                                        \
    case NN4_F64: { using T = double; return call; }   \
    case NN4_F32: { using T = float; return call; }    \
    case NN4_BF16: { using T = bf16; return call; }    \
  }                                                    \
  return set_error(NN4_EINVAL, "bad dtype");

int launch_add_correction(nn4_dtype dt, double* x, const LevelGeom& g64, const void* e, const LevelGeom& gT,
                          cudaStream_t s) {
  NN4_DISPATCH(dt, add_correction_t<T>(x, g64, e, gT, s))
}
int launch_to_inner(nn4_dtype dt, const double* r, const LevelGeom& g64, void* rT, const LevelGeom& gT,
                    cudaStream_t s) {
  NN4_DISPATCH(dt, to_inner_t<T>(r, g64, rT, gT, s))
}
int launch_inv_diag(const double* k, const double* lk, double* invd, const LevelGeom& g, double c0,
                    cudaStream_t s) {
  k_inv_diag<<<pw_grid(g), kPwBlock, 0, s>>>(k, lk, invd, g, c0);
  return check_cuda(cudaGetLastError(), "inverse diagonal");
}

int launch_scalars(double* p, int a, int b, int c, int d, int dst, int src, cudaStream_t s) {
  k_scalars<<<1, 32, 0, s>>>(p, a, b, c, d, dst, src);
  return check_cuda(cudaGetLastError(), "device scalars");
}
int launch_masked_copy(const double* b, double* r, const LevelGeom& g, cudaStream_t s) {
  k_masked_copy<<<pw_grid(g), kPwBlock, 0, s>>>(b, r, g);
  return check_cuda(cudaGetLastError(), "masked copy");
}
int launch_sumsq(const double* v, const LevelGeom& g, double* out, cudaStream_t s) {
  k_sumsq<<<pw_grid(g), kPwBlock, 0, s>>>(v, g, out);
  return check_cuda(cudaGetLastError(), "sum of squares");
}
int launch_norm_masked(const double* v, const LevelGeom& g, double* out, cudaStream_t s) {
  k_norm_masked<<<pw_grid(g), kPwBlock, 0, s>>>(v, g, out);
  return check_cuda(cudaGetLastError(), "norm");
}
#define NN4_DISPATCH2(da, db, call)                                                       \
  switch (da * 3 + db) {                                                                  \
    case NN4_F64 * 3 + NN4_F64: { using A1 = double; using B1 = double; return call; }  \
    case NN4_F32 * 3 + NN4_F64: { using A1 = float; using B1 = double; return call; }   \
    case NN4_BF16 * 3 + NN4_F64: { using A1 = bf16; using B1 = double; return call; }   \
    case NN4_F64 * 3 + NN4_F32: { using A1 = double; using B1 = float; return call; }   \
    case NN4_F32 * 3 + NN4_F32: { using A1 = float; using B1 = float; return call; }    \
    case NN4_BF16 * 3 + NN4_F32: { using A1 = bf16; using B1 = float; return call; }    \
  }                                                                                       \
  return set_error(NN4_EINVAL, "unsupported type pair");

int launch_dot(nn4_dtype tz, const void* z, const LevelGeom& gz, nn4_dtype tv, const void* q, const LevelGeom& gv,
               double* out, cudaStream_t s) {
  NN4_DISPATCH2(tz, tv, (dot_zq_t<A1, B1>(z, gz, q, gv, out, s)))
}
int launch_direction(nn4_dtype tz, const void* z, const LevelGeom& gz, nn4_dtype tv, const void* p_old, void* p,
                     const LevelGeom& gv, const double* zq, const double* pq_old, cudaStream_t s) {
  NN4_DISPATCH2(tz, tv, (new_direction_t<A1, B1>(z, gz, p_old, p, gv, zq, pq_old, s)))
}
int launch_update(nn4_dtype tv, void* x, void* r, const void* p, const void* q, const LevelGeom& gv, nn4_dtype tr,
                  void* rT, const LevelGeom& gT, const double* pr, const double* pq, double* norm2, cudaStream_t s) {
  if (tv == NN4_F64) {
    switch (tr) {
      case NN4_F64: return fcg_update_t<double, double>(x, r, p, q, gv, rT, gT, pr, pq, norm2, s);
      case NN4_F32: return fcg_update_t<double, float>(x, r, p, q, gv, rT, gT, pr, pq, norm2, s);
      case NN4_BF16: return fcg_update_t<double, bf16>(x, r, p, q, gv, rT, gT, pr, pq, norm2, s);
    }
  } else if (tv == NN4_F32) {
    switch (tr) {
      case NN4_F64: return set_error(NN4_EINVAL, "bad type pair");
      case NN4_F32: return fcg_update_t<float, float>(x, r, p, q, gv, rT, gT, pr, pq, norm2, s);
      case NN4_BF16: return fcg_update_t<float, bf16>(x, r, p, q, gv, rT, gT, pr, pq, norm2, s);
    }
  }
  return set_error(NN4_EINVAL, "unsupported type pair");
}
int launch_convert(nn4_dtype ta, const void* a, const LevelGeom& ga, nn4_dtype tb, void* b, const LevelGeom& gb,
                   cudaStream_t s) {
  switch (ta * 3 + tb) {
    case NN4_F64 * 3 + NN4_F32:
      NN4_CHECK_CHUNKS(ga);
      k_convert<double, float><<<cw_grid(k_convert<double, float>, ga), kCwBlock, 0, s>>>(static_cast<const double*>(a), ga, static_cast<float*>(b), gb);
      break;
    case NN4_F64 * 3 + NN4_BF16:
      NN4_CHECK_CHUNKS(ga);
      k_convert<double, bf16><<<cw_grid(k_convert<double, bf16>, ga), kCwBlock, 0, s>>>(static_cast<const double*>(a), ga, static_cast<bf16*>(b), gb);
      break;
    case NN4_F32 * 3 + NN4_BF16:
      NN4_CHECK_CHUNKS(ga);
      k_convert<float, bf16><<<cw_grid(k_convert<float, bf16>, ga), kCwBlock, 0, s>>>(static_cast<const float*>(a), ga, static_cast<bf16*>(b), gb);
      break;
    case NN4_F64 * 3 + NN4_F64:  // a copy between two pitches (dense host layout <-> plan layout)
      NN4_CHECK_CHUNKS(ga);
      k_convert<double, double><<<cw_grid(k_convert<double, double>, ga), kCwBlock, 0, s>>>(static_cast<const double*>(a), ga, static_cast<double*>(b), gb);
      break;
    case NN4_F32 * 3 + NN4_F64:
      NN4_CHECK_CHUNKS(ga);
      k_convert<float, double><<<cw_grid(k_convert<float, double>, ga), kCwBlock, 0, s>>>(static_cast<const float*>(a), ga, static_cast<double*>(b), gb);
      break;
    default:
      return set_error(NN4_EINVAL, "unsupported conversion");
  }
  return check_cuda(cudaGetLastError(), "convert");
}

// FP64-vector forms used by the outer loop
int launch_dot_zq(nn4_dtype dt, const void* z, const LevelGeom& gT, const double* q, const LevelGeom& g64,
                  double* out, cudaStream_t s) {
  return launch_dot(dt, z, gT, NN4_F64, q, g64, out, s);
}
int launch_new_direction(nn4_dtype dt, const void* z, const LevelGeom& gT, const double* p_old, double* p,
                         const LevelGeom& g64, const double* zq, const double* pq_old, cudaStream_t s) {
  return launch_direction(dt, z, gT, NN4_F64, p_old, p, g64, zq, pq_old, s);
}
int launch_fcg_update(nn4_dtype dt, double* x, double* r, const double* p, const double* q, const LevelGeom& g64,
                      void* rT, const LevelGeom& gT, const double* pr, const double* pq, double* norm2,
                      cudaStream_t s) {
  return launch_update(NN4_F64, x, r, p, q, g64, dt, rT, gT, pr, pq, norm2, s);
}

}  // namespace nn4
