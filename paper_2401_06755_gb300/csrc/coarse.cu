// Exact solve on the coarsest multigrid level: e = A_L^+ r with the dense FP64 (pseudo-)inverse
// formed at plan time.  Always FP64 arithmetic, whatever the storage type of r and e.
#include "common.cuh"
#include "internal.h"

namespace nn4 {
namespace {

// One warp per row of the inverse; the right-hand side is gathered into shared memory first.
template <typename T>
__global__ void k_coarse(const double* __restrict__ ainv, const int* __restrict__ free_idx, int nfree,
                         const T* __restrict__ r, T* __restrict__ e, int nall, LevelGeom g, int accumulate) {
  extern __shared__ double rs[];
  for (int t = threadIdx.x; t < nfree; t += blockDim.x) rs[t] = (double)to_acc(r[free_idx[t]]);
  // zero every node of e first (Dirichlet nodes stay zero); block 0 only, before the barrier
  if (blockIdx.x == 0 && !accumulate) {
    for (int t = threadIdx.x; t < nall; t += blockDim.x) {
      const int i = t % g.nx, j = (t / g.nx) % g.ny, k = t / (g.nx * g.ny);
      e[i + g.pitch * ((long long)j + (long long)g.ny * k)] = from_acc<T>(0.0);
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  for (int row = blockIdx.x * nwarps + warp; row < nfree; row += gridDim.x * nwarps) {
    double s = 0.0;
    for (int c = lane; c < nfree; c += 32) s += ainv[(long long)row * nfree + c] * rs[c];
    s = warp_sum(s);
    if (lane == 0) e[free_idx[row]] = from_acc<T>(accumulate ? s + (double)to_acc(e[free_idx[row]]) : s);
  }
}

template <typename T>
int coarse_t(const double* ainv, const int* free_idx, int nfree, const void* r, void* e,
             const LevelGeom& g, int acc, cudaStream_t s) {
  // a single CTA keeps the zero fill ordered before the scattered writes
  k_coarse<T><<<1, 512, nfree * sizeof(double), s>>>(ainv, free_idx, nfree, static_cast<const T*>(r),
                                                     static_cast<T*>(e), g.nx * g.ny * g.nz, g, acc);
  return check_cuda(cudaGetLastError(), "coarse solve launch");
}

}  // namespace

int launch_coarse_solve(nn4_dtype dt, const double* ainv, const int* free_idx, int nfree,
                        const void* r, void* e, const LevelGeom& g, int acc, cudaStream_t s) {
  switch (dt) {
    case NN4_F64: return coarse_t<double>(ainv, free_idx, nfree, r, e, g, acc, s);
    case NN4_F32: return coarse_t<float>(ainv, free_idx, nfree, r, e, g, acc, s);
    case NN4_BF16: return coarse_t<bf16>(ainv, free_idx, nfree, r, e, g, acc, s);
  }
  return set_error(NN4_EINVAL, "bad dtype");
}

}  // namespace nn4
