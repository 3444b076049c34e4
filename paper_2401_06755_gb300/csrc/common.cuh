// Device-side helpers shared by the kernels: storage types, TMA tile loads, bounded mbarrier
// waits, the device error word and the mirror indexing that realises natural boundaries.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nn4.h"

namespace nn4 {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------- storage types
// Storage type T is held in memory; arithmetic runs in Acc<T> (FP64 for double, FP32 else).
template <typename T> struct Acc;
template <> struct Acc<double> { using type = double; };
template <> struct Acc<float> { using type = float; };
template <> struct Acc<bf16> { using type = float; };

__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ float to_acc(bf16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_acc(double v);
template <> __device__ __forceinline__ double from_acc<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_acc<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ bf16 from_acc<bf16>(double v) { return __double2bfloat16(v); }
template <typename T> __device__ __forceinline__ T from_acc(float v);
template <> __device__ __forceinline__ float from_acc<float>(float v) { return v; }
template <> __device__ __forceinline__ bf16 from_acc<bf16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ double from_acc<double>(float v) { return (double)v; }

// A value the compiler treats as opaque: a loop-invariant conversion (e.g. of an FP64 kernel
// argument) is then computed once and kept, not recomputed at each use.
__device__ __forceinline__ float opaque(float v) {
  float r;
  asm volatile("mov.b32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ double opaque(double v) {
  double r;
  asm volatile("mov.b64 %0, %1;" : "=d"(r) : "d"(v));
  return r;
}

// ---------------------------------------------------------------- device error word
// Bit 0: a bounded wait gave up.  Bit 1: a checked index was out of range.  Each translation
// unit has its own word (no relocatable device code); NN4_DEFINE_ERROR_ACCESSOR(name) gives the
// unit a host function that reads and clears it, and nn4_device_error() polls all of them.
static __device__ unsigned int g_error_word = 0;

#define NN4_DEFINE_ERROR_ACCESSOR(fname)                                   \
  unsigned int fname() {                                                   \
    unsigned int w = 0, z = 0;                                             \
    if (cudaMemcpyFromSymbol(&w, g_error_word, sizeof(w)) != cudaSuccess) \
      return 0u;                                                           \
    if (w) cudaMemcpyToSymbol(g_error_word, &z, sizeof(z));                \
    return w;                                                              \
  }

__device__ __forceinline__ void raise_error(unsigned int bit) { atomicOr(&g_error_word, bit); }

// ---------------------------------------------------------------- mirror indexing
// Natural (zero-derivative) faces are realised by finite-element truncation.  On a vertex grid
// the truncated row at a boundary node equals the interior stencil applied to the field mirrored
// about that node (x_{-1} = x_1, x_n = x_{n-2}), times 1/2 per natural boundary the node lies on.
__device__ __forceinline__ int mirror(int i, int n) {
  return i < 0 ? -i : (i >= n ? 2 * (n - 1) - i : i);
}

// ---------------------------------------------------------------- mbarrier + TMA (sm_90+ PTX)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// One test of phase `parity`; a thread whose phase is not complete may be suspended until it
// completes, for at most about a millisecond (the suspend-time hint), instead of spinning and
// taking issue slots from the warps that compute.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of `bar` for at most ~2 s of wall time.  Returns false on timeout
// (after latching the error bit); the caller then stops issuing work and drains.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > 2000000000ull) {
      raise_error(1u);
      return false;
    }
  }
}

// 3D tiled TMA load of box (bx, by, 1) at element coordinates (x, y, z) into shared memory,
// completing on `bar`.  x must be a multiple of 16 bytes / sizeof(element) (checked by callers
// through their tiling); y and z may be negative or past the end (zero fill).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// 4D tiled TMA load of box (bx, by, 1, bd) at element coordinates (x, y, z, w); same rules.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------- block reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum v over the block and add it to *out with one atomic per block.  `scratch` holds >= 32
// doubles of shared memory.  Every thread of the block must call this.
__device__ __forceinline__ void block_sum_atomic(double v, double* out, double* scratch) {
  v = warp_sum(v);
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < nwarps ? scratch[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) atomicAdd(out, s);
  }
}

}  // namespace nn4
