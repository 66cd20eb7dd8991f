// tc_prims.cuh — warp/block building blocks used by several kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tc {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Exclusive scan over the block; every thread must call it.  `ws` is shared scratch of blockDim.x/32 (<= 32)
// entries.  Returns the thread's exclusive prefix; *total receives the block sum.  Ends with __syncthreads(), so
// ws may be reused right away.
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* ws, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  T x = warp_inclusive_scan(v);
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T s = lane < nw ? ws[lane] : T(0);
    s = warp_inclusive_scan(s);
    if (lane < nw) ws[lane] = s;
  }
  __syncthreads();
  const T prefix = warp > 0 ? ws[warp - 1] : T(0);
  *total = ws[nw - 1];
  __syncthreads();
  return prefix + x - v;
}

}  // namespace tc
