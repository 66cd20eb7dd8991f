// gg_dev.cu — device evaluation of the generators in gg.h (C ABI; device pointers, caller's stream).
// Bit-identical to gg_host.cpp: both call the same per-edge functions.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gg.h"

namespace {

__global__ void k_er(uint64_t seed, uint32_t n, int64_t e0, int64_t len, int32_t* src, int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    gg_er_edge(seed, n, (uint64_t)(e0 + i), &src[i], &dst[i]);
}

__global__ void k_rmat(uint64_t seed, int scale, uint32_t n, const uint32_t* __restrict__ thr_g, int64_t e0,
                       int64_t len, int32_t* src, int32_t* dst) {
  __shared__ uint32_t thr[3 * 32];
  for (int i = threadIdx.x; i < 3 * scale; i += blockDim.x) thr[i] = thr_g[i];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    gg_rmat_edge(seed, scale, n, thr, (uint64_t)(e0 + i), &src[i], &dst[i]);
}

__global__ void k_perm(uint64_t seed, uint32_t n, int32_t* ids, int64_t len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
    ids[i] = (int32_t)gg_permute(seed, n, (uint32_t)ids[i]);
}

// Row i's pair count into cnt[i + 1] (cnt[0] = 0), for an inclusive scan into row offsets.
__global__ void k_gnp_count(uint64_t seed, uint32_t n, uint64_t lq, int64_t* cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    cnt[i + 1] = gg_gnp_row(seed, n, lq, (uint32_t)i, nullptr, nullptr);
    if (i == 0) cnt[0] = 0;
  }
}

__global__ void k_gnp_write(uint64_t seed, uint32_t n, uint64_t lq, const int64_t* __restrict__ off, int32_t* src,
                            int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    gg_gnp_row(seed, n, lq, (uint32_t)i, src + off[i], dst + off[i]);
}

int grid_for(int64_t len) {
  int64_t b = (len + 255) / 256;
  if (b > 152 * 64) b = 152 * 64;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

extern "C" {

int gg_er_dev(uint64_t seed, uint32_t n, int64_t e0, int64_t len, int32_t* src, int32_t* dst, void* stream) {
  if (n == 0 || len < 0) return 1;
  if (len == 0) return 0;
  k_er<<<grid_for(len), 256, 0, (cudaStream_t)stream>>>(seed, n, e0, len, src, dst);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// thr: DEVICE pointer to 3*scale uint32 thresholds.
int gg_rmat_dev(uint64_t seed, int scale, uint32_t n, const uint32_t* thr, int64_t e0, int64_t len, int32_t* src,
                int32_t* dst, void* stream) {
  if (n == 0 || scale < 1 || scale > 31 || (1ULL << scale) < n || len < 0) return 1;
  if (len == 0) return 0;
  k_rmat<<<grid_for(len), 256, 0, (cudaStream_t)stream>>>(seed, scale, n, thr, e0, len, src, dst);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// G(n, p), first step: cnt (n + 1 int64, device) receives 0 and the per-row pair counts; the caller scans it
// inclusively into row offsets.
int gg_gnp_count_dev(uint64_t seed, uint32_t n, uint64_t lq, int64_t* cnt, void* stream) {
  if (n == 0 || !cnt) return 1;
  k_gnp_count<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(seed, n, lq, cnt);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

// G(n, p), second step: row i's pairs written at off[i] (off: n + 1 int64 row offsets, device).
int gg_gnp_write_dev(uint64_t seed, uint32_t n, uint64_t lq, const int64_t* off, int32_t* src, int32_t* dst,
                     void* stream) {
  if (n == 0 || !off) return 1;
  k_gnp_write<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(seed, n, lq, off, src, dst);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int gg_permute_dev(uint64_t seed, uint32_t n, int32_t* ids, int64_t len, void* stream) {
  if (n == 0 || len < 0) return 1;
  if (len == 0) return 0;
  k_perm<<<grid_for(len), 256, 0, (cudaStream_t)stream>>>(seed, n, ids, len);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

}  // extern "C"
