// Partition arena kernels: grouping rows into contiguous partitions
// (index install after build or load).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace qk {

__global__ void histogram_kernel(const int32_t* __restrict__ lab, int64_t n, int32_t K, int32_t* __restrict__ counts,
                                 int32_t* __restrict__ status, bool skip_unlabelled) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = lab[i];
    if (c == -1 && skip_unlabelled) continue;
    if (c < 0 || c >= K) {
      atomicExch(status, DEV_BAD_ARG);
      continue;
    }
    atomicAdd(&counts[c], 1);
  }
}

// One warp per row: the row's slot is taken from the partition cursor and the
// row is copied with 16-byte accesses (d is a multiple of 32).
__global__ void scatter_kernel(const float* __restrict__ X, const int64_t* __restrict__ ids, int64_t n, int d,
                               const int32_t* __restrict__ lab, const int64_t* __restrict__ off,
                               int32_t* __restrict__ cursor, float* __restrict__ vec, int64_t* __restrict__ ids_out) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w; r < n; r += nw) {
    int32_t c = lab[r];
    if (c < 0) continue;   // unlabelled rows (reserved arena rows) are left out
    int64_t pos = 0;
    if (lane == 0) pos = off[c] + atomicAdd(&cursor[c], 1);
    pos = __shfl_sync(0xffffffffu, pos, 0);
    const float4* src = reinterpret_cast<const float4*>(X + r * d);
    float4* dst = reinterpret_cast<float4*>(vec + pos * d);
    for (int j = lane; j < d / 4; j += 32) dst[j] = src[j];
    if (lane == 0) ids_out[pos] = ids[r];
  }
}

qk_status launch_histogram(const int32_t* lab, int64_t n, int32_t K, int32_t* counts, int32_t* status,
                           cudaStream_t s, bool skip_unlabelled) {
  if (n <= 0) return QK_OK;
  int64_t grid = (n + 255) / 256;
  if (grid > 148 * 32) grid = 148 * 32;
  histogram_kernel<<<(unsigned)grid, 256, 0, s>>>(lab, n, K, counts, status, skip_unlabelled);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_scatter(const float* X, const int64_t* ids, int64_t n, int d, const int32_t* lab, const int64_t* off,
                         int32_t* cursor, float* vec, int64_t* ids_out, cudaStream_t s) {
  if (n <= 0) return QK_OK;
  int64_t grid = (n * 32 + 255) / 256;
  if (grid > 148 * 64) grid = 148 * 64;
  scatter_kernel<<<(unsigned)grid, 256, 0, s>>>(X, ids, n, d, lab, off, cursor, vec, ids_out);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
