// Low-precision copies of the level-0 arena (BF16, or FP8 E4M3 with one scale
// per partition), kept beside the FP32 master rows that the re-rank reads.
//
//   BF16   round to nearest even (cvt.rn.bf16.f32).
//   E4M3   s_p = max|x| / 448 over the partition (FP32; 1 for an all-zero
//          partition), codes = E4M3(x / s_p) rounded to nearest even and
//          saturated at +-448 (cvt.rn.satfinite.e4m3x2.f32).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace qk {

// One CTA per partition: s_p = max |x| / 448.
__global__ void partition_scale_kernel(const float* __restrict__ vec, const int64_t* __restrict__ off,
                                       const int32_t* __restrict__ size, int d, float* __restrict__ scale) {
  int j = blockIdx.x;
  const float* x = vec + off[j] * d;
  int64_t n = (int64_t)size[j] * d;
  float m = 0.f;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) m = fmaxf(m, fabsf(x[e]));
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    scale[j] = t > 0.f ? t / 448.0f : 1.0f;
  }
}

__device__ __forceinline__ void quantize_one(const float* x, int64_t slot, int d, int storage, float scale,
                                             unsigned char* lp, int lane, int nlanes) {
  if (storage == 1) {
    __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(lp) + slot * d;
    for (int j = lane; j < d; j += nlanes) o[j] = __float2bfloat16_rn(x[j]);
  } else {
    __nv_fp8_storage_t* o = reinterpret_cast<__nv_fp8_storage_t*>(lp) + slot * d;
    for (int j = lane; j < d; j += nlanes) o[j] = __nv_cvt_float_to_fp8(x[j] / scale, __NV_SATFINITE, __NV_E4M3);
  }
}

// Every stored row of every partition (one CTA per partition).
__global__ void quantize_arena_kernel(const float* __restrict__ vec, const int64_t* __restrict__ off,
                                      const int32_t* __restrict__ size, int d, int storage,
                                      const float* __restrict__ scale, unsigned char* __restrict__ lp) {
  int j = blockIdx.x;
  float s = storage == 2 ? scale[j] : 1.f;
  for (int64_t r = threadIdx.x >> 5; r < size[j]; r += blockDim.x >> 5)
    quantize_one(vec + (off[j] + r) * d, off[j] + r, d, storage, s, lp, threadIdx.x & 31, 32);
}

// Rows X[i] stored at arena slot dst[i] of partition part[i] (one warp per row).
__global__ void quantize_rows_kernel(const float* __restrict__ X, int64_t n, int d, const int64_t* __restrict__ dst,
                                     const int32_t* __restrict__ part, int storage, const float* __restrict__ scale,
                                     unsigned char* __restrict__ lp) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  float s = storage == 2 ? scale[part[w]] : 1.f;
  quantize_one(X + w * d, dst[w], d, storage, s, lp, threadIdx.x & 31, 32);
}

// Byte rows: src slots -> temp, then temp -> dst slots (two launches, so
// overlapping moves read the old contents).
__global__ void gather_bytes_kernel(const unsigned char* __restrict__ a, const int64_t* __restrict__ src, int64_t m,
                                    int rb, unsigned char* __restrict__ tmp) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= m) return;
  const uint4* s = reinterpret_cast<const uint4*>(a + src[w] * rb);
  uint4* o = reinterpret_cast<uint4*>(tmp + w * rb);
  for (int j = threadIdx.x & 31; j < rb / 16; j += 32) o[j] = s[j];
}

__global__ void place_bytes_kernel(const unsigned char* __restrict__ tmp, const int64_t* __restrict__ dst, int64_t m,
                                   int rb, unsigned char* __restrict__ a) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= m) return;
  const uint4* s = reinterpret_cast<const uint4*>(tmp + w * rb);
  uint4* o = reinterpret_cast<uint4*>(a + dst[w] * rb);
  for (int j = threadIdx.x & 31; j < rb / 16; j += 32) o[j] = s[j];
}

// Partition j's first size[j] byte rows from old_off[j] to new_off[j].
__global__ void relayout_bytes_kernel(const unsigned char* __restrict__ old_a, const int64_t* __restrict__ old_off,
                                      const int64_t* __restrict__ new_off, const int32_t* __restrict__ size, int rb,
                                      unsigned char* __restrict__ new_a) {
  int j = blockIdx.x;
  int64_t n16 = (int64_t)size[j] * rb / 16;
  const uint4* s = reinterpret_cast<const uint4*>(old_a + old_off[j] * rb);
  uint4* o = reinterpret_cast<uint4*>(new_a + new_off[j] * rb);
  for (int64_t e = threadIdx.x; e < n16; e += blockDim.x) o[e] = s[e];
}

// Loads this file's kernels into the context (see preload_update_kernels).
void preload_quant_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, partition_scale_kernel);
  cudaFuncGetAttributes(&fa, quantize_arena_kernel);
  cudaFuncGetAttributes(&fa, quantize_rows_kernel);
  cudaFuncGetAttributes(&fa, gather_bytes_kernel);
  cudaFuncGetAttributes(&fa, place_bytes_kernel);
  cudaFuncGetAttributes(&fa, relayout_bytes_kernel);
}

qk_status launch_quantize_arena(const float* vec, const int64_t* off, const int32_t* size, int32_t n_part, int d,
                                int storage, float* scale, unsigned char* lp, cudaStream_t s) {
  if (n_part <= 0) return QK_OK;
  if (storage == 2) {
    partition_scale_kernel<<<n_part, 256, 0, s>>>(vec, off, size, d, scale);
    QK_CUDA(cudaGetLastError());
  }
  quantize_arena_kernel<<<n_part, 256, 0, s>>>(vec, off, size, d, storage, scale, lp);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_quantize_rows(const float* X, int64_t n, int d, const int64_t* dst, const int32_t* part, int storage,
                               const float* scale, unsigned char* lp, cudaStream_t s) {
  if (n <= 0) return QK_OK;
  quantize_rows_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, dst, part, storage, scale, lp);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_move_bytes(unsigned char* a, const int64_t* src, const int64_t* dst, int64_t m, int rb,
                            unsigned char* tmp, cudaStream_t s) {
  if (m <= 0) return QK_OK;
  unsigned grid = (unsigned)((m * 32 + 255) / 256);
  gather_bytes_kernel<<<grid, 256, 0, s>>>(a, src, m, rb, tmp);
  QK_CUDA(cudaGetLastError());
  place_bytes_kernel<<<grid, 256, 0, s>>>(tmp, dst, m, rb, a);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_relayout_bytes(const unsigned char* old_a, const int64_t* old_off, const int64_t* new_off,
                                const int32_t* size, int32_t n_part, int rb, unsigned char* new_a, cudaStream_t s) {
  if (n_part <= 0) return QK_OK;
  relayout_bytes_kernel<<<n_part, 256, 0, s>>>(old_a, old_off, new_off, size, rb, new_a);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
