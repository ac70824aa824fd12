// Lloyd k-means on the GPU (Sec. 3, "Index Structure": partitions and the
// centroids of upper levels come from k-means).
//
//   assign  argmin_c ||x - c||^2 with ties to the lower centroid index.  The
//           squared distance is accumulated in FP32 from the differences
//           (x_j - c_j), never through ||x||^2 - 2<x,c> + ||c||^2, so near
//           ties resolve as they do in exact arithmetic up to FP32 rounding.
//           A CTA holds 64 rows and sweeps the centroids in tiles of 64; both
//           tiles are staged in shared memory 64 dimensions at a time, and
//           each thread keeps a 4 x 4 block of distances in registers.
//   update  per-cluster FP64 sums and counts, then the FP64 mean rounded once
//           to FP32; an empty cluster keeps its previous centroid.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace qk {

constexpr int kAsgRows = 64;
constexpr int kAsgCents = 64;
constexpr int kAsgChunk = 64;
constexpr int kAsgPad = 68;   // row stride of the transposed tiles (float4 aligned)

__global__ void __launch_bounds__(256) kmeans_assign_kernel(const float* __restrict__ X, int64_t n, int d,
                                                            const float* __restrict__ C, int K,
                                                            int32_t* __restrict__ assign,
                                                            float* __restrict__ best_dist) {
  __shared__ __align__(16) float Xs[kAsgChunk][kAsgPad];
  __shared__ __align__(16) float Cs[kAsgChunk][kAsgPad];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * kAsgRows;
  float bd[4];
  int bi[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    bd[i] = INFINITY;
    bi[i] = 0x7fffffff;
  }
  for (int c0 = 0; c0 < K; c0 += kAsgCents) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < d; k0 += kAsgChunk) {
      int kc = d - k0 < kAsgChunk ? d - k0 : kAsgChunk;
      // stage 64 rows x kc dims and 64 centroids x kc dims, transposed
      for (int e = threadIdx.x; e < kAsgRows * kAsgChunk; e += 256) {
        int rr = e / kAsgChunk, kk = e % kAsgChunk;
        int64_t gr = row0 + rr;
        float xv = 0.f, cv = 0.f;
        if (kk < kc) {
          if (gr < n) xv = X[gr * d + k0 + kk];
          if (c0 + rr < K) cv = C[(int64_t)(c0 + rr) * d + k0 + kk];
        }
        Xs[kk][rr] = xv;
        Cs[kk][rr] = cv;
      }
      __syncthreads();
      for (int kk = 0; kk < kc; ++kk) {
        float4 xa = *reinterpret_cast<const float4*>(&Xs[kk][ty * 4]);
        float4 ca = *reinterpret_cast<const float4*>(&Cs[kk][tx * 4]);
        float xr[4] = {xa.x, xa.y, xa.z, xa.w};
        float cr[4] = {ca.x, ca.y, ca.z, ca.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float df = xr[i] - cr[j];
            acc[i][j] = fmaf(df, df, acc[i][j]);
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = c0 + tx * 4 + j;
      if (c < K) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (acc[i][j] < bd[i] || (acc[i][j] == bd[i] && c < bi[i])) {
            bd[i] = acc[i][j];
            bi[i] = c;
          }
      }
    }
  }
  // reduce over the 16 threads that share these rows
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      float d2 = __shfl_xor_sync(0xffffffffu, bd[i], o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi[i], o);
      if (d2 < bd[i] || (d2 == bd[i] && i2 < bi[i])) {
        bd[i] = d2;
        bi[i] = i2;
      }
    }
  }
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t gr = row0 + ty * 4 + i;
      if (gr < n) {
        assign[gr] = bi[i];
        if (best_dist) best_dist[gr] = bd[i];
      }
    }
  }
}

__global__ void kmeans_accumulate_kernel(const float* __restrict__ X, int64_t n, int d,
                                         const int32_t* __restrict__ assign, double* __restrict__ sums,
                                         int32_t* __restrict__ counts) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = n * d;
  for (; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / d;
    int j = (int)(e - r * d);
    int c = assign[r];
    atomicAdd(&sums[(int64_t)c * d + j], (double)X[e]);
    if (j == 0) atomicAdd(&counts[c], 1);
  }
}

// C_new may be the same buffer as C_prev (each element is read, then written,
// by one thread), so those two are not marked __restrict__.
__global__ void kmeans_finalize_kernel(const double* __restrict__ sums, const int32_t* __restrict__ counts,
                                       const float* C_prev, float* C_new, int K, int d) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)K * d) return;
  int c = (int)(e / d);
  int cnt = counts[c];
  C_new[e] = cnt > 0 ? (float)(sums[e] / (double)cnt) : C_prev[e];
}

__global__ void gather_rows_kernel(const float* __restrict__ X, int d, const int64_t* __restrict__ rows, int K,
                                   float* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)K * d) return;
  int c = (int)(e / d);
  int j = (int)(e - (int64_t)c * d);
  out[e] = X[rows[c] * d + j];
}

qk_status launch_kmeans_assign(const float* X, int64_t n, int d, const float* C, int K, int32_t* assign,
                               float* best_dist, cudaStream_t s) {
  if (n <= 0) return QK_OK;
  int64_t grid = (n + kAsgRows - 1) / kAsgRows;
  kmeans_assign_kernel<<<(unsigned)grid, 256, 0, s>>>(X, n, d, C, K, assign, best_dist);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

// sums (K x d doubles) and counts (K) are scratch supplied by the caller.
qk_status launch_kmeans_update(const float* X, int64_t n, int d, const int32_t* assign, const float* C_prev, int K,
                               float* C_new, double* sums, int32_t* counts, cudaStream_t s) {
  QK_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)K * d, s));
  QK_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)K, s));
  if (n > 0) {
    int64_t total = n * d;
    int64_t grid = (total + 255) / 256;
    if (grid > 148 * 64) grid = 148 * 64;
    kmeans_accumulate_kernel<<<(unsigned)grid, 256, 0, s>>>(X, n, d, assign, sums, counts);
    QK_CUDA(cudaGetLastError());
  }
  int64_t kd = (int64_t)K * d;
  kmeans_finalize_kernel<<<(unsigned)((kd + 255) / 256), 256, 0, s>>>(sums, counts, C_prev, C_new, K, d);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_gather_rows(const float* X, int d, const int64_t* rows, int K, float* out, cudaStream_t s) {
  int64_t kd = (int64_t)K * d;
  if (kd == 0) return QK_OK;
  gather_rows_kernel<<<(unsigned)((kd + 255) / 256), 256, 0, s>>>(X, d, rows, K, out);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
