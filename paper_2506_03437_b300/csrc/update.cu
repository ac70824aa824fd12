// Insert and delete kernels (Sec. 3, "Adaptive Incremental Maintenance":
// inserts descend the tree to the nearest leaf and append; deletes remove the
// vector with immediate compaction).  The host runtime plans slots and moves;
// these kernels move the rows.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace qk {

void preload_quant_kernels();

// Second step of the greedy descent for a two-level index: among the leaf
// centroids grouped under parent[r] (rows [off1[p], off1[p] + size1[p]) of the
// level-1 arena, ids = leaf index), the nearest one; ties to the lower leaf.
// One warp per inserted row.
__global__ void descend_children_kernel(const float* __restrict__ X, int64_t n, int d,
                                        const int32_t* __restrict__ parent, const float* __restrict__ vec1,
                                        const int64_t* __restrict__ ids1, const int64_t* __restrict__ off1,
                                        const int32_t* __restrict__ size1, int32_t n_parent,
                                        int32_t* __restrict__ leaf) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  int p = parent[w];
  if (p < 0 || p >= n_parent) {   // no parent (a row the assignment could not place): no leaf
    if (lane == 0) leaf[w] = -1;
    return;
  }
  const float* x = X + w * d;
  float best = INFINITY;
  int64_t best_leaf = INT64_MAX;
  for (int32_t t = 0; t < size1[p]; ++t) {
    const float* c = vec1 + (off1[p] + t) * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) {
      float df = x[j] - c[j];
      acc = fmaf(df, df, acc);
    }
    acc = warp_sum_f(acc);
    int64_t lf = ids1[off1[p] + t];
    if (acc < best || (acc == best && lf < best_leaf)) {
      best = acc;
      best_leaf = lf;
    }
  }
  if (lane == 0) leaf[w] = best_leaf == INT64_MAX ? -1 : (int32_t)best_leaf;
}

__global__ void nan_check_kernel(const float* __restrict__ X, int64_t total, int32_t* __restrict__ flag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (; i < total; i += (int64_t)gridDim.x * blockDim.x)
    if (isnan(X[i])) atomicExch(flag, 1);
}

// Copies partition j's first size[j] rows from old_off[j] to new_off[j]
// (one CTA per partition; regions of different partitions do not overlap).
__global__ void relayout_kernel(const float* __restrict__ old_vec, const int64_t* __restrict__ old_ids,
                                const int64_t* __restrict__ old_off, const int64_t* __restrict__ new_off,
                                const int32_t* __restrict__ size, int d, float* __restrict__ new_vec,
                                int64_t* __restrict__ new_ids) {
  int j = blockIdx.x;
  int64_t so = old_off[j], dn = new_off[j];
  int64_t nf4 = (int64_t)size[j] * d / 4;
  const float4* src = reinterpret_cast<const float4*>(old_vec + so * d);
  float4* dst = reinterpret_cast<float4*>(new_vec + dn * d);
  for (int64_t e = threadIdx.x; e < nf4; e += blockDim.x) dst[e] = src[e];
  for (int64_t e = threadIdx.x; e < size[j]; e += blockDim.x) new_ids[dn + e] = old_ids[so + e];
}

// Writes row r of X (and its id) to arena row dst[r].  One warp per row.
__global__ void place_rows_kernel(const float* __restrict__ X, const int64_t* __restrict__ ids, int64_t n, int d,
                                  const int64_t* __restrict__ dst, float* __restrict__ vec,
                                  int64_t* __restrict__ ids_out) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  const float4* s = reinterpret_cast<const float4*>(X + w * d);
  float4* o = reinterpret_cast<float4*>(vec + dst[w] * d);
  for (int j = lane; j < d / 4; j += 32) o[j] = s[j];
  if (lane == 0) ids_out[dst[w]] = ids[w];
}

// Arena rows src[m] -> tmp row m (first phase of a set of moves).
__global__ void gather_moves_kernel(const float* __restrict__ vec, const int64_t* __restrict__ ids,
                                    const int64_t* __restrict__ src, int64_t m, int d, float* __restrict__ tvec,
                                    int64_t* __restrict__ tids) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= m) return;
  const float4* s = reinterpret_cast<const float4*>(vec + src[w] * d);
  float4* o = reinterpret_cast<float4*>(tvec + w * d);
  for (int j = lane; j < d / 4; j += 32) o[j] = s[j];
  if (lane == 0) tids[w] = ids[src[w]];
}

// Loads the update kernels into the context.  With lazy module loading a
// kernel is loaded at its first launch, and that load waits for the work in
// flight on the device; an index loads them when it is installed, so that its
// first insert or delete does not wait for the searches running beside it.
void preload_update_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, descend_children_kernel);
  cudaFuncGetAttributes(&fa, nan_check_kernel);
  cudaFuncGetAttributes(&fa, relayout_kernel);
  cudaFuncGetAttributes(&fa, place_rows_kernel);
  cudaFuncGetAttributes(&fa, gather_moves_kernel);
  preload_quant_kernels();
  cudaGetLastError();
}

qk_status launch_descend_children(const float* X, int64_t n, int d, const int32_t* parent, const float* vec1,
                                  const int64_t* ids1, const int64_t* off1, const int32_t* size1, int32_t n_parent,
                                  int32_t* leaf, cudaStream_t s) {
  if (n <= 0) return QK_OK;
  descend_children_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, parent, vec1, ids1, off1, size1,
                                                                           n_parent, leaf);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_nan_check(const float* X, int64_t total, int32_t* flag, cudaStream_t s) {
  if (total <= 0) return QK_OK;
  int64_t grid = (total + 255) / 256;
  if (grid > 148 * 16) grid = 148 * 16;
  nan_check_kernel<<<(unsigned)grid, 256, 0, s>>>(X, total, flag);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_relayout(const float* old_vec, const int64_t* old_ids, const int64_t* old_off, const int64_t* new_off,
                          const int32_t* size, int32_t n_part, int d, float* new_vec, int64_t* new_ids,
                          cudaStream_t s) {
  if (n_part <= 0) return QK_OK;
  relayout_kernel<<<n_part, 256, 0, s>>>(old_vec, old_ids, old_off, new_off, size, d, new_vec, new_ids);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_place_rows(const float* X, const int64_t* ids, int64_t n, int d, const int64_t* dst, float* vec,
                            int64_t* ids_out, cudaStream_t s) {
  if (n <= 0) return QK_OK;
  place_rows_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, ids, n, d, dst, vec, ids_out);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_gather_moves(const float* vec, const int64_t* ids, const int64_t* src, int64_t m, int d, float* tvec,
                              int64_t* tids, cudaStream_t s) {
  if (m <= 0) return QK_OK;
  gather_moves_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(vec, ids, src, m, d, tvec, tids);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
