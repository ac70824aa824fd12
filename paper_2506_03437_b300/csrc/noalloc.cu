// Allocation-free variant of one Lloyd step (qk_kmeans_step_noalloc).
//
// Some callers cannot allocate device memory while they run: code inside a
// memory pool that forbids cudaMalloc/cudaFree (which would synchronise the
// device and stall a latency-critical serving loop), code that runs while a
// custom allocator owns all free memory, or embedders that must keep a fixed
// device footprint.  qk_kmeans_step allocates its FP64 per-cluster sums and
// staging buffers on every call; this variant takes only device buffers from
// the caller and keeps its one piece of scratch, the sums, in a fixed array
// that lives in the library's own device image.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its 8 MiB until the process exits.  In host code its name is
// only a host-side stand-in, not a device address (a kernel given it would
// fault, or on systems where the GPU can reach host memory silently use the
// wrong memory), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.cuh"

namespace qk {

qk_status launch_kmeans_assign(const float* X, int64_t n, int d, const float* C, int K, int32_t* assign,
                               float* best_dist, cudaStream_t s);
qk_status launch_kmeans_update(const float* X, int64_t n, int d, const int32_t* assign, const float* C_prev, int K,
                               float* C_new, double* sums, int32_t* counts, cudaStream_t s);
bool is_device_ptr(const void* p);

// Maximum K * d of one call: 2^20 FP64 sums (8 MiB).
constexpr int64_t kNoAllocMaxSums = int64_t(1) << 20;

static __device__ __align__(256) double g_noalloc_sums[kNoAllocMaxSums];

constexpr int kMaxDevices = 64;
static double* g_sums_addr[kMaxDevices] = {nullptr};
static std::mutex g_setup_mutex;

// Device address of the scratch array on the current device, looked up on
// the first call made on that device.
static qk_status scratch_address(double** out) {
  int dev = 0;
  QK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the allocation-free path");
    return QK_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_sums_addr[dev]) {
    void* p = nullptr;
    QK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_sums));
    g_sums_addr[dev] = static_cast<double*>(p);
  }
  *out = g_sums_addr[dev];
  return QK_OK;
}

}  // namespace qk

using namespace qk;

extern "C" qk_status qk_kmeans_step_noalloc(const float* x, int64_t n, int32_t d, const float* c, int32_t K,
                                            float* c_new, int32_t* assign, int32_t* counts, void* stream) {
  QK_GUARD_BEGIN
  if (!x || !c || !c_new || !assign || !counts || n < 1 || d < 1 || K < 1) {
    set_error("qk_kmeans_step_noalloc: null buffer or empty size");
    return QK_ERR_ARG;
  }
  if ((int64_t)K * d > kNoAllocMaxSums) {
    set_error("qk_kmeans_step_noalloc: K * d = " + std::to_string((int64_t)K * d) +
              " exceeds the fixed scratch of " + std::to_string(kNoAllocMaxSums) + " sums");
    return QK_ERR_ARG;
  }
  if (!is_device_ptr(x) || !is_device_ptr(c) || !is_device_ptr(c_new) || !is_device_ptr(assign) ||
      !is_device_ptr(counts)) {
    set_error("qk_kmeans_step_noalloc: every buffer must be device memory (no staging is allocated)");
    return QK_ERR_ARG;
  }
  double* sums = nullptr;
  QK_TRY(scratch_address(&sums));
  cudaStream_t s = (cudaStream_t)stream;
  // launch_kmeans_update zeroes the sums and counts before accumulating, so
  // nothing left in the array by an earlier call reaches this one.
  QK_TRY(launch_kmeans_assign(x, n, d, c, K, assign, nullptr, s));
  QK_TRY(launch_kmeans_update(x, n, d, assign, c, K, c_new, sums, counts, s));
  return QK_OK;
  QK_GUARD_END
}
