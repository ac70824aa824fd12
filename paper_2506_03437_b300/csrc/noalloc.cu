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
// The array is a file-scope __device__ variable of this file's module.  CUDA
// loads modules lazily, so a GPU holds the 8 MiB from the first call made on
// it (which loads the module) until the process exits.  In host code the
// array's name is only a host-side stand-in, not a device address (a kernel
// given it would fault, or on systems where the GPU can reach host memory
// silently use the wrong memory), so its device address is looked up with
// cudaGetSymbolAddress, with the device current, and passed to the kernels.
// The lookup is redone whenever the current CUDA context differs from the one
// the address was taken in (after a cudaDeviceReset the module is loaded
// again, possibly elsewhere).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "common.cuh"
#include "devmem.h"

namespace qk {

qk_status launch_kmeans_assign(const float* X, int64_t n, int d, const float* C, int K, int32_t* assign,
                               float* best_dist, cudaStream_t s);
qk_status launch_kmeans_update(const float* X, int64_t n, int d, const int32_t* assign, const float* C_prev, int K,
                               float* C_new, double* sums, int32_t* counts, cudaStream_t s);

// Maximum K * d of one call: 2^20 FP64 sums (8 MiB).
constexpr int64_t kNoAllocMaxSums = int64_t(1) << 20;

static __device__ __align__(256) double g_noalloc_sums[kNoAllocMaxSums];

constexpr int kMaxDevices = 64;
struct ScratchSlot {
  double* addr = nullptr;
  unsigned long long ctx_id = 0;   // context the address was taken in
};
static ScratchSlot g_slots[kMaxDevices];
static std::mutex g_setup_mutex;

// The id of the current CUDA context through the driver's entry points
// (resolved at run time, so the library does not link the driver library).
// False when they are unavailable or no context is current yet.
static bool current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    resolved = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(f1);
      get_id = reinterpret_cast<GetId>(f2);
    } else {
      cudaGetLastError();
    }
  }
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array on the current device: looked up on
// the first call made on that device, and again if the context changed.
static qk_status scratch_address(double** out) {
  int dev = 0;
  QK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the allocation-free path");
    return QK_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchSlot& sl = g_slots[dev];
  unsigned long long id = 0;
  if (sl.addr && current_context_id(&id) && id == sl.ctx_id) {
    *out = sl.addr;
    return QK_OK;
  }
  void* p = nullptr;
  QK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_sums));
  *out = static_cast<double*>(p);
  // cached only under a known context id; otherwise looked up again next call
  sl.addr = current_context_id(&id) ? *out : nullptr;
  sl.ctx_id = id;
  return QK_OK;
}

// Every buffer must be device memory of the current GPU (or managed memory):
// nothing is staged, so host memory cannot be used, and another GPU's memory
// would need peer access.
static qk_status check_buffer(const void* p, int dev, const char* name) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("qk_kmeans_step_noalloc: ") + name + " is not memory CUDA knows");
    return QK_ERR_ARG;
  }
  if (!usable_on_device(at, dev)) {
    set_error(std::string("qk_kmeans_step_noalloc: ") + name +
              (at.type == cudaMemoryTypeDevice ? " is device memory of another GPU"
                                               : " must be device memory (no staging is allocated)"));
    return QK_ERR_ARG;
  }
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
  int dev = 0;
  QK_CUDA(cudaGetDevice(&dev));
  QK_TRY(check_buffer(x, dev, "x"));
  QK_TRY(check_buffer(c, dev, "c"));
  QK_TRY(check_buffer(c_new, dev, "c_new"));
  QK_TRY(check_buffer(assign, dev, "assign"));
  QK_TRY(check_buffer(counts, dev, "counts"));
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
