// Shared device helpers: status plumbing, mbarrier and bulk-copy (TMA) PTX
// wrappers with bounded waits, warp/block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <new>
#include <string>

#include "../../include/quake_b300.h"

namespace qk {

// ------------------------------------------------------------------ status

void set_error(const std::string& msg);
qk_status cuda_status(cudaError_t e, const char* what);

#define QK_CUDA(call)                                              \
  do {                                                             \
    cudaError_t e__ = (call);                                      \
    if (e__ != cudaSuccess) return ::qk::cuda_status(e__, #call);  \
  } while (0)

// Host exceptions (std::bad_alloc from a container, above all) must not cross
// the C interface: the body of every qk_status entry point runs inside
// QK_GUARD_BEGIN ... QK_GUARD_END.
#define QK_GUARD_BEGIN try {
#define QK_GUARD_END                                                     \
  }                                                                      \
  catch (const std::bad_alloc&) {                                        \
    ::qk::set_error("out of host memory");                               \
    return QK_ERR_OOM;                                                   \
  }                                                                      \
  catch (const std::exception& e__) {                                    \
    ::qk::set_error(std::string("unexpected host exception: ") + e__.what()); \
    return QK_ERR_INTERNAL;                                              \
  }

#define QK_TRY(call)                         \
  do {                                       \
    qk_status s__ = (call);                  \
    if (s__ != QK_OK) return s__;            \
  } while (0)

// Lanes that sum one row in the per-query search kernel (TPR of the launch
// table in search.cu).  A row's float4 chunk c belongs to lane c % lanes, which
// keeps two packed FMA chains over its chunks in order; the lanes' sums are
// added by a butterfly.  The grouped scans sum every row in exactly this
// order, so a row's distance is bitwise the same whichever kernel scans it.
constexpr int row_lanes(int d) { return d <= 256 ? 8 : 32; }

// Device-side error codes written to the index's status word.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD_ARG = 2, DEV_BAD_INDEX = 3 };

// Number of int64 words in the device diagnostic record (code, query, a, b, c, d).
constexpr int kDiagWords = 16;   // [0..7] first failure, [8] longest tile wait

// A device wait gives up after this many SM cycles (about one second).
constexpr long long kWaitBudget = 2000000000LL;

// ------------------------------------------------------------- PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete; false after the budget.
// `waited` receives the cycles spent when the first test failed (else 0).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long* waited = nullptr) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitBudget) {
      if (waited) *waited = clock64() - t0;
      return false;
    }
  }
  if (waited) *waited = clock64() - t0;
  return true;
}

__device__ __forceinline__ uint64_t mbar_raw(uint64_t* bar) {
  uint64_t v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(smem_u32(bar)) : "memory");
  return v;
}

// One-dimensional bulk copy global -> shared, completing `bytes` on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// --------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_prod_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (value, index) arg-max with ties to the lower index.
__device__ __forceinline__ void warp_argmax(double& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (v2 > v || (v2 == v && i2 < i)) {
      v = v2;
      i = i2;
    }
  }
}

}  // namespace qk
