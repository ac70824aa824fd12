// Which caller buffers a kernel launched on the current GPU may be handed
// directly (host code only; no CUDA call here, so the rule can be checked on
// a machine without a GPU).
#pragma once

#include <cuda_runtime_api.h>

namespace qk {

// Device memory of GPU `dev` itself, or managed memory, which migrates on
// demand.  Device memory of another GPU would need peer access, which this
// library never enables: a kernel given it faults.  Host memory, pinned or
// not, is not device memory.
inline bool usable_on_device(const cudaPointerAttributes& at, int dev) {
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace qk
