// Dispatch of the search kernel by dimension, and the FP64 cap-volume
// kernels (beta table, cap-fraction probe).  The search kernel itself is in
// search_impl.cuh; each dimension is instantiated in its own file
// (search_d<d>.cu) so that the ten instantiations compile in parallel.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "capvol.cuh"
#include "common.cuh"
#include "index.cuh"

namespace qk {

// Defined in search_impl.cuh, instantiated in search_d<d>.cu.
template <int TPR, int NV>
qk_status launch_one(const SearchArgs& a, cudaStream_t stream);

qk_status launch_search(const SearchArgs& a, cudaStream_t stream) {
  switch (a.d) {
    case 32: return launch_one<8, 1>(a, stream);
    case 64: return launch_one<8, 2>(a, stream);
    case 96: return launch_one<8, 3>(a, stream);
    case 128: return launch_one<8, 4>(a, stream);
    case 192: return launch_one<8, 6>(a, stream);
    case 256: return launch_one<8, 8>(a, stream);
    case 384: return launch_one<32, 3>(a, stream);
    case 512: return launch_one<32, 4>(a, stream);
    case 768: return launch_one<32, 6>(a, stream);
    case 1024: return launch_one<32, 8>(a, stream);
    default:
      set_error("unsupported dimension");
      return QK_ERR_ARG;
  }
}

// ------------------------------------------------------- cap-fraction probe

__global__ void cap_fraction_kernel(int mode, double a_, double lnB, const double* table, const double* t,
                                    const double* rho, int64_t n, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = mode == QK_BETA_EXACT ? cap_fraction_exact(t[i], rho[i], a_, lnB) : cap_fraction_table(t[i], rho[i], table);
}

__global__ void beta_table_kernel(double a_, double lnB, double* table) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= kBetaTablePoints) return;
  table[j] = inc_beta(a_, 0.5, (double)j / (kBetaTablePoints - 1), lnB);
}

qk_status launch_beta_table(double a_, double lnB, double* table, cudaStream_t stream) {
  beta_table_kernel<<<(kBetaTablePoints + 255) / 256, 256, 0, stream>>>(a_, lnB, table);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_cap_fraction(int mode, double a_, double lnB, const double* table, const double* t,
                              const double* rho, int64_t n, double* out, cudaStream_t stream) {
  if (n <= 0) return QK_OK;
  cap_fraction_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(mode, a_, lnB, table, t, rho, n, out);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
