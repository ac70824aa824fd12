// Scan-latency profile lambda(s) for the maintenance cost model (Sec. 4,
// "Cost Model": the latency of scanning s vectors comes from offline
// profiling; Sec. 9 profiles it again for another device or for compressed
// partitions).
//
// On the GPU a search batch is throughput-bound, so lambda(s) is the device
// time that one more scanned partition of s rows adds to a batch of
// fixed-nprobe searches, per (query, partition) item.  A throwaway one-level
// index of P partitions of s rows each, in the configuration's dimension,
// metric and storage format, is searched by Q queries at nprobe = 1 and at
// nprobe = 1 + m:
//     lambda(s) = (T(1 + m) - T(1)) / (m Q).
// The difference removes the costs that do not grow with the number of
// partitions scanned: the launch, the centroid scoring and selection, the
// result write and the exact re-rank of low-precision storage.  P is at least
// 4 per SM and the rows of one size at least about 1 GiB (more than L2)
// where 24 GiB allows, so the queries in flight read different partitions
// from HBM, as in a large index.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace qk {
namespace {

constexpr int kExtraProbes = 8;                        // m
constexpr double kRowsBytes = 1024.0 * 1024 * 1024;    // target rows per size
constexpr double kMaxRowsBytes = 24.0 * kRowsBytes;    // cap on P x rows; fewer than 9 partitions refused
constexpr double kScanBytes = 16.0 * kRowsBytes;       // target bytes scanned per launch at nprobe 1 + m
constexpr int64_t kMaxParts = 4096;
constexpr int64_t kMaxQueries = 4096;

// SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform in [-1, 1) from the top 24 bits of a hash.
__device__ __forceinline__ float unit(uint64_t key) {
  return (float)(mix64(key) >> 40) * (2.0f / 16777216.0f) - 1.0f;
}

// Partition p has centre 4 u_p (u uniform in [-1, 1)^d) and its s rows are
// centre + u_r.  C receives the centres (the leaf centroids), row r gets id r
// and label r / s.
__global__ void profile_rows_kernel(float* X, int64_t* ids, int32_t* lab, float* C, int64_t s, int64_t P, int d,
                                    uint64_t seed) {
  const int64_t n = s * P;
  const int64_t total = (n + P) * d;
  const uint64_t noise = mix64(seed + 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / d;
    const int j = (int)(i - r * d);
    const int64_t p = r < n ? r / s : r - n;
    const float centre = 4.f * unit(seed ^ mix64(((uint64_t)p << 20) + (uint64_t)j));
    if (r < n) {
      X[i] = centre + unit(noise ^ mix64((uint64_t)i));
      if (j == 0) {
        ids[r] = r;
        lab[r] = (int32_t)p;
      }
    } else {
      C[p * d + j] = centre;
    }
  }
}

// Query j sits on the centre of partition j mod P, so its first probe is
// that partition and the next ones are other, unrelated partitions.
__global__ void profile_queries_kernel(const float* C, int64_t P, int d, float* Q, int64_t nq) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq * d; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / d;
    const int j = (int)(i - r * d);
    Q[i] = C[(r % P) * d + j];
  }
}

struct Buf {
  void* p = nullptr;
  cudaStream_t s;
  explicit Buf(cudaStream_t st) : s(st) {}
  Buf(const Buf&) = delete;
  ~Buf() { release(); }
  qk_status alloc(size_t bytes) {
    QK_CUDA(cudaMallocAsync(&p, std::max<size_t>(bytes, 256), s));
    return QK_OK;
  }
  void release() {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct IndexGuard {
  qk_index* ix = nullptr;
  ~IndexGuard() { qk_destroy(ix); }
};

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

int grid_for(int64_t work, int n_sm) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)n_sm * 16));
}

// Median over `reps` timed searches at one nprobe (one untimed search first).
qk_status time_search(qk_index* ix, const float* Q, int64_t nq, int32_t k, int32_t nprobe, int reps, int64_t* oi,
                      float* od, const EventPair& ev, cudaStream_t s, double* ms) {
  QK_TRY(qk_search(ix, Q, nq, k, 0.f, nprobe, oi, od, nullptr, nullptr, s));
  std::vector<double> t;
  for (int r = 0; r < reps; ++r) {
    QK_CUDA(cudaEventRecord(ev.a, s));
    QK_TRY(qk_search(ix, Q, nq, k, 0.f, nprobe, oi, od, nullptr, nullptr, s));
    QK_CUDA(cudaEventRecord(ev.b, s));
    QK_CUDA(cudaEventSynchronize(ev.b));
    float e = 0.f;
    QK_CUDA(cudaEventElapsedTime(&e, ev.a, ev.b));
    t.push_back(e);
  }
  QK_TRY(qk_check(ix, s));
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return QK_OK;
}

qk_status profile_one(const qk_config& base, int32_t k, int64_t s_rows, int reps, int n_sm, cudaStream_t s,
                      const EventPair& ev, double* out_us) {
  const int d = base.d;
  const double part_bytes = (double)s_rows * d * sizeof(float);
  // at least 4 partitions per SM, so that the queries in flight mostly read
  // different partitions (no L2 sharing a large index would not have)
  int64_t P = std::max<int64_t>((int64_t)std::ceil(kRowsBytes / part_bytes), 4 * (int64_t)n_sm);
  P = std::min<int64_t>({P, kMaxParts, (int64_t)std::floor(kMaxRowsBytes / part_bytes)});
  if (P < kExtraProbes + 1) {
    set_error("qk_profile_scan: partition size too large to profile");
    return QK_ERR_ARG;
  }
  const int64_t nq = std::min<int64_t>(
      kMaxQueries, std::max<int64_t>(4 * (int64_t)n_sm, (int64_t)(kScanBytes / ((kExtraProbes + 1) * part_bytes))));
  const int64_t n = s_rows * P;
  qk_config c = base;
  c.n_leaf = (int32_t)P;
  c.n_parent = 0;
  IndexGuard g;
  QK_TRY(qk_create(&c, &g.ix));
  Buf X(s), ids(s), lab(s), C(s), Q(s), oi(s), od(s);
  QK_TRY(X.alloc(sizeof(float) * (size_t)n * d));
  QK_TRY(ids.alloc(sizeof(int64_t) * (size_t)n));
  QK_TRY(lab.alloc(sizeof(int32_t) * (size_t)n));
  QK_TRY(C.alloc(sizeof(float) * (size_t)P * d));
  profile_rows_kernel<<<grid_for((n + P) * d, n_sm), 256, 0, s>>>(X.as<float>(), ids.as<int64_t>(),
                                                                    lab.as<int32_t>(), C.as<float>(), s_rows, P, d,
                                                                    base.seed);
  QK_CUDA(cudaGetLastError());
  QK_TRY(qk_load(g.ix, X.as<float>(), ids.as<int64_t>(), n, C.as<float>(), lab.as<int32_t>(), nullptr, nullptr, s));
  X.release();
  ids.release();
  lab.release();
  QK_TRY(Q.alloc(sizeof(float) * (size_t)nq * d));
  QK_TRY(oi.alloc(sizeof(int64_t) * (size_t)nq * k));
  QK_TRY(od.alloc(sizeof(float) * (size_t)nq * k));
  profile_queries_kernel<<<grid_for(nq * d, n_sm), 256, 0, s>>>(C.as<float>(), P, d, Q.as<float>(), nq);
  QK_CUDA(cudaGetLastError());
  double t1 = 0, t2 = 0;
  QK_TRY(time_search(g.ix, Q.as<float>(), nq, k, 1, reps, oi.as<int64_t>(), od.as<float>(), ev, s, &t1));
  QK_TRY(time_search(g.ix, Q.as<float>(), nq, k, 1 + kExtraProbes, reps, oi.as<int64_t>(), od.as<float>(), ev, s,
                     &t2));
  *out_us = std::max(0.0, t2 - t1) * 1e3 / ((double)kExtraProbes * (double)nq);
  QK_CUDA(cudaStreamSynchronize(s));
  return QK_OK;
}

}  // namespace
}  // namespace qk

using namespace qk;

extern "C" qk_status qk_profile_scan(const qk_config* cfg, int32_t k, const int64_t* sizes, int32_t n_sizes,
                                     int32_t reps, double* out_us, void* stream) {
  QK_GUARD_BEGIN
  if (!cfg || !sizes || !out_us || n_sizes < 1 || k < 1 || k > 1024 || reps < 1) {
    set_error("qk_profile_scan: invalid arguments");
    return QK_ERR_ARG;
  }
  for (int32_t i = 0; i < n_sizes; ++i)
    if (sizes[i] < 1 || (i > 0 && sizes[i] <= sizes[i - 1])) {
      set_error("qk_profile_scan: sizes must be positive and increasing");
      return QK_ERR_ARG;
    }
  if (cfg->d < 1) {
    set_error("qk_profile_scan: invalid dimension");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, n_sm = 0;
  QK_CUDA(cudaGetDevice(&dev));
  QK_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  EventPair ev;
  QK_CUDA(cudaEventCreate(&ev.a));
  QK_CUDA(cudaEventCreate(&ev.b));
  for (int32_t i = 0; i < n_sizes; ++i) QK_TRY(profile_one(*cfg, k, sizes[i], reps, n_sm, s, ev, &out_us[i]));
  return QK_OK;
  QK_GUARD_END
}
