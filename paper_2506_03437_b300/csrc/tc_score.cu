// Tensor-core centroid scoring (5th-generation tensor cores: tcgen05 + TMEM).
//
// For rows X (n x d) and centroids C (K x d) the kernel forms the dot
// products X C^T with tcgen05.mma kind::tf32 (FP32 operands read as TF32,
// FP32 accumulation in tensor memory), turns them into approximate distances
//   L2: ||c||^2 - 2 <x, c>      IP: -<x, c>
// (||x||^2 is the same for every centroid of a row) and keeps, per row, the
// kT candidates with the smallest approximate distance.  An exact FP32 pass
// then re-scores those candidates from the direct differences and keeps the
// k best, so the result is the exact FP32 k-nearest set whenever the true
// neighbours are among the kT approximate ones: TF32 rounds each operand to
// 11 significant bits, which moves an approximate distance by at most about
// 2^-10 * ||x|| * ||c||.
//
// The kernel is persistent (one CTA per SM) and warp-specialised:
//   warp 0     the producer: one thread streams K-slices of 32 elements of
//              the CTA's 128 rows and of 256 centroids into a ring of shared
//              memory stages with TMA tensor copies (cp.async.bulk.tensor,
//              128-byte swizzle), each stage completing on its "full" mbarrier;
//   warp 1     the MMA issuer: one thread waits for a full stage, issues four
//              K = 8 MMAs into a 128 x 256 FP32 accumulator in TMEM and commits
//              them to the stage's "empty" mbarrier, which frees the stage for
//              the producer when the MMAs have read it;
//   warps 2.. the epilogue: several warps per quarter of the TMEM lanes (the
//              quarter a warp may read is its number mod 4), each thread one
//              row and one part of the columns; it reads the accumulator with
//              tcgen05.ld and keeps its row's candidates, and the parts' lists
//              are merged through shared memory at the end of a row tile.
// Two accumulators (all 512 TMEM columns) alternate between the MMA issuer
// and the epilogue ("acc full" / "acc empty" mbarriers), so the epilogue of
// one tile of centroids runs while the MMAs of the next one do.  No CTA-wide
// barrier sits in the main loop.  Every wait is bounded: on expiry the kernel
// records a timeout in the status word, every role leaves its loop, copies
// and MMAs still in flight are waited for (bounded), and TMEM is freed.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <mutex>
#include <stdint.h>
#include <string>

#include "common.cuh"
#include "tc_common.cuh"

namespace qk {

namespace tc {

constexpr int kT = 16;         // approximate candidates kept per row (k <= 8)
constexpr int kT1 = 4;         // ... when only the nearest centroid is wanted

// Threads of one kernel shape: warp 0 the producer, warp 1 the MMA issuer,
// then EW epilogue warps, EW / 4 per quarter of the TMEM lanes; each of
// those P = EW / 4 warps takes kN / P columns of every tile.  Keeping the
// k = 1 candidates (T = 4) is the lighter epilogue, so it gets 16 warps; the
// others 8.  Shared memory: the stages (1024-byte aligned for the swizzle),
// the candidate lists of parts 1..P-1 (distances and indices), the mbarriers
// and the TMEM address.
template <int T, bool kStore>
struct Shape {
  static constexpr int EW = (!kStore && T <= 4) ? 16 : 8;
  static constexpr int P = EW / 4;
  static constexpr int kThreads = 64 + 32 * EW;
  static constexpr int kEpi = 32 * EW;
  static constexpr int kMerge = kStore ? 0 : (P - 1) * kM * T * 8;
  static constexpr int kSmem = kStages * kStageBytes + kMerge + 1024 + 256;
};

}  // namespace tc

// Squared norm of every centroid row (one warp per row).
__global__ void row_norms_kernel(const float* __restrict__ C, int64_t K, int d, float* __restrict__ out) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= K) return;
  float acc = 0.f;
  for (int j = lane; j < d; j += 32) acc = fmaf(C[w * d + j], C[w * d + j], acc);
  acc = warp_sum_f(acc);
  if (lane == 0) out[w] = acc;
}

// Approximate top-T candidates per row (see the file comment), or with
// kStore every approximate distance written to dout (row r, centroid c at
// dout[r * ldd + c]).  Work item i is row tile i / splits and the range of
// `span` centroids (whole tiles) number i % splits; the CTAs take items i =
// blockIdx.x, blockIdx.x + gridDim.x, ...  mapX / mapC are TMA tensor maps
// of X (n x d) and C (K x d) with boxes of 32 x 128 and 32 x 256 elements.
template <int T, bool kStore, int kMetric>
__global__ void __launch_bounds__(tc::Shape<T, kStore>::kThreads, 1)
    tc_score_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapC, int64_t n,
                    int d, int K, const float* __restrict__ cnorm, int metric, int32_t* __restrict__ cand,
                    int32_t* __restrict__ status, float* __restrict__ dout, int64_t ldd, int splits, int span,
                    int64_t n_items) {
  using namespace tc;
  using S = Shape<T, kStore>;
  constexpr int kMerge = S::kMerge;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the stages must sit on 1024-byte boundaries (the swizzle atom)
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* mrg_d = reinterpret_cast<float*>(smem + kStages * kStageBytes);   // (P - 1) x kM x T
  int32_t* mrg_i = reinterpret_cast<int32_t*>(mrg_d + (S::P - 1) * kM * T);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + kMerge);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int32_t* s_abort = reinterpret_cast<volatile int32_t*>(tmem_holder + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nslices = d / kKS;

  if (warp == 1) tmem_alloc(tmem_holder, 2 * kN);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], S::kEpi);
    }
    mbar_init(drain, 1);
    *s_abort = 0;
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;
  auto fail = [&]() {
    *s_abort = 1;
    atomicExch(status, DEV_TIMEOUT);
  };
  auto range = [&](int64_t item, int64_t& row0, int& n_begin, int& n_end) {
    row0 = (item / splits) * kM;
    n_begin = (int)(item % splits) * span;
    n_end = min(K, n_begin + span);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t fills[kStages] = {};
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t item = blockIdx.x; item < n_items && !*s_abort; item += gridDim.x) {
        int64_t row0;
        int n_begin, n_end;
        range(item, row0, n_begin, n_end);
        for (int n0 = n_begin; n0 < n_end && !*s_abort; n0 += kN) {
          for (int ks = 0; ks < nslices; ++ks) {
            if (!mbar_wait_bounded(&empty[stage], phase ^ 1u)) {
              fail();
              break;
            }
            const uint32_t a_dst = smem_u32(smem + stage * kStageBytes);
            mbar_arrive_expect_tx(&full[stage], kStageBytes);
            tma_load_2d(a_dst, &mapX, ks * kKS, (int)row0, &full[stage]);
            tma_load_2d(a_dst + kStageA, &mapC, ks * kKS, n0, &full[stage]);
            ++fills[stage];
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      // copies still in flight land before the CTA leaves (the n-th fill of a
      // stage completes the phase of parity (n - 1) & 1)
      for (int i = 0; i < kStages; ++i)
        if (fills[i]) mbar_wait_bounded(&full[i], (fills[i] - 1u) & 1u);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0, acc = 0;
      uint32_t phase = 0, acc_phase = 0;
      bool issued = false;
      for (int64_t item = blockIdx.x; item < n_items && !*s_abort; item += gridDim.x) {
        int64_t row0;
        int n_begin, n_end;
        range(item, row0, n_begin, n_end);
        for (int n0 = n_begin; n0 < n_end && !*s_abort; n0 += kN) {
          if (!mbar_wait_bounded(&acc_empty[acc], acc_phase ^ 1u)) {   // the epilogue freed this accumulator
            fail();
            break;
          }
          fence_after_sync();
          const uint32_t d_tmem = tmem + (uint32_t)(acc * kN);
          for (int ks = 0; ks < nslices; ++ks) {
            if (!mbar_wait_bounded(&full[stage], phase)) {
              fail();
              break;
            }
            fence_after_sync();
            const uint32_t a_base = smem_u32(smem + stage * kStageBytes), b_base = a_base + kStageA;
#pragma unroll
            for (int i = 0; i < kKS / 8; ++i)   // K = 8 per TF32 MMA: 32 bytes into the swizzle row
              mma_tf32(d_tmem, smem_desc_sw128(a_base + 32 * i), smem_desc_sw128(b_base + 32 * i), kIdesc,
                       (ks > 0 || i > 0) ? 1u : 0u);
            mma_commit(&empty[stage]);   // the stage is free once these MMAs have read it
            issued = true;
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (*s_abort) break;
          mma_commit(&acc_full[acc]);   // the accumulator is complete
          if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1u;
          }
        }
      }
      // every MMA completes before TMEM is freed
      if (issued) {
        mma_commit(drain);
        mbar_wait_bounded(drain, 0);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;                 // the TMEM lanes this warp may read
    const int part = (warp - 2) >> 2;             // the part of the columns this warp takes
    constexpr int kPart = kN / S::P;
    const int my_lane = quarter * 32 + lane;      // this thread's row within the tile
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    int acc = 0;
    uint32_t acc_phase = 0;
    // every epilogue thread walks every item, even after an abort (then
    // without waiting), so all of them reach the named barriers equally often
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
      int64_t row0;
      int n_begin, n_end;
      range(item, row0, n_begin, n_end);
      const int64_t my_row = row0 + my_lane;
      // this row's best T (distance, column) in ascending order.  A thread
      // meets its columns in increasing order, so a strict comparison keeps
      // equal distances in column order.
      float bd[T];
      int32_t bi[T];
#pragma unroll
      for (int i = 0; i < T; ++i) {
        bd[i] = INFINITY;
        bi[i] = -1;
      }
      for (int n0 = n_begin; n0 < n_end; n0 += kN) {
        if (*s_abort || !mbar_wait_bounded(&acc_full[acc], acc_phase)) {
          fail();
          break;
        }
        fence_after_sync();
        for (int c0 = part * kPart; c0 < (part + 1) * kPart; c0 += 32) {
          float v[32];
          tc::tmem_ld32(lane_addr + (uint32_t)(acc * kN + c0), v);
          const int cbase = n0 + c0;
          if (cbase + 32 <= K && kMetric == QK_METRIC_L2) {   // all 32 columns exist: vector loads of the norms
            const float4* c4 = reinterpret_cast<const float4*>(cnorm + cbase);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float4 c = __ldg(c4 + i);
              v[4 * i] = fmaf(-2.f, v[4 * i], c.x);
              v[4 * i + 1] = fmaf(-2.f, v[4 * i + 1], c.y);
              v[4 * i + 2] = fmaf(-2.f, v[4 * i + 2], c.z);
              v[4 * i + 3] = fmaf(-2.f, v[4 * i + 3], c.w);
            }
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const int col = cbase + i;
              v[i] = col >= K ? INFINITY : (kMetric == QK_METRIC_L2 ? fmaf(-2.f, v[i], __ldg(&cnorm[col])) : -v[i]);
            }
          }
          if (kStore) {
            if (my_row < n) {
              float* dst = dout + my_row * ldd + cbase;
              if (cbase + 32 <= K && (ldd & 3) == 0) {   // 16-byte aligned stores
#pragma unroll
                for (int i = 0; i < 32; i += 4)
                  reinterpret_cast<float4*>(dst + i)[0] = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
              } else {
#pragma unroll
                for (int i = 0; i < 32; ++i)
                  if (cbase + i < K) dst[i] = v[i];
              }
            }
            continue;
          }
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const bool pass = v[i] < bd[T - 1];
            if (__any_sync(0xffffffffu, pass) && pass) {   // the insertion only where some lane needs it
              float cd = v[i];
              int32_t ci = cbase + i;
#pragma unroll
              for (int j = 0; j < T; ++j) {
                const bool lt = cd < bd[j];
                const float td = bd[j];
                const int32_t ti = bi[j];
                bd[j] = lt ? cd : td;
                bi[j] = lt ? ci : ti;
                cd = lt ? td : cd;
                ci = lt ? ti : ci;
              }
            }
          }
        }
        fence_before_sync();
        mbar_arrive(&acc_empty[acc]);   // this thread's reads of the accumulator are done
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
      if (!kStore) {
        // parts 1..P-1 leave their lists in shared memory; part 0 merges them
        // into its own by (distance, column) and writes the row's candidates
        if (part > 0) {
          float* od = mrg_d + ((part - 1) * kM + my_lane) * T;
          int32_t* oi = mrg_i + ((part - 1) * kM + my_lane) * T;
#pragma unroll
          for (int i = 0; i < T; ++i) {
            od[i] = bd[i];
            oi[i] = bi[i];
          }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(S::kEpi) : "memory");
        if (part == 0 && my_row < n && !*s_abort) {
          for (int o = 1; o < S::P; ++o) {
            const float* od = mrg_d + ((o - 1) * kM + my_lane) * T;
            const int32_t* oi = mrg_i + ((o - 1) * kM + my_lane) * T;
            for (int e = 0; e < T; ++e) {
              float cd = od[e];
              int32_t ci = oi[e];
              if (!(cd < INFINITY)) break;
#pragma unroll
              for (int j = 0; j < T; ++j) {
                const bool lt = cd < bd[j] || (cd == bd[j] && ci < bi[j]);
                const float td = bd[j];
                const int32_t ti = bi[j];
                bd[j] = lt ? cd : td;
                bi[j] = lt ? ci : ti;
                cd = lt ? td : cd;
                ci = lt ? ti : ci;
              }
            }
          }
#pragma unroll
          for (int i = 0; i < T; ++i) cand[my_row * kT + i] = bd[i] < INFINITY ? bi[i] : -1;
          for (int i = T; i < kT; ++i) cand[my_row * kT + i] = -1;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(S::kEpi) : "memory");   // the lists are read before reuse
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) tmem_dealloc(tmem, 2 * kN);
}

// Exact FP32 re-score of the kT candidates of every row (direct differences),
// keeping the k best by (distance, index).  One warp per row.
__global__ void rescore_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ C,
                               const int32_t* __restrict__ cand, int metric, int k, int32_t* __restrict__ out_idx,
                               float* __restrict__ out_dist) {
  using namespace tc;
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  const float* x = X + w * d;
  float dd = INFINITY;
  int32_t di = 0x7fffffff;
  for (int i = 0; i < kT; ++i) {
    int32_t c = cand[w * kT + i];
    if (c < 0) continue;
    const float* cc = C + (int64_t)c * d;
    float acc = 0.f;
    if (metric == QK_METRIC_L2) {
      for (int j = lane; j < d; j += 32) {
        float df = x[j] - cc[j];
        acc = fmaf(df, df, acc);
      }
    } else {
      for (int j = lane; j < d; j += 32) acc = fmaf(x[j], cc[j], acc);
    }
    acc = warp_sum_f(acc);
    if (metric != QK_METRIC_L2) acc = -acc;
    if (lane == i) {
      dd = acc;
      di = c;
    }
  }
  // rank the kT (distance, index) pairs held one per lane
  int rank = 0;
  for (int j = 0; j < kT; ++j) {
    float oj = __shfl_sync(0xffffffffu, dd, j);
    int32_t ij = __shfl_sync(0xffffffffu, di, j);
    if (j != lane && (oj < dd || (oj == dd && ij < di))) ++rank;
  }
  if (lane < kT && rank < k && di != 0x7fffffff) {
    out_idx[w * k + rank] = di;
    if (out_dist) out_dist[w * k + rank] = dd;
  }
  if (lane < k) {   // fewer than k valid candidates: pad
    int valid = __popc(__ballot_sync(0xffffffffu, lane < kT && di != 0x7fffffff));
    if (lane >= valid) {
      out_idx[w * k + lane] = -1;
      if (out_dist) out_dist[w * k + lane] = INFINITY;
    }
  }
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point, so the
// library does not link the driver library.
EncodeTiled encode_fn() {
  static const EncodeTiled fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiled) nullptr;
    }
    return reinterpret_cast<EncodeTiled>(f);
  }();
  return fn;
}

// Tensor map of a row-major FP32 matrix (rows x d) read in boxes of 32
// elements x box_rows rows with the 128-byte swizzle; rows past the end read
// as zeros.
qk_status make_map(CUtensorMap* m, const float* base, int64_t rows, int d, int box_rows) {
  const EncodeTiled enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available");
    return QK_ERR_CUDA;
  }
  if (reinterpret_cast<uintptr_t>(base) % 16 != 0) {
    set_error("tensor-core operands must be 16-byte aligned");
    return QK_ERR_ARG;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)d * 4};
  const cuuint32_t box[2] = {(cuuint32_t)tc::kKS, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return QK_ERR_CUDA;
  }
  return QK_OK;
}

// Sets the kernel's shared-memory limit once (the first call is never inside a
// stream capture) and returns the number of SMs of the current device.
template <int T, bool kStore, int kMetric>
qk_status prepare_kernel(int* n_sm) {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(tc_score_kernel<T, kStore, kMetric>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               tc::Shape<T, kStore>::kSmem);
  });
  QK_CUDA(err);
  int dev = 0;
  QK_CUDA(cudaGetDevice(&dev));
  QK_CUDA(cudaDeviceGetAttribute(n_sm, cudaDevAttrMultiProcessorCount, dev));
  return QK_OK;
}

template <int T, bool kStore, int kMetric>
qk_status launch_score_m(const float* X, int64_t n, int d, const float* C, int K, const float* cnorm, int32_t* cand,
                         int32_t* status, float* dout, int64_t ldd, int splits, int span, cudaStream_t s) {
  using S = tc::Shape<T, kStore>;
  CUtensorMap mx, mc;
  QK_TRY(make_map(&mx, X, n, d, tc::kM));
  QK_TRY(make_map(&mc, C, K, d, tc::kN));
  int n_sm = 0;
  QK_TRY((prepare_kernel<T, kStore, kMetric>(&n_sm)));
  const int64_t items = (n + tc::kM - 1) / tc::kM * splits;
  const unsigned grid = (unsigned)std::min<int64_t>(items, n_sm);
  tc_score_kernel<T, kStore, kMetric><<<grid, S::kThreads, S::kSmem, s>>>(mx, mc, n, d, K, cnorm, kMetric, cand,
                                                                          status, dout, ldd, splits, span, items);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

template <int T, bool kStore>
qk_status launch_score(const float* X, int64_t n, int d, const float* C, int K, const float* cnorm, int metric,
                       int32_t* cand, int32_t* status, float* dout, int64_t ldd, int splits, int span,
                       cudaStream_t s) {
  if (metric == QK_METRIC_L2)
    return launch_score_m<T, kStore, QK_METRIC_L2>(X, n, d, C, K, cnorm, cand, status, dout, ldd, splits, span, s);
  return launch_score_m<T, kStore, QK_METRIC_IP>(X, n, d, C, K, cnorm, cand, status, dout, ldd, splits, span, s);
}

}  // namespace

qk_status launch_tc_nearest(const float* X, int64_t n, int d, const float* C, int K, int metric, int k,
                            int32_t* out_idx, float* out_dist, float* cnorm, int32_t* cand, int32_t* status,
                            cudaStream_t s) {
  if (n <= 0) return QK_OK;
  if (d % tc::kKS != 0 || k < 1 || k > tc::kT || K < 1) return QK_ERR_ARG;
  row_norms_kernel<<<(unsigned)(((int64_t)K * 32 + 255) / 256), 256, 0, s>>>(C, K, d, cnorm);
  QK_CUDA(cudaGetLastError());
  const int span = (K + tc::kN - 1) / tc::kN * tc::kN;
  if (k == 1)
    QK_TRY((launch_score<tc::kT1, false>(X, n, d, C, K, cnorm, metric, cand, status, nullptr, 0, 1, span, s)));
  else
    QK_TRY((launch_score<tc::kT, false>(X, n, d, C, K, cnorm, metric, cand, status, nullptr, 0, 1, span, s)));
  rescore_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, C, cand, metric, k, out_idx, out_dist);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

int tc_candidates_per_row() { return tc::kT; }

// Approximate distance matrix (L2: ||c||^2 - 2 <x, c>, without ||x||^2; IP:
// -<x, c>) of every row against every centroid, written to dout with row
// stride ldd (>= K).  cnorm must hold the centroids' squared norms.  The
// centroids are split into ranges of whole tiles so that a small number of
// 128-row tiles still gives every SM work.
qk_status launch_tc_distances(const float* X, int64_t n, int d, const float* C, int K, const float* cnorm, int metric,
                              float* dout, int64_t ldd, int32_t* status, int n_sm, cudaStream_t s) {
  if (n <= 0 || K <= 0) return QK_OK;
  if (d % tc::kKS != 0 || ldd < K) return QK_ERR_ARG;
  const int64_t row_tiles = (n + tc::kM - 1) / tc::kM;
  const int col_tiles = (K + tc::kN - 1) / tc::kN;
  int splits = (int)std::min<int64_t>(col_tiles, std::max<int64_t>(1, (2LL * n_sm + row_tiles - 1) / row_tiles));
  const int tiles_per_split = (col_tiles + splits - 1) / splits;
  splits = (col_tiles + tiles_per_split - 1) / tiles_per_split;
  return launch_score<1, true>(X, n, d, C, K, cnorm, metric, nullptr, status, dout, ldd, splits,
                               tiles_per_split * tc::kN, s);
}

qk_status launch_row_norms(const float* C, int64_t K, int d, float* out, cudaStream_t s) {
  if (K <= 0) return QK_OK;
  row_norms_kernel<<<(unsigned)((K * 32 + 255) / 256), 256, 0, s>>>(C, K, d, out);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
