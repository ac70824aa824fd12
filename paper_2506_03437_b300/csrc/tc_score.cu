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
// neighbours are among the kT approximate ones: TF32 keeps 11 significant
// bits of each operand, which moves an approximate distance by at most about
// 2^-9 * ||x|| * ||c||.  For the nearest centroid alone the kernel keeps, per
// row, just the smallest approximate distance, its column and the runner-up
// (branch-free, so a warp's 32 rows never diverge), and a certificate on the
// gap makes the answer exact (see launch_tc_nearest).
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
// Two modes for the nearest centroid alone (k = 1), see launch_tc_nearest:
constexpr int kTop1 = 1;       // the smallest approximate distance, its column and the runner-up
constexpr int kCollect = 0;    // every column within a per-row threshold
constexpr int kCollectCap = 8; // ... at most this many per row and part of the columns
constexpr int kCollectStride = 4 + 4 * kCollectCap;   // per row: a count per part, then the lists

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
  static constexpr int kTD = (!kStore && T == kTop1) ? 2 : T;   // distances kept per row (the runner-up too)
  static constexpr int kMerge = (kStore || T == kCollect) ? 0 : (P - 1) * kM * (kTD + T) * 4;
  static constexpr int kSmem = kStages * kStageBytes + kMerge + 1024 + 256;
  static constexpr int kStride = T == kCollect ? kCollectStride : kT;   // candidate words per row
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
// dout[r * ldd + c]).  T = kTop1 keeps per row the smallest approximate
// distance, its column and the second smallest distance (cand words 0, 1, 2);
// T = kCollect lists every column whose approximate distance is <= thr[row],
// up to kCollectCap per part of the columns (words 0..3 the counts, which may
// exceed the cap, then the lists).  Work item i is row tile i / splits and the range of
// `span` centroids (whole tiles) number i % splits; the CTAs take items i =
// blockIdx.x, blockIdx.x + gridDim.x, ...  mapX / mapC are TMA tensor maps
// of X (n x d) and C (K x d) with boxes of 32 x 128 and 32 x 256 elements.
template <int T, bool kStore, int kMetric>
__global__ void __launch_bounds__(tc::Shape<T, kStore>::kThreads, 1)
    tc_score_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapC, int64_t n,
                    int d, int K, const float* __restrict__ cnorm, int metric, int32_t* __restrict__ cand,
                    int32_t* __restrict__ status, float* __restrict__ dout, int64_t ldd, int splits, int span,
                    int64_t n_items, const float* __restrict__ thr) {
  using namespace tc;
  using S = Shape<T, kStore>;
  constexpr int kMerge = S::kMerge;
  constexpr bool kTop = !kStore && T == kTop1;      // the modes of k = 1 (the store mode also has T = 1)
  constexpr bool kColl = !kStore && T == kCollect;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the stages must sit on 1024-byte boundaries (the swizzle atom)
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* mrg_d = reinterpret_cast<float*>(smem + kStages * kStageBytes);   // (P - 1) x kM x kTD
  int32_t* mrg_i = reinterpret_cast<int32_t*>(mrg_d + (S::P - 1) * kM * S::kTD);
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
      float bd[S::kTD > 0 ? S::kTD : 1];
      int32_t bi[T > 0 ? T : 1];
#pragma unroll
      for (int i = 0; i < (S::kTD > 0 ? S::kTD : 1); ++i) bd[i] = INFINITY;
#pragma unroll
      for (int i = 0; i < (T > 0 ? T : 1); ++i) bi[i] = -1;
      // kCollect: this row's threshold and how many of its columns met it
      const float my_thr = (kColl && my_row < n) ? thr[my_row] : -INFINITY;
      int n_hit = 0;
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
          if constexpr (kTop) {
            // branch-free: runner-up first (it takes the old smallest value or x)
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const float x = v[i];
              bd[1] = fminf(bd[1], fmaxf(bd[0], x));
              bi[0] = x < bd[0] ? cbase + i : bi[0];
              bd[0] = fminf(bd[0], x);
            }
            continue;
          }
          if constexpr (kColl) {
            if (my_row < n) {
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (v[i] <= my_thr) {   // rare: only columns near the row's best
                  if (n_hit < kCollectCap) cand[my_row * S::kStride + 4 + part * kCollectCap + n_hit] = cbase + i;
                  ++n_hit;
                }
            }
            continue;
          }
          // the chunk's smallest value decides whether any of its 32 can enter
          // the list; after the first chunks of a row tile most chunks cannot
          float m16[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) m16[i] = fminf(v[i], v[i + 16]);   // a tree, for independent operations
#pragma unroll
          for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
            for (int i = 0; i < w; ++i) m16[i] = fminf(m16[i], m16[i + w]);
          if (!__any_sync(0xffffffffu, m16[0] < bd[T - 1])) continue;
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
      if constexpr (kColl) {
        if (my_row < n && !*s_abort) cand[my_row * S::kStride + part] = n_hit;
      } else if constexpr (kTop) {
        // parts 1..P-1 leave (smallest, runner-up, column) in shared memory;
        // part 0 combines them (equal smallest values make the runner-up equal)
        if (part > 0) {
          mrg_d[((part - 1) * kM + my_lane) * 2] = bd[0];
          mrg_d[((part - 1) * kM + my_lane) * 2 + 1] = bd[1];
          mrg_i[(part - 1) * kM + my_lane] = bi[0];
        }
        asm volatile("bar.sync 1, %0;" ::"n"(S::kEpi) : "memory");
        if (part == 0 && my_row < n && !*s_abort) {
          for (int o = 1; o < S::P; ++o) {
            const float o0 = mrg_d[((o - 1) * kM + my_lane) * 2], o1 = mrg_d[((o - 1) * kM + my_lane) * 2 + 1];
            const int32_t oi = mrg_i[(o - 1) * kM + my_lane];
            const float nb1 = fminf(fmaxf(bd[0], o0), fminf(bd[1], o1));
            if (o0 < bd[0] || (o0 == bd[0] && oi < bi[0])) bi[0] = oi;
            bd[0] = fminf(bd[0], o0);
            bd[1] = nb1;
          }
          cand[my_row * kT] = bd[0] < INFINITY ? bi[0] : -1;
          cand[my_row * kT + 1] = __float_as_int(bd[0]);
          cand[my_row * kT + 2] = __float_as_int(bd[1]);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(S::kEpi) : "memory");   // the lists are read before reuse
      } else if (!kStore) {
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

// Exact FP32 distance of row x to centroid cc, from the direct differences
// (L2) or the products (IP, negated): each lane takes float4 j = lane,
// lane + 32, ... and the warp sums the lanes.  Every exact score of this file
// comes from here, so equal inputs give equal distances whichever path scored
// them.  With xn2, also the row's squared norm (the same loads).
__device__ __forceinline__ float exact_dist(const float* __restrict__ x, const float* __restrict__ cc, int d,
                                            int metric, int lane, float* xn2 = nullptr) {
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* c4 = reinterpret_cast<const float4*>(cc);
  float acc = 0.f, nrm = 0.f;
  for (int j = lane; j < d / 4; j += 32) {
    const float4 a = x4[j];
    if (xn2) nrm = fmaf(a.w, a.w, fmaf(a.z, a.z, fmaf(a.y, a.y, fmaf(a.x, a.x, nrm))));
    if (!cc) continue;
    const float4 b = c4[j];
    if (metric == QK_METRIC_L2) {
      const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
      acc = fmaf(dw, dw, fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, acc))));
    } else {
      acc = fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
    }
  }
  if (xn2) *xn2 = warp_sum_f(nrm);
  if (!cc) return 0.f;
  acc = warp_sum_f(acc);
  return metric == QK_METRIC_L2 ? acc : -acc;
}

// Exact FP32 re-score of the kT candidates of every row, keeping the k best by
// (distance, index).  One warp per row.
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
    const float acc = exact_dist(x, C + (int64_t)c * d, d, metric, lane);
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

// ---- the nearest centroid (k = 1), exact by certificate --------------------
// Error of an approximate distance (TF32 operands, FP32 accumulation):
//   TF32 keeps 10 of the 23 mantissa bits, so each operand is off by less
//   than 2^-10 of itself (truncated or rounded); the product of two TF32
//   values is exact in FP32, so a product is off by less than
//   (2^-9 + 2^-20) |x_i c_i|, and the FP32 accumulation of d <= 1024 terms
//   adds at most (d - 1) 2^-24 <= 2^-14 of sum |x_i c_i|.  With
//   sum |x_i c_i| <= ||x|| ||c|| (Cauchy-Schwarz) the dot product is off by
//   less than 1.035 * 2^-9 ||x|| ||c||.  ||c||^2 - 2 <x,c> doubles that and
//   adds the FP32 norm (2^-14 ||c||^2) and one rounding, so
//     |approximate - real| <= E_tc = 1.05 * 2^-8 ||x|| cmax + 2^-13 (||x|| + cmax)^2.
//   An exact FP32 score (exact_dist: d/128 + 7 roundings deep) is off by at
//   most E_ex = 2^-17 (||x|| + cmax)^2.
// If the runner-up's approximate distance exceeds the smallest one by more
// than 2 (E_tc + E_ex), no other centroid can score at or below the smallest
// one's exact score: its column is the exact FP32 nearest centroid.  The
// rows this does not settle are scored again, collecting every centroid
// within the same margin of the smallest approximate distance; the exact
// nearest centroid is among them, and is found by exact scores.
__device__ __forceinline__ float nearest_margin(float xn, float cmax) {
  const float s = xn + cmax;
  // 1%: the bound itself evaluated in FP32
  return 1.01f * 2.f * (1.05f * ldexpf(xn * cmax, -8) + (ldexpf(1.f, -13) + ldexpf(1.f, -17)) * s * s);
}

__device__ __forceinline__ float largest_norm(const float* __restrict__ cnorm, int K) {
  __shared__ float s_cmax;
  if (threadIdx.x < 32) {
    float m = 0.f;
    for (int j = threadIdx.x; j < K; j += 32) m = fmaxf(m, cnorm[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) s_cmax = sqrtf(m);
  }
  __syncthreads();
  return s_cmax;
}

// Certified rows get their nearest centroid (and its exact distance); the
// others are listed in retry with the threshold of the second pass (the
// smallest approximate distance plus the margin).  A warp takes 32 rows at a
// time: lane l decides row r0 + l, the row norms are read by the whole warp
// (coalesced float4), and the rows to retry take one slot range per warp.
__global__ void certify_top1_kernel(const float* __restrict__ X, int64_t n, int d, const float* __restrict__ C,
                                    int K, const float* __restrict__ cnorm, const int32_t* __restrict__ cand,
                                    int metric, int32_t* __restrict__ out_idx, float* __restrict__ out_dist,
                                    int32_t* __restrict__ retry, float* __restrict__ thr,
                                    int32_t* __restrict__ n_retry) {
  const float cmax = largest_norm(cnorm, K);
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; r0 < n; r0 += warps * 32) {
    const int64_t row = r0 + lane;
    int32_t i0 = -1;
    float b0 = INFINITY, b1 = INFINITY;
    if (row < n) {
      i0 = cand[row * tc::kT];
      b0 = __int_as_float(cand[row * tc::kT + 1]);
      b1 = __int_as_float(cand[row * tc::kT + 2]);
    }
    const bool valid = row < n && i0 >= 0 && i0 < K;
    // squared norms of the 32 rows and, when distances are wanted, the exact
    // distance to the row's candidate (the arithmetic of exact_dist), four
    // rows per step for loads in flight
    float my_s2 = 0.f, my_dd = 0.f;
    const int rows = (int)(n - r0 < 32 ? n - r0 : 32);
    for (int j = 0; j < rows; j += 4) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f}, dst[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (j + u >= rows) break;
        const float4* x4 = reinterpret_cast<const float4*>(X + (r0 + j + u) * d);
        const int32_t c = __shfl_sync(0xffffffffu, valid ? i0 : -1, j + u);
        const float4* c4 = reinterpret_cast<const float4*>(C + (int64_t)(c < 0 ? 0 : c) * d);
        for (int q = lane; q < d / 4; q += 32) {
          const float4 a = x4[q];
          acc[u] = fmaf(a.w, a.w, fmaf(a.z, a.z, fmaf(a.y, a.y, fmaf(a.x, a.x, acc[u]))));
          if (out_dist && c >= 0) {
            const float4 b = c4[q];
            if (metric == QK_METRIC_L2) {
              const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z, dw = a.w - b.w;
              dst[u] = fmaf(dw, dw, fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, dst[u]))));
            } else {
              dst[u] = fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, dst[u]))));
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float t = warp_sum_f(acc[u]);
        const float e = out_dist ? warp_sum_f(dst[u]) : 0.f;
        if (lane == j + u) {
          my_s2 = t;
          my_dd = metric == QK_METRIC_L2 ? e : -e;
        }
      }
    }
    const float m = nearest_margin(sqrtf(my_s2), cmax);
    const bool certified = valid && b1 - b0 > m;   // false for NaN
    if (certified) {
      out_idx[row] = i0;
      if (out_dist) out_dist[row] = my_dd;
    }
    const bool again = row < n && !certified;
    const uint32_t mask = __ballot_sync(0xffffffffu, again);
    int32_t base = 0;
    if (lane == 0 && mask) base = atomicAdd(n_retry, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (again) {
      const int32_t slot = base + __popc(mask & ((1u << lane) - 1u));
      retry[slot] = (int32_t)row;
      thr[slot] = b0 + m;
    }
  }
}

// Rows retry[0..r) of X, gathered into consecutive rows of Xg (one warp per row).
__global__ void gather_retry_kernel(const float* __restrict__ X, int d, const int32_t* __restrict__ retry, int64_t r,
                                    float* __restrict__ Xg) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= r) return;
  const float4* src = reinterpret_cast<const float4*>(X + (int64_t)retry[w] * d);
  float4* dst = reinterpret_cast<float4*>(Xg + w * d);
  for (int j = lane; j < d / 4; j += 32) dst[j] = src[j];
}

// One warp per retried row: the exact nearest among the collected centroids,
// or among all K when a part's list overflowed.  Ties go to the lower index.
__global__ void resolve_retry_kernel(const float* __restrict__ X, int d, const float* __restrict__ C, int K,
                                     const int32_t* __restrict__ retry, int64_t r, const int32_t* __restrict__ cand2,
                                     int metric, int32_t* __restrict__ out_idx, float* __restrict__ out_dist) {
  using namespace tc;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= r) return;
  const int64_t row = retry[w];
  const float* x = X + row * d;
  const int32_t* lst = cand2 + w * kCollectStride;
  // a count outside [0, cap] (a full list, or a pass that stopped on a
  // timeout, which the status word reports) means: score every centroid
  bool overflow = false;
  for (int p = 0; p < 4; ++p) overflow |= lst[p] < 0 || lst[p] > kCollectCap;
  float bd = INFINITY;
  int32_t bi = 0x7fffffff;
  auto consider = [&](int32_t c) {
    const float dd = exact_dist(x, C + (int64_t)c * d, d, metric, lane);
    if (dd < bd || (dd == bd && c < bi)) {
      bd = dd;
      bi = c;
    }
  };
  if (overflow) {
    for (int32_t c = 0; c < K; ++c) consider(c);
  } else {
    for (int p = 0; p < 4; ++p)
      for (int j = 0; j < lst[p]; ++j) {
        const int32_t c = lst[4 + p * kCollectCap + j];
        if (c >= 0 && c < K) consider(c);
      }
  }
  if (lane == 0) {
    out_idx[row] = bi == 0x7fffffff ? -1 : bi;
    if (out_dist) out_dist[row] = bi == 0x7fffffff ? INFINITY : bd;
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
                         int32_t* status, float* dout, int64_t ldd, int splits, int span, cudaStream_t s,
                         const float* thr) {
  using S = tc::Shape<T, kStore>;
  CUtensorMap mx, mc;
  QK_TRY(make_map(&mx, X, n, d, tc::kM));
  QK_TRY(make_map(&mc, C, K, d, tc::kN));
  int n_sm = 0;
  QK_TRY((prepare_kernel<T, kStore, kMetric>(&n_sm)));
  const int64_t items = (n + tc::kM - 1) / tc::kM * splits;
  const unsigned grid = (unsigned)std::min<int64_t>(items, n_sm);
  tc_score_kernel<T, kStore, kMetric><<<grid, S::kThreads, S::kSmem, s>>>(mx, mc, n, d, K, cnorm, kMetric, cand,
                                                                          status, dout, ldd, splits, span, items, thr);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

template <int T, bool kStore>
qk_status launch_score(const float* X, int64_t n, int d, const float* C, int K, const float* cnorm, int metric,
                       int32_t* cand, int32_t* status, float* dout, int64_t ldd, int splits, int span,
                       cudaStream_t s, const float* thr = nullptr) {
  if (metric == QK_METRIC_L2)
    return launch_score_m<T, kStore, QK_METRIC_L2>(X, n, d, C, K, cnorm, cand, status, dout, ldd, splits, span, s,
                                                   thr);
  return launch_score_m<T, kStore, QK_METRIC_IP>(X, n, d, C, K, cnorm, cand, status, dout, ldd, splits, span, s,
                                                 thr);
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
  if (k > 1) {
    QK_TRY((launch_score<tc::kT, false>(X, n, d, C, K, cnorm, metric, cand, status, nullptr, 0, 1, span, s)));
    rescore_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, C, cand, metric, k, out_idx, out_dist);
    QK_CUDA(cudaGetLastError());
    return QK_OK;
  }
  // k = 1: the smallest approximate distance and the runner-up of every row,
  // then the certificate, then a second pass over the rows it leaves open
  QK_TRY((launch_score<tc::kTop1, false>(X, n, d, C, K, cnorm, metric, cand, status, nullptr, 0, 1, span, s)));
  void* scratch = nullptr;
  QK_CUDA(cudaMallocAsync(&scratch, (size_t)n * 8 + 256, s));
  int32_t* retry = static_cast<int32_t*>(scratch);
  float* thr = reinterpret_cast<float*>(retry + n);
  int32_t* n_retry = reinterpret_cast<int32_t*>(thr + n);
  int n_sm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMemsetAsync(n_retry, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 8));
    certify_top1_kernel<<<grid, 256, 0, s>>>(X, n, d, C, K, cnorm, cand, metric, out_idx, out_dist, retry, thr,
                                             n_retry);
    e = cudaGetLastError();
  }
  int32_t h_retry = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_retry, n_retry, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  qk_status st = e == cudaSuccess ? QK_OK : cuda_status(e, "nearest-centroid certificate");
  if (st == QK_OK && h_retry > 0) {
    // second pass in chunks of about 256 MiB of scratch: gathered rows, the columns
    // within each row's threshold, exact scores of those
    const int64_t R = std::min<int64_t>(h_retry, std::max<int64_t>(8192, (256ll << 20) / (d * 4 + tc::kCollectStride * 4)));
    void* scratch2 = nullptr;
    e = cudaMallocAsync(&scratch2, (size_t)R * d * 4 + (size_t)R * tc::kCollectStride * 4 + 256, s);
    if (e != cudaSuccess) st = cuda_status(e, "cudaMallocAsync");
    float* Xg = static_cast<float*>(scratch2);
    int32_t* cand2 = reinterpret_cast<int32_t*>(Xg + R * d);
    for (int64_t base = 0; st == QK_OK && base < h_retry; base += R) {
      const int64_t r = std::min<int64_t>(R, h_retry - base);
      const unsigned g = (unsigned)((r * 32 + 255) / 256);
      gather_retry_kernel<<<g, 256, 0, s>>>(X, d, retry + base, r, Xg);
      st = launch_score<tc::kCollect, false>(Xg, r, d, C, K, cnorm, metric, cand2, status, nullptr, 0, 1, span, s,
                                             thr + base);
      if (st == QK_OK) {
        resolve_retry_kernel<<<g, 256, 0, s>>>(X, d, C, K, retry + base, r, cand2, metric, out_idx, out_dist);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_status(e, "nearest-centroid second pass");
      }
    }
    if (scratch2) cudaFreeAsync(scratch2, s);
  }
  cudaFreeAsync(scratch, s);
  return st;
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
