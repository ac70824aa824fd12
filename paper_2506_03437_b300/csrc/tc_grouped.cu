// Tensor-core grouped scan of the batched APS rounds (FP32 storage, L2).
//
// A round's (query, partition) items are grouped by partition as in
// grouped.cuh, but a unit now holds up to 128 queries (one per TMEM lane) and
// a chunk of the partition's rows.  Per unit the kernel forms the dot
// products of the unit's queries with its rows on the tensor cores
// (tcgen05.mma kind::tf32, FP32 accumulation in TMEM), turns them into
// approximate squared distances ||q||^2 + ||x||^2 - 2 <q, x> and keeps, per
// query, the T rows with the smallest approximate distance among those below
// the query's bound (the k-th distance of the results Algorithm 1 has already
// taken in, plus the TF32 error margin E).  An exact pass then re-scores
// every kept row from the FP32 rows (direct differences) and keeps the k best,
// which is the item's exact top-k below the bound whenever
//   - fewer than T rows passed (every row left out is approximately above
//     bound + E, so exactly above the bound, and cannot enter R), or
//   - the T-th kept approximate distance exceeds the k-th by more than 2E
//     (every row left out is exactly worse than the k-th kept one).
// Otherwise the exact pass scans that query's rows of the unit directly.
// The candidates it leaves are those the SIMT grouped scan would leave, so the
// replay of Algorithm 1 is unchanged.
//
// E bounds the error of the approximate distance.  kind::tf32 reads the 10
// leading mantissa bits of each FP32 operand, dropping the rest, so each
// product q_i x_i moves by at most (2^-9 + 2^-20) |q_i x_i| and <q, x> by at
// most 2^-9 sum |q_i x_i| <= 2^-9 ||q|| ||x|| (Cauchy-Schwarz); the FP32
// accumulation over K <= 1024 terms adds at most 2^-14 of the same sum, and
// the norms and the final additions less than 2^-18 (||q||^2 + ||x||^2).
// The distance carries twice the dot product's error, so
//   E = 2^-8 ||q|| xmax + 2^-16 (||q||^2 + xmax^2),
// with xmax the largest row norm of the index, covers it with room to spare.
//
// The kernel has the structure of the centroid scoring kernel (tc_score.cu):
// persistent, warp 0 streams K-slices of the unit's 128 queries (gathered
// into list order beforehand) and 256 of its rows through a 4-stage TMA ring
// with the 128-byte swizzle, warp 1 issues the MMAs into one of two TMEM
// accumulators, eight epilogue warps (two per TMEM lane quarter, each half of
// the columns) read the other.  The units are taken round-robin by the CTAs,
// largest partitions first.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <stdint.h>

#include "common.cuh"
#include "grouped.cuh"
#include "tc_common.cuh"

namespace qk {
namespace tg {

constexpr int kT = 16;                    // approximate candidates kept per (query, unit)
constexpr int kEW = 8;                    // epilogue warps
constexpr int kP = kEW / 4;               // parts of the columns
constexpr int kThreads = 64 + 32 * kEW;
constexpr int kEpi = 32 * kEW;
constexpr int kG = tc::kM;                // queries per unit
constexpr int kMerge = (kP - 1) * tc::kM * kT * 8;
constexpr int kSmem = tc::kStages * tc::kStageBytes + kMerge + 1024 + 256;
constexpr int kSlot = kT + 1;             // candidate entries per (query, unit): a header, then T

struct Args {
  // the units, numbered as grouped.cuh numbers them
  const int32_t* order = nullptr;
  const int64_t* ustart = nullptr;
  int32_t K = 0;
  const int64_t* n_units = nullptr;
  const int32_t* pstart = nullptr;
  const int32_t* pcount = nullptr;
  const int32_t* size = nullptr;
  const int64_t* off = nullptr;
  int CH = 4096;
  // the round's items in list order
  const int32_t* qlist = nullptr;
  const int32_t* qpos = nullptr;
  const float* qn = nullptr;         // ||q||^2 per list entry
  const uint32_t* gtau = nullptr;    // per query: the bound (bits of a float >= 0)
  const float* xn = nullptr;         // ||x||^2 per arena row
  float xmax = 0.f;                  // the largest row norm
  const int64_t* qcoff = nullptr;
  int32_t* qcnt = nullptr;
  float* cd = nullptr;
  int64_t* ci = nullptr;
  int32_t* cpos = nullptr;
  int64_t cand_cap = 0;
  int64_t nq = 0;
  int32_t* status = nullptr;
  int64_t* diag = nullptr;
};

struct Unit {
  int64_t base;     // arena row of the chunk's first row
  int32_t qb, nq, rows, p;
};

__device__ __forceinline__ void decode(const Args& a, int64_t u, Unit& U) {
  int lo = 0, hi = a.K;   // rank: the last with ustart[rank] <= u
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.ustart[mid] <= u) lo = mid; else hi = mid;
  }
  const int p = a.order[lo];
  const int64_t local = u - a.ustart[lo];
  const int32_t sp = a.size[p];
  const int32_t nch = (sp + a.CH - 1) / a.CH;
  const int32_t g = (int32_t)(local / nch), c = (int32_t)(local % nch);
  U.p = p;
  U.qb = a.pstart[p] + g * kG;
  U.nq = min(kG, a.pcount[p] - g * kG);
  const int32_t row0 = c * a.CH;
  U.rows = min(a.CH, sp - row0);
  U.base = a.off[p] + row0;
}

__device__ __forceinline__ float error_margin(float qn, float xmax) {
  return 0.00390625f * sqrtf(qn) * xmax + 1.52587890625e-05f * (qn + xmax * xmax);   // 2^-8, 2^-16
}

// Exact FP32 squared distance of one row to the query held in shared memory,
// summed in element order by one thread (both exact paths below use it, so a
// row's distance does not depend on the path).
__device__ __forceinline__ float exact_dist(const float* __restrict__ x, const float* sq, int d) {
  float acc = 0.f;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  const float4* q4 = reinterpret_cast<const float4*>(sq);
  for (int j = 0; j < d / 4; ++j) {
    const float4 a = __ldg(x4 + j), b = q4[j];
    float df = a.x - b.x;
    acc = fmaf(df, df, acc);
    df = a.y - b.y;
    acc = fmaf(df, df, acc);
    df = a.z - b.z;
    acc = fmaf(df, df, acc);
    df = a.w - b.w;
    acc = fmaf(df, df, acc);
  }
  return acc;
}

__global__ void __launch_bounds__(kThreads, 1)
    tc_grouped_kernel(const __grid_constant__ CUtensorMap mapQ, const __grid_constant__ CUtensorMap mapX, int d,
                      Args a) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* mrg_d = reinterpret_cast<float*>(smem + kStages * kStageBytes);   // (P - 1) x kM x T
  int32_t* mrg_i = reinterpret_cast<int32_t*>(mrg_d + (kP - 1) * kM * kT);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + kMerge);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int32_t* s_abort = reinterpret_cast<volatile int32_t*>(tmem_holder + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nslices = d / kKS;
  const int64_t n_units = *a.n_units;

  if (warp == 1) tmem_alloc(tmem_holder, 2 * kN);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], kEpi);
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
    atomicExch(a.status, DEV_TIMEOUT);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t fills[kStages] = {};
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t u = blockIdx.x; u < n_units && !*s_abort; u += gridDim.x) {
        Unit U;
        decode(a, u, U);
        for (int r0 = 0; r0 < U.rows && !*s_abort; r0 += kN) {
          for (int ks = 0; ks < nslices; ++ks) {
            if (!mbar_wait_bounded(&empty[stage], phase ^ 1u)) {
              fail();
              break;
            }
            const uint32_t dst = smem_u32(smem + stage * kStageBytes);
            mbar_arrive_expect_tx(&full[stage], kStageBytes);
            tma_load_2d(dst, &mapQ, ks * kKS, U.qb, &full[stage]);
            tma_load_2d(dst + kStageA, &mapX, ks * kKS, (int)(U.base + r0), &full[stage]);
            ++fills[stage];
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
      }
      for (int i = 0; i < kStages; ++i)
        if (fills[i]) mbar_wait_bounded(&full[i], (fills[i] - 1u) & 1u);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0, acc = 0;
      uint32_t phase = 0, acc_phase = 0;
      bool issued = false;
      for (int64_t u = blockIdx.x; u < n_units && !*s_abort; u += gridDim.x) {
        Unit U;
        decode(a, u, U);
        for (int r0 = 0; r0 < U.rows && !*s_abort; r0 += kN) {
          if (!mbar_wait_bounded(&acc_empty[acc], acc_phase ^ 1u)) {
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
            for (int i = 0; i < kKS / 8; ++i)
              mma_tf32(d_tmem, smem_desc_sw128(a_base + 32 * i), smem_desc_sw128(b_base + 32 * i), kIdesc,
                       (ks > 0 || i > 0) ? 1u : 0u);
            mma_commit(&empty[stage]);
            issued = true;
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (*s_abort) break;
          mma_commit(&acc_full[acc]);
          if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1u;
          }
        }
      }
      if (issued) {
        mma_commit(drain);
        mbar_wait_bounded(drain, 0);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int quarter = warp & 3;
    const int part = (warp - 2) >> 2;
    constexpr int kPart = kN / kP;
    const int my_lane = quarter * 32 + lane;      // this thread's query within the unit
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    int acc = 0;
    uint32_t acc_phase = 0;
    // every epilogue thread walks every unit, even after an abort, so all of
    // them reach the named barriers equally often
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
      Unit U;
      decode(a, u, U);
      const bool valid = my_lane < U.nq;
      const bool warp_busy = quarter * 32 < U.nq;   // some lane of this warp holds a query
      int32_t q = -1, pos = 0;
      float qn = 0.f, thr0 = -INFINITY;
      if (valid) {
        q = a.qlist[U.qb + my_lane];
        if (q < 0 || q >= a.nq) {   // never expected: record and skip the query
          bt::report_once(a.status, a.diag, DEV_BAD_INDEX, -23, q, U.qb);
          q = 0;
        }
        pos = a.qpos[U.qb + my_lane];
        qn = a.qn[U.qb + my_lane];
        const float bound = __uint_as_float(a.gtau[q]);
        thr0 = bound >= 3.0e38f ? INFINITY : bound + error_margin(qn, a.xmax);
      }
      float bd[kT];
      int32_t bi[kT];
#pragma unroll
      for (int i = 0; i < kT; ++i) {
        bd[i] = INFINITY;
        bi[i] = -1;
      }
      float thr = thr0;   // min(bound + E, the T-th kept): a row enters only below it
      for (int r0 = 0; r0 < U.rows; r0 += kN) {
        if (*s_abort || !mbar_wait_bounded(&acc_full[acc], acc_phase)) {
          fail();
          break;
        }
        fence_after_sync();
        if (warp_busy) {
          for (int c0 = part * kPart; c0 < (part + 1) * kPart; c0 += 32) {
            const int cb = r0 + c0;   // first row of the chunk within the unit
            if (cb >= U.rows) break;
            float v[32];
            tc::tmem_ld32(lane_addr + (uint32_t)(acc * kN + c0), v);
            const float* xr = a.xn + U.base + cb;
            if (cb + 32 <= U.rows) {
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = fmaf(-2.f, v[i], qn + __ldg(xr + i));
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i) v[i] = cb + i < U.rows ? fmaf(-2.f, v[i], qn + __ldg(xr + i)) : INFINITY;
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
              const bool pass = v[i] < thr;
              if (__any_sync(0xffffffffu, pass) && pass) {
                float cdv = v[i];
                int32_t civ = cb + i;
#pragma unroll
                for (int j = 0; j < kT; ++j) {   // rows arrive in increasing order: a strict comparison
                  const bool lt = cdv < bd[j];
                  const float td = bd[j];
                  const int32_t ti = bi[j];
                  bd[j] = lt ? cdv : td;
                  bi[j] = lt ? civ : ti;
                  cdv = lt ? td : cdv;
                  civ = lt ? ti : civ;
                }
                thr = fminf(thr0, bd[kT - 1]);
              }
            }
          }
        }
        fence_before_sync();
        mbar_arrive(&acc_empty[acc]);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1u;
        }
      }
      // parts 1..P-1 leave their lists in shared memory; part 0 merges them by
      // (approximate distance, row) and writes the unit's list of the query
      if (part > 0) {
        float* od = mrg_d + ((part - 1) * kM + my_lane) * kT;
        int32_t* oi = mrg_i + ((part - 1) * kM + my_lane) * kT;
#pragma unroll
        for (int i = 0; i < kT; ++i) {
          od[i] = bd[i];
          oi[i] = bi[i];
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kEpi) : "memory");
      if (part == 0 && valid && !*s_abort) {
        for (int o = 1; o < kP; ++o) {
          const float* od = mrg_d + ((o - 1) * kM + my_lane) * kT;
          const int32_t* oi = mrg_i + ((o - 1) * kM + my_lane) * kT;
          for (int e = 0; e < kT; ++e) {
            float cdv = od[e];
            int32_t civ = oi[e];
            if (!(cdv < bd[kT - 1] || (cdv == bd[kT - 1] && civ >= 0 && civ < bi[kT - 1]))) break;
#pragma unroll
            for (int j = 0; j < kT; ++j) {
              const bool lt = cdv < bd[j] || (cdv == bd[j] && (bi[j] < 0 || civ < bi[j]));
              const float td = bd[j];
              const int32_t ti = bi[j];
              bd[j] = lt ? cdv : td;
              bi[j] = lt ? civ : ti;
              cdv = lt ? td : cdv;
              civ = lt ? ti : civ;
            }
          }
        }
        const int64_t slot = a.qcoff[q] + atomicAdd(&a.qcnt[q], kSlot);
        if (slot < 0 || slot + kSlot > a.qcoff[q + 1] || slot + kSlot > a.cand_cap) {   // never expected
          bt::report_once(a.status, a.diag, DEV_BAD_INDEX, -24, slot, a.qcoff[q + 1]);
        } else {
        a.cd[slot] = __int_as_float(U.rows);     // the header: the chunk's rows and first row
        a.ci[slot] = U.base;
        a.cpos[slot] = -2 - pos;
#pragma unroll
        for (int i = 0; i < kT; ++i) {
          a.cd[slot + 1 + i] = bd[i];
          a.ci[slot + 1 + i] = bi[i] >= 0 ? U.base + bi[i] : -1;   // arena rows for now
          a.cpos[slot + 1 + i] = pos;
        }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kEpi) : "memory");
    }
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) tmem_dealloc(tmem, 2 * kN);
}

// The round's queries in list order with their squared norms (one warp per item).
__global__ void gather_kernel(const float* __restrict__ Q, int d, const int32_t* __restrict__ qlist,
                              const int32_t* __restrict__ pstart, const int32_t* __restrict__ pcount, int K,
                              int64_t cap, int64_t nq_total, float* __restrict__ Qg, float* __restrict__ qn) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t total = (int64_t)pstart[K - 1] + pcount[K - 1];
  if (w >= total || w >= cap) return;
  const int32_t qi = qlist[w];
  if (qi < 0 || (int64_t)qi >= nq_total) return;   // never expected (the scan reports it)
  const float* src = Q + (int64_t)qi * d;
  float* dst = Qg + w * d;
  float acc = 0.f;
  for (int j = lane; j < d; j += 32) {
    const float x = src[j];
    dst[j] = x;
    acc = fmaf(x, x, acc);
  }
  acc = warp_sum_f(acc);
  if (lane == 0) qn[w] = acc;
}

// Squared norms of the live rows of every partition (one block per
// partition, one warp per row), and the largest norm (float bits).
__global__ void live_norms_kernel(const float* __restrict__ X, int d, const int64_t* __restrict__ off,
                                  const int32_t* __restrict__ size, float* __restrict__ xn, uint32_t* __restrict__ xmax2) {
  const int p = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int64_t o = off[p];
  uint32_t m = 0;
  for (int r = warp; r < size[p]; r += nw) {
    const float* x = X + (o + r) * d;
    float acc = 0.f;
    for (int j = lane; j < d; j += 32) acc = fmaf(x[j], x[j], acc);
    acc = warp_sum_f(acc);
    if (lane == 0) xn[o + r] = acc;
    m = max(m, __float_as_uint(acc));
  }
  if (lane == 0) atomicMax(xmax2, m);
}

// Exact re-score: one warp per query.  Every (query, unit) list of the round
// becomes the unit's exact top-k of the rows that may still enter R (see the
// file comment), as (distance, id) pairs tagged with the item's position; the
// header entry is left with a negative position, the unused entries get id -1.
// Each lane scores one row, so the rows of a list (or 32 rows of a fallback
// scan) are fetched together.
__global__ void __launch_bounds__(256) rescore_kernel(const float* __restrict__ Q, const float* __restrict__ X,
                                                       const int64_t* __restrict__ ids, int d, int64_t nq, int k,
                                                       const int64_t* __restrict__ qcoff,
                                                       const int32_t* __restrict__ qcnt, const uint32_t* __restrict__ gtau,
                                                       float xmax, float* cd, int64_t* ci, int32_t* cpos,
                                                       unsigned long long* fallbacks, int64_t x_rows,
                                                       int64_t cand_cap, int32_t* status, int64_t* diag) {
  extern __shared__ __align__(16) float s_q[];   // 8 x d
  __shared__ float s_bd[8][64];
  __shared__ int64_t s_bi[8][64];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = blockIdx.x * (int64_t)8 + warp;
  if (q >= nq) return;
  const int n = qcnt[q];
  if (n == 0) return;
  float* sq = s_q + warp * d;
  const float* qv = Q + q * d;
  float qn = 0.f;
  for (int j = lane; j < d; j += 32) {
    const float v = qv[j];
    sq[j] = v;
    qn = fmaf(v, v, qn);
  }
  qn = warp_sum_f(qn);
  __syncwarp();
  const float E = error_margin(qn, xmax);
  const float bound = __uint_as_float(gtau[q]);
  float* bd = s_bd[warp];
  int64_t* bi = s_bi[warp];
  if (qcoff[q] < 0 || qcoff[q] + n > cand_cap || n % kSlot != 0) {   // never expected: record and skip
    if (lane == 0) bt::report_once(status, diag, DEV_BAD_INDEX, -20, q, n);
    return;
  }
  for (int64_t g = qcoff[q]; g < qcoff[q] + n; g += kSlot) {
    int rows = __float_as_int(cd[g]);
    const int64_t base = ci[g];
    const int pos = -2 - cpos[g];
    if (base < 0 || rows < 0 || base + rows > x_rows || pos < 0) {
      if (lane == 0) bt::report_once(status, diag, DEV_BAD_INDEX, -21, base, rows);
      rows = 0;
    }
    // the approximate list: entry `lane` (lanes < T)
    const float ad = lane < kT ? cd[g + 1 + lane] : INFINITY;
    int64_t arow = lane < kT ? ci[g + 1 + lane] : -1;
    if (arow >= x_rows) {
      bt::report_once(status, diag, DEV_BAD_INDEX, -22, arow, x_rows);
      arow = -1;
    }
    const float akth = __shfl_sync(0xffffffffu, ad, k - 1);
    const float alast = __shfl_sync(0xffffffffu, ad, kT - 1);
    const bool full = __shfl_sync(0xffffffffu, arow, kT - 1) >= 0;
    float dd = INFINITY;
    int64_t did = INT64_MAX;
    if (!full || alast - akth > 2.f * E) {
      if (arow >= 0) {
        dd = exact_dist(X + arow * d, sq, d);
        did = ids[arow];
      }
      bt::warp_sort32(dd, did, lane);
    } else {
      // the list cannot vouch for the top-k: every row of the unit, exactly
      if (lane == 0 && fallbacks) atomicAdd(fallbacks, 1ull);
      int cnt = 0;
      float kd = INFINITY;
      int64_t kid = INT64_MAX;
      for (int r0 = 0; r0 < rows; r0 += 32) {
        const int r = r0 + lane;
        float acc = INFINITY;
        int64_t id = INT64_MAX;
        if (r < rows) {
          acc = exact_dist(X + (base + r) * d, sq, d);
          id = ids[base + r];
        }
        const bool s = r < rows && acc <= bound && bt::pair_less(acc, id, kd, kid);
        const unsigned m = __ballot_sync(0xffffffffu, s);
        if (s) {
          const int at = cnt + __popc(m & ((1u << lane) - 1u));
          bd[at] = acc;
          bi[at] = id;
        }
        cnt += __popc(m);
        __syncwarp();
        if (cnt > 32) {
          cnt = bt::warp_compact(bd, bi, cnt, k, lane);
          if (cnt == k) {
            kd = bd[k - 1];
            kid = bi[k - 1];
          }
        }
      }
      cnt = bt::warp_compact(bd, bi, cnt, k, lane);
      dd = lane < cnt ? bd[lane] : INFINITY;
      did = lane < cnt ? bi[lane] : INT64_MAX;
      __syncwarp();
    }
    if (lane < kT) {
      const bool keep = lane < k && dd < INFINITY;
      cd[g + 1 + lane] = keep ? dd : INFINITY;
      ci[g + 1 + lane] = keep ? did : -1;
      cpos[g + 1 + lane] = pos;
    }
    __syncwarp();
  }
}

}  // namespace tg

int tg_slot() { return tg::kSlot; }
int tg_max_k() { return 12; }   // k <= 12 leaves T - k >= 4 rows of margin for the gap check

// Squared norms of the live arena rows into xn and the largest norm into *xmax
// (synchronous: the maximum is read back).  Host work outside any capture.
qk_status tg_prepare_norms(const float* X, int d, const int64_t* off, const int32_t* size, int K, float* xn,
                           uint32_t* scratch, float* xmax, cudaStream_t s) {
  QK_CUDA(cudaMemsetAsync(scratch, 0, sizeof(uint32_t), s));
  tg::live_norms_kernel<<<K, 256, 0, s>>>(X, d, off, size, xn, scratch);
  QK_CUDA(cudaGetLastError());
  uint32_t h = 0;
  QK_CUDA(cudaMemcpyAsync(&h, scratch, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));
  float m2 = 0.f;
  std::memcpy(&m2, &h, sizeof(float));
  *xmax = sqrtf(m2);
  return QK_OK;
}

// One round's scan on the tensor cores: gather, grouped TF32 scan, exact re-score.
qk_status tg_scan(const float* Q, int64_t nq, int d, int k, const float* X, int64_t x_rows, const int64_t* ids,
                  const bt::ScanArgs& sc, const int32_t* qpos, const float* xn, float xmax, float* Qg, float* qn,
                  int64_t qg_cap, int32_t* cpos, unsigned long long* fallbacks, int64_t cand_cap, int64_t* diag,
                  int n_sm, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(tg::tc_grouped_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tg::kSmem);
  });
  QK_CUDA(err);
  tg::gather_kernel<<<(unsigned)((qg_cap * 32 + 255) / 256), 256, 0, s>>>(Q, d, sc.qlist, sc.pstart, sc.pcount,
                                                                         sc.K, qg_cap, nq, Qg, qn);
  QK_CUDA(cudaGetLastError());
  CUtensorMap mq, mx;
  QK_TRY(make_map(&mq, Qg, qg_cap, d, tc::kM));
  QK_TRY(make_map(&mx, X, x_rows, d, tc::kN));
  tg::Args a;
  a.order = sc.order;
  a.ustart = sc.ustart;
  a.K = sc.K;
  a.n_units = sc.n_units;
  a.pstart = sc.pstart;
  a.pcount = sc.pcount;
  a.size = sc.size;
  a.off = sc.off;
  a.CH = sc.CH;
  a.qlist = sc.qlist;
  a.qpos = qpos;
  a.qn = qn;
  a.gtau = sc.gtau;
  a.xn = xn;
  a.xmax = xmax;
  a.qcoff = sc.qcoff;
  a.qcnt = sc.qcnt;
  a.cd = sc.cd;
  a.ci = sc.ci;
  a.cpos = cpos;
  a.cand_cap = cand_cap;
  a.nq = nq;
  a.status = sc.status;
  a.diag = diag;
  tg::tc_grouped_kernel<<<n_sm, tg::kThreads, tg::kSmem, s>>>(mq, mx, d, a);
  QK_CUDA(cudaGetLastError());
  tg::rescore_kernel<<<(unsigned)((nq + 7) / 8), 256, sizeof(float) * 8 * d, s>>>(
      Q, X, ids, d, nq, k, sc.qcoff, sc.qcnt, sc.gtau, xmax, sc.cd, sc.ci, cpos, fallbacks, x_rows, cand_cap,
      sc.status, diag);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
