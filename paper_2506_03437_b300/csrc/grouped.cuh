// Grouped scan of (query, partition) work: the pieces shared by the batched
// fixed-nprobe search (batch.cu) and the batched APS search (aps_batch.cu).
//
// A unit is one partition x one group of G queries x one chunk of CH rows;
// one persistent launch scans the units, reading every row tile from HBM once
// for all G queries (each warp holds QW of them in registers) and writing
// each query's top-k of the unit to a candidate buffer.  The grouping kernels
// list every partition's queries contiguously and number the units; the
// merge kernel takes each query's top-k over its units.
//
// Included by more than one .cu file: the kernels that are not templates are
// static, so every object file holds its own copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "tc_common.cuh"

namespace qk {
namespace bt {

// Records the first device-side failure of a launch (code and details) in the
// index's status word and diagnostic record.
static __device__ void report_once(int32_t* status, int64_t* diag, int code, int64_t a0, int64_t a1, int64_t a2) {
  if (atomicCAS(status, DEV_OK, code) == DEV_OK) {
    diag[0] = code;
    diag[1] = a0;
    diag[2] = a1;
    diag[3] = a2;
  }
}

constexpr int kThreads = 256;     // 8 warps
constexpr int kWarps = kThreads / 32;
constexpr int kStages = 3;        // row tiles in flight per CTA
constexpr int kBuf = 64;          // per-query candidate buffer of a warp (entries)
constexpr int kMaxK = 32;
constexpr int kSelThreads = 256;
constexpr int kSelCap = 4096;     // candidates a selection may re-score
constexpr int kMaxNprobe = kSelCap / 2;

// Order-preserving map of a float onto uint32 (negative values included).
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

__device__ __forceinline__ bool pair_less(float da, int64_t ia, float db, int64_t ib) {
  return da < db || (da == db && ia < ib);
}

// Bitonic sort of 64 (distance, index) pairs held two per lane (positions
// lane and lane + 32), ascending by (distance, index).
template <class I>
__device__ __forceinline__ void warp_sort64(float& d0, I& i0, float& d1, I& i1, int lane) {
#pragma unroll
  for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride == 32) {   // size == 64: the partner of position p is p + 32, in the same lane
        const bool sw = pair_less(d1, i1, d0, i0);
        const float td = d0;
        const I ti = i0;
        d0 = sw ? d1 : d0;
        i0 = sw ? i1 : i0;
        d1 = sw ? td : d1;
        i1 = sw ? ti : i1;
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float& d = h ? d1 : d0;
          I& i = h ? i1 : i0;
          const int p = lane + 32 * h;
          const float od = __shfl_xor_sync(0xffffffffu, d, stride);
          const I oi = __shfl_xor_sync(0xffffffffu, i, stride);
          const bool up = (p & size) == 0;
          const bool lower = (p & stride) == 0;
          // in an ascending pair the lower position keeps the smaller element
          const bool keep_small = lower == up;
          const bool other_smaller = pair_less(od, oi, d, i);
          if (keep_small == other_smaller) {
            d = od;
            i = oi;
          }
        }
      }
    }
  }
}

// Bitonic sort of 32 (distance, index) pairs, one per lane, ascending.
template <class I>
__device__ __forceinline__ void warp_sort32(float& d, I& i, int lane) {
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, d, stride);
      const I oi = __shfl_xor_sync(0xffffffffu, i, stride);
      const bool up = (lane & size) == 0 || size == 32;
      const bool lower = (lane & stride) == 0;
      if ((lower == up) == pair_less(od, oi, d, i)) {
        d = od;
        i = oi;
      }
    }
  }
}

// Sorts the warp's buffer of n <= 64 entries and keeps its first min(n, k).
template <class I>
__device__ __forceinline__ int warp_compact(float* bd, I* bi, int n, int k, int lane) {
  if (n <= 32) {   // one entry per lane: the shorter network
    float d = lane < n ? bd[lane] : INFINITY;
    I i = lane < n ? bi[lane] : (I)0x7fffffff;
    __syncwarp();
    warp_sort32(d, i, lane);
    const int keep = n < k ? n : k;
    if (lane < keep) {
      bd[lane] = d;
      bi[lane] = i;
    }
    __syncwarp();
    return keep;
  }
  float d0 = lane < n ? bd[lane] : INFINITY, d1 = lane + 32 < n ? bd[lane + 32] : INFINITY;
  I i0 = lane < n ? bi[lane] : (I)0x7fffffff, i1 = lane + 32 < n ? bi[lane + 32] : (I)0x7fffffff;
  __syncwarp();
  warp_sort64(d0, i0, d1, i1, lane);
  const int keep = n < k ? n : k;
  if (lane < keep) {
    bd[lane] = d0;
    bi[lane] = i0;
  }
  if (lane + 32 < keep) {
    bd[lane + 32] = d1;
    bi[lane + 32] = i1;
  }
  __syncwarp();
  return keep;
}

// Lanes per row of the grouped scan: the smallest power of two t dividing
// row_lanes(D) with at most 32 query floats per lane (16 when a warp holds
// four queries) and at most 8 (query, per-query-kernel lane) chain pairs per
// lane.  Each lane stands in for row_lanes(D) / t lanes of the per-query
// kernel, so every shape sums a row in that kernel's order.  0: no such t.
constexpr int tpr_for(int D, int QW) {
  const int tp = row_lanes(D), fmax = QW > 2 ? 16 : 32;
  for (int t = 1; t <= tp; t <<= 1)
    if (tp % t == 0 && D / t <= fmax && QW * (tp / t) <= 8) return t;
  return 0;
}

struct ScanArgs {
  const float* vec = nullptr;
  const int64_t* ids = nullptr;
  const int64_t* off = nullptr;
  const int32_t* size = nullptr;
  const float* Q = nullptr;
  int k = 10;
  int CH = 4096;             // rows per unit
  int TR = 32;               // rows per tile
  const int32_t* order = nullptr;    // partitions by decreasing size
  const int64_t* ustart = nullptr;   // K + 1 unit offsets by rank
  int32_t K = 0;
  const int64_t* n_units = nullptr;
  const int32_t* pstart = nullptr;   // query-list offset per partition
  const int32_t* pcount = nullptr;
  const int32_t* qlist = nullptr;
  const int64_t* qcoff = nullptr;    // candidate offset per query
  int32_t* qcnt = nullptr;           // candidates written per query
  uint32_t* gtau = nullptr;          // best reported k-th distance per query (bits of a float >= 0)
  float* cd = nullptr;
  int64_t* ci = nullptr;
  unsigned long long* work = nullptr;
  int32_t* status = nullptr;
  // Rounds of the batched APS search: every (query, partition) item keeps its
  // own exact top-k.  gtau is then a fixed bound per query (the k-th distance
  // of the results the query has already consumed, which no later item can
  // loosen) and is never lowered by a unit; candidates are tagged with the
  // item's position in the query's candidate list.
  int aps = 0;
  const int32_t* qpos = nullptr;     // per query-list entry: the item's position
  int32_t* cpos = nullptr;           // per candidate: that position
  int64_t x_rows = 0;                // rows of the arena vec points to (whole-rows scan)
};

struct UnitInfo {
  int64_t unit;
  int64_t base;     // arena row of the chunk's first row
  int32_t p, qb, nq, row0, rows;
  int32_t nw, rep;  // warps holding distinct queries; copies of each (nw * rep <= 8)
};

template <int D, int QW>
__global__ void __launch_bounds__(kThreads, 2) grouped_scan_kernel(ScanArgs a) {
  constexpr int TPR = tpr_for(D, QW);
  static_assert(TPR > 0, "unsupported dimension for this query count");
  constexpr int TP = row_lanes(D);   // lanes per row of the per-query kernel
  constexpr int V = TP / TPR;        // of those, the lanes this lane stands in for
  constexpr int NV = D / 4 / TP;     // float4 chunks of one per-query-kernel lane
  constexpr int F4 = V * NV;         // float4 chunks per lane, row and query
  constexpr int RS = 32 / TPR;       // rows per warp step
  constexpr int G = kWarps * QW;
  extern __shared__ __align__(128) unsigned char smem[];
  const int tile_floats = a.TR * D;
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + sizeof(float) * kStages * tile_floats);
  float* qbd = reinterpret_cast<float*>(full + kStages);              // G x kBuf
  int32_t* qbr = reinterpret_cast<int32_t*>(qbd + G * kBuf);          // G x kBuf
  UnitInfo* su = reinterpret_cast<UnitInfo*>(qbr + G * kBuf);
  int32_t* s_n = reinterpret_cast<int32_t*>(su + 1);                  // G: list length after the unit
  int32_t* s_done = s_n + G;                 // per stage: busy warps done with its current tile
  uint32_t* s_fills = reinterpret_cast<uint32_t*>(s_done + kStages);   // per stage: copies issued so far
  uint32_t* s_pending = s_fills + kStages;   // stages with a copy in flight
  int32_t* s_abort = reinterpret_cast<int32_t*>(s_pending + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int part = lane % TPR, rsub = lane / TPR;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      s_done[s] = 0;
      s_fills[s] = 0;
    }
    *s_pending = 0;
    *s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase[kStages];
#pragma unroll
  for (int s = 0; s < kStages; ++s) phase[s] = 0u;
  const int64_t n_units = *a.n_units;

  for (;;) {
    if (tid == 0) {
      UnitInfo u;
      u.unit = (int64_t)atomicAdd(a.work, 1ull);
      if (u.unit < n_units) {
        // rank r: the last with ustart[r] <= unit (ustart[0] = 0 <= unit < ustart[K])
        int lo = 0, hi = a.K;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (a.ustart[mid] <= u.unit) lo = mid; else hi = mid;
        }
        const int p = a.order[lo];
        const int64_t local = u.unit - a.ustart[lo];
        const int32_t sp = a.size[p];
        const int32_t nch = (sp + a.CH - 1) / a.CH;
        const int32_t g = (int32_t)(local / nch), c = (int32_t)(local % nch);
        u.p = p;
        u.qb = a.pstart[p] + g * G;
        u.nq = min(G, a.pcount[p] - g * G);
        u.row0 = c * a.CH;
        u.rows = min(a.CH, sp - u.row0);
        u.base = a.off[p] + u.row0;
        u.nw = (u.nq + QW - 1) / QW;
        u.rep = kWarps / u.nw;
        // the first tiles of the unit
        const int ntiles = (u.rows + a.TR - 1) / a.TR;
        for (int t = 0; t < kStages && t < ntiles; ++t) {
          const int rows_t = min(a.TR, u.rows - t * a.TR);
          const uint32_t bytes = (uint32_t)rows_t * D * 4;
          mbar_arrive_expect_tx(&full[t], bytes);
          bulk_g2s(tiles + t * tile_floats, a.vec + (u.base + (int64_t)t * a.TR) * D, bytes, &full[t]);
          ++s_fills[t];
          atomicOr(s_pending, 1u << t);
        }
      }
      *su = u;
    }
    __syncthreads();
    const UnitInfo u = *su;
    if (u.unit >= n_units) break;
    const int ntiles = (u.rows + a.TR - 1) / a.TR;

    // this warp's queries: slots qg * QW + j of the unit's group; copy rc of
    // them scans row steps rc, rc + rep, ... of every tile
    const bool busy = warp < u.nw * u.rep;
    const int qg = busy ? warp % u.nw : 0, rc = busy ? warp / u.nw : 0;
    float4 qv[QW][F4];
    float tau[QW];
    int cnt[QW];
    int64_t qid[QW];
    int32_t qp[QW];
    bool any = false;
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      const int slot = qg * QW + j;
      qid[j] = busy && slot < u.nq ? a.qlist[u.qb + slot] : -1;
      qp[j] = a.qpos && qid[j] >= 0 ? a.qpos[u.qb + slot] : 0;
      // negated: a row element minus the query element is one packed add
      const float4* q4 = reinterpret_cast<const float4*>(a.Q + (qid[j] < 0 ? 0 : qid[j]) * D);
#pragma unroll
      for (int i = 0; i < V; ++i)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 e = q4[part + TPR * i + TP * v];
          qv[j][i * NV + v] = make_float4(-e.x, -e.y, -e.z, -e.w);
        }
      tau[j] = qid[j] < 0 ? -INFINITY : __uint_as_float(a.gtau[qid[j]]);
      cnt[j] = 0;
      any |= qid[j] >= 0;
    }

    // No CTA-wide barrier per tile: each busy warp counts itself done with a
    // stage, and the last of them refills it, so warps may run up to
    // kStages - 1 tiles apart.  Idle warps only keep their phase bits in step.
    const int nbusy = u.nw * u.rep;
    for (int t = 0; t < ntiles; ++t) {
      const int st = t % kStages;
      if (!busy) {
        phase[st] ^= 1u;
        continue;
      }
      const bool arrived = mbar_wait_bounded(&full[st], phase[st]);
      phase[st] ^= 1u;
      if (!__all_sync(0xffffffffu, arrived)) {   // the warp gives up together
        if (lane == 0) {
          atomicExch(a.status, DEV_TIMEOUT);
          atomicExch(s_abort, 1);
        }
        break;
      }
      if (lane == 0) atomicAnd(s_pending, ~(1u << st));
      const int rows_t = min(a.TR, u.rows - t * a.TR);
      const float* tile = tiles + st * tile_floats;
      if (any) {
        for (int r0 = rc * RS; r0 < rows_t; r0 += u.rep * RS) {
          const int rr = r0 + rsub;
          const bool rv = rr < rows_t;
          const float4* x4 = reinterpret_cast<const float4*>(tile + (rv ? rr : 0) * D);
          // per-query-kernel lane s = part + TPR * i sums chunks s, s + TP, ...
          // in two packed chains (elements x, y and z, w of each float4), one
          // such lane after the other
          float val[QW][V];
#pragma unroll
          for (int i = 0; i < V; ++i) {
            float2 c01[QW], c23[QW];
#pragma unroll
            for (int j = 0; j < QW; ++j) c01[j] = c23[j] = make_float2(0.f, 0.f);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              const float4 x = x4[part + TPR * i + TP * v];
#pragma unroll
              for (int j = 0; j < QW; ++j) {
                const float4 nq = qv[j][i * NV + v];
                const float2 d01 = __fadd2_rn(make_float2(x.x, x.y), make_float2(nq.x, nq.y));
                const float2 d23 = __fadd2_rn(make_float2(x.z, x.w), make_float2(nq.z, nq.w));
                c01[j] = __ffma2_rn(d01, d01, c01[j]);
                c23[j] = __ffma2_rn(d23, d23, c23[j]);
              }
            }
#pragma unroll
            for (int j = 0; j < QW; ++j) val[j][i] = (c01[j].x + c01[j].y) + (c23[j].x + c23[j].y);
          }
          // the per-query kernel's butterfly: its levels TP/2 .. TPR pair
          // lanes this lane holds, the levels below pair lanes of the row
          float acc[QW];
#pragma unroll
          for (int j = 0; j < QW; ++j) {
#pragma unroll
            for (int h = V >> 1; h > 0; h >>= 1)
#pragma unroll
              for (int i = 0; i < h; ++i) val[j][i] += val[j][i + h];
            acc[j] = val[j][0];
#pragma unroll
            for (int o = TPR >> 1; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
          }
#pragma unroll
          for (int j = 0; j < QW; ++j) {
            const bool s = part == 0 && rv && acc[j] < tau[j];
            const unsigned m = __ballot_sync(0xffffffffu, s);
            if (m) {
              float* bd = qbd + (warp * QW + j) * kBuf;
              int32_t* br = qbr + (warp * QW + j) * kBuf;
              if (s) {
                const int pos = cnt[j] + __popc(m & ((1u << lane) - 1u));
                bd[pos] = acc[j];
                br[pos] = u.row0 + t * a.TR + rr;
              }
              cnt[j] += __popc(m);
              __syncwarp();
              if (cnt[j] > kBuf - RS) {
                cnt[j] = warp_compact(bd, br, cnt[j], a.k, lane);
                if (cnt[j] == a.k) tau[j] = fminf(tau[j], bd[a.k - 1]);
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();   // this warp's reads of the stage come before its count
        if (atomicAdd(&s_done[st], 1) == nbusy - 1) {   // the last busy warp: the stage is free
          s_done[st] = 0;
          if (t + kStages < ntiles && !*(volatile int32_t*)s_abort) {
            const int tn = t + kStages;
            const int rows_n = min(a.TR, u.rows - tn * a.TR);
            const uint32_t bytes = (uint32_t)rows_n * D * 4;
            mbar_arrive_expect_tx(&full[st], bytes);
            bulk_g2s(tiles + st * tile_floats, a.vec + (u.base + (int64_t)tn * a.TR) * D, bytes, &full[st]);
            ++s_fills[st];
            atomicOr(s_pending, 1u << st);
          }
        }
      }
    }
    __syncthreads();   // every warp is done with the unit's tiles
    if (*s_abort) {
      // copies still in flight: wait for them (bounded) before the CTA leaves;
      // the n-th copy of a stage completes the phase of parity (n - 1) & 1
      if (tid == 0)
        for (int s2 = 0; s2 < kStages; ++s2)
          if (*s_pending & (1u << s2)) mbar_wait_bounded(&full[s2], (s_fills[s2] - 1u) & 1u);
      break;
    }
    // every copy sorts its lists down to k; copy 0 of each query set takes in
    // the other copies' lists and writes the unit's top-k to the candidates
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      if (qid[j] < 0) continue;
      const int n = warp_compact(qbd + (warp * QW + j) * kBuf, qbr + (warp * QW + j) * kBuf, cnt[j], a.k, lane);
      if (lane == 0) s_n[warp * QW + j] = n;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < QW; ++j) {
      if (qid[j] < 0 || rc != 0) continue;
      float* bd = qbd + (warp * QW + j) * kBuf;
      int32_t* br = qbr + (warp * QW + j) * kBuf;
      int n = s_n[warp * QW + j];
      for (int c = 1; c < u.rep; ++c) {   // n <= k and the copy's list <= k: at most 64 entries
        const int w2 = qg + c * u.nw;
        const int n2 = s_n[w2 * QW + j];
        if (lane < n2) {
          bd[n + lane] = qbd[(w2 * QW + j) * kBuf + lane];
          br[n + lane] = qbr[(w2 * QW + j) * kBuf + lane];
        }
        __syncwarp();
        n = warp_compact(bd, br, n + n2, a.k, lane);
      }
      int64_t slot = 0;
      if (lane == 0) slot = a.qcoff[qid[j]] + atomicAdd(&a.qcnt[qid[j]], a.k);
      slot = __shfl_sync(0xffffffffu, slot, 0);
      if (lane < a.k) {
        const int64_t row = a.off[u.p] + br[lane];
        a.cd[slot + lane] = lane < n ? bd[lane] : INFINITY;
        a.ci[slot + lane] = lane < n ? a.ids[row] : -1;
        if (a.cpos) a.cpos[slot + lane] = qp[j];
      }
      // L2 distances are >= 0, so their bit patterns order like the values
      if (lane == 0 && n == a.k && !a.aps) atomicMin(&a.gtau[qid[j]], __float_as_uint(bd[a.k - 1]));
      __syncwarp();
    }
    __syncthreads();
  }
}

// ------------------------------------------------ whole rows per thread

// The grouped scan with the contraction tiled in registers: every thread sums
// two whole rows against the four queries of its warp, so no lane reduction
// is needed and each shared-memory load feeds four (row loads) or eight
// (query loads) packed FP32 operations.  The queries of the unit sit in
// shared memory (read as warp-wide broadcasts).  The rows arrive by TMA tensor
// copies, one per 32-float column block of a 64-row tile, with the 128-byte
// swizzle: 16-byte chunk c of row r lands in chunk c ^ (r & 7) of the row's
// 128-byte line, so the 32 rows a warp reads at once fall on distinct banks.
// A unit holds G = 32 queries (8 warps x 4); warps without queries sit the
// unit out.
//
// Each row is summed in the per-query kernel's order (row_lanes(D) = 8 lanes
// with two packed chains each, then its butterfly), evaluated here lane by
// lane in the order 0, 4, 2, 6, 1, 5, 3, 7 that completes the butterfly's
// pairs as early as possible, so the distances equal the other kernels' bit
// for bit.
constexpr int kRowsG = kWarps * 4;   // queries per unit of the whole-rows layout

template <int D>
struct RowsLayout {
  static constexpr int kQ = 4;                 // queries per warp
  static constexpr int kR = 2;                 // rows per lane
  static constexpr int kTR = 32 * kR;          // rows per tile: one step of every warp
  static constexpr int kStg = 2;               // tiles in flight
  static constexpr int kG = kWarps * kQ;       // queries per unit
  static_assert(kG == kRowsG, "the grouping sizes units by kRowsG");
  static constexpr int kBlock = kTR * 128;     // bytes of one 32-float column block of a tile
  static constexpr int kTile = kBlock * (D / 32);
  // offsets from the 1024-byte aligned start of the dynamic shared memory
  static constexpr size_t tiles = 0;
  static constexpr size_t sq = tiles + (size_t)kStg * kTile;
  static constexpr size_t bars = sq + sizeof(float) * kG * D;
  static constexpr size_t qbd = bars + sizeof(uint64_t) * kStg;
  static constexpr size_t qbr = qbd + sizeof(float) * kG * kBuf;
  static constexpr size_t unit = qbr + sizeof(int32_t) * kG * kBuf;
  static constexpr size_t misc = unit + sizeof(UnitInfo);
  static constexpr size_t total = misc + sizeof(int32_t) * (2 * kStg + 2) + 1024;   // + alignment slack
};

// Distances of rows lane and lane + 32 of a staged tile to the warp's four
// (negated) queries in qn.
template <int D>
__device__ __forceinline__ void rows_distances(const unsigned char* tile, const float* qn, int lane,
                                               float (&out)[2][4]) {
  constexpr int TP = row_lanes(D), NV = D / 4 / TP, D4 = D / 4, BLK = RowsLayout<D>::kBlock;
  static_assert(TP == 8, "the evaluation order below is that of an 8-lane butterfly");
  const unsigned char* r0 = tile + lane * 128;
  const unsigned char* r1 = tile + (lane + 32) * 128;
  const float4* q4 = reinterpret_cast<const float4*>(qn);
  float c0[2][4], b1[2][4], pv[2][4];
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    const int s = ((kk & 1) << 2) | (kk & 2) | ((kk >> 2) & 1);   // 0, 4, 2, 6, 1, 5, 3, 7
    const int coff = (s ^ (lane & 7)) << 4;                       // chunk s of rows lane, lane + 32
    float2 c01[2][4], c23[2][4];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) c01[r][j] = c23[r][j] = make_float2(0.f, 0.f);
#pragma unroll(NV <= 4 ? NV : 2)
    for (int v = 0; v < NV; ++v) {
      // float4 s + 8 v of the row: chunk s of column block v
      const float4 xa = *reinterpret_cast<const float4*>(r0 + v * BLK + coff);
      const float4 xb = *reinterpret_cast<const float4*>(r1 + v * BLK + coff);
      const int f = s + TP * v;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 nq = q4[j * D4 + f];
        const float2 n01 = make_float2(nq.x, nq.y), n23 = make_float2(nq.z, nq.w);
        const float2 a01 = __fadd2_rn(make_float2(xa.x, xa.y), n01);
        const float2 a23 = __fadd2_rn(make_float2(xa.z, xa.w), n23);
        const float2 e01 = __fadd2_rn(make_float2(xb.x, xb.y), n01);
        const float2 e23 = __fadd2_rn(make_float2(xb.z, xb.w), n23);
        c01[0][j] = __ffma2_rn(a01, a01, c01[0][j]);
        c23[0][j] = __ffma2_rn(a23, a23, c23[0][j]);
        c01[1][j] = __ffma2_rn(e01, e01, c01[1][j]);
        c23[1][j] = __ffma2_rn(e23, e23, c23[1][j]);
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float val = (c01[r][j].x + c01[r][j].y) + (c23[r][j].x + c23[r][j].y);
        // butterfly: ((l0 + l4) + (l2 + l6)) + ((l1 + l5) + (l3 + l7))
        if (kk == 0 || kk == 2 || kk == 4 || kk == 6) pv[r][j] = val;
        if (kk == 1) c0[r][j] = pv[r][j] + val;
        if (kk == 3) c0[r][j] = c0[r][j] + (pv[r][j] + val);
        if (kk == 5) b1[r][j] = pv[r][j] + val;
        if (kk == 7) out[r][j] = c0[r][j] + (b1[r][j] + (pv[r][j] + val));
      }
  }
}

template <int D>
__global__ void __launch_bounds__(kThreads, 2)
    grouped_scan_rows_kernel(const __grid_constant__ CUtensorMap xmap, ScanArgs a) {
  using L = RowsLayout<D>;
  constexpr int Q = L::kQ, TR = L::kTR, NS = L::kStg, G = L::kG;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the swizzle pattern follows address bits 7-9: tiles start 1024-byte aligned
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* tiles = smem + L::tiles;
  float* sq = reinterpret_cast<float*>(smem + L::sq);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::bars);
  float* qbd = reinterpret_cast<float*>(smem + L::qbd);
  int32_t* qbr = reinterpret_cast<int32_t*>(smem + L::qbr);
  UnitInfo* su = reinterpret_cast<UnitInfo*>(smem + L::unit);
  int32_t* s_done = reinterpret_cast<int32_t*>(smem + L::misc);   // per stage: busy warps done with its tile
  uint32_t* s_fills = reinterpret_cast<uint32_t*>(s_done + NS);    // per stage: fills issued so far
  uint32_t* s_pending = s_fills + NS;                              // stages with a fill in flight
  int32_t* s_abort = reinterpret_cast<int32_t*>(s_pending + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      s_done[s] = 0;
      s_fills[s] = 0;
    }
    *s_pending = 0;
    *s_abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) phase[s] = 0u;
  const int64_t n_units = *a.n_units;

  for (;;) {
    if (tid == 0) {
      UnitInfo u;
      u.unit = (int64_t)atomicAdd(a.work, 1ull);
      if (u.unit < n_units) {
        int lo = 0, hi = a.K;   // rank: the last with ustart[rank] <= unit
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (a.ustart[mid] <= u.unit) lo = mid; else hi = mid;
        }
        const int p = a.order[lo];
        const int64_t local = u.unit - a.ustart[lo];
        const int32_t sp = a.size[p];
        const int32_t nch = (sp + a.CH - 1) / a.CH;
        const int32_t g = (int32_t)(local / nch), c = (int32_t)(local % nch);
        u.p = p;
        u.qb = a.pstart[p] + g * G;
        u.nq = min(G, a.pcount[p] - g * G);
        u.row0 = c * a.CH;
        u.rows = min(a.CH, sp - u.row0);
        u.base = a.off[p] + u.row0;
        u.nw = (u.nq + Q - 1) / Q;
        u.rep = 1;
      }
      *su = u;
    }
    __syncthreads();
    const UnitInfo& u = *su;   // read in place: stable until the unit's last barrier
    if (u.unit >= n_units) break;
    const int ntiles = (u.rows + TR - 1) / TR;

    // Tile t into stage t % NS (one thread): a TMA copy of 64 rows per
    // 32-float column block.  Rows past the chunk are copied too (rows past
    // the arena read as zeros) and never scored.
    auto fill = [&](int t) {
      const int st = t % NS;
      mbar_arrive_expect_tx(&full[st], (uint32_t)L::kTile);
      ++s_fills[st];
      atomicOr(s_pending, 1u << st);
      const int y = (int)(u.base + (int64_t)t * TR);
#pragma unroll
      for (int b = 0; b < D / 32; ++b)
        tc::tma_load_2d(smem_u32(tiles + (size_t)st * L::kTile + b * L::kBlock), &xmap, 32 * b, y, &full[st]);
    };
    if (tid == 0)
      for (int t = 0; t < NS && t < ntiles; ++t) fill(t);

    // the unit's queries, negated, into slots warp * Q + j (zeros past nq)
    for (int i = tid; i < G * (D / 4); i += kThreads) {
      const int slot = i / (D / 4), f = i % (D / 4);
      float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
      if (slot < u.nq) e = reinterpret_cast<const float4*>(a.Q + (int64_t)a.qlist[u.qb + slot] * D)[f];
      reinterpret_cast<float4*>(sq)[i] = make_float4(-e.x, -e.y, -e.z, -e.w);
    }
    const bool busy = warp < u.nw;
    float tau[Q];
    int cnt[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int slot = warp * Q + j;
      const int64_t qi = busy && slot < u.nq ? a.qlist[u.qb + slot] : -1;
      tau[j] = qi < 0 ? -INFINITY : __uint_as_float(a.gtau[qi]);
      cnt[j] = 0;
    }
    __syncthreads();   // the queries are in place

    const int nbusy = u.nw;
    for (int t = 0; t < ntiles; ++t) {
      const int st = t % NS;
      if (!busy) {
        phase[st] ^= 1u;
        continue;
      }
      const bool arrived = mbar_wait_bounded(&full[st], phase[st]);
      phase[st] ^= 1u;
      if (!__all_sync(0xffffffffu, arrived)) {   // the warp gives up together
        if (lane == 0) {
          atomicExch(a.status, DEV_TIMEOUT);
          atomicExch(s_abort, 1);
        }
        break;
      }
      if (lane == 0) atomicAnd(s_pending, ~(1u << st));
      const int rows_t = min(TR, u.rows - t * TR);
      float dist[2][4];
      rows_distances<D>(tiles + (size_t)st * L::kTile, sq + warp * Q * D, lane, dist);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        float* bd = qbd + (warp * Q + j) * kBuf;
        int32_t* br = qbr + (warp * Q + j) * kBuf;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int rr = lane + 32 * r;
          const bool s = rr < rows_t && dist[r][j] < tau[j];
          const unsigned m = __ballot_sync(0xffffffffu, s);
          if (m) {
            if (s) {
              const int pos = cnt[j] + __popc(m & ((1u << lane) - 1u));
              bd[pos] = dist[r][j];
              br[pos] = u.row0 + t * TR + rr;
            }
            cnt[j] += __popc(m);
            __syncwarp();
            if (cnt[j] > kBuf - 32) {
              cnt[j] = warp_compact(bd, br, cnt[j], a.k, lane);
              if (cnt[j] == a.k) tau[j] = fminf(tau[j], bd[a.k - 1]);
            }
          }
        }
      }
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        __threadfence_block();   // this warp's reads of the stage come before its count
        last = atomicAdd(&s_done[st], 1) == nbusy - 1;
        if (last) s_done[st] = 0;
      }
      if (last && t + NS < ntiles && !*(volatile int32_t*)s_abort) fill(t + NS);   // the stage is free
    }
    __syncthreads();   // every warp is done with the unit's tiles
    if (*s_abort) {
      // fills still in flight: wait for them (bounded) before the CTA leaves;
      // the n-th fill of a stage completes the phase of parity (n - 1) & 1
      if (tid == 0)
        for (int s2 = 0; s2 < NS; ++s2)
          if (*s_pending & (1u << s2)) mbar_wait_bounded(&full[s2], (s_fills[s2] - 1u) & 1u);
      break;
    }
    if (busy) {
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int slot = warp * Q + j;
        if (slot >= u.nq) continue;
        const int64_t qi = a.qlist[u.qb + slot];
        float* bd = qbd + (warp * Q + j) * kBuf;
        int32_t* br = qbr + (warp * Q + j) * kBuf;
        const int n = warp_compact(bd, br, cnt[j], a.k, lane);
        int64_t at = 0;
        if (lane == 0) at = a.qcoff[qi] + atomicAdd(&a.qcnt[qi], a.k);
        at = __shfl_sync(0xffffffffu, at, 0);
        if (lane < a.k) {
          const int64_t row = a.off[u.p] + br[lane];
          a.cd[at + lane] = lane < n ? bd[lane] : INFINITY;
          a.ci[at + lane] = lane < n ? a.ids[row] : -1;
          if (a.cpos) a.cpos[at + lane] = a.qpos[u.qb + slot];
        }
        // L2 distances are >= 0, so their bit patterns order like the values
        if (lane == 0 && n == a.k && !a.aps) atomicMin(&a.gtau[qi], __float_as_uint(bd[a.k - 1]));
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// Launches grouped_scan_rows_kernel with (SMs x CTAs an SM holds) CTAs.  The
// attribute and occupancy queries run outside stream capture and are cached
// in *per_sm; a captured launch reuses the cached value.
template <int D>
qk_status launch_rows_t(const ScanArgs& a, int n_sm, bool capturing, int* per_sm, cudaStream_t s) {
  const size_t smem = RowsLayout<D>::total;
  if (a.x_rows <= 0 || a.x_rows >= (int64_t)1 << 31) {
    set_error("whole-rows scan: the arena must hold 1 to 2^31 - 1 rows");
    return QK_ERR_ARG;
  }
  CUtensorMap xmap;
  QK_TRY(make_map(&xmap, a.vec, a.x_rows, D, RowsLayout<D>::kTR));
  if (!capturing) {
    QK_CUDA(cudaFuncSetAttribute(grouped_scan_rows_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int n = 0;
    QK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, grouped_scan_rows_kernel<D>, kThreads, smem));
    *per_sm = n > 0 ? n : 1;
  } else if (*per_sm < 1) {
    set_error("capture without a prior run of the same tiles");
    return QK_ERR_STATE;
  }
  grouped_scan_rows_kernel<D><<<n_sm * *per_sm, kThreads, smem, s>>>(xmap, a);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

// Whole rows per thread: dimensions with an 8-lane summation order (d <= 256).
inline bool rows_layout_ok(int d) {
  return d == 32 || d == 64 || d == 96 || d == 128 || d == 192 || d == 256;
}

inline qk_status launch_scan_rows(const ScanArgs& a, int d, int n_sm, bool capturing, int* per_sm, cudaStream_t s) {
  switch (d) {
    case 32: return launch_rows_t<32>(a, n_sm, capturing, per_sm, s);
    case 64: return launch_rows_t<64>(a, n_sm, capturing, per_sm, s);
    case 96: return launch_rows_t<96>(a, n_sm, capturing, per_sm, s);
    case 128: return launch_rows_t<128>(a, n_sm, capturing, per_sm, s);
    case 192: return launch_rows_t<192>(a, n_sm, capturing, per_sm, s);
    case 256: return launch_rows_t<256>(a, n_sm, capturing, per_sm, s);
    default: set_error("rows_per_thread 2 needs d <= 256"); return QK_ERR_ARG;
  }
}

// ----------------------------------------------------------------- grouping

// Exclusive scan of n int64 values by one CTA; the total goes to *total.
static __device__ void block_scan(const int64_t* in, int64_t* out, int n, int64_t* total, int64_t* s_part) {
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = (T + 31) >> 5;
  const int per = (n + T - 1) / T;
  const int b = tid * per, e = min(n, b + per);
  int64_t sum = 0;
  for (int i = b; i < e; ++i) sum += in[i];
  // the threads' sums scanned by warp shuffles, then the warps' totals by warp 0
  int64_t x = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_part[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t v = lane < nw ? s_part[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < nw) s_part[lane] = v;   // inclusive totals of warps 0..lane
    if (lane == nw - 1) *total = v;
  }
  __syncthreads();
  int64_t run = x - sum + (warp > 0 ? s_part[warp - 1] : 0);
  for (int i = b; i < e; ++i) {
    const int64_t v = in[i];
    out[i] = run;
    run += v;
  }
  __syncthreads();
}

struct GroupArgs {
  int32_t K = 0;
  int64_t nq = 0;
  int G = 16, CH = 4096, k = 10;
  const int32_t* size = nullptr;
  const int32_t* order = nullptr;
  const int32_t* pcount = nullptr;
  int32_t* pstart = nullptr;
  int64_t* tmp = nullptr;        // max(K, nq) scratch
  int64_t* tmp2 = nullptr;
  int64_t* ustart = nullptr;     // K + 1
  int64_t* n_units = nullptr;
  const int64_t* qslots = nullptr;
  int64_t* qcoff = nullptr;      // nq + 1
  int64_t cand_cap = 0;
  int32_t* status = nullptr;
  int64_t* diag = nullptr;
  const unsigned long long* asked = nullptr;   // items requested for this grouping (null: unknown)
};

static __global__ void __launch_bounds__(1024) group_kernel(GroupArgs a) {
  __shared__ int64_t s_part[1024];
  __shared__ int64_t s_tot;
  if (a.asked && *a.asked == 0ull) {   // nothing requested: no units
    if (threadIdx.x == 0) *a.n_units = 0;
    return;
  }
  // query-list offsets per partition (index order)
  for (int p = threadIdx.x; p < a.K; p += blockDim.x) a.tmp[p] = a.pcount[p];
  __syncthreads();
  block_scan(a.tmp, a.tmp2, a.K, &s_tot, s_part);
  for (int p = threadIdx.x; p < a.K; p += blockDim.x) a.pstart[p] = (int32_t)a.tmp2[p];
  __syncthreads();
  // units per partition, in order of decreasing size
  for (int r = threadIdx.x; r < a.K; r += blockDim.x) {
    const int p = a.order[r];
    const int64_t groups = (a.pcount[p] + a.G - 1) / a.G;
    const int64_t chunks = (a.size[p] + a.CH - 1) / a.CH;
    a.tmp[r] = groups * chunks;
  }
  __syncthreads();
  block_scan(a.tmp, a.ustart, a.K, &s_tot, s_part);
  const int64_t units = s_tot;
  if (threadIdx.x == 0) a.ustart[a.K] = units;
  __syncthreads();
  // candidate slots per query: k per unit that holds it
  for (int64_t q = threadIdx.x; q < a.nq; q += blockDim.x) a.tmp[q] = a.qslots[q] * a.k;
  __syncthreads();
  block_scan(a.tmp, a.qcoff, (int)a.nq, &s_tot, s_part);
  if (threadIdx.x == 0) {
    a.qcoff[a.nq] = s_tot;
    if (s_tot > a.cand_cap) {   // the plan's candidate buffer is too small: scan nothing
      *a.n_units = 0;
      report_once(a.status, a.diag, DEV_BAD_ARG, -2, s_tot, a.cand_cap);
    } else {
      *a.n_units = units;
    }
  }
}

static __global__ void fill_kernel(const int32_t* sel, const int32_t* nsel, int64_t nq, int max_nprobe, const int32_t* pstart,
                            int32_t* pcur, int32_t* qlist) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nq * max_nprobe) return;
  const int64_t q = i / max_nprobe;
  const int j = (int)(i % max_nprobe);
  if (j >= nsel[q]) return;
  const int p = sel[i];
  qlist[pstart[p] + atomicAdd(&pcur[p], 1)] = (int32_t)q;
}

// ------------------------------------------------------------------- merge

static __global__ void __launch_bounds__(kThreads) merge_kernel(const float* cd, const int64_t* ci, const int64_t* qcoff,
                                                         const int32_t* qcnt, int64_t nq, int k, int64_t* out_ids,
                                                         float* out_dist) {
  __shared__ float sbd[kWarps][kBuf];
  __shared__ int64_t sbi[kWarps][kBuf];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = blockIdx.x * (int64_t)kWarps + warp;
  if (q >= nq) return;
  float* bd = sbd[warp];
  int64_t* bi = sbi[warp];
  const int64_t o = qcoff[q];
  const int n = qcnt[q];
  int cnt = 0;
  float tau = INFINITY;
  int64_t tau_id = INT64_MAX;
  for (int b = 0; b < n; b += 32) {
    const int i = b + lane;
    float d = INFINITY;
    int64_t id = -1;
    if (i < n) {
      d = cd[o + i];
      id = ci[o + i];
    }
    const bool s = id >= 0 && pair_less(d, id, tau, tau_id);
    const unsigned m = __ballot_sync(0xffffffffu, s);
    if (s) {
      const int pos = cnt + __popc(m & ((1u << lane) - 1u));
      bd[pos] = d;
      bi[pos] = id;
    }
    cnt += __popc(m);
    __syncwarp();
    if (cnt > kBuf - 32) {
      cnt = warp_compact(bd, bi, cnt, k, lane);
      if (cnt == k) {
        tau = bd[k - 1];
        tau_id = bi[k - 1];
      }
    }
  }
  cnt = warp_compact(bd, bi, cnt, k, lane);
  if (lane < k) {
    out_dist[q * k + lane] = lane < cnt ? bd[lane] : INFINITY;
    out_ids[q * k + lane] = lane < cnt ? bi[lane] : -1;
  }
}

// Maximum squared centroid norm (float bits; every value >= 0).
static __global__ void max_norm_kernel(const float* cnorm, int K, uint32_t* out) {
  uint32_t m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K; i += gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(cnorm[i]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace bt
}  // namespace qk
