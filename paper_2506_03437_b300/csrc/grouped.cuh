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

// ----------------------------------------------------------------- grouping

// Exclusive scan of n int64 values by one CTA; the total goes to *total.
static __device__ void block_scan(const int64_t* in, int64_t* out, int n, int64_t* total, int64_t* s_part) {
  const int tid = threadIdx.x, T = blockDim.x;
  const int per = (n + T - 1) / T;
  const int b = tid * per, e = min(n, b + per);
  int64_t sum = 0;
  for (int i = b; i < e; ++i) sum += in[i];
  s_part[tid] = sum;
  __syncthreads();
  if (tid == 0) {
    int64_t run = 0;
    for (int i = 0; i < T; ++i) {
      const int64_t v = s_part[i];
      s_part[i] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  int64_t run = s_part[tid];
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
};

static __global__ void __launch_bounds__(1024) group_kernel(GroupArgs a) {
  __shared__ int64_t s_part[1024];
  __shared__ int64_t s_tot;
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
