// Query-time hot path: root scoring, Adaptive Partition Scanning at every
// level and the fused distance + top-k partition scan, in one persistent
// kernel.
//
// One CTA runs one query at a time through the whole tree and takes the next
// query from a work-stealing counter, so thousands of queries with different
// APS depths share one launch.  Within a query the CTA follows Algorithm 1
// exactly (Sec. 5): the scan order depends on the k-th distance after every
// partition, so the partitions of one query are scanned one after another,
// while the CTAs of other queries keep the memory system busy.
//
// A partition is a contiguous run of rows in the arena.  It streams through a
// ring of shared-memory stages filled by one-dimensional bulk copies
// (cp.async.bulk, the TMA engine) that complete on per-stage mbarriers; every
// row is read from HBM once per (query, partition) and never from registers
// of another CTA.  Each row is reduced by TPR adjacent lanes that hold the
// matching slice of the query in registers.  Rows whose distance does not beat
// the current k-th distance are dropped at once; the rest are appended to a
// small survivor buffer that is merged into the sorted result set R with a
// bitonic sort, so R always holds the k smallest (distance, id) pairs.
//
// The estimator (Eq. 7-9) runs in FP64 over the candidate list held in shared
// memory, with the cap fraction taken from the 1024-point table or the exact
// continued fraction.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "capvol.cuh"
#include "common.cuh"
#include "index.cuh"

namespace qk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kBufCap = 256;

// Tiles in flight per CTA: four, or three when four tiles would take more than
// 64 KB (large d), so that two CTAs still fit on an SM.
__host__ __device__ constexpr int stages_for(int tile_floats) { return tile_floats * 4 * 4 > 65536 ? 3 : 4; }

__host__ __device__ inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// Shared-memory layout, computed identically on host and device.
struct SmemLayout {
  size_t stages, bars, q, sd, sid, cpart, cD, ct, cp, csc, total;
  int sortn;
  __host__ __device__ SmemLayout(int tile_floats, int d, int kcap, int mcap) {
    sortn = 2 * kcap + kBufCap;   // R, the survivor buffer, the merge output
    size_t o = 0;
    auto take = [&](size_t bytes, size_t align) {
      o = (o + align - 1) / align * align;
      size_t at = o;
      o += bytes;
      return at;
    };
    stages = take(sizeof(float) * (size_t)tile_floats * stages_for(tile_floats), 128);
    bars = take(sizeof(uint64_t) * stages_for(tile_floats), 8);
    q = take(sizeof(float) * d, 16);
    sd = take(sizeof(float) * sortn, 16);
    sid = take(sizeof(int64_t) * sortn, 16);
    cpart = take(sizeof(int32_t) * mcap, 16);
    cD = take(sizeof(float) * mcap, 16);
    ct = take(sizeof(double) * mcap, 16);
    cp = take(sizeof(double) * mcap, 16);
    csc = take(sizeof(uint8_t) * mcap, 16);
    total = o;
  }
};

struct Scalars {
  int64_t qi;
  double rho;        // current k-th radius (APS)
  double r;          // current recall estimate (APS)
  int32_t next;      // next candidate position (APS)
  int32_t go;        // APS continues
  int32_t buf_count;
  int32_t r_count;
  float thr;
  uint32_t issued;   // tiles issued so far (thread 0 writes)
};

// Element types of a scanned row.  load4 returns the 4 consecutive elements
// starting at element 4 * i as FP32 (FP8 multiplied by the partition scale).
struct ElemF32 {
  static constexpr int kBytes = 4;
  __device__ static float4 load4(const unsigned char* row, int i, float) {
    return reinterpret_cast<const float4*>(row)[i];
  }
};
struct ElemBF16 {
  static constexpr int kBytes = 2;
  __device__ static float4 load4(const unsigned char* row, int i, float) {
    uint2 u = reinterpret_cast<const uint2*>(row)[i];
    return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u));
  }
};
struct ElemFP8 {
  static constexpr int kBytes = 1;
  __device__ static float4 load4(const unsigned char* row, int i, float scale) {
    uint32_t u = reinterpret_cast<const uint32_t*>(row)[i];
    __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xffffu), __NV_E4M3);
    __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3);
    const float2 sc = make_float2(scale, scale);
    const float2 a = __fmul2_rn(__half22float2(*reinterpret_cast<__half2*>(&lo)), sc);
    const float2 b = __fmul2_rn(__half22float2(*reinterpret_cast<__half2*>(&hi)), sc);
    return make_float4(a.x, a.y, b.x, b.y);
  }
};

template <int TPR, int NV>
struct Block {
  static constexpr int D = NV * 4 * TPR;
  static_assert(TPR == row_lanes(D), "the grouped scans follow this kernel's summation order");
  // The first lane holding row i of a tile step after the reduce-scatter of rpt rows.
  static __device__ __forceinline__ constexpr int row_judge(int i, int rpt) {
    int lane = 0, o = TPR / 2;
    for (int h = rpt / 2; h >= 1; h >>= 1, o >>= 1)
      if (i & h) lane += o;
    return lane;
  }
  static constexpr int ROWS = kThreads / TPR;
  static constexpr int TILE = ROWS * D;
  static constexpr int STAGES = stages_for(TILE);

  float* stages;
  uint64_t* bars;
  float* sq;
  float* sd;
  int64_t* sid;
  int32_t* cpart;
  float* cD;
  double* ct;
  double* cp;
  uint8_t* csc;
  Scalars* s;
  uint32_t consumed;  // tiles consumed (uniform across the CTA)
  int tid, lane, warp;
  float4 qv[NV];
  int metric, beta_mode;
  double tau_rho, beta_a, beta_lnB;
  const double* beta_table;
  int32_t* status;
  int64_t* diag;
  int64_t qi;
  const unsigned char* lp_vec;   // level-0 low-precision rows (BF16 or FP8), or NULL
  const float* lp_scale;         // FP8 scale per level-0 partition
  float qn;                      // ||q||^2 (inner product radius)
  long long max_wait;   // longest tile wait of this thread, in SM cycles
  bool aborted;         // a tile wait expired (uniform across the CTA)
  int32_t* rec;         // scanned-partition record of the current query and level, or NULL
  int rec_cap, rec_n;   // its length; partitions scanned so far (thread 0)

  // Records the first failure of the launch (code, query, details) and keeps going.
  __device__ void report(int code, int64_t a0, int64_t a1, int64_t a2) {
    if (atomicCAS(status, 0, code) == 0) {
      diag[0] = code;
      diag[1] = qi;
      diag[2] = a0;
      diag[3] = a1;
      diag[4] = a2;
    }
  }

  // -------------------------------------------------------------- top-k
  __device__ static bool key_less(float d1, int64_t i1, float d2, int64_t i2) {
    return d1 < d2 || (d1 == d2 && i1 < i2);
  }

  __device__ void reset_R(int K) {
    for (int i = tid; i < K; i += kThreads) {
      sd[i] = INFINITY;
      sid[i] = INT64_MAX;
    }
    if (tid == 0) {
      s->r_count = 0;
      s->buf_count = 0;
      s->thr = INFINITY;
    }
    __syncthreads();
  }

  // Sorts the survivor buffer [K, K + cnt) in place.  Up to 32 survivors are
  // sorted by one warp with shuffles; more by a CTA bitonic network.
  __device__ void sort_buffer(int K, int cnt) {
    float* bd = sd + K;
    int64_t* bi = sid + K;
    if (cnt > 32 && cnt <= 64) {
      // one warp, two elements per lane (positions 2 lane and 2 lane + 1)
      if (warp == 0) {
        float d0 = 2 * lane < cnt ? bd[2 * lane] : INFINITY;
        int64_t i0 = 2 * lane < cnt ? bi[2 * lane] : INT64_MAX;
        float d1 = 2 * lane + 1 < cnt ? bd[2 * lane + 1] : INFINITY;
        int64_t i1 = 2 * lane + 1 < cnt ? bi[2 * lane + 1] : INT64_MAX;
#pragma unroll
        for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
          for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 1) {   // the pair (2 lane, 2 lane + 1) sits in this lane
              bool up = ((2 * lane) & k) == 0;
              bool sw = up ? key_less(d1, i1, d0, i0) : key_less(d0, i0, d1, i1);
              if (sw) {
                float td = d0;
                int64_t ti = i0;
                d0 = d1;
                i0 = i1;
                d1 = td;
                i1 = ti;
              }
            } else {        // partner positions differ by j: lane ^ (j / 2), same slot
              int pl = j >> 1;
              bool lower = (lane & pl) == 0;
              bool up = ((2 * lane) & k) == 0;
              bool take_min = lower == up;
              float od0 = __shfl_xor_sync(0xffffffffu, d0, pl);
              int64_t oi0 = __shfl_xor_sync(0xffffffffu, i0, pl);
              float od1 = __shfl_xor_sync(0xffffffffu, d1, pl);
              int64_t oi1 = __shfl_xor_sync(0xffffffffu, i1, pl);
              bool l0 = key_less(od0, oi0, d0, i0), l1 = key_less(od1, oi1, d1, i1);
              if (take_min ? l0 : (!l0 && (od0 != d0 || oi0 != i0))) {
                d0 = od0;
                i0 = oi0;
              }
              if (take_min ? l1 : (!l1 && (od1 != d1 || oi1 != i1))) {
                d1 = od1;
                i1 = oi1;
              }
            }
          }
        }
        if (2 * lane < cnt) {
          bd[2 * lane] = d0;
          bi[2 * lane] = i0;
        }
        if (2 * lane + 1 < cnt) {
          bd[2 * lane + 1] = d1;
          bi[2 * lane + 1] = i1;
        }
      }
      __syncthreads();
      return;
    }
    if (cnt <= 32) {
      if (warp == 0) {
        float d = lane < cnt ? bd[lane] : INFINITY;
        int64_t id = lane < cnt ? bi[lane] : INT64_MAX;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
          for (int j = k >> 1; j > 0; j >>= 1) {
            float od = __shfl_xor_sync(0xffffffffu, d, j);
            int64_t oi = __shfl_xor_sync(0xffffffffu, id, j);
            bool take_min = ((lane & j) == 0) == ((lane & k) == 0);
            bool other_less = key_less(od, oi, d, id);
            if (take_min ? other_less : (!other_less && (od != d || oi != id))) {
              d = od;
              id = oi;
            }
          }
        }
        if (lane < cnt) {
          bd[lane] = d;
          bi[lane] = id;
        }
      }
      __syncthreads();
      return;
    }
    int n = next_pow2(cnt);
    for (int i = cnt + tid; i < n; i += kThreads) {
      bd[i] = INFINITY;
      bi[i] = INT64_MAX;
    }
    __syncthreads();
    for (int k = 2; k <= n; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < n; i += kThreads) {
          int p = i ^ j;
          if (p > i) {
            float di = bd[i], dp = bd[p];
            int64_t ii = bi[i], ip = bi[p];
            bool up = (i & k) == 0;
            bool sw = up ? key_less(dp, ip, di, ii) : key_less(di, ii, dp, ip);
            if (sw) {
              bd[i] = dp;
              bd[p] = di;
              bi[i] = ip;
              bi[p] = ii;
            }
          }
        }
        __syncthreads();
      }
    }
  }

  // Merges the survivor buffer [K, K + cnt) into the sorted R = [0, K): the
  // buffer is sorted, then every element of R and of the buffer finds its rank
  // in the union by binary search in the other list (keys (dist, id) are
  // unique) and the first K land in R.  Called by the whole CTA with the same cnt.
  __device__ void merge(int K, int cnt) {
    sort_buffer(K, cnt);
    const int rc = s->r_count;
    const float* bd = sd + K;
    const int64_t* bi = sid + K;
    float* od = sd + K + kBufCap;
    int64_t* oi = sid + K + kBufCap;
    for (int e = tid; e < rc + cnt; e += kThreads) {
      float d;
      int64_t id;
      int rank;
      if (e < rc) {
        d = sd[e];
        id = sid[e];
        int lo = 0, hi = cnt;   // buffer elements below (d, id)
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (key_less(bd[mid], bi[mid], d, id)) lo = mid + 1; else hi = mid;
        }
        rank = e + lo;
      } else {
        int m = e - rc;
        d = bd[m];
        id = bi[m];
        int lo = 0, hi = rc;    // R elements below (d, id)
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (key_less(sd[mid], sid[mid], d, id)) lo = mid + 1; else hi = mid;
        }
        rank = m + lo;
      }
      if (rank < K) {
        od[rank] = d;
        oi[rank] = id;
      }
    }
    __syncthreads();
    const int nc = rc + cnt < K ? rc + cnt : K;
    for (int i = tid; i < nc; i += kThreads) {
      sd[i] = od[i];
      sid[i] = oi[i];
    }
    if (tid == 0) {
      s->r_count = nc;
      s->buf_count = 0;
      s->thr = nc == K ? od[K - 1] : INFINITY;
    }
    __syncthreads();
  }

  // ------------------------------------------------------------ the scan
  // A tile holds ROWS rows of FP32, or as many more narrow rows as fit the same
  // bytes: RPT = 4 / element bytes rows per thread (1 FP32, 2 BF16, 4 FP8).
  template <class E>
  __device__ void issue(const unsigned char* rows, int32_t nrows, int t, uint32_t g) {
    constexpr int RT = ROWS * (4 / E::kBytes);
    int st = g % STAGES;
    int r0 = t * RT;
    int nr = nrows - r0 < RT ? nrows - r0 : RT;
    uint32_t bytes = (uint32_t)nr * D * E::kBytes;
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[st], bytes);
    bulk_g2s(stages + (size_t)st * TILE, rows + (size_t)r0 * D * E::kBytes, bytes, &bars[st]);
  }

  // Scans rows [0, nrows) of `rows` (element type E; ids[r], or base_id + r
  // when ids is NULL), keeping the K best in R.  FP8 rows are multiplied by
  // `scale` as they are read.
  //
  // Every decision that leads to a __syncthreads() is taken on values that are
  // identical in all threads: the survivor count of a tile comes back from the
  // tile's own barrier (__syncthreads_count), so threads that run ahead into
  // the next tile and append its survivors cannot change the merge decision
  // of threads still finishing this one.
  template <class E>
  __device__ void scan(const unsigned char* rows, const int64_t* ids, int64_t base_id, int32_t nrows, int K,
                       float scale) {
    if (nrows <= 0 || aborted) return;
    constexpr int RPT = 4 / E::kBytes;       // rows per thread per tile
    constexpr int RT = ROWS * RPT;           // rows per tile
    static_assert(RPT <= TPR, "each row's survivor flag needs its own lane");
    int ntiles = (nrows + RT - 1) / RT;
    uint32_t g0 = consumed;
    if (tid == 0) {
      int pre = ntiles < STAGES ? ntiles : STAGES;
      for (int t = 0; t < pre; ++t) issue<E>(rows, nrows, t, g0 + t);
      s->issued = g0 + pre;
    }
    const int r = tid / TPR, sub = tid % TPR;
    int buffered = 0;     // survivors in the buffer (uniform)
    bool tmo = false;     // this thread's wait on a tile expired
    for (int t = 0; t < ntiles; ++t) {
      uint32_t g = g0 + t;
      int st = g % STAGES;
      if (!tmo) {
        long long waited = 0;
        if (!mbar_wait_bounded(&bars[st], (g / STAGES) & 1u, &waited)) {
          tmo = true;
          if (atomicCAS(status, 0, DEV_TIMEOUT) == 0) {
            diag[0] = DEV_TIMEOUT;
            diag[1] = qi;
            diag[2] = g;
            diag[3] = t;
            diag[4] = ntiles;
            diag[5] = (int64_t)mbar_raw(&bars[st]);
            diag[6] = s->issued;
            diag[7] = consumed;
          }
        }
        if (waited > max_wait) max_wait = waited;
      }
      int nr = nrows - t * RT < RT ? nrows - t * RT : RT;
      const unsigned char* tile = reinterpret_cast<const unsigned char*>(stages + (size_t)st * TILE);
      float acc[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        acc[i] = 0.f;
        const int rr = r + ROWS * i;
        if (rr < nr) {
          const unsigned char* row = tile + (size_t)rr * D * E::kBytes;
          // four independent FMA chains, as two packed pairs (FADD2 / FFMA2
          // do two FP32 operations per instruction, each rounded as alone)
          float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
          if (metric == QK_METRIC_L2) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              float4 x = E::load4(row, sub + TPR * v, scale);
              const float2 d01 = __fadd2_rn(make_float2(x.x, x.y), make_float2(-qv[v].x, -qv[v].y));
              const float2 d23 = __fadd2_rn(make_float2(x.z, x.w), make_float2(-qv[v].z, -qv[v].w));
              a01 = __ffma2_rn(d01, d01, a01);
              a23 = __ffma2_rn(d23, d23, a23);
            }
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              float4 x = E::load4(row, sub + TPR * v, scale);
              a01 = __ffma2_rn(make_float2(x.x, x.y), make_float2(qv[v].x, qv[v].y), a01);
              a23 = __ffma2_rn(make_float2(x.z, x.w), make_float2(qv[v].z, qv[v].w), a23);
            }
          }
          acc[i] = (a01.x + a01.y) + (a23.x + a23.y);
        }
      }
      // Reduce-scatter over the row group's TPR lanes: the first log2(RPT)
      // butterfly levels also split the RPT rows between the two lane halves
      // (a half keeps its rows and receives the partner's partials of them),
      // the rest are plain butterfly levels.  Every row's total pairs the same
      // partials in the same order as the full butterfly; row i ends in the
      // lanes whose bits TPR/2, TPR/4, ... spell i, and the first of them,
      // row_judge(i), judges it, so each thread raises at most one flag.
      float red;
      {
        float v[RPT];
#pragma unroll
        for (int i = 0; i < RPT; ++i) v[i] = acc[i];
        int o = TPR / 2;
#pragma unroll
        for (int h = RPT / 2; h >= 1; h >>= 1, o >>= 1) {
          const bool up = (sub & o) != 0;
#pragma unroll
          for (int m = 0; m < h; ++m) {
            const float send = up ? v[m] : v[m + h];
            const float keep = up ? v[m + h] : v[m];
            v[m] = keep + __shfl_xor_sync(0xffffffffu, send, o);
          }
        }
#pragma unroll
        for (; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        red = v[0];
      }
      bool surv = false;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        if (sub == row_judge(i, RPT)) {
          const int rr = r + ROWS * i;
          float dist = metric == QK_METRIC_L2 ? red : -red;
          surv = !tmo && rr < nr && dist <= s->thr;
          if (surv) {
            int pos = atomicAdd(&s->buf_count, 1);
            int64_t gr = (int64_t)t * RT + rr;
            sd[K + pos] = dist;
            sid[K + pos] = ids ? ids[gr] : base_id + gr;
          }
        }
      }
      buffered += __syncthreads_count(surv);
      ++consumed;
      if (tid == 0 && !tmo && t + STAGES < ntiles) {
        issue<E>(rows, nrows, t + STAGES, g + STAGES);
        s->issued = g + STAGES + 1;
      }
      // merge when the buffer could overflow, or as soon as R can first be
      // filled (the threshold then turns finite and filters the rest)
      if (buffered > kBufCap - RT || (s->r_count < K && s->r_count + buffered >= K)) {
        merge(K, buffered);
        buffered = 0;
      }
    }
    if (__syncthreads_or(tmo)) {
      aborted = true;
      return;
    }
    if (buffered > 0) merge(K, buffered);
  }

  // ---------------------------------------------------- APS on one level
  // mode: 0 FP32 rows, ids kept; 1 FP32 rows, arena slots kept; 2 BF16 rows,
  // slots kept; 3 FP8 rows (scaled per partition), slots kept.
  __device__ void scan_pos(const DevLevel& lv, int pos, int M, int K, unsigned long long* hits, int mode) {
    if (pos < 0 || pos >= M) {            // never expected: record and skip
      if (tid == 0) report(DEV_BAD_INDEX, 1, pos, M);
      __syncthreads();
      return;
    }
    int part = cpart[pos];
    if (part < 0 || part >= lv.n_part) {
      if (tid == 0) report(DEV_BAD_INDEX, 2, pos, part);
      __syncthreads();
      return;
    }
    int64_t off = lv.off[part];
    int32_t sz = lv.size[part];
    const unsigned char* f32 = reinterpret_cast<const unsigned char*>(lv.vec + off * D);
    switch (mode) {
      case 0: scan<ElemF32>(f32, lv.ids + off, 0, sz, K, 1.f); break;
      case 1: scan<ElemF32>(f32, nullptr, off, sz, K, 1.f); break;
      case 2: scan<ElemBF16>(lp_vec + off * D * 2, nullptr, off, sz, K, 1.f); break;
      default: scan<ElemFP8>(lp_vec + off * D, nullptr, off, sz, K, lp_scale[part]); break;
    }
    if (tid == 0) {
      csc[pos] = 1;
      if (hits) atomicAdd(&hits[part], 1ull);
      if (rec && rec_n < rec_cap) rec[rec_n] = part;
      ++rec_n;
    }
    __syncthreads();
  }

  // Optional record of the scanned partitions (in scan order) of the current
  // query at one level; rec_n is kept by thread 0.
  __device__ void record_start(int32_t* row, int cap) {
    rec = row;
    rec_cap = cap;
    rec_n = 0;
  }
  __device__ void record_finish() {
    __syncthreads();
    const int n = __shfl_sync(0xffffffffu, rec_n, 0);   // warp 0 learns thread 0's count
    if (warp == 0 && rec)
      for (int i = n + lane; i < rec_cap; i += 32) rec[i] = -1;
    rec = nullptr;
    __syncthreads();
  }

  // t_i = (D_i - D_0) / (2 ||c_i - c_0||) with D the squared Euclidean
  // centroid distance, for either metric: the partitions are k-means cells,
  // bounded by the Euclidean bisectors of their centroids.  FP32 like the
  // distances it comes from (one warp per candidate).
  __device__ void bisector(const DevLevel& lv, int M) {
    const float* c0 = lv.cent + (size_t)cpart[0] * D;
    for (int i = 1 + warp; i < M; i += kWarps) {
      const float* ci = lv.cent + (size_t)cpart[i] * D;
      float acc = 0.f;
      for (int j = lane; j < D; j += 32) {
        float df = ci[j] - c0[j];
        acc = fmaf(df, df, acc);
      }
      acc = warp_sum_f(acc);
      if (lane == 0) {
        float cd = sqrtf(acc);
        float den = 2.f * cd;
        float t = den > 0.f ? (cD[i] - cD[0]) / den : 0.f;
        ct[i] = t > 0.f ? (double)t : 0.0;
      }
    }
    if (tid == 0) ct[0] = 0.0;
    __syncthreads();
  }

  // ---- the estimator, run by warp 0 only (the FP64 pipe is narrow on this
  // part, so FP64 work is confined to the cap-volume terms of one warp) ----

  // p_0 = prod (1 - u_j), p_i = (1 - p_0) u_i / sum u (Eq. 8-9, raw caps for
  // p_0) for every candidate; then r = p_0 + sum of the scanned p_i (R5).
  __device__ double w0_probabilities(int M, double rho) {
    double su = 0.0, pr = 1.0;
    const double inv = rho > 0.0 ? 1.0 / rho : 0.0;
    for (int i = 1 + lane; i < M; i += 32) {
      const double u = cap_u(ct[i], rho, inv, beta_mode == QK_BETA_EXACT, beta_table, beta_a, beta_lnB);
      cp[i] = u;
      su += u;
      pr *= 1.0 - u;
    }
    const double U = warp_sum_d(su);
    const double P0 = warp_prod_d(pr);
    const double c = U > 0.0 ? (1.0 - P0) / U : 0.0;
    double rs = 0.0;
    for (int i = 1 + lane; i < M; i += 32) {
      double p = cp[i] * c;
      cp[i] = p;
      if (csc[i]) rs += p;
    }
    if (lane == 0) cp[0] = P0;
    return P0 + warp_sum_d(rs);
  }

  // The unscanned candidate with the largest p (R6: ties to the lower
  // position).  p >= 0, so its IEEE bits order like its value and the
  // comparison runs on the integer pipe.  Returns M if none is left.
  __device__ int w0_next(int M) {
    long long bk = -1;
    int bi = M;
    for (int i = 1 + lane; i < M; i += 32) {
      if (csc[i]) continue;
      long long k = __double_as_longlong(cp[i]);
      if (k > bk) {
        bk = k;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
      int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (k2 > bk || (k2 == bk && i2 < bi)) {
        bk = k2;
        bi = i2;
      }
    }
    return bi;
  }

  // rho from the current k-th result (R1), in FP32 like the distances.  For
  // inner product, rho = ||q - x_k|| = sqrt(||q||^2 + ||x_k||^2 + 2 D_k) with
  // D_k = -<q, x_k>; x_k is row sid[k-1] of krow (called by warp 0).
  __device__ double kth_radius(int k, const float* krow) {
    float dk = sd[k - 1];
    if (metric == QK_METRIC_L2) return (double)sqrtf(dk > 0.f ? dk : 0.f);
    const float* x = krow + (size_t)sid[k - 1] * D;
    float xn = 0.f;
    for (int j = lane; j < D; j += 32) xn = fmaf(x[j], x[j], xn);
    xn = warp_sum_f(xn);
    float r2 = qn + xn + 2.f * dk;
    return (double)sqrtf(r2 > 0.f ? r2 : 0.f);
  }

  // Algorithm 1 over the M candidates in (cpart, cD); result set in R.
  // Returns r (NaN in fixed-nprobe mode) and the number of scanned partitions.
  // K results are kept (K >= k when low-precision candidates are oversized);
  // rho and the "R holds k results" rule use the k-th; krow locates result rows
  // for the inner-product radius; mode selects the scanned rows (see scan_pos).
  __device__ void aps(const DevLevel& lv, int M, int K, int k, double tau, int fixed, unsigned long long* hits,
                      int mode, const float* krow, double& r_out, int& nprobe_out, bool t_given = false) {
    reset_R(K);
    for (int i = tid; i < M; i += kThreads) csc[i] = 0;
    __syncthreads();
    if (fixed > 0) {
      int n = fixed < M ? fixed : M;
      for (int pos = 0; pos < n && !aborted; ++pos) scan_pos(lv, pos, M, K, hits, mode);
      r_out = NAN;
      nprobe_out = n;
      return;
    }
    if (!t_given) bisector(lv, M);
    int ns = 0;
    scan_pos(lv, 0, M, K, hits, mode);
    ns = 1;
    while (s->r_count < k && ns < M && !aborted) {   // R holds fewer than k: centroid order
      scan_pos(lv, ns, M, K, hits, mode);
      ++ns;
    }
    nprobe_out = ns;
    if (s->r_count < k || aborted) {
      r_out = 1.0;
      return;
    }
    // warp 0 owns rho, p and r; the CTA follows its decisions through shared memory
    if (warp == 0) {
      double rho = kth_radius(k, krow);
      double r = w0_probabilities(M, rho);
      int nx = w0_next(M);
      if (lane == 0) {
        s->rho = rho;
        s->r = r;
        s->next = nx;
        s->go = (r < tau && ns < M) ? 1 : 0;
      }
    }
    __syncthreads();
    while (s->go && !aborted) {
      const int best = s->next;
      scan_pos(lv, best, M, K, hits, mode);
      ++ns;
      if (warp == 0) {
        double rho = s->rho, r = s->r;
        double rho2 = kth_radius(k, krow);
        if (fabs(rho2 - rho) > tau_rho * rho) {           // R7: recompute every p
          rho = rho2;
          r = w0_probabilities(M, rho);
        } else {                                          // p unchanged: add the scanned p
          r += cp[best];
        }
        int nx = w0_next(M);
        if (lane == 0) {
          s->rho = rho;
          s->r = r;
          s->next = nx;
          s->go = (r < tau && ns < M) ? 1 : 0;
        }
      }
      __syncthreads();
    }
    r_out = s->r;
    nprobe_out = ns;
  }

  // Sorts sd/sid[0, n) by (dist, id) with a CTA bitonic network (pads to a power of two).
  __device__ void sort_range(int n) {
    int np = next_pow2(n);
    for (int i = n + tid; i < np; i += kThreads) {
      sd[i] = INFINITY;
      sid[i] = INT64_MAX;
    }
    __syncthreads();
    for (int k = 2; k <= np; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < np; i += kThreads) {
          int p = i ^ j;
          if (p > i) {
            float di = sd[i], dp = sd[p];
            int64_t ii = sid[i], ip = sid[p];
            bool up = (i & k) == 0;
            if (up ? key_less(dp, ip, di, ii) : key_less(di, ii, dp, ip)) {
              sd[i] = dp;
              sd[p] = di;
              sid[i] = ip;
              sid[p] = ii;
            }
          }
        }
        __syncthreads();
      }
    }
  }

  // Replaces the arena slots in R by ids with exact FP32 distances computed
  // from the FP32 master rows (the re-rank of low-precision candidates), then
  // sorts R by (distance, id).
  __device__ void rerank(const float* vec0, const int64_t* ids0) {
    const int rc = s->r_count;
    for (int i = warp; i < rc; i += kWarps) {
      const float* x = vec0 + (size_t)sid[i] * D;
      float acc = 0.f;
      if (metric == QK_METRIC_L2) {
        for (int j = lane; j < D; j += 32) {
          float df = x[j] - sq[j];
          acc = fmaf(df, df, acc);
        }
      } else {
        for (int j = lane; j < D; j += 32) acc = fmaf(x[j], sq[j], acc);
      }
      acc = warp_sum_f(acc);
      __syncwarp();
      if (lane == 0) {
        int64_t slot = sid[i];
        sd[i] = metric == QK_METRIC_L2 ? acc : -acc;
        sid[i] = ids0[slot];
      }
    }
    __syncthreads();
    sort_range(rc);
  }

  // SPANN's early-termination rule over the candidates (cpart, cD) sorted by
  // squared distance: how many have a Euclidean distance within (1 + eps) of
  // the nearest one's (a prefix of the list; the same count in every thread).
  __device__ int ratio_count(int M, float eps) {
    const float lim = (1.f + eps) * sqrtf(fmaxf(cD[0], 0.f));
    int n = 0;
    for (int base = 0; base < M; base += kThreads) {
      const int i = base + tid;
      n += __syncthreads_count(i < M && sqrtf(fmaxf(cD[i], 0.f)) <= lim);
    }
    return n;
  }

  // R -> candidate list of the next level.
  __device__ int take_candidates() {
    int M = s->r_count;
    for (int i = tid; i < M; i += kThreads) {
      cpart[i] = (int32_t)sid[i];
      cD[i] = sd[i];
    }
    __syncthreads();
    return M;
  }
};

// Three CTAs per SM keep the memory system busy while each waits on its own
// query's tiles; up to d = 256 their shared memory allows it, so the
// registers are held to a third of the file (beyond, two CTAs fit anyway).
template <int TPR, int NV>
__global__ void __launch_bounds__(kThreads, (NV * 4 * TPR <= 256) ? 3 : 2) aps_search_kernel(SearchArgs args) {
  using B = Block<TPR, NV>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ Scalars sc;
  SmemLayout L(B::TILE, B::D, args.kcap, args.mcap);
  B b;
  b.metric = args.metric;
  b.beta_mode = args.beta_mode;
  b.tau_rho = args.tau_rho;
  b.beta_a = args.beta_a;
  b.beta_lnB = args.beta_lnB;
  b.beta_table = args.beta_table;
  b.status = args.status;
  b.diag = args.diag;
  b.lp_vec = static_cast<const unsigned char*>(args.lp_vec);
  b.lp_scale = args.lp_scale;
  b.qi = -1;
  b.max_wait = 0;
  b.aborted = false;
  b.rec = nullptr;
  b.rec_cap = 0;
  b.rec_n = 0;
  b.stages = reinterpret_cast<float*>(smem + L.stages);
  b.bars = reinterpret_cast<uint64_t*>(smem + L.bars);
  b.sq = reinterpret_cast<float*>(smem + L.q);
  b.sd = reinterpret_cast<float*>(smem + L.sd);
  b.sid = reinterpret_cast<int64_t*>(smem + L.sid);
  b.cpart = reinterpret_cast<int32_t*>(smem + L.cpart);
  b.cD = reinterpret_cast<float*>(smem + L.cD);
  b.ct = reinterpret_cast<double*>(smem + L.ct);
  b.cp = reinterpret_cast<double*>(smem + L.cp);
  b.csc = reinterpret_cast<uint8_t*>(smem + L.csc);
  b.s = &sc;
  b.tid = threadIdx.x;
  b.lane = threadIdx.x & 31;
  b.warp = threadIdx.x >> 5;
  b.consumed = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < B::STAGES; ++i) mbar_init(&b.bars[i], 1);
    fence_mbar_init();
    sc.issued = 0;
  }
  __syncthreads();

  for (;;) {
    if (threadIdx.x == 0) sc.qi = atomicAdd(args.work, 1);
    __syncthreads();
    int64_t qi = sc.qi;
    b.qi = qi;
    if (qi >= args.nq || b.aborted) break;
    const float* q = args.Q + qi * B::D;
    for (int i = threadIdx.x; i < B::D; i += kThreads) b.sq[i] = q[i];
    __syncthreads();
    {
      const float4* q4 = reinterpret_cast<const float4*>(b.sq);
      int sub = threadIdx.x % TPR;
#pragma unroll
      for (int v = 0; v < NV; ++v) b.qv[v] = q4[sub + TPR * v];
      float qn = 0.f;
      for (int j = b.lane; j < B::D; j += 32) qn = fmaf(b.sq[j], b.sq[j], qn);
      b.qn = warp_sum_f(qn);
    }
    // A query with a NaN or infinite element, or whose squared norm exceeds
    // FP32, is refused before any comparison sees it: ids -1, distances NaN,
    // and the status records a bad argument (the other queries are answered).
    if (__syncthreads_or(!(b.qn < INFINITY))) {
      if (threadIdx.x == 0) b.report(DEV_BAD_ARG, 1, 0, 0);
      for (int i = threadIdx.x; i < args.kq; i += kThreads) {
        args.out_dist[qi * args.kq + i] = NAN;
        args.out_ids[qi * args.kq + i] = -1;
      }
      if (threadIdx.x == 0) {
        if (args.out_nprobe) args.out_nprobe[qi] = 0;
        if (args.out_recall) args.out_recall[qi] = NAN;
      }
      for (int i = threadIdx.x; i < args.scan_cap0 && args.scan0; i += kThreads) args.scan0[qi * args.scan_cap0 + i] = -1;
      for (int i = threadIdx.x; i < args.scan_cap1 && args.scan1; i += kThreads) args.scan1[qi * args.scan_cap1 + i] = -1;
      if (threadIdx.x == 0 && args.xs_M) args.xs_M[qi] = -1;
      __syncthreads();
      continue;
    }
    // The tree is searched in the Euclidean geometry it was built in: the top
    // partition and the upper levels rank centroids by squared L2; only the
    // base rows use the index's metric (for inner product, -<q, x>).
    b.metric = QK_METRIC_L2;
    int M = 0;
    double r = 0.0;
    int np = 0;
    const bool imported = args.im_M != nullptr;
    if (imported) {
      // the upper levels were walked by the prepare step: its leaf candidates and t_i
      M = args.im_M[qi];
      if (M < 1 || M > args.mcap) {   // a query the prepare step refused is refused above
        if (threadIdx.x == 0) b.report(DEV_BAD_INDEX, 4, M, args.mcap);
        __syncthreads();
        continue;
      }
      for (int i = threadIdx.x; i < M; i += kThreads) {
        b.cpart[i] = args.im_cand[qi * args.im_mcap + i];
        b.ct[i] = args.im_t[qi * args.im_mcap + i];
      }
      __syncthreads();
    } else {
    // top partition: all centroids of the top level
    b.reset_R(args.M_root);
    b.template scan<ElemF32>(reinterpret_cast<const unsigned char*>(args.root), nullptr, 0, args.n_root, args.M_root, 1.f);
    M = b.take_candidates();
    if (args.L == 2) {
      // level-1 rows are leaf centroids whose id is the leaf index: x_k = cent0[id]
      if (args.scan1) b.record_start(args.scan1 + qi * args.scan_cap1, args.scan_cap1);
      b.aps(args.lv[1], M, args.k1, args.k1, args.tau1, 0, args.hits1, 0, args.lv[0].cent, r, np);
      if (args.scan1) b.record_finish();
      M = b.take_candidates();
    } else if (args.scan1) {
      for (int i = threadIdx.x; i < args.scan_cap1; i += kThreads) args.scan1[qi * args.scan_cap1 + i] = -1;
    }
    }
    if (args.xs_M) {
      // batched APS: export S_0 with its t_i; the leaf level is scanned in
      // rounds by the grouped scan and replayed per query elsewhere
      if (b.aborted) break;
      b.bisector(args.lv[0], M);
      for (int i = threadIdx.x; i < M; i += kThreads) {
        args.xs_cand[qi * args.xs_mcap + i] = b.cpart[i];
        args.xs_t[qi * args.xs_mcap + i] = b.ct[i];
      }
      if (threadIdx.x == 0) args.xs_M[qi] = M;
      __syncthreads();
      continue;
    }
    int fixed = args.nprobe_q ? args.nprobe_q[qi] : args.fixed_nprobe;
    if (args.ratio_eps > 0.f) fixed = b.ratio_count(M, args.ratio_eps);
    b.metric = args.metric;
    if (args.scan0) b.record_start(args.scan0 + qi * args.scan_cap0, args.scan_cap0);
    b.aps(args.lv[0], M, args.k0, args.kq, args.tau0, fixed, args.hits0, args.mode0, args.lv[0].vec, r, np,
          imported);
    if (args.scan0) b.record_finish();
    if (b.aborted) break;
    if (args.mode0 != 0) b.rerank(args.lv[0].vec, args.lv[0].ids);
    int rc = sc.r_count;
    for (int i = threadIdx.x; i < args.kq; i += kThreads) {
      bool ok = i < rc;
      if (ok && (b.sid[i] < 0 || !(b.sd[i] < INFINITY))) b.report(DEV_BAD_INDEX, 3, i, rc);
      args.out_dist[qi * args.kq + i] = ok ? b.sd[i] : INFINITY;
      args.out_ids[qi * args.kq + i] = ok ? b.sid[i] : -1;
    }
    if (threadIdx.x == 0) {
      if (args.out_nprobe) args.out_nprobe[qi] = np;
      if (args.out_recall) args.out_recall[qi] = (float)r;
    }
    __syncthreads();
  }
  if (args.wait_stats && (threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(args.wait_stats), (unsigned long long)b.max_wait);
  // after an abort, wait (bounded) for copies still in flight before exiting
  if (threadIdx.x == 0 && b.aborted) {
    uint32_t lo = sc.issued > B::STAGES ? sc.issued - B::STAGES : 0;
    for (uint32_t g = lo; g < sc.issued; ++g) mbar_wait_bounded(&b.bars[g % B::STAGES], (g / B::STAGES) & 1u);
  }
}

template <int TPR, int NV>
qk_status launch_one(const SearchArgs& a, cudaStream_t stream) {
  using B = Block<TPR, NV>;
  SmemLayout L(B::TILE, B::D, a.kcap, a.mcap);
  size_t smem = L.total;
  int dev;
  QK_CUDA(cudaGetDevice(&dev));
  int max_optin = 0;
  QK_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem + sizeof(Scalars) + 1024 > (size_t)max_optin) {
    set_error("search: k or candidate count too large for shared memory");
    return QK_ERR_UNSUPPORTED;
  }
  auto kern = aps_search_kernel<TPR, NV>;
  QK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int nsm = 0, per_sm = 0;
  QK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  QK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > a.nq) grid = a.nq;
  QK_CUDA(cudaMemsetAsync(a.work, 0, sizeof(int32_t), stream));
  kern<<<(unsigned)grid, kThreads, smem, stream>>>(a);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
