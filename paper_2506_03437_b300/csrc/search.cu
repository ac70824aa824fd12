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
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "capvol.cuh"
#include "common.cuh"
#include "index.cuh"

namespace qk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kStages = 4;
constexpr int kBufCap = 256;

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
    stages = take(sizeof(float) * (size_t)tile_floats * kStages, 128);
    bars = take(sizeof(uint64_t) * kStages, 8);
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

template <int TPR, int NV>
struct Block {
  static constexpr int D = NV * 4 * TPR;
  static constexpr int ROWS = kThreads / TPR;
  static constexpr int TILE = ROWS * D;

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
  long long max_wait;   // longest tile wait of this thread, in SM cycles
  bool aborted;         // a tile wait expired (uniform across the CTA)

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
  __device__ void issue(const float* rows, int32_t nrows, int t, uint32_t g) {
    int st = g % kStages;
    int r0 = t * ROWS;
    int nr = nrows - r0 < ROWS ? nrows - r0 : ROWS;
    uint32_t bytes = (uint32_t)nr * D * sizeof(float);
    fence_proxy_async();
    mbar_arrive_expect_tx(&bars[st], bytes);
    bulk_g2s(stages + (size_t)st * TILE, rows + (size_t)r0 * D, bytes, &bars[st]);
  }

  // Scans rows [0, nrows) of `rows` (ids[r] or base_id + r), keeping the K best in R.
  //
  // Every decision that leads to a __syncthreads() is taken on values that are
  // identical in all threads: the survivor count of a tile comes back from the
  // tile's own barrier (__syncthreads_count), so threads that run ahead into
  // the next tile and append its survivors cannot change the merge decision
  // of threads still finishing this one.
  __device__ void scan(const float* rows, const int64_t* ids, int64_t base_id, int32_t nrows, int K) {
    if (nrows <= 0 || aborted) return;
    int ntiles = (nrows + ROWS - 1) / ROWS;
    uint32_t g0 = consumed;
    if (tid == 0) {
      int pre = ntiles < kStages ? ntiles : kStages;
      for (int t = 0; t < pre; ++t) issue(rows, nrows, t, g0 + t);
      s->issued = g0 + pre;
    }
    const int r = tid / TPR, sub = tid % TPR;
    int buffered = 0;     // survivors in the buffer (uniform)
    bool tmo = false;     // this thread's wait on a tile expired
    for (int t = 0; t < ntiles; ++t) {
      uint32_t g = g0 + t;
      int st = g % kStages;
      if (!tmo) {
        long long waited = 0;
        if (!mbar_wait_bounded(&bars[st], (g / kStages) & 1u, &waited)) {
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
      int nr = nrows - t * ROWS < ROWS ? nrows - t * ROWS : ROWS;
      float acc = 0.f;
      if (r < nr) {
        const float4* row = reinterpret_cast<const float4*>(stages + (size_t)st * TILE + (size_t)r * D);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;   // four independent FMA chains
        if (metric == QK_METRIC_L2) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            float4 x = row[sub + TPR * v];
            float dx = x.x - qv[v].x, dy = x.y - qv[v].y, dz = x.z - qv[v].z, dw = x.w - qv[v].w;
            a0 = fmaf(dx, dx, a0);
            a1 = fmaf(dy, dy, a1);
            a2 = fmaf(dz, dz, a2);
            a3 = fmaf(dw, dw, a3);
          }
        } else {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            float4 x = row[sub + TPR * v];
            a0 = fmaf(x.x, qv[v].x, a0);
            a1 = fmaf(x.y, qv[v].y, a1);
            a2 = fmaf(x.z, qv[v].z, a2);
            a3 = fmaf(x.w, qv[v].w, a3);
          }
        }
        acc = (a0 + a1) + (a2 + a3);
      }
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      float dist = metric == QK_METRIC_L2 ? acc : -acc;
      bool surv = !tmo && sub == 0 && r < nr && dist <= s->thr;
      if (surv) {
        int pos = atomicAdd(&s->buf_count, 1);
        int64_t rr = (int64_t)t * ROWS + r;
        sd[K + pos] = dist;
        sid[K + pos] = ids ? ids[rr] : base_id + rr;
      }
      buffered += __syncthreads_count(surv);
      ++consumed;
      if (tid == 0 && !tmo && t + kStages < ntiles) {
        issue(rows, nrows, t + kStages, g + kStages);
        s->issued = g + kStages + 1;
      }
      // merge when the buffer could overflow, or as soon as R can first be
      // filled (the threshold then turns finite and filters the rest)
      if (buffered > kBufCap - ROWS || (s->r_count < K && s->r_count + buffered >= K)) {
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
  __device__ void scan_pos(const DevLevel& lv, int pos, int M, int K, unsigned long long* hits) {
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
    scan(lv.vec + off * D, lv.ids + off, 0, sz, K);
    if (tid == 0) {
      csc[pos] = 1;
      if (hits) atomicAdd(&hits[part], 1ull);
    }
    __syncthreads();
  }

  // t_i = (D_i - D_0) / (2 ||c_i - c_0||) for L2, / ||c_i - c_0|| for IP, in
  // FP32 like the distances it comes from (one warp per candidate).
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
        float den = metric == QK_METRIC_L2 ? 2.f * cd : cd;
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
      double u = 0.0;
      double t = ct[i];
      if (rho > 0.0 && t < rho) {
        if (beta_mode == QK_BETA_EXACT) {
          u = cap_fraction_exact(t, rho, beta_a, beta_lnB);
        } else {
          double sc = t * inv;
          double x = 1.0 - sc * sc;
          double f = x * (kBetaTablePoints - 1);
          int j = (int)f;
          if (j > kBetaTablePoints - 2) j = kBetaTablePoints - 2;
          double lo = beta_table[j], hi = beta_table[j + 1];
          u = 0.5 * (lo + (f - j) * (hi - lo));
        }
      }
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

  // rho from the current k-th result (R1), in FP32 like the distances.
  __device__ double kth_radius(int K) {
    float dk = sd[K - 1];
    return (double)sqrtf(dk > 0.f ? dk : 0.f);
  }

  // Algorithm 1 over the M candidates in (cpart, cD); result set in R.
  // Returns r (NaN in fixed-nprobe mode) and the number of scanned partitions.
  __device__ void aps(const DevLevel& lv, int M, int K, double tau, int fixed,
                      unsigned long long* hits, double& r_out, int& nprobe_out) {
    reset_R(K);
    for (int i = tid; i < M; i += kThreads) csc[i] = 0;
    __syncthreads();
    if (fixed > 0) {
      int n = fixed < M ? fixed : M;
      for (int pos = 0; pos < n && !aborted; ++pos) scan_pos(lv, pos, M, K, hits);
      r_out = NAN;
      nprobe_out = n;
      return;
    }
    bisector(lv, M);
    int ns = 0;
    scan_pos(lv, 0, M, K, hits);
    ns = 1;
    while (s->r_count < K && ns < M && !aborted) {   // R holds fewer than k: centroid order
      scan_pos(lv, ns, M, K, hits);
      ++ns;
    }
    nprobe_out = ns;
    if (s->r_count < K || aborted) {
      r_out = 1.0;
      return;
    }
    // warp 0 owns rho, p and r; the CTA follows its decisions through shared memory
    if (warp == 0) {
      double rho = kth_radius(K);
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
      scan_pos(lv, best, M, K, hits);
      ++ns;
      if (warp == 0) {
        double rho = s->rho, r = s->r;
        double rho2 = kth_radius(K);
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

template <int TPR, int NV>
__global__ void __launch_bounds__(kThreads) aps_search_kernel(SearchArgs args) {
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
  b.qi = -1;
  b.max_wait = 0;
  b.aborted = false;
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
    for (int i = 0; i < kStages; ++i) mbar_init(&b.bars[i], 1);
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
    }
    // top partition: all centroids of the top level
    b.reset_R(args.M_root);
    b.scan(args.root, nullptr, 0, args.n_root, args.M_root);
    int M = b.take_candidates();
    double r = 0.0;
    int np = 0;
    if (args.L == 2) {
      b.aps(args.lv[1], M, args.k1, args.tau1, 0, args.hits1, r, np);
      M = b.take_candidates();
    }
    b.aps(args.lv[0], M, args.k0, args.tau0, args.fixed_nprobe, args.hits0, r, np);
    if (b.aborted) break;
    int rc = sc.r_count;
    for (int i = threadIdx.x; i < args.k0; i += kThreads) {
      bool ok = i < rc;
      if (ok && (b.sid[i] < 0 || !(b.sd[i] < INFINITY))) b.report(DEV_BAD_INDEX, 3, i, rc);
      args.out_dist[qi * args.k0 + i] = ok ? b.sd[i] : INFINITY;
      args.out_ids[qi * args.k0 + i] = ok ? b.sid[i] : -1;
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
    uint32_t lo = sc.issued > kStages ? sc.issued - kStages : 0;
    for (uint32_t g = lo; g < sc.issued; ++g) mbar_wait_bounded(&b.bars[g % kStages], (g / kStages) & 1u);
  }
}

template <int TPR, int NV>
static qk_status launch_one(const SearchArgs& a, cudaStream_t stream) {
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
