// The first step of a batched APS search with one warp per query: the top
// partition is scanned, the upper level is searched by Algorithm 1 with the
// upper target tau_1, and the leaf candidates S with their bisector distances
// t_i are exported for the rounds.  It computes what aps_search_kernel's
// export mode computes, with the same arithmetic in the same order (the row
// distances of the tile scan, the k-th radius, Eq. 7-9 as its warp 0 runs
// them, the bisectors), so the candidates and t_i are bitwise the same; the
// per-query kernel spends most of this step waiting at CTA barriers while
// one warp works, which this layout does not have.  Indexes whose candidate
// counts exceed the warp's buffers keep using the per-query kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "capvol.cuh"
#include "common.cuh"
#include "grouped.cuh"
#include "index.cuh"

namespace qk {
namespace ap {

constexpr int kWarps = 4;     // queries per block
constexpr int kRCap = 224;    // the largest result set R of a level (K <= kRCap)
constexpr int kBuf = 32;      // survivors waiting for a merge
constexpr int kMCap = 256;    // the most candidates of a level searched by Algorithm 1

// Shared memory of one warp.
struct Ws {
  float* sq;        // D: the query
  float* rd;        // kRCap: R, sorted by (distance, id)
  int64_t* ri;
  float* bd;        // kBuf: survivors
  int64_t* bi;
  float* od;        // kRCap: merge output
  int64_t* oi;
  int32_t* cpart;   // kMCap: candidates of the level, nearest first
  float* cD;
  double* ct;       // kMCap: t_i
  double* cp;       // kMCap: p_i
  uint8_t* csc;     // kMCap: scanned
};

// Bytes of one warp's buffers for results of up to rcap and mcap candidates
// (every piece rounded to 16 bytes).
__host__ __device__ inline size_t warp_bytes(int D, int rcap, int mcap) {
  auto r16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  return r16(8 * (size_t)rcap) * 2 + r16(8 * (size_t)kBuf) + r16(8 * (size_t)mcap) * 2 + r16(4 * (size_t)D) +
         r16(4 * (size_t)rcap) * 2 + r16(4 * (size_t)kBuf) + r16(4 * (size_t)mcap) * 2 + r16(mcap);
}

__device__ inline Ws carve(unsigned char* base, int D, int rcap, int mcap) {
  Ws w;
  unsigned char* p = base;
  auto take = [&](size_t bytes) {
    unsigned char* r = p;
    p += (bytes + 15) & ~size_t(15);
    return r;
  };
  w.ri = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * rcap));
  w.oi = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * rcap));
  w.bi = reinterpret_cast<int64_t*>(take(sizeof(int64_t) * kBuf));
  w.ct = reinterpret_cast<double*>(take(sizeof(double) * mcap));
  w.cp = reinterpret_cast<double*>(take(sizeof(double) * mcap));
  w.sq = reinterpret_cast<float*>(take(sizeof(float) * D));
  w.rd = reinterpret_cast<float*>(take(sizeof(float) * rcap));
  w.od = reinterpret_cast<float*>(take(sizeof(float) * rcap));
  w.bd = reinterpret_cast<float*>(take(sizeof(float) * kBuf));
  w.cpart = reinterpret_cast<int32_t*>(take(sizeof(int32_t) * mcap));
  w.cD = reinterpret_cast<float*>(take(sizeof(float) * mcap));
  w.csc = reinterpret_cast<uint8_t*>(take(mcap));
  return w;
}

__device__ __forceinline__ bool key_less(float d1, int64_t i1, float d2, int64_t i2) {
  return d1 < d2 || (d1 == d2 && i1 < i2);
}

template <int TPR, int NV>
struct Warp {
  static constexpr int D = NV * 4 * TPR;
  static constexpr int RPW = 32 / TPR;   // rows per warp step
  Ws w;
  int lane;
  float4 qv[NV];
  int rn;          // entries in R
  float thr;       // a row enters the buffer at distance <= thr
  int cnt;         // entries in the buffer
  int K;

  __device__ void reset(int K_) {
    K = K_;
    rn = 0;
    cnt = 0;
    thr = INFINITY;
  }

  // The buffer, sorted, rank-merged into R; R keeps its first K.
  __device__ void merge() {
    float d = lane < cnt ? w.bd[lane] : INFINITY;
    int64_t i = lane < cnt ? w.bi[lane] : INT64_MAX;
    __syncwarp();
    bt::warp_sort32(d, i, lane);
    if (lane < cnt) {
      w.bd[lane] = d;
      w.bi[lane] = i;
    }
    __syncwarp();
    for (int e = lane; e < rn; e += 32) {   // R elements: rank among the buffer
      const float de = w.rd[e];
      const int64_t ie = w.ri[e];
      int lo = 0, hi = cnt;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_less(w.bd[mid], w.bi[mid], de, ie)) lo = mid + 1; else hi = mid;
      }
      const int rank = e + lo;
      if (rank < K) {
        w.od[rank] = de;
        w.oi[rank] = ie;
      }
    }
    if (lane < cnt) {   // buffer elements: rank among R
      int lo = 0, hi = rn;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_less(w.rd[mid], w.ri[mid], d, i)) lo = mid + 1; else hi = mid;
      }
      const int rank = lane + lo;
      if (rank < K) {
        w.od[rank] = d;
        w.oi[rank] = i;
      }
    }
    __syncwarp();
    const int n = rn + cnt < K ? rn + cnt : K;
    for (int e = lane; e < n; e += 32) {
      w.rd[e] = w.od[e];
      w.ri[e] = w.oi[e];
    }
    __syncwarp();
    rn = n;
    cnt = 0;
    thr = rn == K ? w.rd[K - 1] : INFINITY;
  }

  // Squared L2 distances of n FP32 rows (ids[r], or base + r without ids)
  // with the tile scan's arithmetic; rows at distance <= thr enter R.
  __device__ void scan(const float* rows, const int64_t* ids, int64_t base, int n) {
    const int grp = lane / TPR, sub = lane % TPR;
    for (int r0 = 0; r0 < n; r0 += RPW) {
      const int row = r0 + grp;
      float acc = 0.f;
      if (row < n) {
        const float4* x4 = reinterpret_cast<const float4*>(rows + (size_t)row * D);
        float2 a01 = make_float2(0.f, 0.f), a23 = make_float2(0.f, 0.f);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 x = x4[sub + TPR * v];
          const float2 d01 = __fadd2_rn(make_float2(x.x, x.y), make_float2(-qv[v].x, -qv[v].y));
          const float2 d23 = __fadd2_rn(make_float2(x.z, x.w), make_float2(-qv[v].z, -qv[v].w));
          a01 = __ffma2_rn(d01, d01, a01);
          a23 = __ffma2_rn(d23, d23, a23);
        }
        acc = (a01.x + a01.y) + (a23.x + a23.y);
      }
#pragma unroll
      for (int o = TPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const bool s = sub == 0 && row < n && acc <= thr;
      const unsigned m = __ballot_sync(0xffffffffu, s);
      if (s) {
        const int at = cnt + __popc(m & ((1u << lane) - 1u));
        w.bd[at] = acc;
        w.bi[at] = ids ? ids[row] : base + row;
      }
      cnt += __popc(m);
      __syncwarp();
      if (cnt > kBuf - RPW) merge();
    }
    if (cnt) merge();
  }

  // t_i = (D_i - D_0) / (2 ||c_i - c_0||) for the M candidates (cpart, cD).
  __device__ void bisector(const float* cent, int M) {
    const float* c0 = cent + (size_t)w.cpart[0] * D;
    for (int i = 1; i < M; ++i) {
      const float* ci = cent + (size_t)w.cpart[i] * D;
      float acc = 0.f;
      for (int j = lane; j < D; j += 32) {
        const float df = ci[j] - c0[j];
        acc = fmaf(df, df, acc);
      }
      acc = warp_sum_f(acc);
      if (lane == 0) {
        const float cd = sqrtf(acc);
        const float den = 2.f * cd;
        const float t = den > 0.f ? (w.cD[i] - w.cD[0]) / den : 0.f;
        w.ct[i] = t > 0.f ? (double)t : 0.0;
      }
    }
    if (lane == 0) w.ct[0] = 0.0;
    __syncwarp();
  }

  // Eq. 8-9 with the raw caps for p_0, then r = p_0 + sum of the scanned p_i.
  __device__ double probabilities(int M, double rho, const SearchArgs& a) {
    double su = 0.0, pr = 1.0;
    const double inv = rho > 0.0 ? 1.0 / rho : 0.0;
    for (int i = 1 + lane; i < M; i += 32) {
      const double u = cap_u(w.ct[i], rho, inv, a.beta_mode == QK_BETA_EXACT, a.beta_table, a.beta_a, a.beta_lnB);
      w.cp[i] = u;
      su += u;
      pr *= 1.0 - u;
    }
    const double U = warp_sum_d(su);
    const double P0 = warp_prod_d(pr);
    const double c = U > 0.0 ? (1.0 - P0) / U : 0.0;
    double rs = 0.0;
    for (int i = 1 + lane; i < M; i += 32) {
      const double p = w.cp[i] * c;
      w.cp[i] = p;
      if (w.csc[i]) rs += p;
    }
    if (lane == 0) w.cp[0] = P0;
    const double r = P0 + warp_sum_d(rs);
    __syncwarp();
    return r;
  }

  // The unscanned candidate with the largest p (ties to the lower position).
  __device__ int next(int M) {
    long long bk = -1;
    int bi = M;
    for (int i = 1 + lane; i < M; i += 32) {
      if (w.csc[i]) continue;
      const long long k = __double_as_longlong(w.cp[i]);
      if (k > bk) {
        bk = k;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long k2 = __shfl_xor_sync(0xffffffffu, bk, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (k2 > bk || (k2 == bk && i2 < bi)) {
        bk = k2;
        bi = i2;
      }
    }
    return bi;
  }

  // Scans candidate partition `pos` of level lv into R.
  __device__ void scan_pos(const DevLevel& lv, int pos, int M, unsigned long long* hits, int32_t* status,
                           int64_t* diag, int64_t qi) {
    const int part = pos >= 0 && pos < M ? w.cpart[pos] : -1;
    if (part < 0 || part >= lv.n_part) {   // never expected: record and skip
      if (lane == 0 && atomicCAS(status, 0, DEV_BAD_INDEX) == 0) {
        diag[0] = DEV_BAD_INDEX;
        diag[1] = qi;
        diag[2] = 40;
        diag[3] = pos;
        diag[4] = part;
      }
      return;
    }
    const int64_t off = lv.off[part];
    scan(lv.vec + off * D, lv.ids + off, 0, lv.size[part]);
    if (lane == 0) {
      w.csc[pos] = 1;
      if (hits) atomicAdd(&hits[part], 1ull);
    }
    __syncwarp();
  }

  // R -> the candidates of the next level (nearest first).
  __device__ int take_candidates() {
    for (int i = lane; i < rn; i += 32) {
      w.cpart[i] = (int32_t)w.ri[i];
      w.cD[i] = w.rd[i];
    }
    __syncwarp();
    return rn;
  }

  // Algorithm 1 on level lv over the M candidates, K = k results (the upper
  // level keeps k' = K candidates for the level below).
  __device__ void aps(const DevLevel& lv, int M, int k, double tau, double tau_rho, unsigned long long* hits,
                      const SearchArgs& a, int64_t qi) {
    reset(k);
    for (int i = lane; i < M; i += 32) w.csc[i] = 0;
    __syncwarp();
    bisector(lv.cent, M);
    scan_pos(lv, 0, M, hits, a.status, a.diag, qi);
    int ns = 1;
    while (rn < k && ns < M) {
      scan_pos(lv, ns, M, hits, a.status, a.diag, qi);
      ++ns;
    }
    if (rn < k) return;
    auto radius = [&]() {
      const float dk = w.rd[k - 1];
      return (double)sqrtf(dk > 0.f ? dk : 0.f);
    };
    double rho = radius();
    double r = probabilities(M, rho, a);
    int nx = next(M);
    bool go = r < tau && ns < M;
    while (go) {
      scan_pos(lv, nx, M, hits, a.status, a.diag, qi);
      ++ns;
      const double rho2 = radius();
      if (fabs(rho2 - rho) > tau_rho * rho) {
        rho = rho2;
        r = probabilities(M, rho, a);
      } else {
        r += w.cp[nx];
      }
      nx = next(M);
      go = r < tau && ns < M;
    }
  }
};

// Buffer sizes of a search: R holds the root's M_root and the upper level's
// k1 results; the candidates of a level are the root's M_root (with one
// level, the leaves exported from the root scan).
inline int rcap_of(const SearchArgs& a) { return ((std::max(a.M_root, a.L == 2 ? a.k1 : 0) + 31) / 32) * 32; }
inline int mcap_of(const SearchArgs& a) { return std::max(1, std::max(a.M_root, a.L == 2 ? a.k1 : 0)); }

template <int TPR, int NV>
__device__ void prepare_query(const SearchArgs& a, Warp<TPR, NV>& b, const int64_t qi, const int lane) {
  constexpr int D = Warp<TPR, NV>::D;
  const float* q = a.Q + qi * D;
  for (int i = lane; i < D; i += 32) b.w.sq[i] = q[i];
  __syncwarp();
  {
    const float4* q4 = reinterpret_cast<const float4*>(b.w.sq);
    const int sub = lane % TPR;
#pragma unroll
    for (int v = 0; v < NV; ++v) b.qv[v] = q4[sub + TPR * v];
  }
  float qn = 0.f;
  for (int j = lane; j < D; j += 32) qn = fmaf(b.w.sq[j], b.w.sq[j], qn);
  qn = warp_sum_f(qn);
  if (!(qn < INFINITY)) {   // refused as the per-query kernel refuses it
    if (lane == 0 && atomicCAS(a.status, 0, DEV_BAD_ARG) == 0) {
      a.diag[0] = DEV_BAD_ARG;
      a.diag[1] = qi;
      a.diag[2] = 1;
      a.diag[3] = 0;
      a.diag[4] = 0;
    }
    for (int i = lane; i < a.kq; i += 32) {
      a.out_dist[qi * a.kq + i] = NAN;
      a.out_ids[qi * a.kq + i] = -1;
    }
    if (lane == 0) {
      if (a.out_nprobe) a.out_nprobe[qi] = 0;
      if (a.out_recall) a.out_recall[qi] = NAN;
      a.xs_M[qi] = -1;
    }
    for (int i = lane; i < a.scan_cap0 && a.scan0; i += 32) a.scan0[qi * a.scan_cap0 + i] = -1;
    return;
  }
  // the top partition: every centroid of the top level, K = M_root
  b.reset(a.M_root);
  b.scan(a.root, nullptr, 0, a.n_root);
  int M = b.take_candidates();
  if (a.L == 2) {
    b.aps(a.lv[1], M, a.k1, a.tau1, a.tau_rho, a.hits1, a, qi);
    M = b.take_candidates();
  }
  b.bisector(a.lv[0].cent, M);
  for (int i = lane; i < M; i += 32) {
    a.xs_cand[qi * a.xs_mcap + i] = b.w.cpart[i];
    a.xs_t[qi * a.xs_mcap + i] = b.w.ct[i];
  }
  if (lane == 0) a.xs_M[qi] = M;
}

// Persistent: each warp takes the next query from a.work (zeroed before the
// launch), so long upper-level walks do not hold a block's other warps.  The
// walks are latency bound, so registers are capped for 6 blocks (24 warps) per
// SM: 0.72 -> 0.64 ms at d = 128 despite a few spills (8 blocks: 0.67 ms).
template <int TPR, int NV>
__global__ void __launch_bounds__(kWarps * 32, 6) aps_prepare_kernel(SearchArgs a, int rcap, int mcap) {
  using W = Warp<TPR, NV>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  W b;
  b.w = carve(smem + (size_t)warp * warp_bytes(W::D, rcap, mcap), W::D, rcap, mcap);
  b.lane = lane;
  for (;;) {
    int qi = 0;
    if (lane == 0) qi = atomicAdd(a.work, 1);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    if ((int64_t)qi >= a.nq) break;
    prepare_query<TPR, NV>(a, b, qi, lane);
    __syncwarp();
  }
}

// Whether the warp layout holds this search's candidate counts.
inline bool fits(const SearchArgs& a) {
  return a.M_root <= kRCap && (a.L == 1 || a.k1 <= kRCap) && mcap_of(a) <= kMCap && a.xs_mcap >= 1;
}

template <int TPR, int NV>
qk_status launch_t(const SearchArgs& a, cudaStream_t s) {
  constexpr int D = NV * 4 * TPR;
  const int rcap = rcap_of(a), mcap = mcap_of(a);
  const size_t smem = warp_bytes(D, rcap, mcap) * kWarps;
  static bool attr = false;   // the largest size, set once per instantiation, outside any capture
  if (!attr) {
    QK_CUDA(cudaFuncSetAttribute(aps_prepare_kernel<TPR, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(warp_bytes(D, kRCap, kMCap) * kWarps)));
    attr = true;
  }
  int per_sm = 1, dev = 0, n_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aps_prepare_kernel<TPR, NV>, kWarps * 32, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  const unsigned grid =
      (unsigned)std::min<int64_t>((a.nq + kWarps - 1) / kWarps, (int64_t)n_sm * std::max(1, per_sm));
  QK_CUDA(cudaMemsetAsync(a.work, 0, sizeof(int32_t), s));
  aps_prepare_kernel<TPR, NV><<<grid, kWarps * 32, smem, s>>>(a, rcap, mcap);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

// The per-query kernel's lane split for each dimension (TPR lanes per row).
inline qk_status launch_prepare(const SearchArgs& a, cudaStream_t s) {
  switch (a.d) {
    case 32: return launch_t<8, 1>(a, s);
    case 64: return launch_t<8, 2>(a, s);
    case 96: return launch_t<8, 3>(a, s);
    case 128: return launch_t<8, 4>(a, s);
    case 192: return launch_t<8, 6>(a, s);
    case 256: return launch_t<8, 8>(a, s);
    case 384: return launch_t<32, 3>(a, s);
    case 512: return launch_t<32, 4>(a, s);
    case 768: return launch_t<32, 6>(a, s);
    case 1024: return launch_t<32, 8>(a, s);
    default:
      set_error("unsupported dimension");
      return QK_ERR_ARG;
  }
}

}  // namespace ap
}  // namespace qk
