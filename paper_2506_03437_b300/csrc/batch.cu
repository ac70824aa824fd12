// Batched fixed-nprobe search: thousands of queries, each with its own
// nprobe, over Zipf-sized partitions (Sec. 3 top-down search with a fixed
// nprobe per query; the multi-query batching of Sec. 6).
//
// One batch runs as a fixed sequence of device steps with no host
// synchronisation, so it can be captured as one CUDA graph:
//   1. Centroid scoring on the tensor cores: the approximate (TF32) distance
//      of every query to every leaf centroid (tcgen05, tc_score.cu).
//   2. Selection, one CTA per query: the nprobe nearest centroids by exact
//      FP32 distance.  A radix select finds theta, the nprobe-th smallest
//      approximate distance.  Every approximate value is within E of the exact
//      one, so every member of the exact top-nprobe has an approximate value
//      <= theta + 2E; those centroids are re-scored exactly from the direct
//      differences and the nprobe smallest (distance, index) pairs are kept.
//      E = 2^-7 ||q|| max||c|| + 2^-14 (||q|| + max||c||)^2 bounds the TF32
//      rounding of both operands (2^-10 relative each), the FP32 accumulation
//      and the norms, with a factor two to spare.
//   3. Grouping: the (query, partition) items are counted per partition and
//      each partition's queries listed contiguously.  A unit is one partition
//      x one group of G queries x one chunk of CH rows; units are numbered
//      partition by partition in order of decreasing size.
//   4. Scan, one persistent launch: CTAs take units from a counter.  A unit's
//      rows stream through a ring of shared-memory tiles filled by bulk copies
//      (a partition is contiguous in the arena, so a tile is one copy); each
//      of the 8 warps holds QW of the unit's queries in registers and keeps
//      their top-k for the unit, so every tile is read from HBM once for all G
//      queries.  When the unit has fewer queries than G, the busy warps'
//      query sets are replicated over the idle warps, the replicas split the
//      rows of every tile, and their lists are merged at the end of the unit.
//      A per-query bound (the best k-th distance any finished unit of the
//      query has reported) prunes candidates across units.
//   5. Merge, one warp per query: the top-k over its units' candidates.
// Distances are FP32 sums of squared differences, like the per-query search.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "index.cuh"
#include "grouped.cuh"
#include "trace.h"

namespace qk {

qk_status launch_tc_distances(const float* X, int64_t n, int d, const float* C, int K, const float* cnorm, int metric,
                              float* dout, int64_t ldd, int32_t* status, int n_sm, cudaStream_t s);
qk_status launch_row_norms(const float* C, int64_t K, int d, float* out, cudaStream_t s);

namespace bt {

// ---------------------------------------------------------------- selection

struct SelArgs {
  float* Dm = nullptr;          // nq x ldd approximate distances (overwritten by exact ones on fallback)
  int64_t ldd = 0;
  int32_t K = 0;
  int d = 0;
  const float* Q = nullptr;
  const float* C = nullptr;
  const uint32_t* cmax2 = nullptr;   // max ||c||^2 (float bits)
  const int32_t* nprobe = nullptr;
  int32_t max_nprobe = 0;
  int32_t* sel = nullptr;        // nq x max_nprobe
  int32_t* nsel = nullptr;
  const int32_t* size = nullptr;
  int CH = 4096;
  int32_t* pcount = nullptr;
  int64_t* qslots = nullptr;     // chunks of the query's partitions
  int32_t* status = nullptr;
  int64_t* diag = nullptr;
};

__device__ float exact_l2(const float* q, const float* c, int d, int lane) {
  float acc = 0.f;
  for (int j = lane; j < d; j += 32) {
    float e = q[j] - c[j];
    acc = fmaf(e, e, acc);
  }
  return warp_sum_f(acc);
}

// Key of the rank-th smallest (1-based) of row[0..K): four 8-bit radix passes
// over a shared histogram.
// The row is read as float4: its stride is a multiple of 4 floats (16-byte
// aligned), and the padding after K is skipped.
__device__ uint32_t radix_select(const float* row, int K, int rank, uint32_t* hist, int* s_b, int* s_rank) {
  const float4* row4 = reinterpret_cast<const float4*>(row);
  const int K4 = (K + 3) >> 2;
  uint32_t prefix = 0, mask = 0;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int c4 = threadIdx.x; c4 < K4; c4 += blockDim.x) {
      const float4 v = row4[c4];
      const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (4 * c4 + t >= K) break;
        const uint32_t key = fkey(e[t]);
        if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t cum = 0;
      int b = 255;
      for (int i = 0; i < 256; ++i) {
        if (cum + hist[i] >= (uint32_t)rank) {
          b = i;
          break;
        }
        cum += hist[i];
      }
      *s_b = b;
      *s_rank = rank - (int)cum;
    }
    __syncthreads();
    prefix |= (uint32_t)(*s_b) << shift;
    mask |= 255u << shift;
    rank = *s_rank;
    __syncthreads();
  }
  return prefix;
}

__global__ void __launch_bounds__(kSelThreads) select_kernel(SelArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float* sq = reinterpret_cast<float*>(smem);                  // d
  float* cdist = sq + a.d;                                     // kSelCap
  int32_t* cidx = reinterpret_cast<int32_t*>(cdist + kSelCap); // kSelCap
  uint32_t* hist = reinterpret_cast<uint32_t*>(cidx + kSelCap);
  int* s_int = reinterpret_cast<int*>(hist + 256);             // [0] count, [1] bin, [2] rank
  float* s_f = reinterpret_cast<float*>(s_int + 4);
  __shared__ long long s_ch[kSelThreads / 32];
  const int q = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nwarps = blockDim.x >> 5;
  float* row = a.Dm + (int64_t)q * a.ldd;
  const int K = a.K;
  int M = a.nprobe[q];
  if (M < 1 || M > a.max_nprobe) {
    if (tid == 0) {
      a.nsel[q] = 0;
      a.qslots[q] = 0;
      report_once(a.status, a.diag, DEV_BAD_ARG, -3, q, M);
    }
    return;
  }
  M = min(M, K);
  for (int j = tid; j < a.d; j += blockDim.x) sq[j] = a.Q[(int64_t)q * a.d + j];
  __syncthreads();
  if (warp == 0) {
    float qn = 0.f;
    for (int j = lane; j < a.d; j += 32) qn = fmaf(sq[j], sq[j], qn);
    qn = warp_sum_f(qn);
    if (lane == 0) {
      const float qnorm = sqrtf(qn), cmax = sqrtf(__uint_as_float(*a.cmax2));
      const float s = qnorm + cmax;
      s_f[0] = 0.0078125f * qnorm * cmax + 6.103515625e-05f * s * s;   // 2^-7 and 2^-14
      s_int[3] = !(qn < INFINITY);
    }
  }
  __syncthreads();
  if (s_int[3]) {   // a NaN or infinite element, or a norm beyond FP32: refused like a bad nprobe
    if (tid == 0) {
      a.nsel[q] = 0;
      a.qslots[q] = 0;
      report_once(a.status, a.diag, DEV_BAD_ARG, -5, q, 0);
    }
    return;
  }
  const float E = s_f[0];
  // with every centroid wanted, or when the bound lets too many through, the
  // exact distances of all centroids replace the approximate row
  bool exact_row = M == K;
  for (int round = 0; round < 2; ++round) {
    if (exact_row) {
      for (int c = warp; c < K; c += nwarps) {
        const float v = exact_l2(sq, a.C + (int64_t)c * a.d, a.d, lane);
        if (lane == 0) row[c] = v;
      }
      __syncthreads();
    }
    const float theta = fkey_inv(radix_select(row, K, M, hist, &s_int[1], &s_int[2]));
    const float lim = exact_row ? theta : __fadd_ru(theta, 2.f * E);
    if (tid == 0) s_int[0] = 0;
    __syncthreads();
    const float4* row4 = reinterpret_cast<const float4*>(row);
    for (int c4 = tid; c4 < ((K + 3) >> 2); c4 += blockDim.x) {
      const float4 v = row4[c4];
      const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = 4 * c4 + t;
        if (c < K && e[t] <= lim) {
          const int pos = atomicAdd(&s_int[0], 1);
          if (pos < kSelCap) cidx[pos] = c;
        }
      }
    }
    __syncthreads();
    const int count = s_int[0];
    if (count <= kSelCap) break;
    if (exact_row) {   // more than kSelCap exact ties at the nprobe-th distance
      if (tid == 0) {
        a.nsel[q] = 0;
        a.qslots[q] = 0;
        report_once(a.status, a.diag, DEV_BAD_INDEX, -4, q, count);
      }
      return;
    }
    exact_row = true;
    __syncthreads();
  }
  const int count = min(s_int[0], kSelCap);
  // exact distances of the candidates (taken from the row when it is exact)
  for (int i = warp; i < count; i += nwarps) {
    const int c = cidx[i];
    const float v = exact_row ? row[c] : exact_l2(sq, a.C + (int64_t)c * a.d, a.d, lane);
    if (lane == 0) cdist[i] = v;
  }
  int P = 1;
  while (P < count) P <<= 1;
  for (int i = count + tid; i < P; i += blockDim.x) {
    cdist[i] = INFINITY;
    cidx[i] = 0x7fffffff;
  }
  __syncthreads();
  // bitonic sort of the P (distance, index) pairs
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const bool j_smaller = pair_less(cdist[j], cidx[j], cdist[i], cidx[i]);
          if (j_smaller == up) {
            const float td = cdist[i];
            cdist[i] = cdist[j];
            cdist[j] = td;
            const int32_t ti = cidx[i];
            cidx[i] = cidx[j];
            cidx[j] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  long long chunks = 0;
  for (int i = tid; i < M; i += blockDim.x) {
    const int p = cidx[i];
    a.sel[(int64_t)q * a.max_nprobe + i] = p;
    atomicAdd(&a.pcount[p], 1);
    chunks += (a.size[p] + a.CH - 1) / a.CH;
  }
  for (int o = 16; o > 0; o >>= 1) chunks += __shfl_xor_sync(0xffffffffu, chunks, o);
  if (lane == 0) s_ch[warp] = chunks;
  __syncthreads();
  if (tid == 0) {
    long long t = 0;
    for (int w = 0; w < nwarps; ++w) t += s_ch[w];
    a.qslots[q] = t;
    a.nsel[q] = M;
  }
}

}  // namespace bt
}  // namespace qk

// ---------------------------------------------------------------- the plan

using namespace qk;

struct qk_batch {
  qk_index* ix = nullptr;
  int64_t max_nq = 0;
  int32_t k = 0, max_nprobe = 0;
  qk_batch_tiles tiles{};
  int n_sm = 148;
  // shape the workspace was sized for
  int32_t K = 0;
  int64_t ldd = 0;
  int64_t cand_cap = 0;
  int32_t ch_min = 0;
  uint64_t version = ~0ull;      // index version the order and sizes were taken from
  // device workspace
  float* Dm = nullptr;
  float* cnorm = nullptr;
  uint32_t* cmax2 = nullptr;
  int32_t* sel = nullptr;
  int32_t* nsel = nullptr;
  int32_t* pcount = nullptr;
  int32_t* pcur = nullptr;
  int32_t* pstart = nullptr;
  int32_t* qlist = nullptr;
  int32_t* order = nullptr;
  int64_t* ustart = nullptr;
  int64_t* tmp = nullptr;
  int64_t* tmp2 = nullptr;
  int64_t* n_units = nullptr;
  int64_t* qslots = nullptr;
  int64_t* qcoff = nullptr;
  int32_t* qcnt = nullptr;
  uint32_t* gtau = nullptr;
  float* cd = nullptr;
  int64_t* ci = nullptr;
  unsigned long long* work = nullptr;
  int scan_blocks = 0;           // CTAs per SM of the scan for scan_tiles
  qk_batch_tiles scan_tiles{};
  // the captured graph
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_version = 0;
  // stage timing of uncaptured batches (events at the stage boundaries)
  bool timing = false;
  bool timed = false;
  cudaEvent_t ev[6] = {};
};

namespace {

template <class T>
qk_status balloc(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  QK_CUDA(cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T)));
  return QK_OK;
}
template <class T>
void bfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_events(qk_batch* b) {
  for (cudaEvent_t& e : b->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
}

void free_workspace(qk_batch* b) {
  bfree(b->Dm);
  bfree(b->cnorm);
  bfree(b->cmax2);
  bfree(b->sel);
  bfree(b->nsel);
  bfree(b->pcount);
  bfree(b->pcur);
  bfree(b->pstart);
  bfree(b->qlist);
  bfree(b->order);
  bfree(b->ustart);
  bfree(b->tmp);
  bfree(b->tmp2);
  bfree(b->n_units);
  bfree(b->qslots);
  bfree(b->qcoff);
  bfree(b->qcnt);
  bfree(b->gtau);
  bfree(b->cd);
  bfree(b->ci);
  bfree(b->work);
}

// Row chunks beyond the first of every partition, summed.
int64_t extra_chunks(const std::vector<int32_t>& sizes, int CH) {
  int64_t x = 0;
  for (int32_t s : sizes) x += std::max<int64_t>(0, ((int64_t)s + CH - 1) / CH - 1);
  return x;
}

bool dim_ok(int d) {
  switch (d) {
    case 32: case 64: case 96: case 128: case 192: case 256: case 384: case 512: case 768: case 1024: return true;
    default: return false;
  }
}

template <int D, int QW>
size_t scan_smem(int TR) {
  return sizeof(float) * bt::kStages * (size_t)TR * D + sizeof(uint64_t) * bt::kStages +
         (sizeof(float) + sizeof(int32_t)) * (size_t)bt::kWarps * QW * bt::kBuf + sizeof(bt::UnitInfo) +
         sizeof(int32_t) * bt::kWarps * QW + sizeof(int32_t) * (2 * bt::kStages + 2) + 16;
}

// Launches the scan with (SMs x CTAs an SM holds) CTAs.  The attribute and
// occupancy queries run outside stream capture and are cached in *per_sm; a
// captured launch reuses the cached value.
template <int D, int QW>
qk_status launch_scan_t(const bt::ScanArgs& a, int n_sm, bool capturing, int* per_sm, cudaStream_t s) {
  if constexpr (bt::tpr_for(D, QW) == 0) {
    set_error("queries_per_warp " + std::to_string(QW) + " is not available for d = " + std::to_string(D));
    return QK_ERR_ARG;
  } else {
    const size_t smem = scan_smem<D, QW>(a.TR);
    if (smem > 227 * 1024) {
      set_error("tile_rows too large for shared memory");
      return QK_ERR_ARG;
    }
    if (!capturing) {
      QK_CUDA(cudaFuncSetAttribute(bt::grouped_scan_kernel<D, QW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
      int n = 0;
      QK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, bt::grouped_scan_kernel<D, QW>, bt::kThreads, smem));
      *per_sm = std::max(1, n);
    } else if (*per_sm < 1) {
      set_error("capture without a prior run of the same tiles");
      return QK_ERR_STATE;
    }
    bt::grouped_scan_kernel<D, QW><<<n_sm * *per_sm, bt::kThreads, smem, s>>>(a);
    QK_CUDA(cudaGetLastError());
    return QK_OK;
  }
}

template <int D>
qk_status launch_scan_d(const bt::ScanArgs& a, int QW, int n_sm, bool cap, int* per_sm, cudaStream_t s) {
  switch (QW) {
    case 1: return launch_scan_t<D, 1>(a, n_sm, cap, per_sm, s);
    case 2: return launch_scan_t<D, 2>(a, n_sm, cap, per_sm, s);
    case 4: return launch_scan_t<D, 4>(a, n_sm, cap, per_sm, s);
    default: set_error("queries_per_warp must be 1, 2 or 4"); return QK_ERR_ARG;
  }
}

qk_status launch_scan(const bt::ScanArgs& a, int d, int QW, int n_sm, bool cap, int* per_sm, cudaStream_t s) {
  switch (d) {
    case 32: return launch_scan_d<32>(a, QW, n_sm, cap, per_sm, s);
    case 64: return launch_scan_d<64>(a, QW, n_sm, cap, per_sm, s);
    case 96: return launch_scan_d<96>(a, QW, n_sm, cap, per_sm, s);
    case 128: return launch_scan_d<128>(a, QW, n_sm, cap, per_sm, s);
    case 192: return launch_scan_d<192>(a, QW, n_sm, cap, per_sm, s);
    case 256: return launch_scan_d<256>(a, QW, n_sm, cap, per_sm, s);
    case 384: return launch_scan_d<384>(a, QW, n_sm, cap, per_sm, s);
    case 512: return launch_scan_d<512>(a, QW, n_sm, cap, per_sm, s);
    case 768: return launch_scan_d<768>(a, QW, n_sm, cap, per_sm, s);
    case 1024: return launch_scan_d<1024>(a, QW, n_sm, cap, per_sm, s);
    default: set_error("unsupported dimension"); return QK_ERR_ARG;
  }
}

bool tiles_valid(const qk_batch* b, const qk_batch_tiles& t, std::string* why) {
  const int d = b->ix->cfg.d;
  if (t.queries_per_warp != 1 && t.queries_per_warp != 2 && t.queries_per_warp != 4) {
    *why = "queries_per_warp must be 1, 2 or 4";
    return false;
  }
  if (bt::tpr_for(d, t.queries_per_warp) == 0) {
    *why = "queries_per_warp " + std::to_string(t.queries_per_warp) + " is not available for d = " + std::to_string(d);
    return false;
  }
  if (t.tile_rows < 1 || (size_t)bt::kStages * t.tile_rows * d * 4 > 200 * 1024) {
    *why = "tile_rows must be >= 1 with 3 tiles of rows within 200 KB";
    return false;
  }
  if (t.chunk_rows < t.tile_rows || t.chunk_rows < b->ch_min) {
    *why = "chunk_rows must be >= tile_rows and >= 1024";
    return false;
  }
  if (t.rows_per_thread != 0 &&
      !(t.rows_per_thread == 2 && bt::rows_layout_ok(d))) {
    *why = "rows_per_thread must be 0, or 2 with d <= 256";
    return false;
  }
  return true;
}

// Re-reads the partition sizes and shape of the index and re-sizes the
// workspace where it no longer fits.  Host work; never inside a capture.
qk_status refresh(qk_batch* b, cudaStream_t s) {
  qk_index* ix = b->ix;
  if (b->version == ix->version && b->K == ix->n_leaf) return QK_OK;
  // the plan's batches still in flight on s use the workspace re-sized below
  QK_CUDA(cudaStreamSynchronize(s));
  const int32_t K = ix->n_leaf;
  const int64_t ldd = ((int64_t)K + 3) / 4 * 4;
  const int64_t need_cand =
      (int64_t)b->k * b->max_nq * ((int64_t)std::min(b->max_nprobe, K) + extra_chunks(ix->h_size0, b->ch_min));
  if (K != b->K) {
    QK_TRY(balloc(&b->Dm, (size_t)b->max_nq * ldd));
    QK_TRY(balloc(&b->cnorm, (size_t)K));
    QK_TRY(balloc(&b->pcount, (size_t)K));
    QK_TRY(balloc(&b->pcur, (size_t)K));
    QK_TRY(balloc(&b->pstart, (size_t)K));
    QK_TRY(balloc(&b->order, (size_t)K));
    QK_TRY(balloc(&b->ustart, (size_t)K + 1));
    QK_TRY(balloc(&b->tmp, (size_t)std::max<int64_t>(K, b->max_nq)));
    QK_TRY(balloc(&b->tmp2, (size_t)std::max<int64_t>(K, b->max_nq)));
    b->K = K;
    b->ldd = ldd;
  }
  if (need_cand > b->cand_cap) {
    const int64_t cap = need_cand + need_cand / 8;
    QK_TRY(balloc(&b->cd, (size_t)cap));
    QK_TRY(balloc(&b->ci, (size_t)cap));
    b->cand_cap = cap;
  }
  std::vector<int32_t> order(K);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t x, int32_t y) { return ix->h_size0[x] > ix->h_size0[y]; });
  QK_CUDA(cudaMemcpyAsync(b->order, order.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
  QK_CUDA(cudaStreamSynchronize(s));
  b->version = ix->version;
  return QK_OK;
}

// The batch's device steps (no host synchronisation, no allocation).
qk_status enqueue(qk_batch* b, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids, float* out_dist,
                  cudaStream_t s) {
  qk_index* ix = b->ix;
  const int d = ix->cfg.d, K = b->K;
  const qk_batch_tiles& t = b->tiles;
  const int G = t.rows_per_thread == 2 ? bt::kRowsG : bt::kWarps * t.queries_per_warp;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  QK_CUDA(cudaStreamIsCapturing(s, &cs));
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  if (capturing && !(b->scan_tiles.queries_per_warp == t.queries_per_warp && b->scan_tiles.tile_rows == t.tile_rows &&
                     b->scan_tiles.rows_per_thread == t.rows_per_thread))
    b->scan_blocks = 0;
  const bool timing = b->timing && !capturing;
  static const char* const kStage[6] = {"start", "scoring", "selection", "grouping", "scan", "merge"};
  Trace tr("batch");
  auto mark = [&](int i) -> qk_status {
    if (i > 0) tr.mark(kStage[i]);
    if (timing) QK_CUDA(cudaEventRecord(b->ev[i], s));
    return QK_OK;
  };
  QK_TRY(mark(0));
  QK_CUDA(cudaMemsetAsync(b->cmax2, 0, sizeof(uint32_t), s));
  QK_CUDA(cudaMemsetAsync(b->pcount, 0, sizeof(int32_t) * K, s));
  QK_CUDA(cudaMemsetAsync(b->pcur, 0, sizeof(int32_t) * K, s));
  QK_CUDA(cudaMemsetAsync(b->qcnt, 0, sizeof(int32_t) * nq, s));
  QK_CUDA(cudaMemsetAsync(b->gtau, 0x7f, sizeof(uint32_t) * nq, s));   // 0x7f7f7f7f = 3.4e38: no bound yet
  QK_CUDA(cudaMemsetAsync(b->work, 0, sizeof(unsigned long long), s));
  QK_TRY(launch_row_norms(ix->cent0, K, d, b->cnorm, s));
  bt::max_norm_kernel<<<std::max(1, std::min(64, (K + 255) / 256)), 256, 0, s>>>(b->cnorm, K, b->cmax2);
  QK_CUDA(cudaGetLastError());
  QK_TRY(launch_tc_distances(q, nq, d, ix->cent0, K, b->cnorm, QK_METRIC_L2, b->Dm, b->ldd, ix->status, b->n_sm, s));
  QK_TRY(mark(1));
  bt::SelArgs sa;
  sa.Dm = b->Dm;
  sa.ldd = b->ldd;
  sa.K = K;
  sa.d = d;
  sa.Q = q;
  sa.C = ix->cent0;
  sa.cmax2 = b->cmax2;
  sa.nprobe = nprobe;
  sa.max_nprobe = b->max_nprobe;
  sa.sel = b->sel;
  sa.nsel = b->nsel;
  sa.size = ix->size0;
  sa.CH = t.chunk_rows;
  sa.pcount = b->pcount;
  sa.qslots = b->qslots;
  sa.status = ix->status;
  sa.diag = ix->diag;
  // at most 4 KB + 32 KB + 1 KB: within the default dynamic shared-memory limit
  const size_t sel_smem = sizeof(float) * d + (sizeof(float) + sizeof(int32_t)) * bt::kSelCap + 256 * 4 + 4 * 4 + 16;
  bt::select_kernel<<<(unsigned)nq, bt::kSelThreads, sel_smem, s>>>(sa);
  QK_CUDA(cudaGetLastError());
  QK_TRY(mark(2));
  bt::GroupArgs ga;
  ga.K = K;
  ga.nq = nq;
  ga.G = G;
  ga.CH = t.chunk_rows;
  ga.k = b->k;
  ga.size = ix->size0;
  ga.order = b->order;
  ga.pcount = b->pcount;
  ga.pstart = b->pstart;
  ga.tmp = b->tmp;
  ga.tmp2 = b->tmp2;
  ga.ustart = b->ustart;
  ga.n_units = b->n_units;
  ga.qslots = b->qslots;
  ga.qcoff = b->qcoff;
  ga.cand_cap = b->cand_cap;
  ga.status = ix->status;
  ga.diag = ix->diag;
  bt::group_kernel<<<1, 1024, 0, s>>>(ga);
  QK_CUDA(cudaGetLastError());
  const int64_t items = nq * b->max_nprobe;
  bt::fill_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(b->sel, b->nsel, nq, b->max_nprobe, b->pstart,
                                                                   b->pcur, b->qlist);
  QK_CUDA(cudaGetLastError());
  QK_TRY(mark(3));
  bt::ScanArgs sc;
  sc.vec = ix->vec0;
  sc.x_rows = ix->cap0;
  sc.ids = ix->ids0;
  sc.off = ix->off0;
  sc.size = ix->size0;
  sc.Q = q;
  sc.k = b->k;
  sc.CH = t.chunk_rows;
  sc.TR = t.tile_rows;
  sc.order = b->order;
  sc.ustart = b->ustart;
  sc.K = K;
  sc.n_units = b->n_units;
  sc.pstart = b->pstart;
  sc.pcount = b->pcount;
  sc.qlist = b->qlist;
  sc.qcoff = b->qcoff;
  sc.qcnt = b->qcnt;
  sc.gtau = b->gtau;
  sc.cd = b->cd;
  sc.ci = b->ci;
  sc.work = b->work;
  sc.status = ix->status;
  if (t.rows_per_thread == 2)
    QK_TRY(bt::launch_scan_rows(sc, d, b->n_sm, capturing, &b->scan_blocks, s));
  else
    QK_TRY(launch_scan(sc, d, t.queries_per_warp, b->n_sm, capturing, &b->scan_blocks, s));
  b->scan_tiles = t;
  QK_TRY(mark(4));
  bt::merge_kernel<<<(unsigned)((nq + bt::kWarps - 1) / bt::kWarps), bt::kThreads, 0, s>>>(
      b->cd, b->ci, b->qcoff, b->qcnt, nq, b->k, out_ids, out_dist);
  QK_CUDA(cudaGetLastError());
  QK_TRY(mark(5));
  if (timing) b->timed = true;
  return QK_OK;
}

qk_status check_call(qk_batch* b, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids,
                     float* out_dist) {
  if (!b) {
    set_error("null plan");
    return QK_ERR_ARG;
  }
  if (!b->ix->ready) {
    set_error("index is empty: build or load it first");
    return QK_ERR_STATE;
  }
  if (b->ix->cfg.storage != QK_STORE_F32 || b->ix->cfg.metric != QK_METRIC_L2) {
    set_error("batched search supports L2 over FP32 storage");
    return QK_ERR_ARG;
  }
  if (nq < 0 || nq > b->max_nq) {
    set_error("nq must be in [0, max_nq]");
    return QK_ERR_ARG;
  }
  if (nq == 0) return QK_OK;
  for (const void* p : {(const void*)q, (const void*)nprobe, (const void*)out_ids, (const void*)out_dist}) {
    if (!p || !is_device_ptr(p) || reinterpret_cast<uintptr_t>(p) % 16 != 0) {
      set_error("batched search takes 16-byte aligned device buffers");
      return QK_ERR_ARG;
    }
  }
  return QK_OK;
}

}  // namespace

extern "C" {

qk_status qk_batch_create(qk_index* ix, int64_t max_nq, int32_t k, int32_t max_nprobe, qk_batch** out) {
  QK_GUARD_BEGIN
  if (!ix || !out) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  *out = nullptr;
  if (!ix->ready) {
    set_error("index is empty: build or load it first");
    return QK_ERR_STATE;
  }
  if (ix->cfg.metric != QK_METRIC_L2 || ix->cfg.storage != QK_STORE_F32) {
    set_error("batched search supports L2 over FP32 storage");
    return QK_ERR_ARG;
  }
  if (!dim_ok(ix->cfg.d)) {
    set_error("unsupported dimension");
    return QK_ERR_ARG;
  }
  if (max_nq < 1 || k < 1 || k > bt::kMaxK || max_nprobe < 1 || max_nprobe > bt::kMaxNprobe) {
    set_error("need max_nq >= 1, 1 <= k <= 32, 1 <= max_nprobe <= 2048");
    return QK_ERR_ARG;
  }
  qk_batch* b = new qk_batch();
  b->ix = ix;
  b->max_nq = max_nq;
  b->k = k;
  b->max_nprobe = max_nprobe;
  b->tiles.queries_per_warp = 2;
  b->tiles.tile_rows = std::max(8, std::min(64, 8192 / ix->cfg.d));
  b->tiles.chunk_rows = 4096;
  b->ch_min = 1024;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
  qk_status st = QK_OK;
  auto run = [&](qk_status s2) {
    if (st == QK_OK) st = s2;
  };
  run(balloc(&b->cmax2, 1));
  run(balloc(&b->sel, (size_t)max_nq * max_nprobe));
  run(balloc(&b->nsel, (size_t)max_nq));
  run(balloc(&b->qlist, (size_t)max_nq * max_nprobe));
  run(balloc(&b->n_units, 1));
  run(balloc(&b->qslots, (size_t)max_nq));
  run(balloc(&b->qcoff, (size_t)max_nq + 1));
  run(balloc(&b->qcnt, (size_t)max_nq));
  run(balloc(&b->gtau, (size_t)max_nq));
  run(balloc(&b->work, 1));
  if (st == QK_OK) st = refresh(b, 0);
  if (st != QK_OK) {
    free_workspace(b);
    delete b;
    return st;
  }
  *out = b;
  return QK_OK;
  QK_GUARD_END
}

void qk_batch_destroy(qk_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  free_events(b);
  free_workspace(b);
  delete b;
}

qk_status qk_batch_set_timing(qk_batch* b, int32_t on) {
  QK_GUARD_BEGIN
  if (!b) {
    set_error("null plan");
    return QK_ERR_ARG;
  }
  if (on && !b->ev[0])
    for (cudaEvent_t& e : b->ev) QK_CUDA(cudaEventCreate(&e));
  b->timing = on != 0;
  b->timed = false;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_batch_stage_times(qk_batch* b, float* ms) {
  QK_GUARD_BEGIN
  if (!b || !ms) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  if (!b->timed) {
    set_error("no timed batch: enable timing and run qk_batch_search first");
    return QK_ERR_STATE;
  }
  QK_CUDA(cudaEventSynchronize(b->ev[5]));
  for (int i = 0; i < 5; ++i) QK_CUDA(cudaEventElapsedTime(&ms[i], b->ev[i], b->ev[i + 1]));
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_batch_get_tiles(const qk_batch* b, qk_batch_tiles* out) {
  QK_GUARD_BEGIN
  if (!b || !out) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  *out = b->tiles;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_batch_set_tiles(qk_batch* b, const qk_batch_tiles* t) {
  QK_GUARD_BEGIN
  if (!b || !t) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  std::string why;
  if (!tiles_valid(b, *t, &why)) {
    set_error(why);
    return QK_ERR_ARG;
  }
  b->tiles = *t;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_batch_search(qk_batch* b, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids,
                          float* out_dist, void* stream) {
  QK_GUARD_BEGIN
  // the index's published structure stays put while this captures and enqueues it
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  QK_TRY(check_call(b, q, nq, nprobe, out_ids, out_dist));
  if (nq == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  QK_TRY(refresh(b, s));
  QK_TRY(enqueue(b, q, nq, nprobe, out_ids, out_dist, s));
  note_readers(b->ix, s);
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_batch_capture(qk_batch* b, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids,
                           float* out_dist, void* stream) {
  QK_GUARD_BEGIN
  // the index's published structure stays put while this captures and enqueues it
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  QK_TRY(check_call(b, q, nq, nprobe, out_ids, out_dist));
  if (nq == 0) {
    set_error("nothing to capture");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (s == 0) {
    set_error("capture needs a created stream, not the legacy default stream");
    return QK_ERR_ARG;
  }
  QK_TRY(refresh(b, s));
  // one ordinary run first: kernel attributes and occupancy are set outside the capture
  QK_TRY(enqueue(b, q, nq, nprobe, out_ids, out_dist, s));
  QK_CUDA(cudaStreamSynchronize(s));
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  QK_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  qk_status st = enqueue(b, q, nq, nprobe, out_ids, out_dist, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != QK_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_status(e, "stream capture");
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return cuda_status(e, "graph instantiate");
  }
  b->graph_version = b->ix->version;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_batch_replay(qk_batch* b, void* stream) {
  QK_GUARD_BEGIN
  // the index's published structure stays put while this captures and enqueues it
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  if (!b || !b->graph) {
    set_error("no captured batch");
    return QK_ERR_STATE;
  }
  if (b->graph_version != b->ix->version) {
    set_error("the index changed since the capture: capture again");
    return QK_ERR_STATE;
  }
  QK_CUDA(cudaGraphLaunch(b->graph, (cudaStream_t)stream));
  note_readers(b->ix, (cudaStream_t)stream);
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_batch_autotune(qk_batch* b, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids,
                            float* out_dist, int32_t reps, qk_batch_tiles* chosen, void* stream) {
  QK_GUARD_BEGIN
  // the index's published structure stays put while this captures and enqueues it
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  QK_TRY(check_call(b, q, nq, nprobe, out_ids, out_dist));
  if (nq == 0) {
    set_error("nothing to tune on");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  QK_TRY(refresh(b, s));
  reps = std::max(1, reps);
  std::vector<qk_batch_tiles> cands;
  for (int rpt : {0, 2})
    for (int qw : {1, 2, 4})
      for (int tr : {16, 32, 64})
        for (int ch : {1024, 4096, 16384}) {
          if (rpt == 2 && (tr != 64 || qw != 2)) continue;   // the whole-rows scan has its own tiles and units
          qk_batch_tiles t{qw, tr, ch, rpt};
          std::string why;
          if (tiles_valid(b, t, &why)) cands.push_back(t);
        }
  cudaEvent_t e0, e1;
  QK_CUDA(cudaEventCreate(&e0));
  QK_CUDA(cudaEventCreate(&e1));
  float best = INFINITY;
  qk_batch_tiles best_t = b->tiles;
  const qk_batch_tiles keep = b->tiles;
  qk_status st = QK_OK;
  for (const qk_batch_tiles& t : cands) {
    b->tiles = t;
    st = enqueue(b, q, nq, nprobe, out_ids, out_dist, s);   // warm-up
    if (st != QK_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == QK_OK; ++r) st = enqueue(b, q, nq, nprobe, out_ids, out_dist, s);
    cudaEventRecord(e1, s);
    if (st != QK_OK) break;
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = cuda_status(e, "autotune");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tiles = st == QK_OK ? best_t : keep;
  if (chosen) *chosen = b->tiles;
  return st;
  QK_GUARD_END
}

}  // extern "C"
