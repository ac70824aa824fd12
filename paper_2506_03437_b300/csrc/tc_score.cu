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
// One CTA = 4 warps owns 128 rows and sweeps the centroids in tiles of 256.
// Each K-slice of 32 elements of both operands is staged in shared memory
// with cp.async in a no-swizzle K-major layout built from 8-row x 16-byte
// core matrices, then thread 0 issues four K=8 MMAs into a 128 x 256 FP32
// accumulator in TMEM and commits them to an mbarrier.  Two slice buffers
// let the loads of slice s+1 overlap the MMAs of slice s.  The epilogue reads
// the accumulator with tcgen05.ld (each warp its 32 TMEM lanes = 32 rows).
#include <cuda_runtime.h>

#include <algorithm>
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace qk {

namespace tc {

constexpr int kM = 128;        // rows per CTA (TMEM lanes)
constexpr int kN = 256;        // centroids per tile (TMEM columns)
constexpr int kKS = 32;        // K elements per staged slice
constexpr int kThreads = 256;  // 8 warps: warps w and w + 4 share TMEM lanes, split the columns
constexpr int kT = 16;         // approximate candidates kept per row (k <= 8)
constexpr int kT1 = 4;         // ... when only the nearest centroid is wanted

constexpr int kSliceA = kM * kKS * 4;    // 16 KB
constexpr int kSliceB = kN * kKS * 4;    // 32 KB
constexpr int kSmem = 2 * (kSliceA + kSliceB) + kN * 4 + 64;

// Instruction descriptor of kind::tf32 (PTX ISA, tcgen05 instruction
// descriptor): D format F32 (bits 4-5 = 1), A and B format TF32 (bits 7-9
// and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22,
// M >> 4 at bits 24-28, dense, no negation.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

// Shared-memory matrix descriptor (PTX ISA, tcgen05 shared memory
// descriptor): start address >> 4 at bits 0-13, leading-dimension byte
// offset >> 4 at bits 16-29, stride-dimension byte offset >> 4 at bits 32-45,
// the fixed value 1 at bits 46-47, base offset 0, no swizzle (bits 61-63 = 0).
// For a K-major operand without swizzle the leading dimension is K (the
// distance between core matrices adjacent in K) and the stride dimension is
// M/N (between core matrices adjacent in rows).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  int n = valid ? 16 : 0;   // src-size 0 fills the 16 bytes with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* holder, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(holder)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

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

// Approximate top-T candidates per row (see the file comment).  With kStore
// the epilogue instead writes every approximate distance to dout (row r,
// centroid c at dout[r * ldd + c]), and blockIdx.y selects the range of
// `span` centroids (a multiple of the tile width) that this CTA sweeps.
template <int T, bool kStore>
__global__ void __launch_bounds__(tc::kThreads) tc_candidates_kernel(const float* __restrict__ X, int64_t n, int d,
                                                                     const float* __restrict__ C, int K,
                                                                     const float* __restrict__ cnorm, int metric,
                                                                     int32_t* __restrict__ cand,
                                                                     int32_t* __restrict__ status,
                                                                     float* __restrict__ dout, int64_t ldd,
                                                                     int span) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* scn = reinterpret_cast<float*>(smem + 2 * (kSliceA + kSliceB));   // ||c||^2 of the tile
  uint64_t* bars = reinterpret_cast<uint64_t*>(scn + kN);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int quarter = warp & 3, half = warp >> 2;   // TMEM lanes 32 * quarter.., columns 128 * half..
  const int64_t row0 = (int64_t)blockIdx.x * kM;

  if (warp == 0) tmem_alloc(tmem_holder, kN);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_holder;

  // this thread's row and its running top-T over its half of every tile (ascending)
  const int my_lane = quarter * 32 + (tid & 31);
  const int64_t my_row = row0 + my_lane;
  float bd[T];
  int32_t bi[T];
#pragma unroll
  for (int i = 0; i < T; ++i) {
    bd[i] = INFINITY;
    bi[i] = -1;
  }
  const int nslices = d / kKS;
  const int n_begin = kStore ? (int)blockIdx.y * span : 0;
  const int n_end = kStore ? min(K, n_begin + span) : K;
  uint32_t phase[2] = {0u, 0u};
  uint32_t issued[2] = {0u, 0u};   // commits outstanding per buffer (0 or 1)
  bool ok = true;

  // a buffer is free once the MMAs that read it have completed
  auto free_buffer = [&](int b) {
    if (!issued[b]) return;
    if (!mbar_wait_bounded(&bars[b], phase[b])) {
      ok = false;
      atomicExch(status, DEV_TIMEOUT);
    }
    phase[b] ^= 1u;
    issued[b] = 0;
  };
  // slice ks into buffer b: 8-row groups, each holding its 8 K-chunks of 16
  // bytes as consecutive core matrices: (row r, chunk c) at
  // ((r / 8) * 8 + c) * 128 + (r % 8) * 16.  K stride 128 B, row-group stride
  // 1024 B, so every address the descriptors can form stays inside the slice.
  // Consecutive threads take consecutive 16-byte chunks of one row, so a warp
  // reads whole 128-byte row segments from global memory.
  auto stage = [&](int n0, int ks, int b) {
    const uint32_t a_base = smem_u32(smem + b * kSliceA), b_base = smem_u32(smem + 2 * kSliceA + b * kSliceB);
    for (int e = tid; e < kM * (kKS / 4); e += kThreads) {
      int c = e % (kKS / 4), r = e / (kKS / 4);
      int64_t gr = row0 + r;
      bool v = gr < n;
      const float* src = X + (v ? gr : 0) * d + ks * kKS + c * 4;
      cp_async16(a_base + ((r >> 3) * (kKS / 4) + c) * 128 + (r & 7) * 16, src, v);
    }
    for (int e = tid; e < kN * (kKS / 4); e += kThreads) {
      int c = e % (kKS / 4), r = e / (kKS / 4);
      int gc = n0 + r;
      bool v = gc < K;
      const float* src = C + (int64_t)(v ? gc : 0) * d + ks * kKS + c * 4;
      cp_async16(b_base + ((r >> 3) * (kKS / 4) + c) * 128 + (r & 7) * 16, src, v);
    }
    cp_async_commit();
  };

  for (int n0 = n_begin; n0 < n_end && ok; n0 += kN) {
    // two slices in flight: slice ks + 1 is copied while slice ks is waited for
    free_buffer(0);
    stage(n0, 0, 0);
    for (int j = tid; j < kN; j += kThreads) scn[j] = n0 + j < K ? cnorm[n0 + j] : INFINITY;
    for (int ks = 0; ks < nslices; ++ks) {
      const int b = ks & 1;
      if (ks + 1 < nslices) {
        free_buffer(b ^ 1);
        stage(n0, ks + 1, b ^ 1);
        cp_async_wait_group<1>();   // this thread's copies of slice ks have landed
      } else {
        cp_async_wait_group<0>();
      }
      fence_proxy_async();        // generic-proxy writes -> tensor-core (async proxy) reads
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (tid == 0) {
        const uint32_t a_base = smem_u32(smem + b * kSliceA), b_base = smem_u32(smem + 2 * kSliceA + b * kSliceB);
#pragma unroll
        for (int i = 0; i < kKS / 8; ++i) {   // K = 8 per tf32 MMA: two 16-byte chunks
          uint64_t ad = smem_desc(a_base + (2 * i) * 128, 128, (kKS / 4) * 128);
          uint64_t bd_ = smem_desc(b_base + (2 * i) * 128, 128, (kKS / 4) * 128);
          mma_tf32(tmem, ad, bd_, kIdesc, (ks > 0 || i > 0) ? 1u : 0u);
        }
        mma_commit(&bars[b]);
      }
      issued[b] = 1;
    }
    // wait for the last slice's MMAs (the commit covers every earlier MMA too)
    const int bl = (nslices - 1) & 1;
    if (!mbar_wait_bounded(&bars[bl], phase[bl])) {
      ok = false;
      atomicExch(status, DEV_TIMEOUT);
    }
    phase[bl] ^= 1u;
    issued[bl] = 0;
    if (nslices > 1 && issued[bl ^ 1]) {   // the other buffer's commit has completed as well
      if (!mbar_wait_bounded(&bars[bl ^ 1], phase[bl ^ 1])) {
        ok = false;
        atomicExch(status, DEV_TIMEOUT);
      }
      phase[bl ^ 1] ^= 1u;
      issued[bl ^ 1] = 0;
    }
    fence_after_sync();
    // epilogue: this thread's TMEM lane = its row, its half of the columns
    const uint32_t lane_addr = tmem + ((uint32_t)(quarter * 32) << 16);
    for (int c0 = half * (kN / 2); c0 < (half + 1) * (kN / 2); c0 += 8) {
      float v[8];
      tc::tmem_ld8(lane_addr + c0, v);
      if (kStore) {
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) o[i] = metric == QK_METRIC_L2 ? fmaf(-2.f, v[i], scn[c0 + i]) : -v[i];
        if (my_row < n) {
          float* dst = dout + my_row * ldd + n0 + c0;
          if (n0 + c0 + 8 <= K && (ldd & 3) == 0) {   // 16-byte aligned: ldd and n0 + c0 are multiples of 4
            reinterpret_cast<float4*>(dst)[0] = make_float4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<float4*>(dst)[1] = make_float4(o[4], o[5], o[6], o[7]);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (n0 + c0 + i < K) dst[i] = o[i];
          }
        }
        continue;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        int col = n0 + c0 + i;
        float dist = metric == QK_METRIC_L2 ? fmaf(-2.f, v[i], scn[c0 + i]) : (col < K ? -v[i] : INFINITY);
        if (dist < bd[T - 1] || (dist == bd[T - 1] && col < bi[T - 1])) {
          // insert into the sorted registers
          float cd = dist;
          int32_t ci = col;
#pragma unroll
          for (int j = 0; j < T; ++j) {
            bool lt = cd < bd[j] || (cd == bd[j] && ci < bi[j]);
            float td = bd[j];
            int32_t ti = bi[j];
            bd[j] = lt ? cd : td;
            bi[j] = lt ? ci : ti;
            cd = lt ? td : cd;
            ci = lt ? ti : ci;
          }
        }
      }
    }
    fence_before_sync();
    __syncthreads();      // every lane read before the next tile's MMAs overwrite TMEM
    fence_after_sync();
  }
  if (kStore) {
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kN);
    return;
  }
  // both halves' lists go to shared memory (the operand buffers are idle now)
  float* xd = reinterpret_cast<float*>(smem) + half * kM * T;
  int32_t* xi = reinterpret_cast<int32_t*>(smem + 2 * kM * T * 4) + half * kM * T;
#pragma unroll
  for (int i = 0; i < T; ++i) {
    xd[my_lane * T + i] = bd[i];
    xi[my_lane * T + i] = bi[i];
  }
  fence_before_sync();
  __syncthreads();
  if (half == 0 && my_row < n) {
    const float* ad = reinterpret_cast<const float*>(smem) + my_lane * T;
    const int32_t* ai = reinterpret_cast<const int32_t*>(smem + 2 * kM * T * 4) + my_lane * T;
    const float* bd2 = ad + kM * T;
    const int32_t* bi2 = ai + kM * T;
    int a = 0, b = 0;
    for (int i = 0; i < T; ++i) {   // merge two ascending lists, keep T
      bool take_b = a >= T || (b < T && (bd2[b] < ad[a] || (bd2[b] == ad[a] && bi2[b] < ai[a])));
      float vd = take_b ? bd2[b] : ad[a];
      int32_t vi = take_b ? bi2[b] : ai[a];
      cand[my_row * kT + i] = vd < INFINITY ? vi : -1;
      if (take_b) ++b; else ++a;
    }
    for (int i = T; i < kT; ++i) cand[my_row * kT + i] = -1;
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kN);
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

qk_status launch_tc_nearest(const float* X, int64_t n, int d, const float* C, int K, int metric, int k,
                            int32_t* out_idx, float* out_dist, float* cnorm, int32_t* cand, int32_t* status,
                            cudaStream_t s) {
  if (n <= 0) return QK_OK;
  if (d % tc::kKS != 0 || k < 1 || k > tc::kT) return QK_ERR_ARG;
  row_norms_kernel<<<(unsigned)(((int64_t)K * 32 + 255) / 256), 256, 0, s>>>(C, K, d, cnorm);
  QK_CUDA(cudaGetLastError());
  unsigned grid = (unsigned)((n + tc::kM - 1) / tc::kM);
  if (k == 1) {
    QK_CUDA(cudaFuncSetAttribute(tc_candidates_kernel<tc::kT1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::kSmem));
    tc_candidates_kernel<tc::kT1, false>
        <<<grid, tc::kThreads, tc::kSmem, s>>>(X, n, d, C, K, cnorm, metric, cand, status, nullptr, 0, 0);
  } else {
    QK_CUDA(cudaFuncSetAttribute(tc_candidates_kernel<tc::kT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::kSmem));
    tc_candidates_kernel<tc::kT, false>
        <<<grid, tc::kThreads, tc::kSmem, s>>>(X, n, d, C, K, cnorm, metric, cand, status, nullptr, 0, 0);
  }
  QK_CUDA(cudaGetLastError());
  rescore_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, C, cand, metric, k, out_idx, out_dist);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

int tc_candidates_per_row() { return tc::kT; }

// Approximate distance matrix (L2: ||c||^2 - 2 <x, c>, without ||x||^2; IP:
// -<x, c>) of every row against every centroid, written to dout with row
// stride ldd (>= K).  cnorm must hold the centroids' squared norms.  The
// centroids are split over blockIdx.y in spans of whole tiles so that a small
// number of 128-row tiles still covers every SM.
qk_status launch_tc_distances(const float* X, int64_t n, int d, const float* C, int K, const float* cnorm, int metric,
                              float* dout, int64_t ldd, int32_t* status, int n_sm, cudaStream_t s) {
  if (n <= 0 || K <= 0) return QK_OK;
  if (d % tc::kKS != 0 || ldd < K) return QK_ERR_ARG;
  const int64_t row_tiles = (n + tc::kM - 1) / tc::kM;
  const int col_tiles = (K + tc::kN - 1) / tc::kN;
  int splits = (int)std::min<int64_t>(col_tiles, std::max<int64_t>(1, (4LL * n_sm + row_tiles - 1) / row_tiles));
  const int tiles_per_split = (col_tiles + splits - 1) / splits;
  splits = (col_tiles + tiles_per_split - 1) / tiles_per_split;
  static bool attr_set = false;   // set once, outside any stream capture (the first call is never captured)
  if (!attr_set) {
    QK_CUDA(cudaFuncSetAttribute(tc_candidates_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::kSmem));
    attr_set = true;
  }
  dim3 grid((unsigned)row_tiles, (unsigned)splits);
  tc_candidates_kernel<1, true><<<grid, tc::kThreads, tc::kSmem, s>>>(X, n, d, C, K, cnorm, metric, nullptr, status,
                                                                      dout, ldd, tiles_per_split * tc::kN);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

qk_status launch_row_norms(const float* C, int64_t K, int d, float* out, cudaStream_t s) {
  if (K <= 0) return QK_OK;
  row_norms_kernel<<<(unsigned)((K * 32 + 255) / 256), 256, 0, s>>>(C, K, d, out);
  QK_CUDA(cudaGetLastError());
  return QK_OK;
}

}  // namespace qk
