// Batched Adaptive Partition Scanning: a batch of queries runs Algorithm 1
// (Sec. 5) together, with the partition scans of all queries grouped by
// partition as in multi-query processing (Sec. 8), so that a partition wanted
// by many queries is read from HBM once per round for all of them.
//
// Algorithm 1 is sequential per query: after every scan the k-th distance rho
// may move, p may be recomputed, and the stop rule r >= tau_R is checked.  Its
// choice at every step depends only on the p values and on the results of the
// partitions already scanned.  So the batch runs in rounds:
//   prepare  one warp per query (aps_prepare.cuh; the per-query kernel's
//            export mode where the warp's buffers are too small) scores the
//            top partition and runs APS on the upper level, then exports each
//            query's leaf candidates S (nearest first) with their bisector
//            distances t_i;
//   round    every unfinished query has asked for a few of its candidates;
//            the (query, partition) items are grouped by partition and one
//            persistent grouped scan computes, for every item, its own exact
//            top-k (bounded only by the k-th distance of the results the query
//            has already taken in, which no later item can loosen);
//   replay   one warp per query walks Algorithm 1 over the items of the round,
//            in exactly the order Algorithm 1 takes them: the partition it
//            chooses next is taken in if it was scanned this round, its top-k
//            merged into R, rho, p and r updated as the per-query kernel
//            does.  When the choice was not scanned, the query asks for it and
//            for the candidates Algorithm 1 would take after it if p stayed as
//            it is (by decreasing p, until r would reach the target); items
//            scanned beyond the point where the query stops are discarded.
// The selections therefore equal those of Algorithm 1 run one query at a
// time.  The last round asks for every candidate a query has not scanned, so a
// fixed number of rounds finishes every query; rounds with nothing to do cost
// only their launches, and the whole batch is one fixed sequence of device
// steps that a CUDA graph can hold.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "capvol.cuh"
#include "common.cuh"
#include "aps_prepare.cuh"
#include "grouped.cuh"
#include "index.cuh"
#include "trace.h"

namespace qk {

namespace ab {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxRounds = 16;

enum : uint8_t { kScanned = 1, kInFlight = 2, kPicked = 4 };
enum : int32_t { kPhaseFill = 0, kPhaseEstimate = 1, kPhaseDone = 2 };

// Per-query state of Algorithm 1 between rounds (device arrays).
struct State {
  int32_t* M = nullptr;        // candidates |S| (-1: refused query)
  int32_t* cand = nullptr;     // nq x mcap leaf partitions, nearest first
  double* t = nullptr;         // nq x mcap bisector distances
  double* p = nullptr;         // nq x mcap p_i (p_0 at position 0)
  uint8_t* flag = nullptr;     // nq x mcap kScanned / kInFlight / kPicked
  float* Rd = nullptr;         // nq x k result set R: distances
  int64_t* Ri = nullptr;       // nq x k ids
  int32_t* Rn = nullptr;       // entries in R
  double* rho = nullptr;
  double* r = nullptr;
  int32_t* phase = nullptr;
  int32_t* ns = nullptr;       // partitions taken in (nprobe)
  int32_t* req = nullptr;      // nq x mcap positions asked for in the next round
  int32_t* nreq = nullptr;
};

struct ReplayArgs {
  State st;
  int64_t nq = 0;
  int mcap = 0;
  int k = 10;
  double tau = 0.9, tau_rho = 0.01;
  bool exact = false;
  const double* table = nullptr;
  double beta_a = 0.0, beta_lnB = 0.0;
  const int32_t* size = nullptr;   // leaf partition sizes
  int CH = 4096;                   // rows per unit chunk
  int first = 0;                   // no round has run yet: set the state up
  int final_request = 0;           // the next round is the last: ask for every unscanned candidate
  int round = 0;
  // the round just scanned
  const float* cd = nullptr;
  const int64_t* ci = nullptr;
  const int32_t* cpos = nullptr;
  const int64_t* qcoff = nullptr;
  const int32_t* qcnt = nullptr;
  // requests for the next round
  int32_t* pcount = nullptr;
  int64_t* qslots = nullptr;
  uint32_t* gtau = nullptr;
  // results
  unsigned long long* hits0 = nullptr;
  int64_t* out_ids = nullptr;
  float* out_dist = nullptr;
  int32_t* out_nprobe = nullptr;
  float* out_recall = nullptr;
  int32_t* scan0 = nullptr;
  int32_t scan_cap0 = 0;
  unsigned long long* rstats = nullptr;   // per round: items asked for, items taken in
  int32_t* status = nullptr;
  int64_t* diag = nullptr;
  unsigned long long* next_q = nullptr;   // the next query a warp takes (zeroed per launch)
  int staged = 0;                         // the walk's state in shared memory (stage_bytes(mcap) per warp)
};

// Shared memory of one warp's staged walk state: t_i and p_i (FP64) and the
// flags of mcap candidates, 16-byte aligned.
__host__ __device__ inline size_t stage_bytes(int mcap) { return ((size_t)mcap * 17 + 15) & ~size_t(15); }
constexpr int kStageMaxCap = 384;   // larger candidate sets walk in global memory

// p from Eq. 8-9 with the raw caps for p_0 (as the per-query kernel computes
// it, lane by lane in the same order), then r = p_0 + sum of the scanned p_i.
__device__ double warp_probabilities(const ReplayArgs& a, const double* t, double* p, const uint8_t* fl, int M,
                                     double rho, int lane) {
  double su = 0.0, pr = 1.0;
  const double inv = rho > 0.0 ? 1.0 / rho : 0.0;
  for (int i = 1 + lane; i < M; i += 32) {
    const double u = cap_u(t[i], rho, inv, a.exact, a.table, a.beta_a, a.beta_lnB);
    p[i] = u;
    su += u;
    pr *= 1.0 - u;
  }
  const double U = warp_sum_d(su);
  const double P0 = warp_prod_d(pr);
  const double c = U > 0.0 ? (1.0 - P0) / U : 0.0;
  double rs = 0.0;
  for (int i = 1 + lane; i < M; i += 32) {
    const double v = p[i] * c;
    p[i] = v;
    if (fl[i] & kScanned) rs += v;
  }
  if (lane == 0) p[0] = P0;
  const double r = P0 + warp_sum_d(rs);
  __syncwarp();
  return r;
}

// The candidate with the largest p among those without any of the `skip`
// flags (ties to the lower position; p >= 0, so its bits order like its
// value).  M if none.
__device__ int warp_next(const double* p, const uint8_t* fl, int M, uint8_t skip, int lane) {
  long long bk = -1;
  int bi = M;
  for (int i = 1 + lane; i < M; i += 32) {
    if (fl[i] & skip) continue;
    const long long key = __double_as_longlong(p[i]);
    if (key > bk) {
      bk = key;
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

// Merges the round's candidates of the item at position `pos` into R
// (bd/bi[0, rn), sorted); returns the new size (<= k).  The scans write a
// query's candidates in blocks of k, one per scanned unit, every entry of a
// block tagged with its item's position, so only the blocks whose first tag
// matches are read.  tag0: lane j's block j tag (-1 past the blocks), read
// once per walk instead of once per step.
__device__ int take_in(float* bd, int64_t* bi, int rn, int k, const float* cd, const int64_t* ci,
                       const int32_t* cpos, int cn, int pos, int32_t tag0, int lane) {
  int cnt = rn;
  float kd = rn == k ? bd[k - 1] : INFINITY;
  int64_t kid = rn == k ? bi[k - 1] : INT64_MAX;
  const int nb = cn / k;
  for (int b0 = 0; b0 < nb; b0 += 32) {
    const int32_t tag = b0 == 0 ? tag0 : (b0 + lane < nb ? cpos[(b0 + lane) * k] : -1);
    unsigned mb = __ballot_sync(0xffffffffu, b0 + lane < nb && tag == pos);
    while (mb) {
      const int i = (b0 + __ffs(mb) - 1) * k + lane;
      mb &= mb - 1;
      bool s = false;
      float d = 0.f;
      int64_t id = -1;
      if (lane < k) {
        d = cd[i];
        id = ci[i];
        s = id >= 0 && bt::pair_less(d, id, kd, kid);
      }
      const unsigned m = __ballot_sync(0xffffffffu, s);
      if (s) {
        const int at = cnt + __popc(m & ((1u << lane) - 1u));
        bd[at] = d;
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
  }
  if (cnt == rn) return rn;   // nothing entered: R is sorted and within k already
  return bt::warp_compact(bd, bi, cnt, k, lane);
}

// Algorithm 1 of query q over the round just scanned, and its next requests
// (one warp; bd / bi its 64-entry buffer in shared memory).
// With `stage`, the query's t_i, p_i and flags are worked on in shared memory
// (stage: mcap doubles, mcap doubles, mcap bytes) and p and the flags written
// back at the end; the walk reads them once per step.
__device__ void replay_query(const ReplayArgs& a, const int64_t q, float* bd, int64_t* bi, const int lane,
                             unsigned char* stage) {
  const State& S = a.st;
  const int M = S.M[q];
  const int k = a.k;
  int phase = a.first ? kPhaseFill : S.phase[q];
  if (M < 0 || phase == kPhaseDone) {   // refused (answered by the prepare step) or finished
    if (lane == 0) {
      S.nreq[q] = 0;
      a.qslots[q] = 0;
      if (M < 0) S.phase[q] = kPhaseDone;
    }
    return;
  }
  int32_t* cand = S.cand + q * a.mcap;
  const double* t = S.t + q * a.mcap;
  double* p = S.p + q * a.mcap;
  uint8_t* fl = S.flag + q * a.mcap;
  double* gp = p;
  uint8_t* gfl = fl;
  if (stage) {
    double* st = reinterpret_cast<double*>(stage);
    double* sp = st + a.mcap;
    uint8_t* sf = reinterpret_cast<uint8_t*>(sp + a.mcap);
    for (int i = lane; i < M; i += 32) {
      st[i] = t[i];
      sp[i] = p[i];
      sf[i] = a.first ? 0 : fl[i];
    }
    t = st;
    p = sp;
    fl = sf;
    __syncwarp();
  }
  int rn = 0, ns = 0;
  double rho = 0.0, r = 0.0;
  if (a.first) {
    for (int i = lane; i < M; i += 32) fl[i] = 0;
  } else {
    rn = S.Rn[q];
    ns = S.ns[q];
    rho = S.rho[q];
    r = S.r[q];
    if (lane < rn) {
      bd[lane] = S.Rd[q * k + lane];
      bi[lane] = S.Ri[q * k + lane];
    }
  }
  __syncwarp();
  const int64_t co = a.first ? 0 : a.qcoff[q];
  const int cn = a.first ? 0 : a.qcnt[q];
  const int32_t tag0 = lane < cn / k ? a.cpos[co + (int64_t)lane * k] : -1;
  int taken = 0;
  bool done = false;
  for (;;) {
    // the partition Algorithm 1 takes next: centroid order until R holds k
    // results, then the largest p
    const int nx = phase == kPhaseFill ? ns : warp_next(p, fl, M, kScanned, lane);
    if (nx >= M) {   // never expected: the stop rules below end the walk first
      if (lane == 0) bt::report_once(a.status, a.diag, DEV_BAD_INDEX, -6, q, ns);
      done = true;
      break;
    }
    if (!(fl[nx] & kInFlight)) break;   // not scanned this round: ask for it
    rn = take_in(bd, bi, rn, k, a.cd + co, a.ci + co, a.cpos + co, cn, nx, tag0, lane);
    if (lane == 0) {
      fl[nx] = kScanned;
      atomicAdd(&a.hits0[cand[nx]], 1ull);
      if (a.scan0 && ns < a.scan_cap0) a.scan0[q * a.scan_cap0 + ns] = cand[nx];
    }
    __syncwarp();
    ++ns;
    ++taken;
    // rho from the k-th result (Euclidean, R1), in FP32 like the distances
    const float dk = rn == k ? bd[k - 1] : 0.f;
    const double rho2 = (double)sqrtf(dk > 0.f ? dk : 0.f);
    if (phase == kPhaseFill) {
      if (rn >= k) {
        phase = kPhaseEstimate;
        rho = rho2;
        r = warp_probabilities(a, t, p, fl, M, rho, lane);
        if (!(r < a.tau && ns < M)) {
          done = true;
          break;
        }
      } else if (ns >= M) {   // S ran out before R held k results
        r = 1.0;
        done = true;
        break;
      }
    } else {
      if (fabs(rho2 - rho) > a.tau_rho * rho) {   // R7: recompute every p
        rho = rho2;
        r = warp_probabilities(a, t, p, fl, M, rho, lane);
      } else {
        r += p[nx];
      }
      if (!(r < a.tau && ns < M)) {
        done = true;
        break;
      }
    }
  }
  if (lane == 0 && a.rstats && taken) atomicAdd(&a.rstats[2 * a.round + 1], (unsigned long long)taken);
  // items of this round not taken in are discarded
  for (int i = lane; i < M; i += 32) fl[i] &= (uint8_t)kScanned;
  __syncwarp();
  if (done) {
    if (lane < k) {
      a.out_dist[q * k + lane] = lane < rn ? bd[lane] : INFINITY;
      a.out_ids[q * k + lane] = lane < rn ? bi[lane] : -1;
    }
    if (a.scan0)
      for (int i = ns + lane; i < a.scan_cap0; i += 32) a.scan0[q * a.scan_cap0 + i] = -1;
    if (lane == 0) {
      if (a.out_nprobe) a.out_nprobe[q] = ns;
      if (a.out_recall) a.out_recall[q] = (float)r;
      S.phase[q] = kPhaseDone;
      S.nreq[q] = 0;
      a.qslots[q] = 0;
    }
    return;
  }
  // Ask for the next round's items, marked kPicked: before R holds k results
  // the next candidates in centroid order until their rows can fill R; after,
  // those Algorithm 1 would take if p stayed as it is, by decreasing p until r
  // would reach the target.  Before the last round: every unscanned candidate.
  int nreq = 0;
  int64_t slots = 0;
  int32_t* req = S.req + q * a.mcap;
  if (phase == kPhaseFill) {
    if (lane == 0) {
      int64_t rows = rn;
      for (int i = ns; i < M; ++i) {
        if (!a.final_request && rows >= k) break;
        req[nreq++] = i;
        rows += a.size[cand[i]];
      }
    }
    nreq = __shfl_sync(0xffffffffu, nreq, 0);
  } else {
    double rs = r;
    for (;;) {
      const int nx = warp_next(p, fl, M, kScanned | kPicked, lane);
      if (nx >= M) break;
      if (lane == 0) {
        fl[nx] |= kPicked;
        req[nreq] = nx;
      }
      __syncwarp();
      ++nreq;
      rs += p[nx];
      if (!a.final_request && !(rs < a.tau)) break;
    }
  }
  __syncwarp();
  for (int j = lane; j < nreq; j += 32) {
    const int pos = req[j];
    const int32_t part = cand[pos];
    fl[pos] = kInFlight;
    atomicAdd(&a.pcount[part], 1);
    slots += (a.size[part] + a.CH - 1) / a.CH;
  }
  for (int o = 16; o > 0; o >>= 1) slots += __shfl_xor_sync(0xffffffffu, slots, o);
  if (stage) {   // the next replay of this query reads them from global memory
    __syncwarp();
    for (int i = lane; i < M; i += 32) {
      gp[i] = p[i];
      gfl[i] = fl[i];
    }
  }
  if (lane < rn) {
    S.Rd[q * k + lane] = bd[lane];
    S.Ri[q * k + lane] = bi[lane];
  }
  if (lane == 0) {
    S.Rn[q] = rn;
    S.ns[q] = ns;
    S.rho[q] = rho;
    S.r[q] = r;
    S.phase[q] = phase;
    S.nreq[q] = nreq;
    a.qslots[q] = slots;
    // the bound of the next round's scans: rows up to R's k-th distance may
    // still enter R (an equal distance with a lower id), so the bound is the
    // next float above it; L2 distances are >= 0, so bits order like values
    a.gtau[q] = rn == k ? __float_as_uint(nextafterf(bd[k - 1], INFINITY)) : 0x7f7f7f7fu;
    if (a.rstats) atomicAdd(&a.rstats[2 * (a.round + 1)], (unsigned long long)nreq);
  }
}

// Persistent: each warp takes the next query from a counter (zeroed before the
// launch), so queries with long walks do not hold a block's other warps.
__global__ void __launch_bounds__(kThreads) aps_replay_kernel(ReplayArgs a) {
  __shared__ float s_bd[kWarps][64];
  __shared__ int64_t s_bi[kWarps][64];
  extern __shared__ __align__(16) unsigned char s_stage[];   // per warp: stage_bytes(mcap), when staged
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* stage = a.staged ? s_stage + (size_t)warp * stage_bytes(a.mcap) : nullptr;
  // a round that asked for nothing: every query had finished before it
  if (a.rstats && a.round >= 0 && a.rstats[2 * a.round] == 0ull) return;
  for (;;) {
    unsigned long long q = 0;
    if (lane == 0) q = atomicAdd(a.next_q, 1ull);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= (unsigned long long)a.nq) break;
    replay_query(a, (int64_t)q, s_bd[warp], s_bi[warp], lane, stage);
    __syncwarp();
  }
}

// Lists every requested item under its partition, with its position.
__global__ void fill_kernel(const int32_t* req, const int32_t* nreq, const int32_t* cand, int64_t nq, int mcap,
                            const int32_t* pstart, int32_t* pcur, int32_t* qlist, int32_t* qpos,
                            const unsigned long long* asked) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nq * mcap || (asked && *asked == 0ull)) return;
  const int64_t q = i / mcap;
  const int j = (int)(i % mcap);
  if (j >= nreq[q]) return;
  const int pos = req[i];
  const int32_t part = cand[q * mcap + pos];
  const int32_t at = pstart[part] + atomicAdd(&pcur[part], 1);
  qlist[at] = (int32_t)q;
  qpos[at] = pos;
}

}  // namespace ab

int32_t prepare_mcap(const SearchArgs& a) { return ap::mcap_of(a); }

qk_status prepare_upper(const SearchArgs& a, cudaStream_t s) {
  if (!ap::fits(a)) {
    set_error("the prepare kernel's buffers do not hold this search's candidate counts");
    return QK_ERR_UNSUPPORTED;
  }
  return ap::launch_prepare(a, s);
}

}  // namespace qk

// ------------------------------------------------------------------ the plan

using namespace qk;

struct qk_aps_batch {
  qk_index* ix = nullptr;
  int64_t max_nq = 0;
  int32_t k = 0;
  int32_t rounds = 4;
  qk_batch_tiles tiles{};
  int n_sm = 148;
  int32_t mcap = 0, K = 0;
  int64_t cand_cap = 0;
  uint64_t version = ~0ull;
  ab::State st;
  int32_t *pcount = nullptr, *pcur = nullptr, *pstart = nullptr, *qlist = nullptr, *qpos = nullptr,
          *order = nullptr, *qcnt = nullptr, *cpos = nullptr;
  int64_t *ustart = nullptr, *tmp = nullptr, *tmp2 = nullptr, *n_units = nullptr, *qslots = nullptr,
          *qcoff = nullptr, *ci = nullptr;
  uint32_t* gtau = nullptr;
  float* cd = nullptr;
  unsigned long long* work = nullptr;
  unsigned long long* rstats = nullptr;
  int scan_blocks = 0;
  int rows_blocks = 0;            // CTAs per SM of the whole-rows scan
  qk_batch_tiles scan_tiles{};
  cudaGraphExec_t graph = nullptr;
  uint64_t graph_version = 0;
  int64_t graph_nq = 0;
  // stage timing of uncaptured batches: events before the prepare step, after
  // it, after the first replay, then per round after grouping, after the scan
  // and after the replay
  bool timing = false, timed = false;
  int timed_rounds = 0;
  cudaEvent_t ev[3 + 3 * ab::kMaxRounds] = {};
  // pinned staging of the partition order (two, used in turn) and the events
  // of their copies to the device
  int32_t* h_order[2] = {};
  int32_t h_order_cap[2] = {};
  cudaEvent_t order_ev[2] = {};
  int order_turn = 0;
};

namespace {

template <class T>
qk_status aalloc(T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  QK_CUDA(cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T)));
  return QK_OK;
}
template <class T>
void afree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_all(qk_aps_batch* b) {
  ab::State& s = b->st;
  afree(s.M), afree(s.cand), afree(s.t), afree(s.p), afree(s.flag), afree(s.Rd), afree(s.Ri), afree(s.Rn);
  afree(s.rho), afree(s.r), afree(s.phase), afree(s.ns), afree(s.req), afree(s.nreq);
  afree(b->pcount), afree(b->pcur), afree(b->pstart), afree(b->qlist), afree(b->qpos), afree(b->order);
  afree(b->qcnt), afree(b->cpos), afree(b->ustart), afree(b->tmp), afree(b->tmp2), afree(b->n_units);
  afree(b->qslots), afree(b->qcoff), afree(b->ci), afree(b->gtau), afree(b->cd), afree(b->work), afree(b->rstats);
  for (int t = 0; t < 2; ++t) {
    if (b->order_ev[t]) cudaEventSynchronize(b->order_ev[t]);   // its copy has read the staging
    if (b->h_order[t]) cudaFreeHost(b->h_order[t]);
    if (b->order_ev[t]) cudaEventDestroy(b->order_ev[t]);
    b->h_order[t] = nullptr;
    b->order_ev[t] = nullptr;
    b->h_order_cap[t] = 0;
  }
}

// Rows per unit in round rd.  The first round asks each query's nearest
// partition only, so its units are few and the largest partitions bound its
// time; they are cut finer there.
constexpr int kFirstRoundChunk = 1024;
int round_chunk(const qk_batch_tiles& t, int rd) {
  return rd == 0 ? std::min(t.chunk_rows, kFirstRoundChunk) : t.chunk_rows;
}

// Re-reads the index's shape and partition sizes; re-sizes the workspace
// where it no longer fits.  Host work, never inside a capture.
qk_status refresh(qk_aps_batch* b, cudaStream_t s) {
  qk_index* ix = b->ix;
  if (b->version == ix->version && b->K == ix->n_leaf) return QK_OK;
  const int32_t K = ix->n_leaf;
  const int32_t mcap = n_candidates(ix->cfg.f_M_leaf, K);
  const int CH = std::min(round_chunk(b->tiles, 0), round_chunk(b->tiles, 1));   // the finest chunking of a round
  int64_t extra = 0;
  for (int32_t sz : ix->h_size0) extra += std::max<int64_t>(0, ((int64_t)sz + CH - 1) / CH - 1);
  const int64_t need_cand =
      (int64_t)b->k * b->max_nq * ((int64_t)mcap + extra);
  const size_t nq = (size_t)b->max_nq;
  // the plan's batches still in flight on s use the workspace re-sized below;
  // a new version of the same shape (inserts, deletes) needs no wait
  if (mcap != b->mcap || K != b->K || need_cand > b->cand_cap) QK_CUDA(cudaStreamSynchronize(s));
  if (mcap != b->mcap) {
    ab::State& st = b->st;
    QK_TRY(aalloc(&st.cand, nq * mcap));
    QK_TRY(aalloc(&st.t, nq * mcap));
    QK_TRY(aalloc(&st.p, nq * mcap));
    QK_TRY(aalloc(&st.flag, nq * mcap));
    QK_TRY(aalloc(&st.req, nq * mcap));
    QK_TRY(aalloc(&b->qlist, nq * mcap));
    QK_TRY(aalloc(&b->qpos, nq * mcap));
    b->mcap = mcap;
  }
  if (K != b->K) {
    QK_TRY(aalloc(&b->pcount, (size_t)K));
    QK_TRY(aalloc(&b->pcur, (size_t)K));
    QK_TRY(aalloc(&b->pstart, (size_t)K));
    QK_TRY(aalloc(&b->order, (size_t)K));
    QK_TRY(aalloc(&b->ustart, (size_t)K + 1));
    QK_TRY(aalloc(&b->tmp, (size_t)std::max<int64_t>(K, b->max_nq)));
    QK_TRY(aalloc(&b->tmp2, (size_t)std::max<int64_t>(K, b->max_nq)));
    b->K = K;
  }
  if (need_cand > b->cand_cap) {
    const int64_t cap = need_cand + need_cand / 8;
    QK_TRY(aalloc(&b->cd, (size_t)cap));
    QK_TRY(aalloc(&b->ci, (size_t)cap));
    QK_TRY(aalloc(&b->cpos, (size_t)cap));
    b->cand_cap = cap;
  }
  // the partitions by decreasing size, copied in stream order from pinned
  // staging the copy before the last has finished reading
  const int tn = b->order_turn;
  b->order_turn ^= 1;
  if (!b->order_ev[tn]) QK_CUDA(cudaEventCreateWithFlags(&b->order_ev[tn], cudaEventDisableTiming));
  QK_CUDA(cudaEventSynchronize(b->order_ev[tn]));
  if (K > b->h_order_cap[tn]) {
    if (b->h_order[tn]) cudaFreeHost(b->h_order[tn]);
    b->h_order[tn] = nullptr;
    b->h_order_cap[tn] = 0;
    QK_CUDA(cudaMallocHost(reinterpret_cast<void**>(&b->h_order[tn]), sizeof(int32_t) * std::max(K, 1)));
    b->h_order_cap[tn] = K;
  }
  int32_t* order = b->h_order[tn];
  std::iota(order, order + K, 0);
  std::stable_sort(order, order + K, [&](int32_t x, int32_t y) { return ix->h_size0[x] > ix->h_size0[y]; });
  QK_CUDA(cudaMemcpyAsync(b->order, order, sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
  QK_CUDA(cudaEventRecord(b->order_ev[tn], s));
  b->version = ix->version;
  return QK_OK;
}

qk_status launch_scan_rounds(const bt::ScanArgs& a, int d, int QW, int n_sm, bool capturing, int* per_sm,
                             cudaStream_t s);

// The batch's device steps: no host synchronisation, no allocation.
qk_status enqueue(qk_aps_batch* b, const float* q, int64_t nq, float recall_target, int64_t* out_ids,
                  float* out_dist, int32_t* out_nprobe, float* out_recall, int32_t* scan0, int32_t cap0,
                  cudaStream_t s) {
  qk_index* ix = b->ix;
  const int d = ix->cfg.d, K = b->K, k = b->k, mcap = b->mcap;
  const qk_batch_tiles& tl = b->tiles;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  QK_CUDA(cudaStreamIsCapturing(s, &cs));
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  if (capturing && !(b->scan_tiles.queries_per_warp == tl.queries_per_warp && b->scan_tiles.tile_rows == tl.tile_rows &&
                     b->scan_tiles.rows_per_thread == tl.rows_per_thread))
    b->scan_blocks = b->rows_blocks = 0;
  Trace tr("aps_batch");
  const bool timing = b->timing && !capturing;
  auto mark = [&](int i) -> qk_status {
    if (timing) QK_CUDA(cudaEventRecord(b->ev[i], s));
    return QK_OK;
  };
  QK_TRY(mark(0));
  // 1. root scoring and upper-level APS per query; S and t_i exported
  SearchArgs sa;
  base_search_args(ix, k, recall_target, 0, sa);
  sa.Q = q;
  sa.nq = nq;
  sa.out_ids = out_ids;   // written only for refused queries
  sa.out_dist = out_dist;
  sa.out_nprobe = out_nprobe;
  sa.out_recall = out_recall;
  sa.scan0 = scan0;
  sa.scan_cap0 = scan0 ? cap0 : 0;
  sa.xs_M = b->st.M;
  sa.xs_cand = b->st.cand;
  sa.xs_t = b->st.t;
  sa.xs_mcap = mcap;
  if (ap::fits(sa))   // one warp per query; the per-query kernel where the warp's buffers are too small
    QK_TRY(ap::launch_prepare(sa, s));
  else
    QK_TRY(launch_search(sa, s));
  tr.mark("prepare");
  QK_TRY(mark(1));
  if (b->rstats) QK_CUDA(cudaMemsetAsync(b->rstats, 0, sizeof(unsigned long long) * 2 * (ab::kMaxRounds + 1), s));
  // 2. the first requests
  ab::ReplayArgs ra;
  ra.st = b->st;
  ra.nq = nq;
  ra.mcap = mcap;
  ra.k = k;
  ra.tau = recall_target;
  ra.tau_rho = ix->cfg.tau_rho;
  ra.exact = ix->cfg.beta_mode == QK_BETA_EXACT;
  ra.table = ix->beta_table;
  ra.beta_a = ix->beta_a;
  ra.beta_lnB = ix->beta_lnB;
  ra.size = ix->size0;
  ra.CH = round_chunk(tl, 0);   // the replay after the prepare step asks for round 0's items
  ra.pcount = b->pcount;
  ra.qslots = b->qslots;
  ra.gtau = b->gtau;
  ra.hits0 = ix->hits0;
  ra.out_ids = out_ids;
  ra.out_dist = out_dist;
  ra.out_nprobe = out_nprobe;
  ra.out_recall = out_recall;
  ra.scan0 = scan0;
  ra.scan_cap0 = scan0 ? cap0 : 0;
  ra.rstats = b->rstats;
  ra.status = ix->status;
  ra.diag = ix->diag;
  ra.cd = b->cd;
  ra.ci = b->ci;
  ra.cpos = b->cpos;
  ra.qcoff = b->qcoff;
  ra.qcnt = b->qcnt;
  // the replay is persistent: as many blocks as the SMs hold at once, at most one per kWarps queries
  ra.staged = mcap <= ab::kStageMaxCap;
  const size_t rsmem = ra.staged ? ab::kWarps * ab::stage_bytes(mcap) : 0;
  if (rsmem > 48 * 1024 && !capturing)
    QK_CUDA(cudaFuncSetAttribute(ab::aps_replay_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem));
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ab::aps_replay_kernel, ab::kThreads, rsmem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  const unsigned rgrid = (unsigned)std::min<int64_t>((nq + ab::kWarps - 1) / ab::kWarps,
                                                     (int64_t)b->n_sm * std::max(1, per_sm));
  ra.next_q = b->work + 1;
  QK_CUDA(cudaMemsetAsync(b->pcount, 0, sizeof(int32_t) * K, s));
  ra.first = 1;
  ra.round = -1;
  ra.final_request = b->rounds == 1;
  QK_CUDA(cudaMemsetAsync(b->work + 1, 0, sizeof(unsigned long long), s));
  ab::aps_replay_kernel<<<rgrid, ab::kThreads, rsmem, s>>>(ra);
  QK_CUDA(cudaGetLastError());
  QK_TRY(mark(2));
  ra.first = 0;
  for (int rd = 0; rd < b->rounds; ++rd) {
    // 3. group the round's items by partition
    bt::GroupArgs ga;
    ga.K = K;
    ga.nq = nq;
    const bool rows_round = tl.rows_per_thread == 2 && rd > 0;   // the first round's partitions hold few queries
    ga.G = rows_round ? bt::kRowsG : bt::kWarps * tl.queries_per_warp;
    ga.CH = round_chunk(tl, rd);
    ga.k = k;
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
    // the items this round asked for, counted by the replay that asked: a round
    // with none (every query finished) skips its grouping, fill and replay
    const unsigned long long* asked = b->rstats ? b->rstats + 2 * rd : nullptr;
    ga.asked = asked;
    bt::group_kernel<<<1, 1024, 0, s>>>(ga);
    QK_CUDA(cudaGetLastError());
    QK_CUDA(cudaMemsetAsync(b->pcur, 0, sizeof(int32_t) * K, s));
    const int64_t items = nq * mcap;
    ab::fill_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(b->st.req, b->st.nreq, b->st.cand, nq, mcap,
                                                                   b->pstart, b->pcur, b->qlist, b->qpos, asked);
    QK_CUDA(cudaGetLastError());
    QK_TRY(mark(3 + 3 * rd));
    // 4. every item's own top-k
    QK_CUDA(cudaMemsetAsync(b->qcnt, 0, sizeof(int32_t) * nq, s));
    QK_CUDA(cudaMemsetAsync(b->work, 0, sizeof(unsigned long long), s));
    bt::ScanArgs sc;
    sc.vec = ix->vec0;
    sc.x_rows = ix->cap0;
    sc.ids = ix->ids0;
    sc.off = ix->off0;
    sc.size = ix->size0;
    sc.Q = q;
    sc.k = k;
    sc.CH = round_chunk(tl, rd);
    sc.TR = tl.tile_rows;
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
    sc.aps = 1;
    sc.qpos = b->qpos;
    sc.cpos = b->cpos;
    if (rows_round) {
      QK_TRY(bt::launch_scan_rows(sc, d, b->n_sm, capturing, &b->rows_blocks, s));
    } else {
      QK_TRY(launch_scan_rounds(sc, d, tl.queries_per_warp, b->n_sm, capturing, &b->scan_blocks, s));
    }
    b->scan_tiles = tl;
    QK_TRY(mark(4 + 3 * rd));
    // 5. Algorithm 1 over the round, and the next requests
    QK_CUDA(cudaMemsetAsync(b->pcount, 0, sizeof(int32_t) * K, s));
    ra.round = rd;
    ra.final_request = rd + 1 == b->rounds - 1;
    ra.CH = round_chunk(tl, rd + 1);   // its requests are the next round's items
    QK_CUDA(cudaMemsetAsync(b->work + 1, 0, sizeof(unsigned long long), s));
    ab::aps_replay_kernel<<<rgrid, ab::kThreads, rsmem, s>>>(ra);
    QK_CUDA(cudaGetLastError());
    QK_TRY(mark(5 + 3 * rd));
  }
  tr.mark("rounds");
  if (timing) {
    b->timed = true;
    b->timed_rounds = b->rounds;
  }
  ix->queries_seen += nq;
  return QK_OK;
}

template <int D, int QW>
qk_status scan_t(const bt::ScanArgs& a, int n_sm, bool capturing, int* per_sm, cudaStream_t s) {
  if constexpr (bt::tpr_for(D, QW) == 0) {
    set_error("queries_per_warp " + std::to_string(QW) + " is not available for d = " + std::to_string(D));
    return QK_ERR_ARG;
  } else {
    const size_t smem = sizeof(float) * bt::kStages * (size_t)a.TR * D + sizeof(uint64_t) * bt::kStages +
                        (sizeof(float) + sizeof(int32_t)) * (size_t)bt::kWarps * QW * bt::kBuf +
                        sizeof(bt::UnitInfo) + sizeof(int32_t) * bt::kWarps * QW +
                        sizeof(int32_t) * (2 * bt::kStages + 2) + 16;
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
qk_status scan_d(const bt::ScanArgs& a, int QW, int n_sm, bool cap, int* per_sm, cudaStream_t s) {
  switch (QW) {
    case 1: return scan_t<D, 1>(a, n_sm, cap, per_sm, s);
    case 2: return scan_t<D, 2>(a, n_sm, cap, per_sm, s);
    case 4: return scan_t<D, 4>(a, n_sm, cap, per_sm, s);
    default: set_error("queries_per_warp must be 1, 2 or 4"); return QK_ERR_ARG;
  }
}

qk_status launch_scan_rounds(const bt::ScanArgs& a, int d, int QW, int n_sm, bool cap, int* per_sm, cudaStream_t s) {
  switch (d) {
    case 32: return scan_d<32>(a, QW, n_sm, cap, per_sm, s);
    case 64: return scan_d<64>(a, QW, n_sm, cap, per_sm, s);
    case 96: return scan_d<96>(a, QW, n_sm, cap, per_sm, s);
    case 128: return scan_d<128>(a, QW, n_sm, cap, per_sm, s);
    case 192: return scan_d<192>(a, QW, n_sm, cap, per_sm, s);
    case 256: return scan_d<256>(a, QW, n_sm, cap, per_sm, s);
    case 384: return scan_d<384>(a, QW, n_sm, cap, per_sm, s);
    case 512: return scan_d<512>(a, QW, n_sm, cap, per_sm, s);
    case 768: return scan_d<768>(a, QW, n_sm, cap, per_sm, s);
    case 1024: return scan_d<1024>(a, QW, n_sm, cap, per_sm, s);
    default: set_error("unsupported dimension"); return QK_ERR_ARG;
  }
}

qk_status check_call(qk_aps_batch* b, const float* q, int64_t nq, float recall_target, int64_t* out_ids,
                     float* out_dist, int32_t* out_nprobe, float* out_recall, int32_t* scan0, int32_t cap0) {
  if (!b) {
    set_error("null plan");
    return QK_ERR_ARG;
  }
  if (!b->ix->ready) {
    set_error("index is empty: build or load it first");
    return QK_ERR_STATE;
  }
  if (b->ix->cfg.storage != QK_STORE_F32 || b->ix->cfg.metric != QK_METRIC_L2) {
    set_error("batched APS search supports L2 over FP32 storage");
    return QK_ERR_ARG;
  }
  if (nq < 0 || nq > b->max_nq) {
    set_error("nq must be in [0, max_nq]");
    return QK_ERR_ARG;
  }
  if (!(recall_target > 0.f)) {
    set_error("batched APS search needs a recall target > 0");
    return QK_ERR_ARG;
  }
  if (scan0 && cap0 < 1) {
    set_error("a scanned-partition record needs a capacity >= 1");
    return QK_ERR_ARG;
  }
  if (nq == 0) return QK_OK;
  for (const void* p : {(const void*)q, (const void*)out_ids, (const void*)out_dist}) {
    if (!p || !is_device_ptr(p) || reinterpret_cast<uintptr_t>(p) % 16 != 0) {
      set_error("batched APS search takes 16-byte aligned device buffers");
      return QK_ERR_ARG;
    }
  }
  for (const void* p : {(const void*)out_nprobe, (const void*)out_recall, (const void*)scan0}) {
    if (p && !is_device_ptr(p)) {
      set_error("batched APS search takes device buffers");
      return QK_ERR_ARG;
    }
  }
  return QK_OK;
}

}  // namespace

extern "C" {

qk_status qk_aps_batch_create(qk_index* ix, int64_t max_nq, int32_t k, qk_aps_batch** out) {
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
    set_error("batched APS search supports L2 over FP32 storage");
    return QK_ERR_ARG;
  }
  if (max_nq < 1 || k < 1 || k > bt::kMaxK) {
    set_error("need max_nq >= 1 and 1 <= k <= 32");
    return QK_ERR_ARG;
  }
  qk_aps_batch* b = new qk_aps_batch();
  b->ix = ix;
  b->max_nq = max_nq;
  b->k = k;
  b->tiles.queries_per_warp = 2;
  b->tiles.tile_rows = std::max(8, std::min(64, 8192 / ix->cfg.d));
  b->tiles.chunk_rows = 4096;
  b->tiles.rows_per_thread = bt::rows_layout_ok(ix->cfg.d) ? 2 : 0;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
  const size_t nq = (size_t)max_nq;
  qk_status st = QK_OK;
  auto run = [&](qk_status s2) {
    if (st == QK_OK) st = s2;
  };
  ab::State& s = b->st;
  run(aalloc(&s.M, nq));
  run(aalloc(&s.Rd, nq * k));
  run(aalloc(&s.Ri, nq * k));
  run(aalloc(&s.Rn, nq));
  run(aalloc(&s.rho, nq));
  run(aalloc(&s.r, nq));
  run(aalloc(&s.phase, nq));
  run(aalloc(&s.ns, nq));
  run(aalloc(&s.nreq, nq));
  run(aalloc(&b->n_units, 1));
  run(aalloc(&b->qslots, nq));
  run(aalloc(&b->qcoff, nq + 1));
  run(aalloc(&b->qcnt, nq));
  run(aalloc(&b->gtau, nq));
  run(aalloc(&b->work, 2));   // [0] the grouped scan's units, [1] the replay's queries
  run(aalloc(&b->rstats, 2 * (ab::kMaxRounds + 1)));   // per round: items asked for, items taken in
  if (st == QK_OK) st = refresh(b, 0);
  if (st != QK_OK) {
    free_all(b);
    delete b;
    return st;
  }
  *out = b;
  return QK_OK;
  QK_GUARD_END
}

void qk_aps_batch_destroy(qk_aps_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (cudaEvent_t& e : b->ev)
    if (e) cudaEventDestroy(e);
  free_all(b);
  delete b;
}

qk_status qk_aps_batch_set_rounds(qk_aps_batch* b, int32_t rounds) {
  QK_GUARD_BEGIN
  if (!b || rounds < 1 || rounds > ab::kMaxRounds) {
    set_error("rounds must be in [1, 16]");
    return QK_ERR_ARG;
  }
  b->rounds = rounds;
  return QK_OK;
  QK_GUARD_END
}

namespace {
bool aps_tiles_valid(int d, const qk_batch_tiles& t) {
  return (t.queries_per_warp == 1 || t.queries_per_warp == 2 || t.queries_per_warp == 4) &&
         bt::tpr_for(d, t.queries_per_warp) > 0 && t.tile_rows >= 1 &&
         (size_t)bt::kStages * t.tile_rows * d * 4 <= 200 * 1024 && t.chunk_rows >= t.tile_rows &&
         t.chunk_rows >= 1024 &&
         (t.rows_per_thread == 0 ||
          (t.rows_per_thread == 2 && bt::rows_layout_ok(d)));
}
}  // namespace

qk_status qk_aps_batch_set_tiles(qk_aps_batch* b, const qk_batch_tiles* t) {
  QK_GUARD_BEGIN
  if (!b || !t) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  if (!aps_tiles_valid(b->ix->cfg.d, *t)) {
    set_error("invalid tiles (queries_per_warp 1, 2 or 4; 3 tiles within 200 KB; chunk_rows >= 1024; "
              "rows_per_thread 0, or 2 with d <= 256)");
    return QK_ERR_ARG;
  }
  b->tiles = *t;
  b->version = ~0ull;   // the candidate buffer depends on chunk_rows
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_aps_batch_autotune(qk_aps_batch* b, const float* q, int64_t nq, float recall_target, int64_t* out_ids,
                                float* out_dist, int32_t reps, qk_batch_tiles* chosen, void* stream) {
  QK_GUARD_BEGIN
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  QK_TRY(check_call(b, q, nq, recall_target, out_ids, out_dist, nullptr, nullptr, nullptr, 0));
  if (nq == 0) {
    set_error("nothing to tune on");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int d = b->ix->cfg.d;
  reps = std::max(1, reps);
  std::vector<qk_batch_tiles> cands;
  for (int rpt : {0, 2})
    for (int qw : {1, 2, 4})
      for (int tr : {16, 32, 64})
        for (int ch : {1024, 4096, 16384}) {
          const qk_batch_tiles t{qw, tr, ch, rpt};
          if (aps_tiles_valid(d, t)) cands.push_back(t);   // every shape gives the same results
        }
  cudaEvent_t e0, e1;
  QK_CUDA(cudaEventCreate(&e0));
  QK_CUDA(cudaEventCreate(&e1));
  float best = INFINITY;
  const qk_batch_tiles keep = b->tiles;
  qk_batch_tiles best_t = keep;
  qk_status st = QK_OK;
  for (const qk_batch_tiles& t : cands) {
    b->tiles = t;
    b->version = ~0ull;
    st = refresh(b, s);
    if (st == QK_OK)   // warm-up
      st = enqueue(b, q, nq, recall_target, out_ids, out_dist, nullptr, nullptr, nullptr, 0, s);
    if (st != QK_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && st == QK_OK; ++r)
      st = enqueue(b, q, nq, recall_target, out_ids, out_dist, nullptr, nullptr, nullptr, 0, s);
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
  b->version = ~0ull;
  if (chosen) *chosen = b->tiles;
  return st;
  QK_GUARD_END
}

qk_status qk_aps_batch_search(qk_aps_batch* b, const float* q, int64_t nq, float recall_target, int64_t* out_ids,
                              float* out_dist, int32_t* out_nprobe, float* out_recall, int32_t* out_scanned0,
                              int32_t cap0, void* stream) {
  QK_GUARD_BEGIN
  // the index's published structure stays put while this captures and enqueues it
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  QK_TRY(check_call(b, q, nq, recall_target, out_ids, out_dist, out_nprobe, out_recall, out_scanned0, cap0));
  if (nq == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  QK_TRY(refresh(b, s));
  QK_TRY(enqueue(b, q, nq, recall_target, out_ids, out_dist, out_nprobe, out_recall, out_scanned0, cap0, s));
  note_readers(b->ix, s);
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_aps_batch_capture(qk_aps_batch* b, const float* q, int64_t nq, float recall_target, int64_t* out_ids,
                               float* out_dist, int32_t* out_nprobe, float* out_recall, void* stream) {
  QK_GUARD_BEGIN
  // the index's published structure stays put while this captures and enqueues it
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  QK_TRY(check_call(b, q, nq, recall_target, out_ids, out_dist, out_nprobe, out_recall, nullptr, 0));
  if (nq == 0) {
    set_error("nothing to capture");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  QK_TRY(refresh(b, s));
  // one run outside the capture sets kernel attributes and occupancy
  QK_TRY(enqueue(b, q, nq, recall_target, out_ids, out_dist, out_nprobe, out_recall, nullptr, 0, s));
  QK_CUDA(cudaStreamSynchronize(s));
  cudaStream_t cs;
  QK_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  qk_status st = QK_OK;
  // relaxed: the prepare launch reads kernel attributes and occupancy, which
  // are not stream work
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaStreamDestroy(cs);
    set_error("stream capture could not start");
    return QK_ERR_CUDA;
  }
  st = enqueue(b, q, nq, recall_target, out_ids, out_dist, out_nprobe, out_recall, nullptr, 0, cs);
  const cudaError_t ce = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (st != QK_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("stream capture failed: ") + cudaGetErrorString(ce));
    return QK_ERR_CUDA;
  }
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("graph instantiation failed: ") + cudaGetErrorString(ie));
    return QK_ERR_CUDA;
  }
  b->graph_version = b->ix->version;
  b->graph_nq = nq;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_aps_batch_replay(qk_aps_batch* b, void* stream) {
  QK_GUARD_BEGIN
  // the index's published structure stays put while this captures and enqueues it
  std::shared_lock<std::shared_mutex> pub;
  if (b && b->ix) pub = std::shared_lock<std::shared_mutex>(b->ix->pub_mu);
  if (!b || !b->graph) {
    set_error("no captured graph");
    return QK_ERR_STATE;
  }
  if (b->graph_version != b->ix->version) {
    set_error("the index changed since the capture: capture again");
    return QK_ERR_STATE;
  }
  QK_CUDA(cudaGraphLaunch(b->graph, (cudaStream_t)stream));
  note_readers(b->ix, (cudaStream_t)stream);
  b->ix->queries_seen += b->graph_nq;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_aps_batch_set_timing(qk_aps_batch* b, int32_t on) {
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

qk_status qk_aps_batch_stage_times(qk_aps_batch* b, float* ms) {
  QK_GUARD_BEGIN
  if (!b || !ms) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  if (!b->timed) {
    set_error("no batch ran with timing on");
    return QK_ERR_STATE;
  }
  const int R = b->timed_rounds;
  QK_CUDA(cudaEventSynchronize(b->ev[2 + 3 * R]));
  auto span = [&](int i, int j) {
    float v = 0.f;
    cudaEventElapsedTime(&v, b->ev[i], b->ev[j]);
    return v;
  };
  ms[0] = span(0, 1);
  ms[1] = span(1, 2);
  ms[2] = ms[3] = 0.f;
  for (int r = 0; r < R; ++r) {
    const int prev = r == 0 ? 2 : 2 + 3 * r;
    const float g = span(prev, 3 + 3 * r), sc = span(3 + 3 * r, 4 + 3 * r), rp = span(4 + 3 * r, 5 + 3 * r);
    ms[1] += rp;
    ms[2] += g;
    ms[3] += sc;
    ms[4 + r] = sc;
  }
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_aps_batch_round_stats(qk_aps_batch* b, int64_t* asked, int64_t* taken) {
  QK_GUARD_BEGIN
  if (!b) {
    set_error("null plan");
    return QK_ERR_ARG;
  }
  unsigned long long h[2 * (ab::kMaxRounds + 1)];
  QK_CUDA(cudaMemcpy(h, b->rstats, sizeof(h), cudaMemcpyDeviceToHost));
  for (int r = 0; r < b->rounds; ++r) {
    if (asked) asked[r] = (int64_t)h[2 * r];
    if (taken) taken[r] = (int64_t)h[2 * r + 1];
  }
  return QK_OK;
  QK_GUARD_END
}

}  // extern "C"
