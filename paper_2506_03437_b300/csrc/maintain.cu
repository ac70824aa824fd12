// The maintenance pass (Sec. 4): cost model, estimate -> verify -> commit /
// reject per level, bottom-up, with 2-means splits, refinement and merges.
//
// The host runtime keeps the bookkeeping: which rows belong to which
// partition, the access frequencies and the action log.  Every computation
// on vectors runs on the GPU: the 2-means of a split, the refinement's Lloyd
// iterations, the reassignment of a merged partition's rows and the
// distances that pick refinement neighbours and merge receivers.  The pass
// ends by re-laying out the arena once from the new partition labels.
//
// Readings (the same as the oracle's, stated in the header of the oracle's
// maintenance module):
//   - lambda(s) is a piecewise-linear table, extended linearly past its ends
//     and floored at 0; Delta O+/- applies lambda to the number of centroids
//     of the level.
//   - Split estimate Eq. 6; merge estimate by uniform redistribution over the
//     n_R = min(r_f, N - 1) nearest centroids (considered for s < s_min).
//   - Candidates with estimate < -tau are processed in ascending order of the
//     estimate (ties: lower index, split first); a partition touched by an
//     earlier committed action of the pass is skipped.
//   - Verify split with Eq. 4 (children's real sizes, alpha A each), verify
//     merge with Eq. 5 (each row to its nearest remaining centroid), both with
//     the current number of live partitions; commit when Delta < -tau.
//   - A committed split keeps the left child in place and appends the right
//     child, then refines: Lloyd iterations seeded by the current centroids
//     over the union of the r_f partitions nearest each child.  A committed
//     merge removes the partition; the dead are compacted out at the end.
//   - In a two-level index the leaves go first; split children stay under
//     their parent, merged leaves leave it; then the parents run their pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "common.cuh"
#include "index.cuh"
#include "trace.h"

namespace qk {

qk_status launch_gather_rows(const float* X, int d, const int64_t* rows, int K, float* out, cudaStream_t s);
qk_status launch_kmeans_assign(const float* X, int64_t n, int d, const float* C, int K, int32_t* assign,
                               float* best_dist, cudaStream_t s);

// Squared distance from x to every row of C (one warp per row of C).
__global__ void dist_to_rows_kernel(const float* __restrict__ C, int64_t n, int d, const float* __restrict__ x,
                                    float* __restrict__ out) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n) return;
  const float* c = C + w * d;
  float acc = 0.f;
  for (int j = lane; j < d; j += 32) {
    float df = c[j] - x[j];
    acc = fmaf(df, df, acc);
  }
  acc = warp_sum_f(acc);
  if (lane == 0) out[w] = acc;
}

namespace {

// Device buffer that grows on demand, stream-ordered like the runtime's
// other temporaries (no call waits for the whole device).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = 0;
  DevBuf() = default;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  DevBuf(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  qk_status reserve(size_t b) {
    if (b <= bytes) return QK_OK;
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
    QK_CUDA(cudaMallocAsync(&p, std::max<size_t>(b, 4096), s));
    bytes = std::max<size_t>(b, 4096);
    return QK_OK;
  }
  template <class T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

struct Lambda {
  std::vector<double> s, us;
  double operator()(double x) const {
    size_t n = s.size();
    if (n == 1) return us[0];
    size_t j;
    if (x <= s[0]) {
      j = 0;
    } else if (x >= s[n - 1]) {
      j = n - 2;
    } else {
      j = std::upper_bound(s.begin(), s.end(), x) - s.begin() - 1;
    }
    double w = (x - s[j]) / (s[j + 1] - s[j]);
    double v = us[j] + w * (us[j + 1] - us[j]);
    return v > 0.0 ? v : 0.0;
  }
};

// One level of the pass: centroids, member row references and frequencies.
struct Level {
  int d = 0;
  const float* rows = nullptr;                 // device rows indexed by the references
  const int64_t* id_of = nullptr;              // id of each reference (NULL: the reference is the id)
  std::vector<std::vector<float>> C;           // centroid per partition (dead ones included)
  std::vector<std::vector<int64_t>> mem;       // member row references per partition
  std::vector<double> A;
  std::vector<char> dead;
};

struct Ctx {
  const qk_maint_params* p;
  Lambda lam;
  uint64_t seed;
  cudaStream_t s;
  DevBuf rows, cent, assign, dist, refs, x;
  std::vector<qk_maint_action>* log;
  explicit Ctx(cudaStream_t st) : s(st), rows(st), cent(st), assign(st), dist(st), refs(st), x(st) {}
};

uint64_t split_seed(uint64_t seed, int level, int64_t j) {
  return seed + 0x9E3779B97F4A7C15ull * (uint64_t)((int64_t)level * 1000003 + j + 1);
}

// Rows of the given references, gathered into ctx.rows (device).
qk_status gather(Ctx& cx, const Level& L, const std::vector<int64_t>& refs) {
  size_t n = refs.size();
  QK_TRY(cx.refs.reserve(sizeof(int64_t) * std::max<size_t>(n, 1)));
  QK_TRY(cx.rows.reserve(sizeof(float) * std::max<size_t>(n, 1) * L.d));
  if (n == 0) return QK_OK;
  QK_CUDA(cudaMemcpyAsync(cx.refs.p, refs.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, cx.s));
  return launch_gather_rows(L.rows, L.d, cx.refs.as<int64_t>(), (int)n, cx.rows.as<float>(), cx.s);
}

// The `count` live partitions whose centroids are nearest x (ties: lower index).
qk_status nearest(Ctx& cx, const Level& L, const std::vector<int32_t>& live, const std::vector<float>& x, int count,
                  int32_t exclude, std::vector<int32_t>& out) {
  out.clear();
  std::vector<int32_t> cand;
  for (int32_t j : live)
    if (j != exclude) cand.push_back(j);
  if (cand.empty() || count <= 0) return QK_OK;
  const int d = L.d;
  size_t n = cand.size();
  std::vector<float> Cc(n * d);
  for (size_t i = 0; i < n; ++i) std::memcpy(&Cc[i * d], L.C[cand[i]].data(), sizeof(float) * d);
  QK_TRY(cx.cent.reserve(sizeof(float) * n * d));
  QK_TRY(cx.x.reserve(sizeof(float) * d));
  QK_TRY(cx.dist.reserve(sizeof(float) * n));
  QK_CUDA(cudaMemcpyAsync(cx.cent.p, Cc.data(), sizeof(float) * n * d, cudaMemcpyHostToDevice, cx.s));
  QK_CUDA(cudaMemcpyAsync(cx.x.p, x.data(), sizeof(float) * d, cudaMemcpyHostToDevice, cx.s));
  dist_to_rows_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, cx.s>>>(cx.cent.as<float>(), (int64_t)n, d,
                                                                           cx.x.as<float>(), cx.dist.as<float>());
  QK_CUDA(cudaGetLastError());
  std::vector<float> dist(n);
  QK_CUDA(cudaMemcpyAsync(dist.data(), cx.dist.p, sizeof(float) * n, cudaMemcpyDeviceToHost, cx.s));
  QK_CUDA(cudaStreamSynchronize(cx.s));
  std::vector<size_t> order(n);
  for (size_t i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
    return dist[a] < dist[b] || (dist[a] == dist[b] && cand[a] < cand[b]);
  });
  for (size_t i = 0; i < n && (int)i < count; ++i) out.push_back(cand[order[i]]);
  return QK_OK;
}

// k-means of the given rows into K clusters on the GPU; C and assignment to host.
qk_status cluster(Ctx& cx, const Level& L, const std::vector<int64_t>& refs, int K, int iters, uint64_t seed,
                  const std::vector<float>* C_init, std::vector<float>& C, std::vector<int32_t>& a) {
  const int d = L.d;
  int64_t n = (int64_t)refs.size();
  QK_TRY(gather(cx, L, refs));
  QK_TRY(cx.assign.reserve(sizeof(int32_t) * std::max<int64_t>(n, 1)));
  DevBuf cout(cx.s), cin(cx.s);
  QK_TRY(cout.reserve(sizeof(float) * K * d));
  if (C_init) {
    QK_TRY(cin.reserve(sizeof(float) * K * d));
    QK_CUDA(cudaMemcpyAsync(cin.p, C_init->data(), sizeof(float) * K * d, cudaMemcpyHostToDevice, cx.s));
  }
  QK_TRY(kmeans(cx.rows.as<float>(), n, d, K, iters, seed, cout.as<float>(), cx.assign.as<int32_t>(), cx.s,
                C_init ? cin.as<float>() : nullptr));
  C.resize((size_t)K * d);
  a.resize(n);
  QK_CUDA(cudaMemcpyAsync(C.data(), cout.p, sizeof(float) * K * d, cudaMemcpyDeviceToHost, cx.s));
  if (n) QK_CUDA(cudaMemcpyAsync(a.data(), cx.assign.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, cx.s));
  QK_CUDA(cudaStreamSynchronize(cx.s));
  return QK_OK;
}

struct Cand {
  double e;
  int32_t j;
  int32_t kind;  // 0 split, 1 merge
  bool operator<(const Cand& o) const {
    if (e != o.e) return e < o.e;
    if (j != o.j) return j < o.j;
    return kind < o.kind;
  }
};

// One estimate / verify / commit pass over a level.  parent_of (leaf level of a
// two-level index) is extended and compacted with the partitions.  On return
// the dead partitions are removed.
qk_status maintain_level(Ctx& cx, Level& L, int level_no, std::vector<int32_t>* parent_of) {
  const qk_maint_params& P = *cx.p;
  const Lambda& lam = cx.lam;
  const int d = L.d;
  const int32_t N0 = (int32_t)L.C.size();
  L.dead.assign(N0, 0);
  std::vector<int32_t> live(N0);
  for (int32_t j = 0; j < N0; ++j) live[j] = j;
  std::vector<int64_t> size(N0);
  for (int32_t j = 0; j < N0; ++j) size[j] = (int64_t)L.mem[j].size();

  // Stage 1: estimates
  std::vector<Cand> cands;
  for (int32_t j = 0; j < N0; ++j) {
    double s = (double)size[j], a = L.A[j];
    if (size[j] >= 2) {
      double e = (lam(N0 + 1) - lam(N0)) - a * lam(s) + 2.0 * P.alpha * a * lam(s / 2.0);
      if (e < -P.tau_us) cands.push_back({e, j, 0});
    }
    if (size[j] < P.s_min && N0 > 1) {
      int nR = std::min<int>(P.refine_radius, N0 - 1);
      std::vector<int32_t> R;
      QK_TRY(nearest(cx, L, live, L.C[j], nR, j, R));
      double e = (lam(N0 - 1) - lam(N0)) - a * lam(s);
      for (int32_t m : R)
        e += (L.A[m] + a / nR) * lam((double)size[m] + s / nR) - L.A[m] * lam((double)size[m]);
      if (e < -P.tau_us) cands.push_back({e, j, 1});
    }
  }
  std::sort(cands.begin(), cands.end());

  std::set<int32_t> touched;
  for (const Cand& c : cands) {
    const int32_t j = c.j;
    if (touched.count(j) || L.dead[j]) continue;
    const int32_t n_live = (int32_t)live.size();
    const double s = (double)size[j], a = L.A[j];
    qk_maint_action act;
    std::memset(&act, 0, sizeof(act));
    act.level = level_no;
    act.kind = c.kind;
    act.partition = j;
    act.estimate = c.e;
    if (c.kind == 0) {
      // 2-means over the partition's rows in ascending id order, so that the
      // seeded rows do not depend on the storage order inside the partition
      std::vector<int64_t> by_id(L.mem[j]);
      auto idv = [&](int64_t r) { return L.id_of ? L.id_of[r] : r; };
      std::stable_sort(by_id.begin(), by_id.end(), [&](int64_t x, int64_t y) { return idv(x) < idv(y); });
      L.mem[j] = by_id;
      std::vector<float> C2;
      std::vector<int32_t> a2;
      QK_TRY(cluster(cx, L, L.mem[j], 2, P.split_iters, split_seed(cx.seed, level_no, j), nullptr, C2, a2));
      std::vector<int64_t> left, right;
      for (size_t r = 0; r < a2.size(); ++r) (a2[r] == 0 ? left : right).push_back(L.mem[j][r]);
      if (left.empty() || right.empty()) {
        act.delta = NAN;
        act.committed = 0;
        cx.log->push_back(act);
        continue;
      }
      double dlt = (lam(n_live + 1) - lam(n_live)) - a * lam(s) + P.alpha * a * lam((double)left.size()) +
                   P.alpha * a * lam((double)right.size());
      act.delta = dlt;
      act.committed = dlt < -P.tau_us;
      cx.log->push_back(act);
      if (!act.committed) continue;
      const int32_t jn = (int32_t)L.C.size();
      L.C[j].assign(C2.begin(), C2.begin() + d);
      L.C.push_back(std::vector<float>(C2.begin() + d, C2.begin() + 2 * d));
      L.mem[j] = left;
      L.mem.push_back(right);
      L.A[j] = P.alpha * a;
      L.A.push_back(P.alpha * a);
      L.dead.push_back(0);
      size[j] = (int64_t)left.size();
      size.push_back((int64_t)right.size());
      live.push_back(jn);
      if (parent_of) parent_of->push_back((*parent_of)[j]);
      touched.insert(j);
      touched.insert(jn);
      if (P.refine && P.refine_iters > 0) {
        std::vector<int32_t> n1, n2;
        QK_TRY(nearest(cx, L, live, L.C[j], P.refine_radius, -1, n1));
        QK_TRY(nearest(cx, L, live, L.C[jn], P.refine_radius, -1, n2));
        std::set<int32_t> ps(n1.begin(), n1.end());
        ps.insert(n2.begin(), n2.end());
        std::vector<int32_t> parts(ps.begin(), ps.end());
        std::vector<int64_t> pooled;
        std::vector<float> Cin;
        for (int32_t p : parts) {
          pooled.insert(pooled.end(), L.mem[p].begin(), L.mem[p].end());
          Cin.insert(Cin.end(), L.C[p].begin(), L.C[p].end());
        }
        std::vector<float> Cr;
        std::vector<int32_t> ar;
        QK_TRY(cluster(cx, L, pooled, (int)parts.size(), P.refine_iters, 0, &Cin, Cr, ar));
        for (size_t n = 0; n < parts.size(); ++n) {
          L.C[parts[n]].assign(Cr.begin() + n * d, Cr.begin() + (n + 1) * d);
          L.mem[parts[n]].clear();
        }
        for (size_t r = 0; r < pooled.size(); ++r) L.mem[parts[ar[r]]].push_back(pooled[r]);
        for (int32_t p : parts) {
          size[p] = (int64_t)L.mem[p].size();
          touched.insert(p);
        }
      }
    } else {
      std::vector<int32_t> others;
      for (int32_t m : live)
        if (m != j) others.push_back(m);
      std::vector<float> Co(others.size() * d);
      for (size_t i = 0; i < others.size(); ++i) std::memcpy(&Co[i * d], L.C[others[i]].data(), sizeof(float) * d);
      int64_t n = (int64_t)L.mem[j].size();
      std::vector<int32_t> am(n);
      if (n > 0) {
        QK_TRY(gather(cx, L, L.mem[j]));
        QK_TRY(cx.cent.reserve(sizeof(float) * Co.size()));
        QK_TRY(cx.assign.reserve(sizeof(int32_t) * n));
        QK_CUDA(cudaMemcpyAsync(cx.cent.p, Co.data(), sizeof(float) * Co.size(), cudaMemcpyHostToDevice, cx.s));
        QK_TRY(assign_nearest(cx.rows.as<float>(), n, d, cx.cent.as<float>(), (int)others.size(),
                              cx.assign.as<int32_t>(), cx.s));
        QK_CUDA(cudaMemcpyAsync(am.data(), cx.assign.p, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, cx.s));
        QK_CUDA(cudaStreamSynchronize(cx.s));
      }
      std::vector<std::vector<int64_t>> recv(others.size());
      for (int64_t r = 0; r < n; ++r) recv[am[r]].push_back(L.mem[j][r]);
      double dlt = (lam(n_live - 1) - lam(n_live)) - a * lam(s);
      for (size_t i = 0; i < others.size(); ++i) {
        if (recv[i].empty()) continue;
        int32_t m = others[i];
        double ds = (double)recv[i].size();
        dlt += (L.A[m] + a * ds / s) * lam((double)size[m] + ds) - L.A[m] * lam((double)size[m]);
      }
      act.delta = dlt;
      act.committed = dlt < -P.tau_us;
      cx.log->push_back(act);
      if (!act.committed) continue;
      for (size_t i = 0; i < others.size(); ++i) {
        if (recv[i].empty()) continue;
        int32_t m = others[i];
        L.mem[m].insert(L.mem[m].end(), recv[i].begin(), recv[i].end());
        L.A[m] += a * (double)recv[i].size() / s;
        size[m] += (int64_t)recv[i].size();
        touched.insert(m);
      }
      L.dead[j] = 1;
      live.erase(std::find(live.begin(), live.end(), j));
      touched.insert(j);
    }
  }
  // compact out the dead partitions, keeping the order of the rest
  Level out;
  out.d = d;
  out.rows = L.rows;
  std::vector<int32_t> po;
  for (size_t j = 0; j < L.C.size(); ++j) {
    if (L.dead[j]) continue;
    out.C.push_back(std::move(L.C[j]));
    out.mem.push_back(std::move(L.mem[j]));
    out.A.push_back(L.A[j]);
    if (parent_of) po.push_back((*parent_of)[j]);
  }
  L = std::move(out);
  if (parent_of) *parent_of = po;
  return QK_OK;
}

}  // namespace
}  // namespace qk

using namespace qk;

// The pass up to its new structure: both levels are planned and the new
// arena, centroids, parent level and id map are built into *out, a fresh
// index object.  ix is only read, so searches of ix may run meanwhile.
static qk_status maintain_plan(qk_index* ix, const qk_maint_params* params, qk_maint_action* log, int32_t log_cap,
                               int32_t* n_log, void* stream, qk_index** out) {
  // planning only reads the published structure; updates wait, searches do not
  std::shared_lock<std::shared_mutex> pub;
  if (ix) pub = std::shared_lock<std::shared_mutex>(ix->pub_mu);
  *out = nullptr;
  if (!ix || !params) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  if (!ix->ready) {
    set_error("index is empty: build or load it first");
    return QK_ERR_STATE;
  }
  const qk_maint_params& P = *params;
  if (P.lambda_points < 1 || !P.lambda_sizes || !P.lambda_us || P.refine_radius < 1 || P.split_iters < 0 ||
      P.refine_iters < 0 || !(P.tau_us >= 0) || !(P.alpha > 0)) {
    set_error("invalid maintenance parameters");
    return QK_ERR_ARG;
  }
  for (int32_t i = 1; i < P.lambda_points; ++i)
    if (!(P.lambda_sizes[i] > P.lambda_sizes[i - 1])) {
      set_error("lambda sizes must increase");
      return QK_ERR_ARG;
    }
  cudaStream_t s = (cudaStream_t)stream;
  const int d = ix->cfg.d;
  const int64_t window = P.window > 0 ? P.window : ix->queries_seen.load();
  if (window < 1) {
    set_error("no queries in the statistics window");
    return QK_ERR_STATE;
  }
  std::vector<qk_maint_action> acts;
  Trace tr("maintain");
  Ctx cx(s);
  cx.p = params;
  cx.lam.s.assign(P.lambda_sizes, P.lambda_sizes + P.lambda_points);
  cx.lam.us.assign(P.lambda_us, P.lambda_us + P.lambda_points);
  cx.seed = ix->cfg.seed;
  cx.log = &acts;

  // Stage 0: statistics (access counts over the window, sizes)
  const int32_t N0 = ix->n_leaf, N1 = ix->n_parent;
  std::vector<int64_t> h0(N0), h1(N1 > 0 ? N1 : 0);
  QK_CUDA(cudaMemcpyAsync(h0.data(), ix->hits0, sizeof(int64_t) * N0, cudaMemcpyDeviceToHost, s));
  if (N1 > 0) QK_CUDA(cudaMemcpyAsync(h1.data(), ix->hits1, sizeof(int64_t) * N1, cudaMemcpyDeviceToHost, s));
  std::vector<float> c0((size_t)N0 * d), c1((size_t)std::max(N1, 0) * d);
  QK_CUDA(cudaMemcpyAsync(c0.data(), ix->cent0, sizeof(float) * c0.size(), cudaMemcpyDeviceToHost, s));
  if (N1 > 0) QK_CUDA(cudaMemcpyAsync(c1.data(), ix->cent1, sizeof(float) * c1.size(), cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));

  Level L0;
  L0.d = d;
  L0.rows = ix->vec0;
  L0.id_of = ix->h_ids0.data();
  for (int32_t j = 0; j < N0; ++j) {
    L0.C.emplace_back(c0.begin() + (size_t)j * d, c0.begin() + (size_t)(j + 1) * d);
    std::vector<int64_t> m((size_t)ix->h_size0[j]);
    for (int32_t t = 0; t < ix->h_size0[j]; ++t) m[t] = ix->h_off0[j] + t;
    L0.mem.push_back(std::move(m));
    L0.A.push_back((double)h0[j] / (double)window);
  }
  std::vector<int32_t> parent_of;
  if (N1 > 0) {
    parent_of.assign(N0, 0);
    std::vector<int64_t> ids1((size_t)N0);
    QK_CUDA(cudaMemcpy(ids1.data(), ix->ids1, sizeof(int64_t) * N0, cudaMemcpyDeviceToHost));
    for (int32_t p = 0; p < N1; ++p)
      for (int32_t t = 0; t < ix->h_size1[p]; ++t) parent_of[ids1[ix->h_off1[p] + t]] = p;
  }
  tr.mark("stats");
  QK_TRY(maintain_level(cx, L0, 0, N1 > 0 ? &parent_of : nullptr));
  tr.mark("leaf_level");
  const int32_t M0 = (int32_t)L0.C.size();
  if (M0 < 1) {
    set_error("maintenance removed every partition");
    return QK_ERR_STATE;
  }

  // new leaf centroids and the label of every arena row
  DevBuf dC0(s), dlab(s), dC1(s), dpol(s);
  std::vector<float> nc0((size_t)M0 * d);
  for (int32_t j = 0; j < M0; ++j) std::memcpy(&nc0[(size_t)j * d], L0.C[j].data(), sizeof(float) * d);
  std::vector<int32_t> lab((size_t)ix->cap0, -1);
  for (int32_t j = 0; j < M0; ++j)
    for (int64_t r : L0.mem[j]) lab[r] = j;
  QK_TRY(dC0.reserve(sizeof(float) * nc0.size()));
  QK_TRY(dlab.reserve(sizeof(int32_t) * lab.size()));
  QK_CUDA(cudaMemcpyAsync(dC0.p, nc0.data(), sizeof(float) * nc0.size(), cudaMemcpyHostToDevice, s));
  QK_CUDA(cudaMemcpyAsync(dlab.p, lab.data(), sizeof(int32_t) * lab.size(), cudaMemcpyHostToDevice, s));

  int32_t M1 = 0;
  std::vector<float> nc1;
  std::vector<int32_t> pol;
  if (N1 > 0) {
    Level L1;
    L1.d = d;
    L1.rows = dC0.as<float>();   // the parents' rows are the new leaf centroids
    for (int32_t p = 0; p < N1; ++p) {
      L1.C.emplace_back(c1.begin() + (size_t)p * d, c1.begin() + (size_t)(p + 1) * d);
      L1.mem.emplace_back();
      L1.A.push_back((double)h1[p] / (double)window);
    }
    for (int32_t lf = 0; lf < M0; ++lf) L1.mem[parent_of[lf]].push_back(lf);
    QK_TRY(maintain_level(cx, L1, 1, nullptr));
    M1 = (int32_t)L1.C.size();
    nc1.resize((size_t)M1 * d);
    pol.assign(M0, 0);
    for (int32_t p = 0; p < M1; ++p) {
      std::memcpy(&nc1[(size_t)p * d], L1.C[p].data(), sizeof(float) * d);
      for (int64_t lf : L1.mem[p]) pol[lf] = p;
    }
    QK_TRY(dC1.reserve(sizeof(float) * nc1.size()));
    QK_TRY(dpol.reserve(sizeof(int32_t) * pol.size()));
    QK_CUDA(cudaMemcpyAsync(dC1.p, nc1.data(), sizeof(float) * nc1.size(), cudaMemcpyHostToDevice, s));
    QK_CUDA(cudaMemcpyAsync(dpol.p, pol.data(), sizeof(int32_t) * pol.size(), cudaMemcpyHostToDevice, s));
  }

  // the level band (off unless asked): keep the top level within
  // sqrt(M0)/4 .. 4 sqrt(M0) centroids by adding, removing or rebuilding the
  // parent level; new parents are the build's k-means (seed + 1) of the leaf
  // centroids into round(sqrt(M0))
  if (P.level_band) {
    const double rt = std::sqrt((double)M0);
    const int32_t np = std::max<int32_t>(1, (int32_t)std::floor(rt + 0.5));
    const int32_t top = N1 > 0 ? M1 : 0;
    int kind = -1;
    if (top == 0) {
      if (M0 > 16) kind = 2;
    } else if (M0 <= 16) {
      kind = 3;
    } else if (top < rt / 4.0 || top > 4.0 * rt) {
      kind = 4;
    }
    if (kind == 2 || kind == 4) {
      QK_TRY(dC1.reserve(sizeof(float) * (size_t)np * d));
      QK_TRY(dpol.reserve(sizeof(int32_t) * (size_t)M0));
      QK_TRY(kmeans(dC0.as<float>(), M0, d, np, std::max(0, P.level_iters), ix->cfg.seed + 1, dC1.as<float>(),
                    dpol.as<int32_t>(), s, nullptr));
      M1 = np;
    } else if (kind == 3) {
      M1 = 0;
    }
    if (kind >= 0) {
      qk_maint_action act;
      std::memset(&act, 0, sizeof(act));
      act.level = 1;
      act.kind = kind;
      act.partition = M1;
      act.committed = 1;
      act.estimate = NAN;
      act.delta = NAN;
      acts.push_back(act);
    }
  }

  tr.mark("parent_level");
  // the new structure, laid out from the labels into a fresh object (the live
  // arena is only read)
  qk_index* nx = new qk_index();
  nx->cfg = ix->cfg;
  nx->cfg.n_leaf = M0;
  nx->cfg.n_parent = M1;
  nx->device = ix->device;
  DevBuf nst(s);             // the install's own status word (the live one may be in use by searches)
  QK_TRY(nst.reserve(sizeof(int32_t)));
  QK_CUDA(cudaMemsetAsync(nst.p, 0, sizeof(int32_t), s));
  nx->status = nst.as<int32_t>();
  qk_status st = install(nx, ix->vec0, ix->ids0, ix->cap0, dC0.as<float>(), dlab.as<int32_t>(),
                         M1 > 0 ? dC1.as<float>() : nullptr, M1 > 0 ? dpol.as<int32_t>() : nullptr, s, true);
  nx->status = nullptr;
  if (st != QK_OK) {
    release_structure(nx);
    delete nx;
    return st;
  }
  nx->n = ix->n;
  *out = nx;
  tr.mark("install");
  if (n_log) *n_log = (int32_t)acts.size();
  if (log)
    for (int32_t i = 0; i < (int32_t)acts.size() && i < log_cap; ++i) log[i] = acts[i];
  return QK_OK;
}

// Makes nx's structure the index's.  The old one is retired: searches still
// in flight keep reading it, and it is freed once they have completed.
static qk_status commit_structure(qk_index* ix, qk_index* nx, cudaStream_t s) {
  QK_CUDA(cudaStreamSynchronize(s));
  reclaim(ix, false);
  std::unique_lock<std::shared_mutex> pub(ix->pub_mu);
  swap_structure(ix, nx);
  Retired r;
  r.version = ix->version;
  r.structure = nx;
  ix->queries_seen = 0;
  ++ix->version;
  pub.unlock();
  retire(ix, std::move(r));
  return QK_OK;
}

static void discard_pending(qk_index* ix) {
  if (!ix->pending) return;
  release_structure(ix->pending);
  delete ix->pending;
  ix->pending = nullptr;
}

extern "C" qk_status qk_maintain(qk_index* ix, const qk_maint_params* params, qk_maint_action* log, int32_t log_cap,
                                 int32_t* n_log, void* stream) {
  QK_GUARD_BEGIN
  qk_index* nx = nullptr;
  QK_TRY(maintain_plan(ix, params, log, log_cap, n_log, stream, &nx));
  discard_pending(ix);
  return commit_structure(ix, nx, (cudaStream_t)stream);
  QK_GUARD_END
}

extern "C" qk_status qk_maintain_prepare(qk_index* ix, const qk_maint_params* params, qk_maint_action* log,
                                         int32_t log_cap, int32_t* n_log, void* stream) {
  QK_GUARD_BEGIN
  if (!ix) {
    set_error("null index");
    return QK_ERR_ARG;
  }
  discard_pending(ix);
  const uint64_t v = ix->version;
  qk_index* nx = nullptr;
  QK_TRY(maintain_plan(ix, params, log, log_cap, n_log, stream, &nx));
  QK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  ix->pending = nx;
  ix->pending_version = v;
  return QK_OK;
  QK_GUARD_END
}

extern "C" qk_status qk_maintain_commit(qk_index* ix, void* stream) {
  QK_GUARD_BEGIN
  if (!ix || !ix->pending) {
    set_error("no prepared maintenance pass");
    return QK_ERR_STATE;
  }
  if (ix->pending_version != ix->version) {
    discard_pending(ix);
    set_error("the index changed after qk_maintain_prepare: the prepared pass was discarded");
    return QK_ERR_STATE;
  }
  qk_index* nx = ix->pending;
  ix->pending = nullptr;
  return commit_structure(ix, nx, (cudaStream_t)stream);
  QK_GUARD_END
}
