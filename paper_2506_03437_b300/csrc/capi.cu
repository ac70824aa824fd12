// Host runtime of the index and the C-ABI entry points declared in
// include/quake_b300.h.  The runtime owns the device arena, the per-level
// partition tables and the id -> (partition, slot) map; every computation on
// vectors runs in the kernels of search.cu, kmeans.cu and arena.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "capvol.cuh"
#include "common.cuh"
#include "index.cuh"
#include "trace.h"

namespace qk {

qk_status launch_search(const SearchArgs& a, cudaStream_t stream);
qk_status launch_beta_table(double a, double lnB, double* table, cudaStream_t stream);
qk_status launch_cap_fraction(int mode, double a, double lnB, const double* table, const double* t,
                              const double* rho, int64_t n, double* out, cudaStream_t stream);
qk_status launch_kmeans_assign(const float* X, int64_t n, int d, const float* C, int K, int32_t* assign,
                               float* best_dist, cudaStream_t s);
qk_status launch_kmeans_update(const float* X, int64_t n, int d, const int32_t* assign, const float* C_prev, int K,
                               float* C_new, double* sums, int32_t* counts, cudaStream_t s);
qk_status launch_gather_rows(const float* X, int d, const int64_t* rows, int K, float* out, cudaStream_t s);
qk_status launch_histogram(const int32_t* lab, int64_t n, int32_t K, int32_t* counts, int32_t* status,
                           cudaStream_t s, bool skip_unlabelled);
qk_status launch_scatter(const float* X, const int64_t* ids, int64_t n, int d, const int32_t* lab,
                         const int64_t* off, int32_t* cursor, float* vec, int64_t* ids_out, cudaStream_t s);

qk_status launch_descend_children(const float* X, int64_t n, int d, const int32_t* parent, const float* vec1,
                                  const int64_t* ids1, const int64_t* off1, const int32_t* size1, int32_t n_parent,
                                  int32_t* leaf, cudaStream_t s);
qk_status launch_nan_check(const float* X, int64_t total, int32_t* flag, cudaStream_t s);
qk_status launch_relayout(const float* old_vec, const int64_t* old_ids, const int64_t* old_off, const int64_t* new_off,
                          const int32_t* size, int32_t n_part, int d, float* new_vec, int64_t* new_ids,
                          cudaStream_t s);
qk_status launch_place_rows(const float* X, const int64_t* ids, int64_t n, int d, const int64_t* dst, float* vec,
                            int64_t* ids_out, cudaStream_t s);
qk_status launch_gather_moves(const float* vec, const int64_t* ids, const int64_t* src, int64_t m, int d, float* tvec,
                              int64_t* tids, cudaStream_t s);

qk_status launch_quantize_arena(const float* vec, const int64_t* off, const int32_t* size, int32_t n_part, int d,
                                int storage, float* scale, unsigned char* lp, cudaStream_t s);
qk_status launch_quantize_rows(const float* X, int64_t n, int d, const int64_t* dst, const int32_t* part, int storage,
                               const float* scale, unsigned char* lp, cudaStream_t s);
qk_status launch_move_bytes(unsigned char* a, const int64_t* src, const int64_t* dst, int64_t m, int rb,
                            unsigned char* tmp, cudaStream_t s);
qk_status launch_relayout_bytes(const unsigned char* old_a, const int64_t* old_off, const int64_t* new_off,
                                const int32_t* size, int32_t n_part, int rb, unsigned char* new_a, cudaStream_t s);

qk_status launch_tc_nearest(const float* X, int64_t n, int d, const float* C, int K, int metric, int k,
                            int32_t* out_idx, float* out_dist, float* cnorm, int32_t* cand, int32_t* status,
                            cudaStream_t s);
int tc_candidates_per_row();
void preload_update_kernels();

static int elem_bytes(int storage) { return storage == QK_STORE_BF16 ? 2 : (storage == QK_STORE_FP8 ? 1 : 4); }

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

qk_status cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return QK_ERR_OOM;
  }
  return QK_ERR_CUDA;
}

static bool supported_dim(int d) {
  switch (d) {
    case 32: case 64: case 96: case 128: case 192: case 256: case 384: case 512: case 768: case 1024:
      return true;
    default:
      return false;
  }
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Temporary device buffer, stream-ordered: taken from the device's memory
// pool on stream s and given back, in stream order, on scope exit, so that
// no call waits for the whole device.
struct Tmp {
  void* p = nullptr;
  cudaStream_t s;
  explicit Tmp(cudaStream_t st) : s(st) {}
  Tmp(const Tmp&) = delete;
  ~Tmp() {
    if (p) cudaFreeAsync(p, s);
  }
  template <class T>
  qk_status alloc(size_t count, T** out) {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    if (count == 0) count = 1;
    QK_CUDA(cudaMallocAsync(&p, count * sizeof(T), s));
    *out = static_cast<T*>(p);
    return QK_OK;
  }
};

template <class T>
static qk_status in_device(const T* src, size_t count, Tmp& tmp, const T** out, cudaStream_t s) {
  if (!src || is_device_ptr(src)) {
    if (reinterpret_cast<uintptr_t>(src) % 16 != 0) {   // rows are read with 16-byte accesses
      set_error("device buffers must be 16-byte aligned");
      return QK_ERR_ARG;
    }
    *out = src;
    return QK_OK;
  }
  T* d = nullptr;
  QK_TRY(tmp.alloc<T>(count, &d));
  QK_CUDA(cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
  *out = d;
  return QK_OK;
}

// Index memory (mem_alloc / mem_free): stream-ordered on a private stream,
// so that handing back an old version's memory never waits for the device.
template <class T>
static void dfree(T*& p) {
  mem_free(p);
  p = nullptr;
}

template <class T>
static qk_status dalloc(T** p, size_t count) {
  dfree(*p);
  if (count == 0) count = 1;
  return mem_alloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

static qk_status ensure(Buffer& b, size_t bytes) {
  if (b.bytes >= bytes) return QK_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = std::max<size_t>(bytes, 1 << 20);
  QK_CUDA(cudaMalloc(&b.p, want));
  b.bytes = want;
  return QK_OK;
}


// Rows reserved per partition: its size plus room for inserts.
static int64_t capacity_for(int64_t size) { return size + std::max<int64_t>(16, size / 4); }

// Free rows behind the last partition of a fresh arena (1/8 of the reserved rows).
static int64_t tail_rows(int64_t reserved) { return std::max<int64_t>(1024, reserved / 8); }

static void free_structure(qk_index* ix) {
  dfree(ix->vec0);
  dfree(ix->ids0);
  dfree(ix->off0);
  dfree(ix->size0);
  dfree(ix->cent0);
  dfree(ix->vec1);
  dfree(ix->ids1);
  dfree(ix->off1);
  dfree(ix->size1);
  dfree(ix->cent1);
  dfree(ix->hits0);
  dfree(ix->hits1);
  dfree(ix->lp0);
  dfree(ix->lp_scale0);
  for (Table& t : ix->spare0) {
    dfree(t.off);
    dfree(t.size);
  }
  ix->spare0.clear();
  ix->free0.clear();
  ix->ready = false;
  ix->where.clear();
}

void release_structure(qk_index* ix) { free_structure(ix); }

void swap_structure(qk_index* a, qk_index* b) {
  using std::swap;
  swap(a->vec0, b->vec0);
  swap(a->ids0, b->ids0);
  swap(a->cap0, b->cap0);
  swap(a->used0, b->used0);
  swap(a->holes0, b->holes0);
  swap(a->off0, b->off0);
  swap(a->size0, b->size0);
  swap(a->cent0, b->cent0);
  swap(a->lp0, b->lp0);
  swap(a->lp_scale0, b->lp_scale0);
  swap(a->h_off0, b->h_off0);
  swap(a->h_cap_part0, b->h_cap_part0);
  swap(a->h_size0, b->h_size0);
  swap(a->h_ids0, b->h_ids0);
  swap(a->arena_id, b->arena_id);
  swap(a->free0, b->free0);
  swap(a->spare0, b->spare0);
  swap(a->vec1, b->vec1);
  swap(a->ids1, b->ids1);
  swap(a->off1, b->off1);
  swap(a->size1, b->size1);
  swap(a->cent1, b->cent1);
  swap(a->h_size1, b->h_size1);
  swap(a->h_off1, b->h_off1);
  swap(a->hits0, b->hits0);
  swap(a->hits1, b->hits1);
  swap(a->where, b->where);
  swap(a->n, b->n);
  swap(a->n_leaf, b->n_leaf);
  swap(a->n_parent, b->n_parent);
  swap(a->cfg.n_leaf, b->cfg.n_leaf);
  swap(a->cfg.n_parent, b->cfg.n_parent);
  swap(a->ready, b->ready);
}

// Groups `rows` (n x d, device) by label into a fresh arena.  Returns the
// arena, its partition offsets/sizes on host and device.
static qk_status group_rows(const float* rows, const int64_t* ids, int64_t n, int d, const int32_t* lab,
                            int32_t K, bool slack, int32_t* status, float** vec, int64_t** ids_out,
                            int64_t** off, int32_t** size, std::vector<int64_t>& h_off,
                            std::vector<int32_t>& h_size, std::vector<int64_t>* h_cap, int64_t* cap_rows,
                            int64_t* used_rows, cudaStream_t s, bool skip_unlabelled) {
  Tmp tc(s);
  int32_t* counts = nullptr;
  QK_TRY(tc.alloc<int32_t>(K, &counts));
  QK_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * K, s));
  QK_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
  QK_TRY(launch_histogram(lab, n, K, counts, status, s, skip_unlabelled));
  h_size.assign(K, 0);
  int32_t st = 0;
  QK_CUDA(cudaMemcpyAsync(h_size.data(), counts, sizeof(int32_t) * K, cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaMemcpyAsync(&st, status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));
  if (st != 0) {
    set_error("partition label out of range");
    return QK_ERR_ARG;
  }
  h_off.assign(K, 0);
  if (h_cap) h_cap->assign(K, 0);
  int64_t o = 0;
  for (int32_t j = 0; j < K; ++j) {
    h_off[j] = o;
    int64_t c = slack ? capacity_for(h_size[j]) : h_size[j];
    if (h_cap) (*h_cap)[j] = c;
    o += c;
  }
  const int64_t total = o + (slack ? tail_rows(o) : 0);
  *cap_rows = total;
  if (used_rows) *used_rows = o;
  QK_TRY(dalloc(vec, (size_t)total * d));
  QK_TRY(dalloc(ids_out, (size_t)total));
  QK_CUDA(cudaMemsetAsync(*ids_out, 0xff, sizeof(int64_t) * (size_t)total, s));   // id -1 in unused rows
  QK_TRY(dalloc(off, (size_t)K));
  QK_TRY(dalloc(size, (size_t)K));
  QK_CUDA(cudaMemcpyAsync(*off, h_off.data(), sizeof(int64_t) * K, cudaMemcpyHostToDevice, s));
  QK_CUDA(cudaMemcpyAsync(*size, h_size.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, s));
  QK_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * K, s));
  QK_TRY(launch_scatter(rows, ids, n, d, lab, *off, counts, *vec, *ids_out, s));
  QK_CUDA(cudaStreamSynchronize(s));
  return QK_OK;
}

// Installs a partitioning given by device arrays (the common end of build,
// load and maintain).  With skip_unlabelled, rows labelled -1 are left out
// (maintain passes the whole arena, reserved rows included).
qk_status install(qk_index* ix, const float* X, const int64_t* ids, int64_t n, const float* C0,
                  const int32_t* leaf_of_row, const float* C1, const int32_t* parent_of_leaf, cudaStream_t s,
                  bool skip_unlabelled) {
  const int d = ix->cfg.d;
  const int32_t N0 = ix->cfg.n_leaf, N1 = ix->cfg.n_parent;
  Trace tr("install");
  // searches in flight keep the structure they were launched on
  if (ix->vec0) retire_structure(ix);
  free_structure(ix);
  QK_TRY(group_rows(X, ids, n, d, leaf_of_row, N0, true, ix->status, &ix->vec0, &ix->ids0, &ix->off0,
                    &ix->size0, ix->h_off0, ix->h_size0, &ix->h_cap_part0, &ix->cap0, &ix->used0, s,
                    skip_unlabelled));
  ix->holes0 = 0;
  ix->arena_id = next_arena_id();
  for (int i = 0; i < 2; ++i) {   // spare partition tables for the updates to come
    Table t;
    t.n = N0;
    QK_TRY(dalloc(&t.off, (size_t)N0));
    qk_status ts = dalloc(&t.size, (size_t)N0);
    if (ts != QK_OK) dfree(t.off);
    QK_TRY(ts);
    ix->spare0.push_back(t);
  }
  QK_TRY(dalloc(&ix->cent0, (size_t)N0 * d));
  QK_CUDA(cudaMemcpyAsync(ix->cent0, C0, sizeof(float) * (size_t)N0 * d, cudaMemcpyDeviceToDevice, s));
  if (ix->cfg.storage != QK_STORE_F32) {
    QK_TRY(dalloc(&ix->lp0, (size_t)ix->cap0 * d * elem_bytes(ix->cfg.storage)));
    QK_TRY(dalloc(&ix->lp_scale0, (size_t)N0));
    QK_TRY(launch_quantize_arena(ix->vec0, ix->off0, ix->size0, N0, d, ix->cfg.storage, ix->lp_scale0, ix->lp0, s));
  }
  QK_TRY(dalloc(&ix->hits0, (size_t)N0));
  QK_CUDA(cudaMemsetAsync(ix->hits0, 0, sizeof(unsigned long long) * N0, s));
  if (N1 > 0) {
    Tmp tl(s);
    int64_t* leaf_ids = nullptr;
    QK_TRY(tl.alloc<int64_t>(N0, &leaf_ids));
    std::vector<int64_t> seq(N0);
    for (int32_t j = 0; j < N0; ++j) seq[j] = j;
    QK_CUDA(cudaMemcpyAsync(leaf_ids, seq.data(), sizeof(int64_t) * N0, cudaMemcpyHostToDevice, s));
    int64_t cap1 = 0;
    QK_TRY(group_rows(C0, leaf_ids, N0, d, parent_of_leaf, N1, false, ix->status, &ix->vec1, &ix->ids1,
                      &ix->off1, &ix->size1, ix->h_off1, ix->h_size1, nullptr, &cap1, nullptr, s, false));
    QK_TRY(dalloc(&ix->cent1, (size_t)N1 * d));
    QK_CUDA(cudaMemcpyAsync(ix->cent1, C1, sizeof(float) * (size_t)N1 * d, cudaMemcpyDeviceToDevice, s));
    QK_TRY(dalloc(&ix->hits1, (size_t)N1));
    QK_CUDA(cudaMemsetAsync(ix->hits1, 0, sizeof(unsigned long long) * N1, s));
  }
  tr.mark("arena");
  // id map, built from the arena so that it records the real slots
  std::vector<int64_t>& h_ids = ix->h_ids0;
  h_ids.assign((size_t)ix->cap0, -1);
  QK_CUDA(cudaMemcpyAsync(h_ids.data(), ix->ids0, sizeof(int64_t) * ix->cap0, cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));
  ix->where.clear();
  ix->where.reserve((size_t)n * 2);
  for (int32_t j = 0; j < N0; ++j) {
    for (int32_t t = 0; t < ix->h_size0[j]; ++t) {
      int64_t id = h_ids[ix->h_off0[j] + t];
      if (!ix->where.emplace(id, ((int64_t)j << 32) | (uint32_t)t).second) {
        free_structure(ix);
        set_error("duplicate id " + std::to_string(id));
        return QK_ERR_DUP_ID;
      }
    }
  }
  tr.mark("id_map");
  preload_update_kernels();
  ++ix->version;
  ix->n = n;
  ix->n_leaf = N0;
  ix->n_parent = N1;
  ix->queries_seen = 0;
  ix->ready = true;
  return QK_OK;
}

// Seeded initial rows: partial Fisher-Yates driven by SplitMix64
// (Steele, Lea, Flood 2014).
static void splitmix_init_rows(int64_t n, int32_t K, uint64_t seed, std::vector<int64_t>& out) {
  std::vector<int64_t> perm((size_t)n);
  for (int64_t i = 0; i < n; ++i) perm[i] = i;
  uint64_t state = seed;
  for (int32_t i = 0; i < K; ++i) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    int64_t j = i + (int64_t)(z % (uint64_t)(n - i));
    std::swap(perm[i], perm[j]);
  }
  out.assign(perm.begin(), perm.begin() + K);
}

// Nearest centroid of every row (L2, ties to the lower index).  With 32 or
// more centroids the candidates come from the tensor-core scoring kernel and
// are re-scored exactly; otherwise the SIMT kernel compares every centroid.
qk_status assign_nearest(const float* X, int64_t n, int d, const float* C, int K, int32_t* assign, cudaStream_t s) {
  if (K < 32 || d % 32 != 0 || n <= 0) return launch_kmeans_assign(X, n, d, C, K, assign, nullptr, s);
  Tmp tn(s), tc_(s), ts(s);
  float* cnorm = nullptr;
  int32_t* cand = nullptr;
  int32_t* st = nullptr;
  QK_TRY(tn.alloc<float>((size_t)K, &cnorm));
  QK_TRY(tc_.alloc<int32_t>((size_t)n * tc_candidates_per_row(), &cand));
  QK_TRY(ts.alloc<int32_t>(1, &st));
  QK_CUDA(cudaMemsetAsync(st, 0, sizeof(int32_t), s));
  QK_TRY(launch_tc_nearest(X, n, d, C, K, QK_METRIC_L2, 1, assign, nullptr, cnorm, cand, st, s));
  int32_t hst = 0;
  QK_CUDA(cudaMemcpyAsync(&hst, st, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));
  if (hst != 0) {
    set_error("tensor-core scoring: a bounded wait expired");
    return QK_ERR_TIMEOUT;
  }
  return QK_OK;
}

// Lloyd k-means of n device rows into K centroids (device, K x d) and the
// final assignment (device, n).  Starts from the seeded rows, or from C_init
// (device, K x d) when it is given.
qk_status kmeans(const float* X, int64_t n, int d, int32_t K, int iters, uint64_t seed, float* C, int32_t* assign,
                 cudaStream_t s, const float* C_init) {
  Tmp t_rows(s), t_c2(s), t_sums(s), t_counts(s);
  int64_t* rows = nullptr;
  float* C2 = nullptr;
  double* sums = nullptr;
  int32_t* counts = nullptr;
  QK_TRY(t_c2.alloc<float>((size_t)K * d, &C2));
  QK_TRY(t_sums.alloc<double>((size_t)K * d, &sums));
  QK_TRY(t_counts.alloc<int32_t>(K, &counts));
  if (C_init) {
    QK_CUDA(cudaMemcpyAsync(C, C_init, sizeof(float) * (size_t)K * d, cudaMemcpyDeviceToDevice, s));
  } else {
    std::vector<int64_t> init;
    splitmix_init_rows(n, K, seed, init);
    QK_TRY(t_rows.alloc<int64_t>(K, &rows));
    QK_CUDA(cudaMemcpyAsync(rows, init.data(), sizeof(int64_t) * K, cudaMemcpyHostToDevice, s));
    QK_TRY(launch_gather_rows(X, d, rows, K, C, s));
  }
  for (int it = 0; it < iters; ++it) {
    QK_TRY(assign_nearest(X, n, d, C, K, assign, s));
    QK_TRY(launch_kmeans_update(X, n, d, assign, C, K, C2, sums, counts, s));
    QK_CUDA(cudaMemcpyAsync(C, C2, sizeof(float) * (size_t)K * d, cudaMemcpyDeviceToDevice, s));
  }
  QK_TRY(assign_nearest(X, n, d, C, K, assign, s));
  QK_CUDA(cudaStreamSynchronize(s));
  return QK_OK;
}

static qk_status check_ready(const qk_index* ix) {
  if (!ix) {
    set_error("null index");
    return QK_ERR_ARG;
  }
  if (!ix->ready) {
    set_error("index is empty: build or load it first");
    return QK_ERR_STATE;
  }
  return QK_OK;
}

// ---- copy-on-write updates of level 0 ----------------------------------
// An update never writes a row or a table entry that a published version can
// read.  It takes free arena rows (take_rows) for every partition whose rows
// change in place, copies the partition there, edits the copy, and publishes
// a fresh partition table; the rows and table the old version used are
// retired until the searches launched on it have completed.

// Lays the arena out again into new memory with every partition keeping its
// room, and a free tail of at least tail_min rows; publishes the result (same
// content, new layout) and retires the old arena.
static qk_status compact(qk_index* ix, int64_t tail_min, cudaStream_t s) {
  const int d = ix->cfg.d;
  const int32_t N0 = ix->n_leaf;
  const int rb = ix->lp0 ? d * elem_bytes(ix->cfg.storage) : 0;
  std::vector<int64_t> off(N0);
  int64_t reserved = 0;
  for (int32_t j = 0; j < N0; ++j) {
    off[j] = reserved;
    reserved += ix->h_cap_part0[j];
  }
  const int64_t total = reserved + std::max(tail_rows(reserved), tail_min);
  float* nvec = nullptr;
  int64_t* nids = nullptr;
  unsigned char* nlp = nullptr;
  Table t;
  qk_status st = dalloc(&nvec, (size_t)total * d);
  if (st == QK_OK) st = dalloc(&nids, (size_t)total);
  if (st == QK_OK && ix->lp0) st = dalloc(&nlp, (size_t)total * rb);
  if (st == QK_OK) st = take_table(ix, &t);
  if (st != QK_OK) {
    dfree(nvec);
    dfree(nids);
    dfree(nlp);
    return st;
  }
  QK_CUDA(cudaMemsetAsync(nids, 0xff, sizeof(int64_t) * (size_t)total, s));
  QK_CUDA(cudaMemcpyAsync(t.off, off.data(), sizeof(int64_t) * N0, cudaMemcpyHostToDevice, s));
  QK_CUDA(cudaMemcpyAsync(t.size, ix->size0, sizeof(int32_t) * N0, cudaMemcpyDeviceToDevice, s));
  QK_TRY(launch_relayout(ix->vec0, ix->ids0, ix->off0, t.off, ix->size0, N0, d, nvec, nids, s));
  if (ix->lp0) QK_TRY(launch_relayout_bytes(ix->lp0, ix->off0, t.off, ix->size0, N0, rb, nlp, s));
  QK_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> mirror((size_t)total, -1);
  for (int32_t j = 0; j < N0; ++j)
    for (int32_t r = 0; r < ix->h_size0[j]; ++r) mirror[off[j] + r] = ix->h_ids0[ix->h_off0[j] + r];
  std::unique_lock<std::shared_mutex> pub(ix->pub_mu);
  Retired old;
  old.version = ix->version;
  old.table = Table{ix->off0, ix->size0, N0};
  old.device = {ix->vec0, ix->ids0};
  if (ix->lp0) old.device.push_back(ix->lp0);
  ix->vec0 = nvec;
  ix->ids0 = nids;
  if (ix->lp0) ix->lp0 = nlp;
  ix->off0 = t.off;
  ix->size0 = t.size;
  ix->h_ids0.swap(mirror);
  ix->h_off0 = off;
  ix->cap0 = total;
  ix->used0 = reserved;
  ix->holes0 = 0;
  ix->free0.clear();
  ix->arena_id = next_arena_id();
  ++ix->version;
  pub.unlock();
  retire(ix, std::move(old));
  return QK_OK;
}

// Gives each partition moved[i] fresh rows of capacity room[i] and copies
// its current rows there.  The new offsets go to off (a working copy of
// h_off0) and the host id mirror; the old rows are added to `old`, to be
// retired when the new table is published.  Compacts first when the free
// ranges and the tail cannot hold them all.
static qk_status relocate(qk_index* ix, const std::vector<int32_t>& moved, const std::vector<int64_t>& room,
                          std::vector<int64_t>& off, std::vector<int64_t>& cap, Retired& old, cudaStream_t s) {
  const int32_t m = (int32_t)moved.size();
  if (m == 0) return QK_OK;
  const int d = ix->cfg.d;
  const int rb = ix->lp0 ? d * elem_bytes(ix->cfg.storage) : 0;
  std::vector<int64_t> dst(m, -1);
  {
    const auto free_saved = ix->free0;
    const int64_t used_saved = ix->used0, holes_saved = ix->holes0;
    bool fits = true;
    for (int32_t i = 0; i < m && fits; ++i) fits = (dst[i] = take_rows(ix, room[i])) >= 0;
    if (!fits) {
      ix->free0 = free_saved;
      ix->used0 = used_saved;
      ix->holes0 = holes_saved;
      int64_t want = 0;
      for (int32_t i = 0; i < m; ++i) want += room[i];
      QK_TRY(compact(ix, want, s));
      off = ix->h_off0;
      cap = ix->h_cap_part0;
      for (int32_t i = 0; i < m; ++i)
        if ((dst[i] = take_rows(ix, room[i])) < 0) {
          set_error("arena: no room after compaction");
          return QK_ERR_INTERNAL;
        }
    }
  }
  std::vector<int64_t> offs(2 * (size_t)m);   // old offsets, then new offsets
  std::vector<int32_t> sz(m);
  for (int32_t i = 0; i < m; ++i) {
    const int32_t j = moved[i];
    offs[i] = off[j];
    offs[m + i] = dst[i];
    sz[i] = ix->h_size0[j];
  }
  Tmp toffs(s), tsz(s);
  int64_t* doffs = nullptr;
  int32_t* dsz = nullptr;
  QK_TRY(toffs.alloc<int64_t>(offs.size(), &doffs));
  QK_TRY(tsz.alloc<int32_t>((size_t)m, &dsz));
  QK_CUDA(cudaMemcpyAsync(doffs, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice, s));
  QK_CUDA(cudaMemcpyAsync(dsz, sz.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
  // the destinations are free rows: no published version reads them
  QK_TRY(launch_relayout(ix->vec0, ix->ids0, doffs, doffs + m, dsz, m, d, ix->vec0, ix->ids0, s));
  if (ix->lp0) QK_TRY(launch_relayout_bytes(ix->lp0, doffs, doffs + m, dsz, m, rb, ix->lp0, s));
  // no wait here: the work that follows is on the same stream, and publish waits for it all
  old.arena = ix->arena_id;
  for (int32_t i = 0; i < m; ++i) {
    const int32_t j = moved[i];
    for (int32_t r = 0; r < sz[i]; ++r) {
      ix->h_ids0[offs[m + i] + r] = ix->h_ids0[offs[i] + r];
      ix->h_ids0[offs[i] + r] = -1;
    }
    old.rows.emplace_back(off[j], cap[j]);
    ix->holes0 += cap[j];
    off[j] = dst[i];
    cap[j] = room[i];
  }
  return QK_OK;
}

// Publishes the level-0 table (off, size) as the next version: uploads it
// into a spare table, waits for the update's own stream, exchanges the
// pointers and retires the previous table with `old`.
static qk_status publish(qk_index* ix, const std::vector<int64_t>& off, const std::vector<int64_t>& cap,
                         const std::vector<int32_t>& size, Retired&& old, int64_t dn, cudaStream_t s) {
  const int32_t N0 = ix->n_leaf;
  Table t;
  QK_TRY(take_table(ix, &t));
  cudaError_t e = cudaMemcpyAsync(t.off, off.data(), sizeof(int64_t) * N0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(t.size, size.data(), sizeof(int32_t) * N0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    ix->spare0.push_back(t);
    return cuda_status(e, "publishing a partition table");
  }
  std::unique_lock<std::shared_mutex> pub(ix->pub_mu);
  old.version = ix->version;
  old.arena = ix->arena_id;
  old.table = Table{ix->off0, ix->size0, N0};
  ix->off0 = t.off;
  ix->size0 = t.size;
  ix->h_off0 = off;
  ix->h_cap_part0 = cap;
  ix->h_size0 = size;
  ix->n += dn;
  ++ix->version;
  pub.unlock();
  retire(ix, std::move(old));
  return QK_OK;
}

template <class T>
static qk_status to_host(const T* src, size_t count, std::vector<T>& out, cudaStream_t s) {
  out.resize(count);
  if (count == 0) return QK_OK;
  if (is_device_ptr(src)) {
    QK_CUDA(cudaMemcpyAsync(out.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost, s));
    QK_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(out.data(), src, sizeof(T) * count);
  }
  return QK_OK;
}

// Synchronises `s`, then reads and clears the device status word and the
// diagnostic record of the index's kernels.
static qk_status read_device_status(qk_index* ix, cudaStream_t s) {
  int32_t st = 0;
  int64_t dg[kDiagWords] = {0};
  QK_CUDA(cudaStreamSynchronize(s));
  QK_CUDA(cudaMemcpy(&st, ix->status, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (std::getenv("QK_DEBUG_WAITS")) {
    int64_t w = 0;
    QK_CUDA(cudaMemcpy(&w, ix->diag + 8, sizeof(int64_t), cudaMemcpyDeviceToHost));
    std::fprintf(stderr, "qk: longest bulk-copy wait %lld cycles\n", (long long)w);
    QK_CUDA(cudaMemset(ix->diag + 8, 0, sizeof(int64_t)));
  }
  if (st == DEV_OK) return QK_OK;
  QK_CUDA(cudaMemcpy(dg, ix->diag, sizeof(dg), cudaMemcpyDeviceToHost));
  QK_CUDA(cudaMemset(ix->status, 0, sizeof(int32_t)));
  QK_CUDA(cudaMemset(ix->diag, 0, sizeof(dg)));
  std::string what = "device status " + std::to_string(st) + " (query " + std::to_string(dg[1]) + ", details " +
                     std::to_string(dg[2]) + " " + std::to_string(dg[3]) + " " + std::to_string(dg[4]) + " " +
                     std::to_string(dg[5]) + " " + std::to_string(dg[6]) + " " + std::to_string(dg[7]) + ")";
  if (st == DEV_TIMEOUT) {
    set_error("a bounded device wait expired: " + what);
    return QK_ERR_TIMEOUT;
  }
  if (st == DEV_BAD_ARG) {   // an argument only the device reads (a per-query nprobe, a buffer bound)
    set_error("invalid argument found on the device: " + what);
    return QK_ERR_ARG;
  }
  set_error("internal consistency check failed: " + what);
  return QK_ERR_INTERNAL;
}


int32_t n_candidates(double f, int32_t n) {
  double m = std::ceil(f * (double)n);
  if (m < 1) m = 1;
  if (m > n) m = n;
  return (int32_t)m;
}

void base_search_args(qk_index* ix, int32_t k, float recall_target, int32_t nprobe, SearchArgs& a) {
  a.d = ix->cfg.d;
  a.metric = ix->cfg.metric;
  a.L = ix->n_parent > 0 ? 2 : 1;
  a.lv[0] = DevLevel{ix->vec0, ix->ids0, ix->off0, ix->size0, ix->cent0, ix->n_leaf};
  a.lv[1] = DevLevel{ix->vec1, ix->ids1, ix->off1, ix->size1, ix->cent1, ix->n_parent};
  const bool fixed = !(recall_target > 0.f);
  a.fixed_nprobe = fixed ? nprobe : 0;
  if (a.L == 1) {
    a.root = ix->cent0;
    a.n_root = ix->n_leaf;
    a.M_root = fixed ? std::min(nprobe, ix->n_leaf) : n_candidates(ix->cfg.f_M_leaf, ix->n_leaf);
    a.k1 = 0;
  } else {
    a.root = ix->cent1;
    a.n_root = ix->n_parent;
    a.M_root = n_candidates(ix->cfg.f_M_parent, ix->n_parent);
    a.k1 = n_candidates(ix->cfg.f_M_leaf, ix->n_leaf);
  }
  const int storage = ix->cfg.storage;
  a.kq = k;
  a.k0 = storage == QK_STORE_F32 ? k : std::min(1024, k * std::max(1, ix->cfg.rerank));
  a.mode0 = storage == QK_STORE_BF16 ? 2 : storage == QK_STORE_FP8 ? 3 : (ix->cfg.metric == QK_METRIC_IP ? 1 : 0);
  a.lp_vec = ix->lp0;
  a.lp_scale = ix->lp_scale0;
  a.tau0 = recall_target;
  a.tau1 = ix->cfg.upper_recall;
  a.tau_rho = ix->cfg.tau_rho;
  a.beta_mode = ix->cfg.beta_mode;
  a.beta_table = ix->beta_table;
  a.beta_a = ix->beta_a;
  a.beta_lnB = ix->beta_lnB;
  a.hits0 = ix->hits0;
  a.hits1 = ix->hits1;
  // every launch takes its own work-stealing counter, so searches on different
  // streams may be in flight together (up to kWorkSlots of them)
  a.work = ix->work + (ix->search_seq++ % kWorkSlots);
  a.status = ix->status;
  a.diag = ix->diag;
  a.wait_stats = ix->diag + 8;
  a.kcap = std::max({a.k0, a.k1, a.M_root});
  a.mcap = std::max({a.M_root, a.k1, 1});
}
}  // namespace qk

using namespace qk;

extern "C" {

void qk_config_default(qk_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->d = 128;
  c->metric = QK_METRIC_L2;
  c->n_leaf = 1000;
  c->n_parent = 0;
  c->kmeans_iters = 10;
  c->beta_mode = QK_BETA_TABLE;
  c->seed = 1234;
  c->f_M_leaf = 0.1;
  c->f_M_parent = 0.25;
  c->tau_rho = 0.01;
  c->upper_recall = 0.99;
  c->storage = QK_STORE_F32;
  c->rerank = 4;
}

const char* qk_last_error(void) { return g_err.c_str(); }

// Freed stream-ordered temporaries stay in the device's default pool (up to
// 1 GiB) instead of going back to the driver at every synchronisation.
static void keep_pool_memory(int dev) {
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = 1ull << 30;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
}

qk_status qk_create(const qk_config* cfg, qk_index** out) {
  QK_GUARD_BEGIN
  if (!cfg || !out) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  *out = nullptr;
  if (!supported_dim(cfg->d)) {
    set_error("unsupported dimension " + std::to_string(cfg->d));
    return QK_ERR_ARG;
  }
  if (cfg->metric != QK_METRIC_L2 && cfg->metric != QK_METRIC_IP) {
    set_error("unknown metric");
    return QK_ERR_ARG;
  }
  if (cfg->n_leaf < 1 || cfg->n_parent < 0 || cfg->n_parent > cfg->n_leaf || cfg->kmeans_iters < 0 ||
      !(cfg->f_M_leaf > 0) || !(cfg->f_M_parent > 0) || !(cfg->tau_rho >= 0) ||
      (cfg->beta_mode != QK_BETA_TABLE && cfg->beta_mode != QK_BETA_EXACT) || cfg->storage < QK_STORE_F32 ||
      cfg->storage > QK_STORE_FP8 || cfg->rerank < 1) {
    set_error("invalid configuration");
    return QK_ERR_ARG;
  }
  qk_index* ix = new qk_index();
  ix->cfg = *cfg;
  cudaGetDevice(&ix->device);
  keep_pool_memory(ix->device);
  ix->beta_a = 0.5 * (cfg->d + 1);
  ix->beta_lnB = std::lgamma(ix->beta_a) + std::lgamma(0.5) - std::lgamma(ix->beta_a + 0.5);
  qk_status st = QK_OK;
  if ((st = dalloc(&ix->beta_table, kBetaTablePoints)) != QK_OK || (st = dalloc(&ix->work, kWorkSlots)) != QK_OK ||
      (st = dalloc(&ix->status, 1)) != QK_OK || (st = dalloc(&ix->diag, kDiagWords)) != QK_OK) {
    qk_destroy(ix);
    return st;
  }
  cudaMemset(ix->status, 0, sizeof(int32_t));
  cudaMemset(ix->diag, 0, sizeof(int64_t) * kDiagWords);
  st = launch_beta_table(ix->beta_a, ix->beta_lnB, ix->beta_table, 0);
  if (st == QK_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_status(e, "beta table");
  }
  if (st != QK_OK) {
    qk_destroy(ix);
    return st;
  }
  *out = ix;
  return QK_OK;
  QK_GUARD_END
}

void qk_destroy(qk_index* ix) {
  if (!ix) return;
  reclaim(ix, true);
  if (ix->pending) {
    free_structure(ix->pending);
    delete ix->pending;
    ix->pending = nullptr;
  }
  free_structure(ix);
  dfree(ix->beta_table);
  dfree(ix->work);
  dfree(ix->status);
  dfree(ix->diag);
  if (ix->stage_in.p) cudaFree(ix->stage_in.p);
  if (ix->stage_out.p) cudaFree(ix->stage_out.p);
  delete ix;
}

qk_status qk_build(qk_index* ix, const float* x, const int64_t* ids, int64_t n, void* stream) {
  QK_GUARD_BEGIN
  if (ix) ix->pub_mu.lock();   // the structure is replaced: no search captures it meanwhile
  struct Unlock {
    qk_index* ix;
    ~Unlock() {
      if (ix) ix->pub_mu.unlock();
    }
  } unlock_pub{ix};
  if (!ix || !x || !ids || n < 1) {
    set_error("null argument or empty input");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int d = ix->cfg.d;
  const int32_t N0 = ix->cfg.n_leaf, N1 = ix->cfg.n_parent;
  if (n < N0) {
    set_error("fewer vectors than leaf partitions");
    return QK_ERR_ARG;
  }
  Tmp tx(s), ti(s), tc0(s), ta0(s), tc1(s), ta1(s);
  const float* X = nullptr;
  const int64_t* I = nullptr;
  QK_TRY(in_device(x, (size_t)n * d, tx, &X, s));
  QK_TRY(in_device(ids, (size_t)n, ti, &I, s));
  float* C0 = nullptr;
  int32_t* a0 = nullptr;
  QK_TRY(tc0.alloc<float>((size_t)N0 * d, &C0));
  QK_TRY(ta0.alloc<int32_t>((size_t)n, &a0));
  QK_TRY(kmeans(X, n, d, N0, ix->cfg.kmeans_iters, ix->cfg.seed, C0, a0, s, nullptr));
  float* C1 = nullptr;
  int32_t* a1 = nullptr;
  if (N1 > 0) {
    QK_TRY(tc1.alloc<float>((size_t)N1 * d, &C1));
    QK_TRY(ta1.alloc<int32_t>((size_t)N0, &a1));
    QK_TRY(kmeans(C0, N0, d, N1, ix->cfg.kmeans_iters, ix->cfg.seed + 1, C1, a1, s, nullptr));
  }
  return install(ix, X, I, n, C0, a0, C1, a1, s, false);
  QK_GUARD_END
}

qk_status qk_load(qk_index* ix, const float* x, const int64_t* ids, int64_t n, const float* leaf_centroids,
                  const int32_t* leaf_of_row, const float* parent_centroids, const int32_t* parent_of_leaf,
                  void* stream) {
  QK_GUARD_BEGIN
  if (ix) ix->pub_mu.lock();   // the structure is replaced: no search captures it meanwhile
  struct Unlock {
    qk_index* ix;
    ~Unlock() {
      if (ix) ix->pub_mu.unlock();
    }
  } unlock_pub{ix};
  if (!ix || !x || !ids || n < 0 || !leaf_centroids || !leaf_of_row) {
    set_error("null argument");
    return QK_ERR_ARG;
  }
  const int d = ix->cfg.d;
  const int32_t N0 = ix->cfg.n_leaf, N1 = ix->cfg.n_parent;
  if (N1 > 0 && (!parent_centroids || !parent_of_leaf)) {
    set_error("two-level index needs parent centroids and parent_of_leaf");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Tmp tx(s), ti(s), tc0(s), ta0(s), tc1(s), ta1(s);
  const float *X = nullptr, *C0 = nullptr, *C1 = nullptr;
  const int64_t* I = nullptr;
  const int32_t *a0 = nullptr, *a1 = nullptr;
  QK_TRY(in_device(x, (size_t)n * d, tx, &X, s));
  QK_TRY(in_device(ids, (size_t)n, ti, &I, s));
  QK_TRY(in_device(leaf_centroids, (size_t)N0 * d, tc0, &C0, s));
  QK_TRY(in_device(leaf_of_row, (size_t)n, ta0, &a0, s));
  if (N1 > 0) {
    QK_TRY(in_device(parent_centroids, (size_t)N1 * d, tc1, &C1, s));
    QK_TRY(in_device(parent_of_leaf, (size_t)N0, ta1, &a1, s));
  }
  return install(ix, X, I, n, C0, a0, C1, a1, s, false);
  QK_GUARD_END
}


// The search of qk_search; nprobe_q (device, optional) gives fixed-nprobe
// mode one nprobe per query, nprobe then being their maximum.
static qk_status search_impl(qk_index* ix, const float* q, int64_t nq, int32_t k, float recall_target, int32_t nprobe,
                             const int32_t* nprobe_q, int64_t* out_ids, float* out_dist, int32_t* out_nprobe,
                             float* out_recall, void* stream, int32_t* scan0 = nullptr, int32_t cap0 = 0,
                             int32_t* scan1 = nullptr, int32_t cap1 = 0, float ratio_eps = 0.f) {
  if (!ix) return check_ready(ix);
  // the published structure stays put while the launch captures it
  std::shared_lock<std::shared_mutex> pub(ix->pub_mu);
  QK_TRY(check_ready(ix));
  if (nq < 0 || k < 1 || k > 1024 || (nq > 0 && (!q || !out_ids || !out_dist))) {
    set_error("invalid search arguments");
    return QK_ERR_ARG;
  }
  if ((scan0 && cap0 < 1) || (scan1 && cap1 < 1)) {
    set_error("a scanned-partition record needs a capacity >= 1");
    return QK_ERR_ARG;
  }
  if (!scan0) cap0 = 0;
  if (!scan1) cap1 = 0;
  if (!(recall_target > 0.f) && nprobe < 1) {
    set_error("fixed-nprobe search needs nprobe >= 1");
    return QK_ERR_ARG;
  }
  if (nq == 0) return QK_OK;
  Trace tr("search");
  cudaStream_t s = (cudaStream_t)stream;
  const int d = ix->cfg.d;
  const bool q_dev = is_device_ptr(q);
  const bool ids_dev = is_device_ptr(out_ids), dist_dev = is_device_ptr(out_dist);
  const bool np_dev = !out_nprobe || is_device_ptr(out_nprobe);
  const bool rc_dev = !out_recall || is_device_ptr(out_recall);
  const bool s0_dev = !scan0 || is_device_ptr(scan0);
  const bool s1_dev = !scan1 || is_device_ptr(scan1);
  const bool all_dev = q_dev && ids_dev && dist_dev && np_dev && rc_dev && s0_dev && s1_dev;
  // staging for host buffers
  const size_t bq = sizeof(float) * (size_t)nq * d;
  const size_t bi = sizeof(int64_t) * (size_t)nq * k, bd = sizeof(float) * (size_t)nq * k;
  const size_t bn = sizeof(int32_t) * (size_t)nq, br = sizeof(float) * (size_t)nq;
  const size_t bs0 = sizeof(int32_t) * (size_t)nq * cap0, bs1 = sizeof(int32_t) * (size_t)nq * cap1;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  if (!all_dev) {
    QK_TRY(ensure(ix->stage_in, al(bq)));
    QK_TRY(ensure(ix->stage_out, al(bi) + al(bd) + al(bn) + al(br) + al(bs0) + al(bs1)));
  }
  unsigned char* so = static_cast<unsigned char*>(ix->stage_out.p);
  const float* dq = q;
  if (!q_dev) {
    QK_CUDA(cudaMemcpyAsync(ix->stage_in.p, q, bq, cudaMemcpyHostToDevice, s));
    dq = static_cast<const float*>(ix->stage_in.p);
  }
  int64_t* dids = ids_dev ? out_ids : reinterpret_cast<int64_t*>(so);
  float* ddist = dist_dev ? out_dist : reinterpret_cast<float*>(so + al(bi));
  int32_t* dnp = np_dev ? out_nprobe : reinterpret_cast<int32_t*>(so + al(bi) + al(bd));
  float* drc = rc_dev ? out_recall : reinterpret_cast<float*>(so + al(bi) + al(bd) + al(bn));
  const size_t o_s0 = al(bi) + al(bd) + al(bn) + al(br);
  int32_t* ds0 = s0_dev ? scan0 : reinterpret_cast<int32_t*>(so + o_s0);
  int32_t* ds1 = s1_dev ? scan1 : reinterpret_cast<int32_t*>(so + o_s0 + al(bs0));

  SearchArgs a;
  base_search_args(ix, k, recall_target, nprobe, a);
  a.Q = dq;
  a.nq = nq;
  a.nprobe_q = a.fixed_nprobe > 0 ? nprobe_q : nullptr;
  if (ratio_eps > 0.f) {   // SPANN's rule within the candidate set APS uses
    a.ratio_eps = ratio_eps;
    if (a.L == 1) a.M_root = n_candidates(ix->cfg.f_M_leaf, ix->n_leaf);
    a.kcap = std::max({a.k0, a.k1, a.M_root});
    a.mcap = std::max({a.M_root, a.k1, 1});
  }
  a.out_ids = dids;
  a.out_dist = ddist;
  a.out_nprobe = out_nprobe ? dnp : nullptr;
  a.out_recall = out_recall ? drc : nullptr;
  a.scan0 = scan0 ? ds0 : nullptr;
  a.scan_cap0 = cap0;
  a.scan1 = scan1 ? ds1 : nullptr;
  a.scan_cap1 = cap1;
  // Where rows are short (d <= 256: a warp sums 4 rows per step) the upper
  // levels go to the warp-per-query prepare kernel first: it walks them
  // bitwise as the query's CTA would, without the CTA's barriers, and the
  // search kernel imports its candidates and t_i (1M x 128, 1,000 leaves:
  // 466k -> 494k queries/s).  For longer rows a warp sums one row per step
  // and the CTA's 8 warps walk faster (d = 768: 265k against 139k).
  // The exported candidates take 12 bytes per (query, candidate): batches
  // whose export would pass 1 GiB keep the CTA walk.
  void* xs = nullptr;
  const size_t xs_bytes = (size_t)nq * ((size_t)prepare_mcap(a) * 12 + 4);
  if (a.L == 2 && !a.scan1 && !(a.ratio_eps > 0.f) && xs_bytes <= (size_t(1) << 30) &&
      (ix->upper_mode == 1 || (ix->upper_mode < 0 && ix->cfg.d <= 256))) {
    SearchArgs pa = a;
    pa.xs_mcap = prepare_mcap(a);
    const size_t n = (size_t)nq * (size_t)pa.xs_mcap;
    const size_t b_t = sizeof(double) * n, b_c = sizeof(int32_t) * n, b_m = sizeof(int32_t) * (size_t)nq;
    QK_CUDA(cudaMallocAsync(&xs, b_t + b_c + b_m, s));
    pa.xs_t = static_cast<double*>(xs);
    pa.xs_cand = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(xs) + b_t);
    pa.xs_M = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(xs) + b_t + b_c);
    const qk_status ps = prepare_upper(pa, s);
    if (ps == QK_OK) {
      a.im_M = pa.xs_M;
      a.im_cand = pa.xs_cand;
      a.im_t = pa.xs_t;
      a.im_mcap = pa.xs_mcap;
    } else if (ps != QK_ERR_UNSUPPORTED) {
      cudaFreeAsync(xs, s);
      return ps;
    }
  }
  const qk_status ls = launch_search(a, s);
  if (xs) QK_CUDA(cudaFreeAsync(xs, s));
  QK_TRY(ls);
  note_readers(ix, s);
  pub.unlock();
  tr.mark("launch");
  ix->queries_seen += nq;
  if (!all_dev) {
    if (!ids_dev) QK_CUDA(cudaMemcpyAsync(out_ids, dids, bi, cudaMemcpyDeviceToHost, s));
    if (!dist_dev) QK_CUDA(cudaMemcpyAsync(out_dist, ddist, bd, cudaMemcpyDeviceToHost, s));
    if (!np_dev) QK_CUDA(cudaMemcpyAsync(out_nprobe, dnp, bn, cudaMemcpyDeviceToHost, s));
    if (!rc_dev) QK_CUDA(cudaMemcpyAsync(out_recall, drc, br, cudaMemcpyDeviceToHost, s));
    if (!s0_dev) QK_CUDA(cudaMemcpyAsync(scan0, ds0, bs0, cudaMemcpyDeviceToHost, s));
    if (!s1_dev) QK_CUDA(cudaMemcpyAsync(scan1, ds1, bs1, cudaMemcpyDeviceToHost, s));
    const qk_status st = read_device_status(ix, s);
    tr.mark("results");
    return st;
  }
  return QK_OK;
}

qk_status qk_set_search_upper(qk_index* ix, int32_t mode) {
  QK_GUARD_BEGIN
  if (!ix || mode < -1 || mode > 1) {
    set_error("upper-level mode is -1 (auto), 0 (in the query's CTA) or 1 (prepare kernel)");
    return QK_ERR_ARG;
  }
  ix->upper_mode = mode;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_search(qk_index* ix, const float* q, int64_t nq, int32_t k, float recall_target, int32_t nprobe,
                    int64_t* out_ids, float* out_dist, int32_t* out_nprobe, float* out_recall, void* stream) {
  QK_GUARD_BEGIN
  return search_impl(ix, q, nq, k, recall_target, nprobe, nullptr, out_ids, out_dist, out_nprobe, out_recall, stream);
  QK_GUARD_END
}

qk_status qk_search_scanned(qk_index* ix, const float* q, int64_t nq, int32_t k, float recall_target, int32_t nprobe,
                            int64_t* out_ids, float* out_dist, int32_t* out_nprobe, float* out_recall,
                            int32_t* out_scanned0, int32_t cap0, int32_t* out_scanned1, int32_t cap1, void* stream) {
  QK_GUARD_BEGIN
  return search_impl(ix, q, nq, k, recall_target, nprobe, nullptr, out_ids, out_dist, out_nprobe, out_recall, stream,
                     out_scanned0, cap0, out_scanned1, cap1);
  QK_GUARD_END
}

qk_status qk_search_ratio(qk_index* ix, const float* q, int64_t nq, int32_t k, float eps, int64_t* out_ids,
                          float* out_dist, int32_t* out_nprobe, int32_t* out_scanned0, int32_t cap0, void* stream) {
  QK_GUARD_BEGIN
  if (!(eps > 0.f) || !(eps < INFINITY)) {
    set_error("the ratio rule needs a finite eps > 0");
    return QK_ERR_ARG;
  }
  return search_impl(ix, q, nq, k, 0.0f, 1, nullptr, out_ids, out_dist, out_nprobe, nullptr, stream, out_scanned0,
                     cap0, nullptr, 0, eps);
  QK_GUARD_END
}

qk_status qk_search_nprobe(qk_index* ix, const float* q, int64_t nq, int32_t k, const int32_t* nprobe,
                           int64_t* out_ids, float* out_dist, void* stream) {
  QK_GUARD_BEGIN
  QK_TRY(check_ready(ix));
  if (nq < 0 || (nq > 0 && !nprobe)) {
    set_error("invalid search arguments");
    return QK_ERR_ARG;
  }
  if (nq == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> h;
  QK_TRY(to_host(nprobe, (size_t)nq, h, s));
  int32_t mx = 0;
  for (int32_t v : h) {
    if (v < 1) {
      set_error("every nprobe must be >= 1");
      return QK_ERR_ARG;
    }
    mx = std::max(mx, v);
  }
  Tmp tn(s);
  const int32_t* dn = nullptr;
  QK_TRY(in_device(nprobe, (size_t)nq, tn, &dn, s));
  return search_impl(ix, q, nq, k, 0.0f, std::min(mx, ix->n_leaf), dn, out_ids, out_dist, nullptr, nullptr, stream);
  QK_GUARD_END
}

qk_status qk_insert(qk_index* ix, const float* x, const int64_t* ids, int64_t n, void* stream) {
  QK_GUARD_BEGIN
  QK_TRY(check_ready(ix));
  if (n < 0 || (n > 0 && (!x || !ids))) {
    set_error("invalid insert arguments");
    return QK_ERR_ARG;
  }
  if (n == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int d = ix->cfg.d;
  Trace tr("insert");
  reclaim(ix, false);
  std::vector<int64_t> hid;
  QK_TRY(to_host(ids, (size_t)n, hid, s));
  {
    std::unordered_map<int64_t, int> seen;
    seen.reserve((size_t)n * 2);
    for (int64_t r = 0; r < n; ++r) {
      if (ix->where.count(hid[r]) || !seen.emplace(hid[r], 1).second) {
        set_error("insert: id " + std::to_string(hid[r]) + " is already present; nothing was inserted");
        return QK_ERR_DUP_ID;
      }
    }
  }
  Tmp tx(s), ti(s), tflag(s), tleaf(s), tpar(s), tdst(s);
  const float* X = nullptr;
  const int64_t* I = nullptr;
  QK_TRY(in_device(x, (size_t)n * d, tx, &X, s));
  QK_TRY(in_device(ids, (size_t)n, ti, &I, s));
  int32_t* flag = nullptr;
  QK_TRY(tflag.alloc<int32_t>(1, &flag));
  QK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
  QK_TRY(launch_nan_check(X, n * d, flag, s));
  // greedy descent (Sec. 3): nearest centroid at each level, ties to the lower
  // index; a row with NaN gets no leaf, and the flag refuses the whole batch
  int32_t* leaf = nullptr;
  QK_TRY(tleaf.alloc<int32_t>((size_t)n, &leaf));
  if (ix->n_parent == 0) {
    QK_TRY(assign_nearest(X, n, d, ix->cent0, ix->n_leaf, leaf, s));
  } else {
    int32_t* par = nullptr;
    QK_TRY(tpar.alloc<int32_t>((size_t)n, &par));
    QK_TRY(assign_nearest(X, n, d, ix->cent1, ix->n_parent, par, s));
    QK_TRY(launch_descend_children(X, n, d, par, ix->vec1, ix->ids1, ix->off1, ix->size1, ix->n_parent, leaf, s));
  }
  std::vector<int32_t> hleaf((size_t)n);
  int32_t hflag = 0;
  QK_CUDA(cudaMemcpyAsync(hleaf.data(), leaf, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));
  if (hflag) {
    set_error("insert: NaN in vectors; nothing was inserted");
    return QK_ERR_ARG;
  }
  tr.mark("checks_descent");
  std::vector<int32_t> need(ix->h_size0);
  for (int64_t r = 0; r < n; ++r) {
    int32_t j = hleaf[r];
    if (j < 0 || j >= ix->n_leaf) {
      set_error("insert: descent reached an empty parent partition");
      return QK_ERR_STATE;
    }
    ++need[j];
  }
  // appends go to rows behind every partition's live rows, which no version
  // reads; a partition whose room runs out moves to fresh rows first
  std::vector<int64_t> off(ix->h_off0), cap(ix->h_cap_part0);
  std::vector<int32_t> moved;
  std::vector<int64_t> room;
  for (int32_t j = 0; j < ix->n_leaf; ++j)
    if (need[j] > cap[j]) {
      moved.push_back(j);
      room.push_back(capacity_for(need[j]));
    }
  Retired old;
  QK_TRY(relocate(ix, moved, room, off, cap, old, s));
  tr.mark("grow");
  std::vector<int64_t> dst((size_t)n);
  std::vector<int32_t> cur(ix->h_size0);
  for (int64_t r = 0; r < n; ++r) {
    int32_t j = hleaf[r];
    int32_t slot = cur[j]++;
    dst[r] = off[j] + slot;
  }
  int64_t* ddst = nullptr;
  QK_TRY(tdst.alloc<int64_t>((size_t)n, &ddst));
  QK_CUDA(cudaMemcpyAsync(ddst, dst.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
  QK_TRY(launch_place_rows(X, I, n, d, ddst, ix->vec0, ix->ids0, s));
  if (ix->lp0)   // FP8 rows use their partition's current scale (values beyond it saturate)
    QK_TRY(launch_quantize_rows(X, n, d, ddst, leaf, ix->cfg.storage, ix->lp_scale0, ix->lp0, s));
  QK_TRY(publish(ix, off, cap, cur, std::move(old), n, s));
  for (int64_t r = 0; r < n; ++r) {
    int32_t j = hleaf[r];
    int64_t slot = dst[r] - off[j];
    ix->where[hid[r]] = ((int64_t)j << 32) | (uint32_t)slot;
    ix->h_ids0[dst[r]] = hid[r];
  }
  tr.mark("place");
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_delete(qk_index* ix, const int64_t* ids, int64_t n, int64_t* n_removed, void* stream) {
  QK_GUARD_BEGIN
  QK_TRY(check_ready(ix));
  if (n < 0 || (n > 0 && !ids)) {
    set_error("invalid delete arguments");
    return QK_ERR_ARG;
  }
  if (n_removed) *n_removed = 0;
  if (n == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const int d = ix->cfg.d;
  Trace tr("delete");
  reclaim(ix, false);
  std::vector<int64_t> hid;
  QK_TRY(to_host(ids, (size_t)n, hid, s));
  // Every partition that loses a row is first copied to fresh rows (the rows
  // a search in flight may read stay as they are); the deletes are then
  // replayed in order on the copy, each moving the partition's last row
  // into the freed slot.
  std::vector<int32_t> moved;
  std::vector<int64_t> room;
  {
    std::vector<char> hit(ix->n_leaf, 0);
    for (int64_t r = 0; r < n; ++r) {
      auto it = ix->where.find(hid[r]);
      if (it == ix->where.end()) continue;
      const int32_t j = (int32_t)(it->second >> 32);
      if (!hit[j]) {
        hit[j] = 1;
        moved.push_back(j);
        room.push_back(ix->h_cap_part0[j]);
      }
    }
  }
  if (moved.empty()) return QK_OK;
  std::vector<int64_t> off(ix->h_off0), cap(ix->h_cap_part0);
  Retired old;
  QK_TRY(relocate(ix, moved, room, off, cap, old, s));
  tr.mark("copy");
  // for every slot that changed, the slot its final content came from
  std::unordered_map<int32_t, std::unordered_map<int32_t, int32_t>> src_of;
  std::vector<int32_t> size(ix->h_size0);
  int64_t removed = 0;
  for (int64_t r = 0; r < n; ++r) {
    auto it = ix->where.find(hid[r]);
    if (it == ix->where.end()) continue;
    int32_t j = (int32_t)(it->second >> 32), slot = (int32_t)(it->second & 0xffffffff);
    int32_t last = size[j] - 1;
    auto& m = src_of[j];
    if (slot != last) {
      auto lt = m.find(last);
      m[slot] = lt == m.end() ? last : lt->second;
      int64_t mv = ix->h_ids0[off[j] + last];
      ix->h_ids0[off[j] + slot] = mv;
      ix->where[mv] = ((int64_t)j << 32) | (uint32_t)slot;
    }
    m.erase(last);
    ix->h_ids0[off[j] + last] = -1;
    ix->where.erase(it);
    size[j] = last;
    ++removed;
  }
  std::vector<int64_t> src, dst;
  for (auto& kv : src_of)
    for (auto& mv : kv.second)
      if (mv.first < size[kv.first] && mv.first != mv.second) {
        src.push_back(off[kv.first] + mv.second);
        dst.push_back(off[kv.first] + mv.first);
      }
  tr.mark("replay");
  const int64_t m = (int64_t)src.size();
  if (m > 0) {
    Tmp tsrc(s), tdst(s), tvec(s), tids(s);
    int64_t *dsrc = nullptr, *ddst = nullptr, *dtid = nullptr;
    float* dtv = nullptr;
    QK_TRY(tsrc.alloc<int64_t>((size_t)m, &dsrc));
    QK_TRY(tdst.alloc<int64_t>((size_t)m, &ddst));
    QK_TRY(tvec.alloc<float>((size_t)m * d, &dtv));
    QK_TRY(tids.alloc<int64_t>((size_t)m, &dtid));
    QK_CUDA(cudaMemcpyAsync(dsrc, src.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    QK_CUDA(cudaMemcpyAsync(ddst, dst.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    QK_TRY(launch_gather_moves(ix->vec0, ix->ids0, dsrc, m, d, dtv, dtid, s));
    QK_TRY(launch_place_rows(dtv, dtid, m, d, ddst, ix->vec0, ix->ids0, s));
    if (ix->lp0) {   // the temporary FP32 rows are free again once place_rows ran (same stream)
      QK_TRY(launch_move_bytes(ix->lp0, dsrc, ddst, m, d * elem_bytes(ix->cfg.storage),
                               reinterpret_cast<unsigned char*>(dtv), s));
    }
  }
  QK_TRY(publish(ix, off, cap, size, std::move(old), -removed, s));
  tr.mark("moves");
  if (n_removed) *n_removed = removed;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_check(qk_index* ix, void* stream) {
  QK_GUARD_BEGIN
  if (!ix) {
    set_error("null index");
    return QK_ERR_ARG;
  }
  return read_device_status(ix, (cudaStream_t)stream);
  QK_GUARD_END
}

qk_status qk_info(const qk_index* ix, int64_t* n_vectors, int32_t* n_leaf, int32_t* n_parent, int32_t* d) {
  QK_GUARD_BEGIN
  std::shared_lock<std::shared_mutex> pub;
  if (ix) pub = std::shared_lock<std::shared_mutex>(ix->pub_mu);
  if (!ix) {
    set_error("null index");
    return QK_ERR_ARG;
  }
  if (n_vectors) *n_vectors = ix->n;
  if (n_leaf) *n_leaf = ix->ready ? ix->n_leaf : ix->cfg.n_leaf;
  if (n_parent) *n_parent = ix->ready ? ix->n_parent : ix->cfg.n_parent;
  if (d) *d = ix->cfg.d;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_stats(const qk_index* ix, qk_index_stats* out) {
  QK_GUARD_BEGIN
  std::shared_lock<std::shared_mutex> pub;
  if (ix) pub = std::shared_lock<std::shared_mutex>(ix->pub_mu);
  QK_TRY(check_ready(ix));
  if (!out) {
    set_error("null output");
    return QK_ERR_ARG;
  }
  qk_index_stats st{};
  st.n_vectors = ix->n;
  st.levels = ix->n_parent > 0 ? 2 : 1;
  st.n_partitions[0] = ix->n_leaf;
  st.n_partitions[1] = ix->n_parent;
  st.d = ix->cfg.d;
  st.metric = ix->cfg.metric;
  st.storage = ix->cfg.storage;
  if (!ix->h_size0.empty()) {
    st.min_size = *std::min_element(ix->h_size0.begin(), ix->h_size0.end());
    st.max_size = *std::max_element(ix->h_size0.begin(), ix->h_size0.end());
  }
  st.mean_size = ix->n_leaf > 0 ? (double)ix->n / ix->n_leaf : 0.0;
  st.arena_rows = ix->cap0;
  st.arena_used = ix->used0;
  st.arena_holes = ix->holes0;
  st.arena_free = ix->cap0 - ix->used0;
  const int64_t lp = ix->cfg.storage == QK_STORE_BF16 ? 2 : ix->cfg.storage == QK_STORE_FP8 ? 1 : 0;
  st.arena_bytes = ix->cap0 * ((int64_t)ix->cfg.d * (4 + lp) + 8);
  for (int l = 0; l < 2; ++l) {
    const unsigned long long* src = l == 0 ? ix->hits0 : ix->hits1;
    const int32_t n = l == 0 ? ix->n_leaf : ix->n_parent;
    if (!src || n <= 0) continue;
    std::vector<unsigned long long> h((size_t)n);
    QK_CUDA(cudaMemcpy(h.data(), src, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost));
    for (unsigned long long v : h) st.hits[l] += (int64_t)v;
  }
  st.queries_seen = ix->queries_seen.load();
  st.version = ix->version;
  st.searches_in_flight = readers_in_flight(const_cast<qk_index*>(ix));
  st.retired_rows = retired_rows(const_cast<qk_index*>(ix));
  *out = st;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_export_level(const qk_index* ix, int32_t level, int32_t* sizes, float* centroids, int64_t* ids,
                          float* vectors) {
  QK_GUARD_BEGIN
  std::shared_lock<std::shared_mutex> pub;
  if (ix) pub = std::shared_lock<std::shared_mutex>(ix->pub_mu);
  QK_TRY(check_ready(ix));
  const int d = ix->cfg.d;
  if (level == 0) {
    if (sizes) std::copy(ix->h_size0.begin(), ix->h_size0.end(), sizes);
    if (centroids)
      QK_CUDA(cudaMemcpy(centroids, ix->cent0, sizeof(float) * (size_t)ix->n_leaf * d, cudaMemcpyDeviceToHost));
    if (ids) {
      std::vector<int64_t> h((size_t)ix->cap0);
      QK_CUDA(cudaMemcpy(h.data(), ix->ids0, sizeof(int64_t) * ix->cap0, cudaMemcpyDeviceToHost));
      int64_t o = 0;
      for (int32_t j = 0; j < ix->n_leaf; ++j)
        for (int32_t t = 0; t < ix->h_size0[j]; ++t) ids[o++] = h[ix->h_off0[j] + t];
    }
    if (vectors) {
      int64_t o = 0;
      for (int32_t j = 0; j < ix->n_leaf; ++j) {
        size_t rows = (size_t)ix->h_size0[j];
        if (rows)
          QK_CUDA(cudaMemcpy(vectors + o * d, ix->vec0 + ix->h_off0[j] * d, sizeof(float) * rows * d,
                             cudaMemcpyDeviceToHost));
        o += rows;
      }
    }
    return QK_OK;
  }
  if (level == 1 && ix->n_parent > 0) {
    if (sizes) std::copy(ix->h_size1.begin(), ix->h_size1.end(), sizes);
    if (centroids)
      QK_CUDA(cudaMemcpy(centroids, ix->cent1, sizeof(float) * (size_t)ix->n_parent * d, cudaMemcpyDeviceToHost));
    if (ids) {
      std::vector<int64_t> h((size_t)ix->n_leaf);
      QK_CUDA(cudaMemcpy(h.data(), ix->ids1, sizeof(int64_t) * ix->n_leaf, cudaMemcpyDeviceToHost));
      int64_t o = 0;
      for (int32_t j = 0; j < ix->n_parent; ++j)
        for (int32_t t = 0; t < ix->h_size1[j]; ++t) ids[o++] = h[ix->h_off1[j] + t];
    }
    return QK_OK;
  }
  set_error("no such level");
  return QK_ERR_ARG;
  QK_GUARD_END
}

qk_status qk_export_quantized(const qk_index* ix, uint8_t* codes, float* scales) {
  QK_GUARD_BEGIN
  std::shared_lock<std::shared_mutex> pub;
  if (ix) pub = std::shared_lock<std::shared_mutex>(ix->pub_mu);
  QK_TRY(check_ready(ix));
  if (!ix->lp0) {
    set_error("the index stores FP32 only");
    return QK_ERR_STATE;
  }
  const size_t rb = (size_t)ix->cfg.d * elem_bytes(ix->cfg.storage);
  if (scales) QK_CUDA(cudaMemcpy(scales, ix->lp_scale0, sizeof(float) * ix->n_leaf, cudaMemcpyDeviceToHost));
  if (codes) {
    int64_t o = 0;
    for (int32_t j = 0; j < ix->n_leaf; ++j) {
      size_t rows = (size_t)ix->h_size0[j];
      if (rows) QK_CUDA(cudaMemcpy(codes + o * rb, ix->lp0 + ix->h_off0[j] * rb, rows * rb, cudaMemcpyDeviceToHost));
      o += (int64_t)rows;
    }
  }
  if (scales && ix->cfg.storage == QK_STORE_BF16)
    for (int32_t j = 0; j < ix->n_leaf; ++j) scales[j] = 1.0f;
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_get_hits(qk_index* ix, int32_t level, int64_t* hits, int32_t reset) {
  QK_GUARD_BEGIN
  std::shared_lock<std::shared_mutex> pub;
  if (ix) pub = std::shared_lock<std::shared_mutex>(ix->pub_mu);
  QK_TRY(check_ready(ix));
  unsigned long long* src = level == 0 ? ix->hits0 : (level == 1 ? ix->hits1 : nullptr);
  int32_t n = level == 0 ? ix->n_leaf : ix->n_parent;
  if (!src || n <= 0) {
    set_error("no such level");
    return QK_ERR_ARG;
  }
  if (hits) QK_CUDA(cudaMemcpy(hits, src, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
  if (reset) QK_CUDA(cudaMemset(src, 0, sizeof(unsigned long long) * n));
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_cap_fraction(int32_t d, int32_t mode, const double* t, const double* rho, int64_t n, double* out_u,
                          void* stream) {
  QK_GUARD_BEGIN
  if (d < 1 || n < 0 || (n > 0 && (!t || !rho || !out_u)) || (mode != QK_BETA_EXACT && mode != QK_BETA_TABLE)) {
    set_error("invalid arguments");
    return QK_ERR_ARG;
  }
  if (n == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  double a = 0.5 * (d + 1);
  double lnB = std::lgamma(a) + std::lgamma(0.5) - std::lgamma(a + 0.5);
  Tmp tt(s), tr(s), tb(s), to(s);
  const double *dt = nullptr, *dr = nullptr;
  QK_TRY(in_device(t, (size_t)n, tt, &dt, s));
  QK_TRY(in_device(rho, (size_t)n, tr, &dr, s));
  double* table = nullptr;
  QK_TRY(tb.alloc<double>(kBetaTablePoints, &table));
  QK_TRY(launch_beta_table(a, lnB, table, s));
  bool out_dev = is_device_ptr(out_u);
  double* dout = out_u;
  if (!out_dev) QK_TRY(to.alloc<double>((size_t)n, &dout));
  QK_TRY(launch_cap_fraction(mode, a, lnB, table, dt, dr, n, dout, s));
  if (!out_dev) QK_CUDA(cudaMemcpyAsync(out_u, dout, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_nearest_centroids(const float* x, int64_t n, int32_t d, const float* c, int32_t K, int32_t metric,
                               int32_t k, int32_t* out_idx, float* out_dist, void* stream) {
  QK_GUARD_BEGIN
  if (!x || !c || !out_idx || n < 0 || K < 1 || d < 32 || d % 32 != 0 || k < 1 || k > 8 || k > K ||
      (metric != QK_METRIC_L2 && metric != QK_METRIC_IP)) {
    set_error("qk_nearest_centroids: invalid arguments (d a multiple of 32, 1 <= k <= min(8, K))");
    return QK_ERR_ARG;
  }
  if (n == 0) return QK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    keep_pool_memory(dev);   // the scratch of repeated calls stays in the pool
  }
  Tmp tx(s), tcen(s), ti(s), td(s), tn(s), tcand(s), ts(s);
  const float *X = nullptr, *C = nullptr;
  QK_TRY(in_device(x, (size_t)n * d, tx, &X, s));
  QK_TRY(in_device(c, (size_t)K * d, tcen, &C, s));
  const bool idx_dev = is_device_ptr(out_idx), dist_dev = !out_dist || is_device_ptr(out_dist);
  int32_t* di = out_idx;
  float* dd = out_dist;
  if (!idx_dev) QK_TRY(ti.alloc<int32_t>((size_t)n * k, &di));
  if (!dist_dev) QK_TRY(td.alloc<float>((size_t)n * k, &dd));
  float* cnorm = nullptr;
  int32_t* cand = nullptr;
  int32_t* st = nullptr;
  QK_TRY(tn.alloc<float>((size_t)K, &cnorm));
  QK_TRY(tcand.alloc<int32_t>((size_t)n * tc_candidates_per_row(), &cand));
  QK_TRY(ts.alloc<int32_t>(1, &st));
  QK_CUDA(cudaMemsetAsync(st, 0, sizeof(int32_t), s));
  QK_TRY(launch_tc_nearest(X, n, d, C, K, metric, k, di, dd, cnorm, cand, st, s));
  if (!idx_dev) QK_CUDA(cudaMemcpyAsync(out_idx, di, sizeof(int32_t) * n * k, cudaMemcpyDeviceToHost, s));
  if (!dist_dev) QK_CUDA(cudaMemcpyAsync(out_dist, dd, sizeof(float) * n * k, cudaMemcpyDeviceToHost, s));
  int32_t hst = 0;
  QK_CUDA(cudaMemcpyAsync(&hst, st, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  QK_CUDA(cudaStreamSynchronize(s));
  if (hst != 0) {
    set_error("tensor-core scoring: a bounded wait expired");
    return QK_ERR_TIMEOUT;
  }
  return QK_OK;
  QK_GUARD_END
}

qk_status qk_kmeans_step(const float* x, int64_t n, int32_t d, const float* c, int32_t K, float* c_new,
                         int32_t* assign, int32_t* counts, void* stream) {
  QK_GUARD_BEGIN
  if (!x || !c || n < 1 || d < 1 || K < 1) {
    set_error("invalid arguments");
    return QK_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Tmp tx(s), tc(s), ta(s), tn(s), tsum(s), tcnt(s);
  const float *X = nullptr, *C = nullptr;
  QK_TRY(in_device(x, (size_t)n * d, tx, &X, s));
  QK_TRY(in_device(c, (size_t)K * d, tc, &C, s));
  int32_t* a = nullptr;
  float* Cn = nullptr;
  double* sums = nullptr;
  int32_t* cnt = nullptr;
  QK_TRY(ta.alloc<int32_t>((size_t)n, &a));
  QK_TRY(tn.alloc<float>((size_t)K * d, &Cn));
  QK_TRY(tsum.alloc<double>((size_t)K * d, &sums));
  QK_TRY(tcnt.alloc<int32_t>((size_t)K, &cnt));
  QK_TRY(assign_nearest(X, n, d, C, K, a, s));
  QK_TRY(launch_kmeans_update(X, n, d, a, C, K, Cn, sums, cnt, s));
  if (c_new) QK_CUDA(cudaMemcpyAsync(c_new, Cn, sizeof(float) * (size_t)K * d, cudaMemcpyDefault, s));
  if (assign) QK_CUDA(cudaMemcpyAsync(assign, a, sizeof(int32_t) * (size_t)n, cudaMemcpyDefault, s));
  if (counts) QK_CUDA(cudaMemcpyAsync(counts, cnt, sizeof(int32_t) * (size_t)K, cudaMemcpyDefault, s));
  QK_CUDA(cudaStreamSynchronize(s));
  return QK_OK;
  QK_GUARD_END
}

}  // extern "C"
