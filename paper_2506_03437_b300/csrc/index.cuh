// Device layout of the multi-level partitioned index and the host object
// that owns it.
//
// HBM layout (all arrays cudaMalloc'd, 256-byte aligned):
//   level 0  arena vec0[cap0 x d] FP32 rows, ids0[cap0] int64; partition j
//            owns rows [off0[j], off0[j] + size0[j]) of the arena, contiguous,
//            so a partition streams with one-dimensional bulk copies, and
//            reserves room for inserts behind them; a free tail after the
//            last reservation takes partitions that outgrow their room;
//            cent0[n_leaf x d] its centroids.
//   level 1  vec1[n_leaf x d] the leaf centroids regrouped by parent,
//            ids1[n_leaf] the leaf index of each row, off1/size1 per parent,
//            cent1[n_parent x d] the parent centroids.
//   root     the centroids of the top level (cent1, or cent0 for one level),
//            scanned as one partition whose row index is the id.
//   beta     the FP64 1024-point table of I_x((d+1)/2, 1/2).
//   hits     int64 access counters per partition and level.
//
// Copy-on-write views (Sec. 9, "Concurrency"): a search reads the partition
// table (off0, size0) and the arena pointers it was launched with.  Inserts,
// deletes, compaction and maintenance never write a row or a table entry that
// a published version can read: they fill free rows and a spare table, then
// publish the new table with a pointer exchange.  What the older versions
// used is retired and handed back only once every search launched on them
// has completed (their completion events are recorded per launch).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <shared_mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/quake_b300.h"

namespace qk {

struct DevLevel {
  const float* vec = nullptr;
  const int64_t* ids = nullptr;
  const int64_t* off = nullptr;
  const int32_t* size = nullptr;
  const float* cent = nullptr;
  int32_t n_part = 0;
};

struct SearchArgs {
  const float* Q = nullptr;
  int64_t nq = 0;
  int32_t d = 0;
  int32_t metric = 0;
  int32_t L = 1;
  DevLevel lv[2];
  const float* root = nullptr;   // top-level centroids, scanned as one partition
  int32_t n_root = 0;
  int32_t M_root = 0;            // candidates kept from the root
  int32_t k0 = 10;               // results kept at level 0 (k, or rerank * k for low-precision scans)
  int32_t kq = 10;               // k returned
  int32_t mode0 = 0;             // level-0 rows: 0 FP32 + ids, 1 FP32 + slots, 2 BF16, 3 FP8 (slots)
  const void* lp_vec = nullptr;  // level-0 low-precision arena
  const float* lp_scale = nullptr;
  int32_t k1 = 0;                // k' at level 1 (= M of level 0)
  double tau0 = 0.9;             // recall target of level 0
  double tau1 = 0.99;            // recall target of level 1
  double tau_rho = 0.01;
  int32_t fixed_nprobe = 0;      // > 0: fixed-nprobe mode at level 0
  const int32_t* nprobe_q = nullptr;   // fixed-nprobe mode: one nprobe per query (else fixed_nprobe)
  int32_t beta_mode = 0;
  const double* beta_table = nullptr;
  double beta_a = 0.0, beta_lnB = 0.0;
  int64_t* out_ids = nullptr;
  float* out_dist = nullptr;
  int32_t* out_nprobe = nullptr;
  float* out_recall = nullptr;
  unsigned long long* hits0 = nullptr;
  unsigned long long* hits1 = nullptr;
  int32_t* work = nullptr;       // work-stealing counter (zeroed before launch)
  int32_t* status = nullptr;     // device status word
  int64_t* diag = nullptr;       // first failure: code, query, details
  int64_t* wait_stats = nullptr; // longest bulk-copy wait of the launch (cycles), optional
  int32_t* scan0 = nullptr;      // optional: level-0 partitions scanned per query, nq x scan_cap0, -1 padded
  int32_t scan_cap0 = 0;
  int32_t* scan1 = nullptr;      // optional: level-1 partitions scanned per query, nq x scan_cap1, -1 padded
  int32_t scan_cap1 = 0;
  float ratio_eps = 0.f;         // > 0: SPANN's rule at level 0 (scan the prefix of S within (1 + eps) of the nearest)
  int32_t* xs_M = nullptr;       // batched APS: per query, leaf candidates exported (-1: refused query)
  int32_t* xs_cand = nullptr;    // nq x xs_mcap leaf candidate partitions, nearest first
  double* xs_t = nullptr;        // nq x xs_mcap their bisector distances t_i
  int32_t xs_mcap = 0;
  // import: the upper levels were searched by the prepare step (the same walk,
  // bitwise); per query M, the leaf candidates and their t_i (nq x im_mcap)
  const int32_t* im_M = nullptr;
  const int32_t* im_cand = nullptr;
  const double* im_t = nullptr;
  int32_t im_mcap = 0;
  int32_t kcap = 16;             // capacity of the result set (>= every k used)
  int32_t mcap = 16;             // capacity of the candidate list
};

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

// A level-0 partition table: offsets and sizes of n_leaf partitions.
struct Table {
  int64_t* off = nullptr;
  int32_t* size = nullptr;
  int32_t n = 0;
};

// A search launch that may still be in flight, and the index version it reads.
struct ViewReader {
  cudaEvent_t ev = nullptr;
  uint64_t version = 0;
};

// Memory that searches of versions up to `version` may still read.
struct Retired {
  uint64_t version = 0;
  uint64_t arena = 0;                                 // arena the row ranges belong to
  std::vector<std::pair<int64_t, int64_t>> rows;      // (first row, rows) of that arena
  Table table;                                        // a partition table
  std::vector<void*> device;                          // allocations (a replaced arena)
  qk_index* structure = nullptr;                      // a whole replaced structure
};

struct qk_index_impl;

}  // namespace qk

struct qk_index {
  qk_config cfg;
  int device = 0;
  bool ready = false;
  int64_t n = 0;                 // live vectors
  int32_t n_leaf = 0, n_parent = 0;
  // level 0
  float* vec0 = nullptr;
  int64_t* ids0 = nullptr;
  int64_t cap0 = 0;              // arena rows
  int64_t used0 = 0;             // rows [0, used0) belong to partitions or holes; the rest is the free tail
  int64_t holes0 = 0;            // rows left behind by partitions that moved to the tail
  int64_t* off0 = nullptr;
  int32_t* size0 = nullptr;
  float* cent0 = nullptr;
  unsigned char* lp0 = nullptr;  // low-precision copy of the arena (BF16 / FP8)
  float* lp_scale0 = nullptr;    // FP8 scale per partition
  std::vector<int64_t> h_off0, h_cap_part0;
  std::vector<int32_t> h_size0;
  std::vector<int64_t> h_ids0;   // host mirror of ids0 (arena slot -> id)
  uint64_t arena_id = 0;         // names the arena that free0 and retired row ranges refer to
  std::map<int64_t, int64_t> free0;   // arena rows free to take again: first row -> rows
  std::vector<qk::Table> spare0; // partition tables no published version uses
  // level 1
  float* vec1 = nullptr;
  int64_t* ids1 = nullptr;
  int64_t* off1 = nullptr;
  int32_t* size1 = nullptr;
  float* cent1 = nullptr;
  std::vector<int32_t> h_size1;
  std::vector<int64_t> h_off1;
  // shared
  double* beta_table = nullptr;
  unsigned long long* hits0 = nullptr;
  unsigned long long* hits1 = nullptr;
  int32_t* work = nullptr;
  int32_t upper_mode = -1;        // upper levels of qk_search: -1 auto, 0 in the query's CTA, 1 prepare kernel
  int32_t* status = nullptr;
  int64_t* diag = nullptr;
  double beta_a = 0.0, beta_lnB = 0.0;
  // scratch for host <-> device staging
  qk::Buffer stage_in, stage_out;
  // id -> (partition, slot) for deletes
  std::unordered_map<int64_t, int64_t> where;
  std::atomic<int64_t> queries_seen{0};   // searched queries since the last install/maintain (the window |W|)
  std::atomic<uint64_t> search_seq{0};   // launches so far (selects the work counter)
  uint64_t version = 0;          // bumped by every change of the partitions (install, insert, delete)
  // a maintenance pass planned and built by qk_maintain_prepare, not yet
  // committed, and the index version it was planned from
  qk_index* pending = nullptr;
  uint64_t pending_version = 0;
  // Publication lock: searches (and other readers of the published structure)
  // hold it shared while they capture pointers and enqueue work; an update
  // holds it exclusively only to exchange pointers and host tables, so one
  // updating thread and any number of searching threads may run together.
  mutable std::shared_mutex pub_mu;
  // copy-on-write views: searches in flight and what older versions still use
  std::mutex view_mu;
  std::vector<qk::ViewReader> readers;
  std::vector<cudaEvent_t> idle_events;
  std::vector<qk::Retired> retired;
};

namespace qk {
constexpr int kWorkSlots = 16;   // searches of one index that may be in flight together
}

namespace qk {
// Shared by capi.cu and maintain.cu.
qk_status kmeans(const float* X, int64_t n, int d, int32_t K, int iters, uint64_t seed, float* C, int32_t* assign,
                 cudaStream_t s, const float* C_init);
qk_status install(qk_index* ix, const float* X, const int64_t* ids, int64_t n, const float* C0,
                  const int32_t* leaf_of_row, const float* C1, const int32_t* parent_of_leaf, cudaStream_t s,
                  bool skip_unlabelled);
bool is_device_ptr(const void* p);
// Exchanges the partition structure (arena, levels, host mirrors, id map,
// counters) of two index objects; frees an object's structure.
void swap_structure(qk_index* a, qk_index* b);
void release_structure(qk_index* ix);
qk_status assign_nearest(const float* X, int64_t n, int d, const float* C, int K, int32_t* assign, cudaStream_t s);
// M = ceil(f n) in double precision, clamped to [1, n] (the candidate count of a level).
int32_t n_candidates(double f, int32_t n);
// The search kernel's arguments that follow from the index and the call's k,
// recall target and fixed nprobe (queries, outputs and records not set).
void base_search_args(qk_index* ix, int32_t k, float recall_target, int32_t nprobe, SearchArgs& a);
qk_status launch_search(const SearchArgs& a, cudaStream_t stream);
// The upper levels of a search by the warp-per-query prepare kernel, exporting
// each query's leaf candidates and t_i into a.xs_*; QK_ERR_UNSUPPORTED when
// its per-warp buffers cannot hold the search's candidate counts.
qk_status prepare_upper(const SearchArgs& a, cudaStream_t stream);
// The xs_mcap a search's export needs.
int32_t prepare_mcap(const SearchArgs& a);

// Copy-on-write views (views.cu).
// Records that the work just enqueued on `s` reads the current version
// (no-op while `s` is capturing a graph: a replay records itself).
void note_readers(qk_index* ix, cudaStream_t s);
// Hands back what no search in flight can read any more: row ranges of the
// current arena go to free0, tables to spare0, the rest is freed.  With
// wait, first waits for every search in flight.
void reclaim(qk_index* ix, bool wait);
// Keeps `r` until the searches of versions up to r.version have completed.
void retire(qk_index* ix, Retired&& r);
// Moves the index's whole structure into a fresh object and retires it.
void retire_structure(qk_index* ix);
// Searches recorded and not yet known complete; arena rows kept for them.
int64_t readers_in_flight(qk_index* ix);
int64_t retired_rows(qk_index* ix);
// Arena rows for a partition of `rows` rows: the smallest free range that
// fits, else the free tail; -1 when neither has room.
int64_t take_rows(qk_index* ix, int64_t rows);
// A partition table of n_leaf entries that no published version uses.
qk_status take_table(qk_index* ix, Table* t);
// A fresh arena id.
uint64_t next_arena_id();
// Device memory of the index structure (arena, tables, levels): allocated and
// freed in stream order on a private stream of the current device; a free
// never waits for other work on the device.  The memory must no longer be in
// use by any kernel when it is freed.
qk_status mem_alloc(void** p, size_t bytes);
void mem_free(void* p);
}  // namespace qk
