/*
 * quake_b300.h -- C ABI of a single-GPU (B300, sm_103a) implementation of the
 * query-time hot path of Quake's adaptive partitioned vector index
 * (Mohoney et al., "Quake: Adaptive Indexing for Vector Search", OSDI'25).
 *
 * Conventions shared by every entry point
 *  - Every buffer argument may be a host or a device pointer; the library asks
 *    the CUDA driver which one it is.  Host buffers are copied in and out inside
 *    the call, which then returns only once the results are in host memory.
 *    With device buffers the call is stream-ordered on `stream` (a
 *    cudaStream_t; NULL = the legacy default stream) and may return before the
 *    GPU has finished.
 *  - The caller owns every buffer it passes; the index owns all of its device
 *    state and frees it in qk_destroy.
 *  - Vectors are row-major FP32, `d` values per row.  Ids are int64.
 *  - Distances: metric L2 reports the squared Euclidean distance; metric IP
 *    reports the NEGATED inner product, so smaller is nearer for both.  Results
 *    are ordered by (distance, id) ascending.  Unfilled result slots hold
 *    id = -1 and distance = +inf.
 *  - Supported dimensions: 32, 64, 96, 128, 192, 256, 384, 512, 768, 1024.
 *  - No C++ exception crosses the ABI.  A failing call returns a non-zero
 *    qk_status and leaves a message for qk_last_error() (thread-local).
 *  - Device buffers must be memory of the current GPU (or managed memory).
 *  - Threads: one host thread may update an index (insert, delete, build,
 *    load, maintain, maintain_commit; one such call at a time) while other
 *    threads search it (qk_search*, the batch plans, each plan used by one
 *    thread at a time) and inspect it (qk_info, qk_stats, qk_export_*,
 *    qk_get_hits).  An update holds the index exclusively only while it
 *    exchanges the published pointers (build and load: for the whole call).
 *    qk_maintain_prepare must not overlap an insert or delete.  Searches with
 *    device buffers may be in flight on up to 16 streams at once; searches
 *    with host buffers share staging memory, one at a time.
 *  - Copy-on-write views (Sec. 9, "Concurrency"): every search reads the
 *    version of the index that was current when it was launched, to its end.
 *    Insert, delete, build, load and a maintenance commit need not wait for
 *    the searches in flight: they build the next version beside the current
 *    one and publish it when they return; what the older versions use is
 *    freed once the searches launched on them have completed (checked at the
 *    next update, and waited for by qk_destroy).  A search launched after an
 *    update returns reads the updated version.  A search that the caller
 *    captured into a CUDA graph is not tracked: replay such a graph only
 *    while the version it captured is current (qk_stats' version).
 */
#ifndef QUAKE_B300_H
#define QUAKE_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qk_index qk_index;

typedef enum {
  QK_OK = 0,
  QK_ERR_ARG = 1,         /* invalid argument (sizes, pointers, NaN input, unsupported d) */
  QK_ERR_OOM = 2,         /* device memory exhausted */
  QK_ERR_CUDA = 3,        /* a CUDA runtime call failed */
  QK_ERR_TIMEOUT = 4,     /* a bounded device wait expired; results are not valid */
  QK_ERR_DUP_ID = 5,      /* insert of an id that is already present; nothing applied */
  QK_ERR_STATE = 6,       /* call not valid in the index's current state (e.g. search before build) */
  QK_ERR_UNSUPPORTED = 7, /* configuration not supported by this library */
  QK_ERR_INTERNAL = 8,    /* a kernel's own consistency check failed; results are not valid */
  QK_ERR_IO = 9           /* a checkpoint file could not be written or read, or is not valid */
} qk_status;

enum { QK_METRIC_L2 = 0, QK_METRIC_IP = 1 };
enum { QK_BETA_TABLE = 0, QK_BETA_EXACT = 1 };
enum { QK_STORE_F32 = 0, QK_STORE_BF16 = 1, QK_STORE_FP8 = 2 };

/*
 * Index configuration.  Paper parameters (Sec. 3, Sec. 5, Sec. 8.1):
 *   n_leaf, n_parent   partitions at level 0 and level 1 (n_parent = 0: one level).
 *   f_M_leaf, f_M_parent  initial candidate fractions f_M (Algorithm 1): the
 *                      search keeps M = ceil(f_M * N_l) candidates, computed in
 *                      double precision and clamped to [1, N_l].
 *   tau_rho            recompute threshold of Algorithm 1 (paper: 1%).
 *   upper_recall       fixed recall target of the upper level (paper: 99%).
 *   beta_mode          QK_BETA_TABLE: regularised incomplete beta from a
 *                      1024-point table at x_j = j/1023 with linear
 *                      interpolation (Sec. 5, "Performance Optimizations");
 *                      QK_BETA_EXACT: evaluated per candidate.
 *   kmeans_iters, seed Lloyd iterations and the SplitMix64 seed of the build.
 *   storage            QK_STORE_F32: the leaf scan reads the FP32 rows.
 *                      QK_STORE_BF16 / QK_STORE_FP8: it reads a BF16 copy, or
 *                      an FP8 E4M3 copy with one scale per partition
 *                      (s = max|x| / 448), accumulating in FP32, keeps
 *                      rerank * k candidates and re-ranks them exactly from
 *                      the FP32 rows.  Upper levels always use FP32.
 *   rerank             candidate multiple of the low-precision scan (>= 1).
 */
typedef struct {
  int32_t d;
  int32_t metric;
  int32_t n_leaf;
  int32_t n_parent;
  int32_t kmeans_iters;
  int32_t beta_mode;
  uint64_t seed;
  double f_M_leaf;
  double f_M_parent;
  double tau_rho;
  double upper_recall;
  int32_t storage;
  int32_t rerank;
} qk_config;

/* Fills `cfg` with the paper's defaults: L2, one level, f_M = 0.1 / 0.25,
 * tau_rho = 0.01, upper_recall = 0.99, table mode, 10 Lloyd iterations,
 * FP32 storage, rerank 4. */
void qk_config_default(qk_config* cfg);

/* Creates an empty index on the current CUDA device.  Errors: QK_ERR_ARG for
 * an unsupported d or metric, QK_ERR_CUDA / QK_ERR_OOM. */
qk_status qk_create(const qk_config* cfg, qk_index** out);

/* Frees all device and host state of the index.  NULL is accepted. */
void qk_destroy(qk_index* index);

/* Message of the last failing call on this host thread ("" if none). */
const char* qk_last_error(void);

/*
 * Builds the index from n vectors x (n x d) with ids (Sec. 3, "Index
 * Structure"): Lloyd k-means into n_leaf partitions (seeded rows chosen by a
 * SplitMix64 partial Fisher-Yates shuffle; assignment to the nearest
 * centroid with ties to the lower index; FP64 member means rounded to FP32;
 * empty clusters keep their centroid), then, if n_parent > 0, k-means of the
 * leaf centroids into n_parent parents.  Every row is finally placed in the
 * partition of its nearest final centroid.  Ids must be unique (QK_ERR_DUP_ID).
 * Synchronous: returns after the index is ready.
 */
qk_status qk_build(qk_index* index, const float* x, const int64_t* ids, int64_t n, void* stream);

/*
 * Installs a given partitioning instead of clustering: leaf_centroids
 * (n_leaf x d), leaf_of_row[n] in [0, n_leaf); for two levels also
 * parent_centroids (n_parent x d) and parent_of_leaf[n_leaf] in [0, n_parent)
 * (both NULL / 0 for one level).  The counts must match the configuration.
 * Synchronous.
 */
qk_status qk_load(qk_index* index, const float* x, const int64_t* ids, int64_t n,
                  const float* leaf_centroids, const int32_t* leaf_of_row,
                  const float* parent_centroids, const int32_t* parent_of_leaf, void* stream);

/* Where qk_search walks the upper levels (the top partition and APS on the
 * parent level, Sec. 5) of a two-level index: 1 = a warp-per-query prepare
 * kernel ahead of the search kernel, 0 = inside each query's CTA, -1
 * (default) = 1 for d <= 256 (a warp sums 4 rows per step there), else 0.
 * Both give the same candidates and t_i bit for bit, hence the same
 * results; qk_search_scanned's upper-level record, the ratio rule and
 * batches whose exported candidates would pass 1 GiB (12 bytes per query
 * and candidate, stream-ordered scratch) always use 0.  QK_ERR_ARG for
 * another value. */
qk_status qk_set_search_upper(qk_index* index, int32_t mode);

/*
 * Searches nq queries q (nq x d) for their k nearest neighbours (k <= 1024).
 *
 * recall_target > 0: Adaptive Partition Scanning (Sec. 5, Eq. 7-9, Algorithm 1)
 *   at every level.  The top partition (all centroids of the top level) is
 *   scored and the M = ceil(f_M * N) nearest kept; an upper level runs APS with
 *   k' = M of the level below and `upper_recall`; the leaf level runs APS with
 *   k and recall_target.  Per query, partitions are scanned nearest first until
 *   k results are held, then in decreasing p_i; p is recomputed when the k-th
 *   distance rho moves by more than tau_rho * rho; the scan stops when the
 *   estimate r = p_0 + sum of the scanned p_i reaches the target or the
 *   candidates run out.
 * recall_target <= 0: fixed nprobe (Faiss-IVF style): the nprobe nearest leaf
 *   partitions are scanned (found through the upper level when there is one).
 *
 * Outputs (nq x k, row-major): out_ids, out_dist.  Optional (NULL to skip):
 * out_nprobe[nq] leaf partitions scanned, out_recall[nq] the final estimate r
 * (NaN in fixed-nprobe mode).  Per-partition access counts are accumulated in
 * the index (see qk_get_hits).  A query with a NaN or infinite element (or a
 * squared norm beyond FP32) is refused by the kernel: its ids are -1, its
 * distances and recall NaN, its nprobe 0, the other queries are answered, and
 * the call (or, with device buffers, the next qk_check) returns QK_ERR_ARG.
 * With low-precision
 * storage the leaf scan keeps rerank * k candidates by their approximate
 * distance (rho is the k-th of them) and the k returned are re-ranked with
 * exact FP32 distances.  Inner product: rho is ||q - x_k|| of the k-th result.
 */
qk_status qk_search(qk_index* index, const float* q, int64_t nq, int32_t k, float recall_target,
                    int32_t nprobe, int64_t* out_ids, float* out_dist, int32_t* out_nprobe,
                    float* out_recall, void* stream);

/*
 * qk_search that also reports each query's partition selection: the
 * partitions Algorithm 1 (Sec. 5) scanned, in the order it scanned them.
 * out_scanned0 (nq x cap0 int32, optional) receives the leaf partitions
 * scanned by query j in row j; out_scanned1 (nq x cap1, optional) the parent
 * partitions scanned by the upper-level APS (all -1 for a one-level index).
 * Entries past the number scanned, or a whole row of a refused query, are -1;
 * a query that scanned more than cap partitions keeps the first cap.
 * Either record may be NULL; a non-NULL record needs cap >= 1 (QK_ERR_ARG
 * otherwise).  Host or device buffers, like every other output.
 */
qk_status qk_search_scanned(qk_index* index, const float* q, int64_t nq, int32_t k, float recall_target,
                            int32_t nprobe, int64_t* out_ids, float* out_dist, int32_t* out_nprobe,
                            float* out_recall, int32_t* out_scanned0, int32_t cap0, int32_t* out_scanned1,
                            int32_t cap1, void* stream);

/*
 * Waits for the index's work on `stream` and reports what its kernels found:
 * QK_ERR_TIMEOUT if a bounded device wait expired, QK_ERR_INTERNAL if a
 * kernel's consistency check failed (details in qk_last_error), QK_OK
 * otherwise.  Clears the device status.  Calls with host buffers do this
 * themselves; calls with device buffers return before the kernels finish, so
 * their callers use qk_check to learn the outcome.
 */
qk_status qk_check(qk_index* index, void* stream);

/* Index shape.  Any output pointer may be NULL. */
qk_status qk_info(const qk_index* index, int64_t* n_vectors, int32_t* n_leaf, int32_t* n_parent,
                  int32_t* d);

/*
 * Index statistics: what the maintenance planner (Sec. 4) and an operator
 * read.  Partition sizes and the access counts A_l,j of the cost model (Eq. 1)
 * accumulate per partition (qk_get_hits returns them one by one); this call
 * sums them, together with the arena's occupancy.  Reads the hit counters
 * from the device (synchronous).  QK_ERR_STATE before the index is built.
 */
typedef struct {
  int64_t n_vectors;          /* live vectors */
  int32_t levels;             /* 1, or 2 with a parent level */
  int32_t n_partitions[2];    /* leaf partitions; parent partitions (0 without) */
  int32_t d, metric, storage;
  int32_t min_size, max_size; /* smallest and largest leaf partition */
  double mean_size;           /* live vectors per leaf partition */
  int64_t arena_rows;         /* rows reserved in the leaf arena */
  int64_t arena_used;         /* rows below the free tail: partitions' rooms and holes */
  int64_t arena_holes;        /* rows below the tail that no partition holds (moved-out rooms) */
  int64_t arena_free;         /* rows of the free tail */
  int64_t arena_bytes;        /* device bytes of the arena (FP32 rows, ids, low-precision copy) */
  int64_t hits[2];            /* scanned (query, partition) pairs since the last reset, per level */
  int64_t queries_seen;       /* queries searched since the last build or maintenance (|W|) */
  uint64_t version;           /* changes with every build, insert, delete and maintenance commit */
  int64_t searches_in_flight; /* search launches not yet known to have completed */
  int64_t retired_rows;       /* arena rows kept, among the holes, for searches of older versions */
} qk_index_stats;
qk_status qk_stats(const qk_index* index, qk_index_stats* out);

/*
 * Inserts n vectors x (n x d) with new ids (Sec. 3, "Adaptive Incremental
 * Maintenance"): each descends the tree greedily (the nearest parent
 * centroid, then the nearest leaf centroid under it; ties to the lower
 * index; centroids are not moved) and is appended to that leaf partition,
 * in batch order.  An id already in the index or repeated in the batch gives
 * QK_ERR_DUP_ID and NaN gives QK_ERR_ARG; in both cases nothing is inserted.
 * The new rows go behind each partition's live rows, which no published
 * version reads.  A partition whose reserved rows run out is copied to free
 * arena rows with more room (a range a finished version gave back, else the
 * free tail); when none is large enough the arena is first laid out again
 * into new memory.  Returns once the new version is published; searches in
 * flight keep the old one.  Synchronous.
 */
qk_status qk_insert(qk_index* index, const float* x, const int64_t* ids, int64_t n, void* stream);

/*
 * Deletes the vectors with the given ids (Sec. 3: the map locates the
 * partition, the vector is removed with immediate compaction).  Deletes apply
 * in order; each moves the partition's last row into the freed slot.  Unknown
 * ids are skipped; *n_removed (if not NULL) receives the number removed.
 * Every partition that loses a row is first copied to free arena rows, and
 * the deletes edit the copy, so searches in flight keep the old version.
 * Synchronous.
 */
qk_status qk_delete(qk_index* index, const int64_t* ids, int64_t n, int64_t* n_removed, void* stream);

/*
 * Copies the structure of one level to host arrays for inspection:
 * level 0: sizes[n_leaf], centroids (n_leaf x d), ids[n_vectors] and
 *   vectors (n_vectors x d) grouped by partition in partition order;
 * level 1: sizes[n_parent], centroids (n_parent x d), ids[n_leaf] = leaf
 *   indices grouped by parent (vectors must be NULL).
 * All outputs are host pointers; any may be NULL.
 */
qk_status qk_export_level(const qk_index* index, int32_t level, int32_t* sizes, float* centroids,
                          int64_t* ids, float* vectors);

/*
 * Copies the low-precision copy of level 0 to host memory: codes holds every
 * vector's d elements (2 bytes each for BF16, 1 for FP8) grouped by partition
 * in partition order, as qk_export_level orders ids; scales[n_leaf] the FP8
 * scale of every partition (1 for BF16).  QK_ERR_STATE for FP32 storage.
 */
qk_status qk_export_quantized(const qk_index* index, uint8_t* codes, float* scales);

/* Copies the access counts of `level` (one int64 per partition, summed over
 * searches since the last reset) to a host array; reset != 0 zeroes them. */
qk_status qk_get_hits(qk_index* index, int32_t level, int64_t* hits, int32_t reset);

/*
 * Checkpoint and resume.  The paper has no counterpart (its indexes live in
 * memory).  qk_save writes one file (host byte order) with everything a
 * search or maintenance pass reads: the configuration with the current
 * partition counts, the partitions of both levels (sizes, centroids, ids and
 * FP32 rows grouped by partition; with BF16 / FP8 storage also the
 * low-precision rows and FP8 scales as they are, since rows inserted after the
 * build keep the scale they were quantized with), the access counters of both
 * levels and the statistics window, and a 64-bit FNV-1a checksum.  The index
 * is only read; it must not be modified meanwhile.
 * qk_restore creates an index on the current device from such a file: it
 * searches, updates and maintains exactly as the saved one.  Partition
 * numbers and contents are kept; the arena layout is fresh.  cfg_out
 * (optional) receives the configuration.  Errors: QK_ERR_ARG (null
 * arguments), QK_ERR_STATE (qk_save of an empty index), QK_ERR_IO (the file
 * cannot be opened, written or read, is not a checkpoint, is truncated, fails
 * the checksum or is inconsistent), QK_ERR_OOM / QK_ERR_CUDA.  Synchronous.
 */
qk_status qk_save(qk_index* index, const char* path);
qk_status qk_restore(const char* path, qk_config* cfg_out, qk_index** out);

/*
 * Exact cap volume fraction u = 1/2 I_x((d+1)/2, 1/2), x = 1 - (t/rho)^2 for
 * t < rho and 0 otherwise (Sec. 5, "Intersection Volume Approximation", after
 * Li 2010), evaluated in FP64 on the GPU with the library's continued fraction
 * (mode QK_BETA_EXACT) or its 1024-point table (QK_BETA_TABLE), for n pairs
 * (t[i], rho[i]).  Exposed so the estimator's arithmetic can be checked.
 */
qk_status qk_cap_fraction(int32_t d, int32_t mode, const double* t, const double* rho, int64_t n,
                          double* out_u, void* stream);

/*
 * For each of the n rows of x (n x d), the k nearest of the K centroids c
 * (K x d), 1 <= k <= min(8, K), d a multiple of 32: out_idx (n x k) and, if
 * not NULL, out_dist (n x k, exact FP32 distances: squared L2, or the negated
 * inner product) in (distance, index) order.  This is the centroid scoring of
 * the top-down search and of k-means assignment (Sec. 3): tensor cores
 * (tcgen05, TF32 operands, FP32 accumulation) score every centroid.
 *  - k = 1: the result is the exact FP32 nearest centroid (ties to the lower
 *    index), as an exact scan with the same FP32 arithmetic gives it.  Each
 *    row keeps its smallest approximate distance and the runner-up; when the
 *    gap exceeds a proven bound on the TF32 and FP32 errors (about 2^-6
 *    ||x|| max||c||) the smallest is the answer; the other rows are scored
 *    again, every centroid within that bound of their smallest approximate
 *    distance is scored exactly, and the best is kept.  Synchronises the
 *    stream once (to size the second pass).
 *  - k > 1: the 16 best approximate candidates of a row are re-scored
 *    exactly in FP32 and the k best are kept.  TF32 moves an approximate
 *    distance by at most about 2^-9 ||x|| ||c||; keeping twice the largest k
 *    as approximate candidates leaves a margin for that, and a true neighbour
 *    outside the 16 approximate candidates is the only way the result can
 *    differ from an exact scan.
 */
qk_status qk_nearest_centroids(const float* x, int64_t n, int32_t d, const float* c, int32_t K, int32_t metric,
                               int32_t k, int32_t* out_idx, float* out_dist, void* stream);

/*
 * One Lloyd step on the GPU (Sec. 3; k-means as in qk_build): assigns each of
 * the n rows of x to the nearest of the K centroids c (ties to the lower
 * index) and returns the FP64 member means rounded to FP32 in c_new (empty
 * clusters keep c), the assignment in assign[n] and the member counts in
 * counts[K].  c_new, assign and counts may be NULL.
 */
qk_status qk_kmeans_step(const float* x, int64_t n, int32_t d, const float* c, int32_t K,
                         float* c_new, int32_t* assign, int32_t* counts, void* stream);

/*
 * Maintenance parameters (Sec. 4 and Sec. 8.1).
 *   lambda_sizes/us   the latency function lambda(s): lambda_points profiled
 *                     (size, microseconds) pairs with strictly increasing
 *                     sizes, interpolated linearly, extended linearly past
 *                     both ends and floored at 0.  It is applied to partition
 *                     sizes and to centroid counts (Delta O+ = lambda(N + 1) -
 *                     lambda(N), Delta O- = lambda(N - 1) - lambda(N)).
 *   tau_us            decision threshold tau (paper: 250 ns = 0.25).
 *   alpha             split access scaling (paper: 0.9).
 *   refine_radius     r_f (paper: 50); also the merge estimate's receiver count.
 *   refine_iters      Lloyd iterations of the refinement (paper: 1); refine = 0 skips it.
 *   split_iters       Lloyd iterations of the 2-means that splits a partition.
 *   s_min             partitions smaller than this are merge candidates.
 *   window            |W| in queries; 0 = the queries searched since the last
 *                     build, load or maintain.
 *   level_band        1: after the levels' passes, keep the top level within
 *                     sqrt(N0)/4 .. 4 sqrt(N0) centroids (N0 = leaves; the
 *                     paper adds and removes levels, Sec. 3 and Sec. 4, with
 *                     thresholds given only in its technical report): a
 *                     single-level index with N0 > 16 gets a parent level, a
 *                     two-level one with N0 <= 16 loses it, and a parent level
 *                     outside the band is rebuilt.  New parents: k-means
 *                     (level_iters Lloyd iterations, seed + 1 like the build)
 *                     of the leaf centroids into round(sqrt(N0)).  0: off.
 *   level_iters       Lloyd iterations of that k-means.
 */
typedef struct {
  const double* lambda_sizes;
  const double* lambda_us;
  int32_t lambda_points;
  int32_t refine_radius;
  int32_t refine_iters;
  int32_t split_iters;
  int32_t s_min;
  int32_t refine;
  double tau_us;
  double alpha;
  int64_t window;
  int32_t level_band;
  int32_t level_iters;
} qk_maint_params;

/* One considered action: kind 0 = split, 1 = merge; partition is the index
 * at the start of the level's pass; estimate is Eq. 6 (split) or the uniform
 * redistribution estimate (merge); delta is Eq. 4 or Eq. 5 after the
 * tentative action (NaN if a split left a child empty).  With level_band,
 * kind 2 = parent level added, 3 = removed, 4 = rebuilt (level 1, partition =
 * the new parent count, committed = 1, estimate and delta NaN). */
typedef struct {
  int32_t level;
  int32_t kind;
  int32_t partition;
  int32_t committed;
  double estimate;
  double delta;
} qk_maint_action;

/*
 * The maintenance pass of Sec. 4 ("Decision Workflow"), bottom-up over the
 * levels.  Stage 0: A = access count / |W| from the counters the searches
 * accumulated, sizes from the index.  Stage 1: split estimate (Eq. 6) for
 * every partition and merge estimate for partitions smaller than s_min; the
 * candidates below -tau are taken in ascending order of the estimate.
 * Stage 2: a tentative split runs 2-means on the partition (rows seeded by
 * SplitMix64 from the index seed, the level and the partition), a tentative
 * merge sends every row to its nearest remaining centroid; Eq. 4 / Eq. 5 are
 * evaluated with the real sizes and the current partition count.  Stage 3:
 * commit when Delta < -tau, otherwise the partition is left as it was.  A
 * committed split is followed by refinement (Lloyd iterations over the r_f
 * partitions nearest each child); partitions touched by a committed action
 * are not considered again in the same pass.  Stage 4: in a two-level index
 * the parent level is then maintained the same way over the updated leaf
 * centroids.  The arena is re-laid out once, partition indices are
 * renumbered (survivors keep their order; split children are appended) and
 * the access counters restart.  Up to log_cap actions are written to log;
 * *n_log receives the number considered.  Synchronous.
 */
qk_status qk_maintain(qk_index* index, const qk_maint_params* params, qk_maint_action* log, int32_t log_cap,
                      int32_t* n_log, void* stream);

/* The same pass in two steps, so that searches need not wait for it (a
 * copy-on-write view of the index; the paper runs maintenance beside the
 * searches, Sec. 4 and Sec. 8):
 *  - qk_maintain_prepare plans the pass and builds the resulting partitions
 *    (arena, centroids, parent level, id map) into separate device memory.
 *    It only reads the index, so searches of the index may run on other
 *    streams (or other host threads) meanwhile; inserts and deletes must
 *    not.  The log arguments are as for qk_maintain.  Returns when the new
 *    structure is complete.  It needs room for a second arena.
 *  - qk_maintain_commit makes the prepared structure the index's.  Searches
 *    in flight keep reading the old one, which is freed once they have
 *    completed.  It is quick (pointer and host-state exchange).
 *    QK_ERR_STATE if nothing was prepared, or if the index changed (insert,
 *    delete, build, load, maintenance) after the prepare: the prepared pass
 *    is then discarded.
 * The statistics window of the next pass starts at the commit.  Preparing
 * again discards an earlier prepared pass. */
qk_status qk_maintain_prepare(qk_index* index, const qk_maint_params* params, qk_maint_action* log,
                              int32_t log_cap, int32_t* n_log, void* stream);
qk_status qk_maintain_commit(qk_index* index, void* stream);

/*
 * Scan-latency profile lambda(s) of the cost model (Sec. 4, "Cost Model":
 * lambda is measured by offline profiling; Sec. 9 profiles it again for other
 * devices and for compressed partitions).  For every size sizes[i] (rows,
 * positive, strictly increasing) a throwaway one-level index of P partitions
 * of that many rows is made on the current device, in cfg's dimension, metric,
 * storage format and rerank (n_leaf and n_parent are ignored).  Its rows are
 * seeded synthetic data (cfg->seed): P = max(4 x SMs, rows of about 1 GiB),
 * capped at 4096 partitions and 24 GiB of FP32 rows.  Q queries (4 x SMs ..
 * 4096, fewer for large partitions)
 * each sit on one partition's centre, and fixed-nprobe searches with k
 * results are timed with CUDA events on `stream` (median of `reps` after one
 * untimed search) at nprobe 1 and 9.
 *   out_us[i] = (T(9) - T(1)) / (8 Q), in microseconds, floored at 0:
 * the device time one more scanned partition of sizes[i] rows adds per
 * (query, partition) item of a search batch.  The differences remove the
 * launch, centroid scoring, result write and re-rank.  The table can be passed
 * to qk_maintain as lambda_sizes / lambda_us; tau_us is then in the same unit.
 * Synchronous.  Errors: QK_ERR_ARG for bad arguments or a size whose 9
 * partitions exceed 24 GiB of FP32 rows; QK_ERR_OOM / QK_ERR_CUDA from the
 * device.  The index of each size is freed before the next.
 */
qk_status qk_profile_scan(const qk_config* cfg, int32_t k, const int64_t* sizes, int32_t n_sizes, int32_t reps,
                          double* out_us, void* stream);

/*
 * Allocation-free Lloyd step.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory while they run
 * (a serving loop that cannot afford the device-wide synchronisation of
 * cudaMalloc/cudaFree, a process whose custom allocator owns all free
 * memory, an embedder with a fixed device footprint).  It allocates nothing:
 * no cudaMalloc, no cudaFree, no allocating library routine.
 *
 *  - What it computes: one Lloyd step with the exact FP32 assignment (every
 *    point to its nearest centroid by direct differences, ties to the lower
 *    index) and FP64 member sums.  qk_kmeans_step assigns through tensor-core
 *    scoring when K >= 32 and d % 32 == 0, keeping a short candidate list that
 *    it re-checks exactly in FP32; the two agree whenever that list contains
 *    the nearest centroid.  Centroids then agree to within the summation
 *    order of the FP64 sums (a few FP32 ulp at most).
 *  - Every buffer must be device memory of the current GPU, or managed
 *    memory: x (n x d), c (K x d) in; c_new (K x d), assign[n], counts[K] out,
 *    all required.  Host memory and another GPU's memory are refused
 *    (QK_ERR_ARG).  c_new may be the same buffer as c.
 *  - Its only scratch, the FP64 per-cluster sums, lives in a fixed 8 MiB
 *    array inside the library.  K * d may not exceed 1,048,576 (QK_ERR_ARG
 *    otherwise).  CUDA loads the array's module lazily: the first call on a
 *    GPU loads it and looks up its device address, and the GPU then keeps the
 *    8 MiB until the process exits.  Make that first call at start-up: before
 *    handing the GPU's free memory to another allocator, and before any
 *    stream capture.  After a cudaDeviceReset the next call looks the address
 *    up again.
 *  - All calls share the one array and each call clears the sums it uses
 *    before accumulating.  Calls that overlap on the GPU (different streams,
 *    or different host threads, at the same time) race on it: serialise them.
 *  - Stream-ordered on `stream`; returns before the GPU has finished.
 */
qk_status qk_kmeans_step_noalloc(const float* x, int64_t n, int32_t d, const float* c, int32_t K,
                                 float* c_new, int32_t* assign, int32_t* counts, void* stream);

/* ------------------------------------------------------------------------
 * Batched fixed-nprobe search (Sec. 3 top-down search with a fixed nprobe per
 * query, for a batch of queries each with its own nprobe; single level: the
 * nprobe nearest leaf centroids of each query are scanned).
 *
 * A plan owns the device workspace of batches of up to max_nq queries with
 * k results and nprobe values up to max_nprobe, so that a batch allocates
 * nothing and never waits on the host: the whole batch is one fixed sequence
 * of device steps, which qk_batch_capture records as one CUDA graph.
 *
 * Steps of a batch (all on the GPU):
 *   1. approximate distances of every query to every leaf centroid on the
 *      tensor cores (tcgen05, TF32 operands, FP32 accumulation);
 *   2. per query, the nprobe nearest centroids by exact FP32 distance: every
 *      centroid whose approximate distance is within a bound of the TF32
 *      error of the nprobe-th one is re-scored exactly, ties to the lower
 *      index, so the selection equals an exact FP32 selection;
 *   3. the (query, partition) pairs grouped by partition into units of one
 *      partition x G queries x chunk_rows rows, largest partitions first;
 *   4. one persistent launch scans the units: each row tile is read once from
 *      HBM for the unit's G queries, each query keeping its top-k;
 *   5. per query, the top-k over its units by (distance, id).
 * Distances are FP32 squared L2 from the direct differences.  Outputs are
 * nq x k rows sorted by (distance, id); a query whose scanned partitions hold
 * fewer than k rows gets (id -1, +inf) in the remaining slots.
 *
 * Conventions: every buffer is 16-byte aligned device memory; calls are
 * stream-ordered and return before the GPU finishes; device-side errors
 * (an nprobe outside [1, max_nprobe], a query with a NaN or infinite
 * element, a bounded wait that expired) are recorded in the index's status
 * word and reported by qk_check; a refused query gets (id -1, +inf) rows and
 * the others are answered.  A plan
 * follows the index's inserts, deletes and maintenance by itself on the next
 * qk_batch_search; a captured graph does not (qk_batch_replay then returns
 * QK_ERR_STATE: capture again).  Calls on one plan must not overlap.  L2
 * metric and FP32 storage only.
 * ------------------------------------------------------------------------ */
typedef struct qk_batch qk_batch;

/* Tile shapes of the grouped scan. */
typedef struct {
  int32_t queries_per_warp;  /* 1, 2 or 4 (4 needs d <= 128 or d = 384, 512): G = 8 x this queries per unit */
  int32_t tile_rows;         /* rows per shared-memory tile (3 tiles in flight, <= 200 KB together) */
  int32_t chunk_rows;        /* rows per unit (>= tile_rows, >= 1024) */
  int32_t rows_per_thread;   /* 0: each row is summed by 1-32 lanes holding the warp's queries in
                                registers; 2: each thread sums 2 whole rows against its warp's 4
                                queries, read from shared memory (d <= 256; units of 32 queries and
                                tiles of 64 rows whatever queries_per_warp and tile_rows say; in the
                                batched APS search it applies to the rounds after the first, which
                                keeps the other fields).  Both give the same results. */
} qk_batch_tiles;

/* Creates a plan for the (built or loaded) index.  max_nq >= 1, 1 <= k <= 32,
 * 1 <= max_nprobe <= 2048.  Errors: QK_ERR_ARG (sizes, IP metric or
 * low-precision storage), QK_ERR_STATE (empty index), QK_ERR_OOM. */
qk_status qk_batch_create(qk_index* index, int64_t max_nq, int32_t k, int32_t max_nprobe, qk_batch** out);
void qk_batch_destroy(qk_batch* plan);

/* Current tile shapes / set them (QK_ERR_ARG for an invalid shape). */
qk_status qk_batch_get_tiles(const qk_batch* plan, qk_batch_tiles* out);
qk_status qk_batch_set_tiles(qk_batch* plan, const qk_batch_tiles* tiles);

/* One batch: q (nq x d FP32), nprobe[nq] (int32, each in [1, max_nprobe];
 * values above the number of leaves scan every leaf), out_ids (nq x k int64),
 * out_dist (nq x k FP32).  0 <= nq <= max_nq. */
qk_status qk_batch_search(qk_batch* plan, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids,
                          float* out_dist, void* stream);

/* Runs the batch once, then records it on `stream` (a created stream, not
 * the legacy default stream) as a CUDA graph bound to these buffers. */
qk_status qk_batch_capture(qk_batch* plan, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids,
                           float* out_dist, void* stream);
/* Launches the captured graph on `stream`. */
qk_status qk_batch_replay(qk_batch* plan, void* stream);

/* Times every valid tile shape (queries_per_warp x tile_rows x chunk_rows
 * from {1,2,4} x {16,32,64} x {1024,4096,16384} with rows_per_thread 0, and
 * the whole-rows layout with each chunk_rows) on this batch, reps runs each
 * after one warm-up, keeps the fastest in the plan and returns it.  Every
 * shape gives the same results.  Synchronises the stream. */
qk_status qk_batch_autotune(qk_batch* plan, const float* q, int64_t nq, const int32_t* nprobe, int64_t* out_ids,
                            float* out_dist, int32_t reps, qk_batch_tiles* chosen, void* stream);

/* Stage timing of uncaptured batches: with timing on, qk_batch_search records
 * CUDA events on its stream between its steps; qk_batch_stage_times waits for
 * the last batch and writes five durations in milliseconds: centroid scoring
 * (norms + tensor-core distances), selection, grouping, grouped scan, merge.
 * QK_ERR_STATE if no batch ran with timing on. */
qk_status qk_batch_set_timing(qk_batch* plan, int32_t on);
qk_status qk_batch_stage_times(qk_batch* plan, float* ms);

/* ------------------------------------------------------------------------
 * Batched Adaptive Partition Scanning: Algorithm 1 (Sec. 5) for every query
 * of a batch, with the leaf scans of all queries grouped by partition
 * (multi-query processing, Sec. 8), so that a partition several queries need
 * is read from HBM once per round for all of them.
 *
 * Steps (all on the GPU, no host synchronisation):
 *   1. per query: the top partition is scored and the upper level searched by
 *      APS exactly as qk_search does; the leaf candidates S, nearest first,
 *      and their bisector distances t_i are kept;
 *   2. rounds: every unfinished query has asked for some of its candidates;
 *      the (query, partition) items are grouped by partition and one
 *      persistent scan computes every item's own exact top-k;
 *   3. after each round one warp per query walks Algorithm 1 over what was
 *      scanned, in the order Algorithm 1 takes the partitions (centroid order
 *      until R holds k results, then decreasing p, with rho, the recompute
 *      rule and r as in qk_search).  When the partition it takes next was not
 *      scanned, the query asks for it and for those Algorithm 1 would take
 *      after it if p stayed as it is, until r would reach the target.  Items
 *      scanned beyond a query's stop are discarded.
 * The results, nprobe, r and the partitions scanned therefore equal
 * qk_search's with the same recall target.  The last of the plan's rounds
 * (4 unless set) asks for every candidate not yet scanned, so every query
 * finishes; unused rounds cost only their launches.
 *
 * Conventions: L2 metric and FP32 storage; k <= 32; q, out_ids and out_dist
 * are 16-byte aligned device buffers, out_nprobe[nq], out_recall[nq] and
 * out_scanned0 (nq x cap0, as qk_search_scanned) optional device buffers.
 * Calls are stream-ordered and return before the GPU finishes; device-side
 * errors land in the index's status word (qk_check).  A query with a NaN or
 * infinite element is refused as in qk_search.  Access counts accumulate as
 * in qk_search.  A plan follows inserts, deletes and maintenance by itself on
 * the next qk_aps_batch_search; a captured graph does not (replay then returns
 * QK_ERR_STATE).  Calls on one plan must not overlap.
 * ------------------------------------------------------------------------ */
typedef struct qk_aps_batch qk_aps_batch;

/* A plan for batches of up to max_nq queries with k results (device workspace:
 * per query the candidate list, its p values and R, plus one round's candidate
 * buffer of k per item chunk). */
qk_status qk_aps_batch_create(qk_index* index, int64_t max_nq, int32_t k, qk_aps_batch** out);
void qk_aps_batch_destroy(qk_aps_batch* plan);
/* Number of rounds, 1 to 16 (default 4). */
qk_status qk_aps_batch_set_rounds(qk_aps_batch* plan, int32_t rounds);
/* Times the tile shapes (queries_per_warp x tile_rows x chunk_rows from
 * {1,2,4} x {16,32,64} x {1024,4096,16384}, each with rows_per_thread 0 and
 * 2) that are valid here, reps batches each after one warm-up, keeps the
 * fastest in the plan and returns it.  Every shape sums each row in the
 * per-query kernel's order, so the results do not depend on the choice.
 * Synchronises the stream. */
qk_status qk_aps_batch_autotune(qk_aps_batch* plan, const float* q, int64_t nq, float recall_target,
                                int64_t* out_ids, float* out_dist, int32_t reps, qk_batch_tiles* chosen,
                                void* stream);
/* Tiles of the grouped scan (as qk_batch_set_tiles; default 2 queries per
 * warp, tile_rows 8192 / d capped to [8, 64], chunk_rows 4096, and whole rows
 * per thread after the first round where d <= 256). */
qk_status qk_aps_batch_set_tiles(qk_aps_batch* plan, const qk_batch_tiles* tiles);
qk_status qk_aps_batch_search(qk_aps_batch* plan, const float* q, int64_t nq, float recall_target,
                              int64_t* out_ids, float* out_dist, int32_t* out_nprobe, float* out_recall,
                              int32_t* out_scanned0, int32_t cap0, void* stream);
/* Runs the batch once, then records it as one CUDA graph (buffers fixed). */
qk_status qk_aps_batch_capture(qk_aps_batch* plan, const float* q, int64_t nq, float recall_target,
                               int64_t* out_ids, float* out_dist, int32_t* out_nprobe, float* out_recall,
                               void* stream);
qk_status qk_aps_batch_replay(qk_aps_batch* plan, void* stream);
/* Stage timing of uncaptured batches: with timing on, qk_aps_batch_search
 * records CUDA events on its stream between its steps; qk_aps_batch_stage_times
 * waits for the last timed batch and writes 4 + rounds durations in
 * milliseconds: the prepare step (root scoring and upper level), every replay
 * together, every grouping together, every grouped scan together, then the
 * grouped scan of each round.  QK_ERR_STATE if no batch ran with timing on. */
qk_status qk_aps_batch_set_timing(qk_aps_batch* plan, int32_t on);
qk_status qk_aps_batch_stage_times(qk_aps_batch* plan, float* ms);
/* For the last batch (synchronous): per round, the items asked for and the
 * items Algorithm 1 took in (the rest were scanned beyond a query's stop);
 * arrays of the plan's round count. */
qk_status qk_aps_batch_round_stats(qk_aps_batch* plan, int64_t* asked, int64_t* taken);

/* SPANN's early-termination rule, the comparator of Sec. 2 "Early Termination"
 * and Table 6: query i scans the candidates of its set S (the same S as APS
 * builds: the ceil(f_M_leaf * n_leaf) nearest leaves with one level, the upper
 * level's APS result with two), nearest first, whose Euclidean centroid
 * distance is at most (1 + eps) times the nearest one's; eps > 0 is the rule's
 * tuned parameter.  out_nprobe[nq] (optional) receives the count scanned,
 * out_scanned0 (optional, nq x cap0) the leaves scanned, as in
 * qk_search_scanned.  Host or device buffers. */
qk_status qk_search_ratio(qk_index* index, const float* q, int64_t nq, int32_t k, float eps, int64_t* out_ids,
                          float* out_dist, int32_t* out_nprobe, int32_t* out_scanned0, int32_t cap0, void* stream);

/* Fixed-nprobe search with one nprobe per query through the per-query search
 * kernel (one CTA per query; the comparison point of the batched path and of
 * the per-query "oracle nprobe"): like qk_search with recall_target <= 0, but
 * query i scans the first nprobe[i] leaves of its candidate list S (with one
 * level: its nprobe[i] nearest leaves; with two: the upper level's APS result,
 * so at most ceil(f_M_leaf * n_leaf) leaves).  nprobe may be host or device
 * memory (read on the host: the call synchronises on a device array); every
 * value >= 1. */
qk_status qk_search_nprobe(qk_index* index, const float* q, int64_t nq, int32_t k, const int32_t* nprobe,
                           int64_t* out_ids, float* out_dist, void* stream);

/* ------------------------------------------------------------------------
 * The serving loop (continuous batching over one index; the paper serves
 * queries and updates together with maintenance beside them, Sec. 4 and
 * Sec. 8).  Callers submit searches, inserts and deletes from any host thread
 * and get a ticket per request; a scheduler thread owned by the server does
 * all GPU work through this ABI:
 *  - waiting searches launch together as one batch whenever one of `streams`
 *    slots is free (pinned staging, device buffers, one stream per slot), so
 *    batches overlap and new requests join the next free slot; a batch is held
 *    back while free device memory is below min_free_bytes;
 *  - updates wait until update_batch are pending or the oldest has waited
 *    update_wait_s, then the group is applied as its net effect (one delete
 *    call, one insert call) by the server's update thread on its own stream,
 *    while the scheduler keeps launching batches; every batch reads the
 *    version current at its launch (copy-on-write views);
 *  - every maintain_every requests a maintenance pass runs with *maint: with
 *    concurrent_maintenance it is prepared by a worker thread beside the
 *    searches (qk_maintain_prepare; updates wait meanwhile) and committed
 *    when ready, otherwise it runs in place; neither waits for the batches
 *    in flight.
 * A request's latency runs from its submission to the moment its result is in
 * host memory.  Inserted ids must be new (a duplicate fails the whole group and
 * stops the server).  The index must not be used directly while a server runs
 * on it.
 * ------------------------------------------------------------------------ */
typedef struct qk_server qk_server;

typedef struct {
  int32_t k;                       /* results per search (<= 1024) */
  float recall_target;             /* APS target of every search */
  int32_t max_batch;               /* searches per batch */
  int32_t streams;                 /* batch slots (1..16) */
  int64_t min_free_bytes;          /* admission: free device memory needed to launch a batch */
  int64_t maintain_every;          /* requests between maintenance passes (0: never) */
  int32_t update_batch;            /* pending updates that trigger a group */
  double update_wait_s;            /* longest wait of a pending update before its group is applied */
  int32_t concurrent_maintenance;  /* 1: prepare passes beside the searches */
  const qk_maint_params* maint;    /* pass parameters (copied; required when maintain_every > 0) */
  int32_t batched_from;            /* batches of at least this many searches run through each slot's
                                      batched APS plan (qk_aps_batch_*; FP32 L2 indexes with k <= 32),
                                      smaller ones through qk_search; 0 (default): always qk_search.
                                      The two give the same results bit for bit.  The plan's persistent
                                      kernels hold every SM for milliseconds, so update kernels wait
                                      behind them: several times the search throughput, at tens of
                                      milliseconds more update latency. */
} qk_server_config;

typedef struct {
  int64_t searches, inserts, deletes;   /* completed requests */
  int64_t batches, update_groups, maintenance_passes;
  double update_s;                      /* scheduler time spent draining and applying update groups */
  double maintenance_stall_s;           /* scheduler time spent draining and committing passes */
  double maintenance_prepare_s;         /* passes prepared beside the searches (wall time) */
} qk_server_stats;

void qk_server_config_default(qk_server_config* cfg);
/* Starts the scheduler thread on the current device.  Errors: QK_ERR_ARG,
 * QK_ERR_STATE (empty index), QK_ERR_CUDA / QK_ERR_OOM. */
qk_status qk_server_create(qk_index* index, const qk_server_config* cfg, qk_server** out);
/* Finishes every submitted request, stops the scheduler and frees the server. */
void qk_server_destroy(qk_server* server);
/* q / x: d FP32 host values, copied at submission.  Tickets count from 0 in
 * submission order.  QK_ERR_ARG (no ticket; the server keeps running) for a
 * vector with a NaN or infinite element or a squared norm beyond FP32, which
 * the kernels would refuse.  QK_ERR_STATE once the server stopped after an
 * error. */
qk_status qk_server_submit_search(qk_server* server, const float* q, int64_t* ticket);
qk_status qk_server_submit_insert(qk_server* server, const float* x, int64_t id, int64_t* ticket);
qk_status qk_server_submit_delete(qk_server* server, int64_t id, int64_t* ticket);
/* Open-loop playback of a request stream from the calling thread: request j
 * (kind 0 search, 1 insert, 2 delete; ref the id of an insert or delete; vec
 * n x d FP32, row j the query or the inserted vector) is submitted at t_s[j]
 * seconds after the call starts (t_s non-decreasing), as the submit calls
 * would, and its latency counts from that scheduled time.  lag_s (optional,
 * n) receives how late each submission was.  Returns once every request is
 * submitted (tickets continue from those already issued); errors as the
 * submit calls, for the first request that fails. */
qk_status qk_server_play(qk_server* server, int64_t n, const int8_t* kind, const int64_t* ref, const float* vec,
                         const double* t_s, double* lag_s);
/* Results of tickets [first, first + count): done flags, search results
 * (count x k ids and distances, -1 / +inf where not a search or not done) and
 * latencies in seconds (-1 where not done).  Any output may be NULL. */
qk_status qk_server_results(qk_server* server, int64_t first, int64_t count, int32_t* done, int64_t* ids,
                            float* dist, double* latency_s);
/* Waits until every request submitted so far is done and a maintenance pass
 * they made due has run (timeout_s <= 0: no limit; QK_ERR_TIMEOUT after it).
 * QK_ERR_STATE if the server stopped after an error (the message names it). */
qk_status qk_server_drain(qk_server* server, double timeout_s);
qk_status qk_server_get_stats(const qk_server* server, qk_server_stats* out);

#ifdef __cplusplus
}
#endif

#endif /* QUAKE_B300_H */
