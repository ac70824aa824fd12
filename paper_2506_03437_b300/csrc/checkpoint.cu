// Checkpoint and resume of an index (qk_save / qk_restore).  The paper has no
// counterpart: its indexes live in memory.  A checkpoint is one flat file of
// the state a search and a maintenance pass read, so a restored index answers
// and maintains exactly as the saved one did:
//   "QKB300CK", format 1, sizeof(qk_config), the configuration (with the
//   current partition counts), n, n_leaf, n_parent, the statistics window
//   |W| (queries seen), then
//   level 0: sizes[n_leaf] int32, centroids[n_leaf x d] FP32, ids[n] int64
//            and rows[n x d] FP32 grouped by partition; with BF16 / FP8
//            storage also the low-precision rows (same order) and the FP8
//            scale of every partition (1 for BF16);
//   level 1 (n_parent > 0): sizes[n_parent] int32, centroids[n_parent x d]
//            FP32, member leaves[n_leaf] int64 grouped by parent;
//   hits0[n_leaf], hits1[n_parent] uint64;
//   FNV-1a 64 of every byte after the magic.
// Host byte order.  The low-precision rows are stored rather than recomputed:
// rows inserted after the build carry their partition's scale at insert time,
// which re-quantizing would not reproduce.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "index.cuh"

namespace qk {
namespace {

constexpr char kMagic[8] = {'Q', 'K', 'B', '3', '0', '0', 'C', 'K'};
constexpr uint32_t kFormat = 1;

int row_bytes_lp(int storage) { return storage == QK_STORE_BF16 ? 2 : (storage == QK_STORE_FP8 ? 1 : 0); }

// FNV-1a, 64-bit (Fowler, Noll and Vo).
struct Fnv {
  uint64_t h = 0xcbf29ce484222325ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 0x100000001b3ull;
  }
};

struct Writer {
  FILE* f = nullptr;
  Fnv sum;
  bool ok = true;
  void put(const void* p, size_t n) {
    if (!n || !ok) return;
    sum.add(p, n);
    ok = std::fwrite(p, 1, n, f) == n;
  }
  template <class T>
  void val(const T& v) {
    put(&v, sizeof(T));
  }
};

struct Reader {
  FILE* f = nullptr;
  Fnv sum;
  bool ok = true;
  void get(void* p, size_t n) {
    if (!n || !ok) return;
    ok = std::fread(p, 1, n, f) == n;
    if (ok) sum.add(p, n);
  }
  template <class T>
  T val() {
    T v{};
    get(&v, sizeof(T));
    return v;
  }
};

struct FileGuard {
  FILE* f = nullptr;
  ~FileGuard() {
    if (f) std::fclose(f);
  }
};

qk_status io_error(const std::string& what) {
  set_error(what);
  return QK_ERR_IO;
}

}  // namespace
}  // namespace qk

using namespace qk;

static qk_status save_impl(qk_index* ix, const char* path) {
  if (!ix || !path) {
    set_error("qk_save: null argument");
    return QK_ERR_ARG;
  }
  if (!ix->ready) {
    set_error("qk_save: index is empty");
    return QK_ERR_STATE;
  }
  const int d = ix->cfg.d;
  const int32_t N0 = ix->n_leaf, N1 = ix->n_parent;
  const int64_t n = ix->n;
  const int lpb = row_bytes_lp(ix->cfg.storage);
  std::vector<int32_t> s0(N0), s1(N1);
  std::vector<float> c0((size_t)N0 * d), c1((size_t)N1 * d), x((size_t)n * d), sc(N0);
  std::vector<int64_t> id0(n), mem1(N1 > 0 ? N0 : 0);
  std::vector<uint8_t> lp(lpb ? (size_t)n * d * lpb : 0);
  std::vector<uint64_t> h0(N0), h1(N1);
  QK_TRY(qk_export_level(ix, 0, s0.data(), c0.data(), id0.data(), x.data()));
  if (N1 > 0) QK_TRY(qk_export_level(ix, 1, s1.data(), c1.data(), mem1.data(), nullptr));
  if (lpb) QK_TRY(qk_export_quantized(ix, lp.data(), sc.data()));
  QK_TRY(qk_get_hits(ix, 0, reinterpret_cast<int64_t*>(h0.data()), 0));
  if (N1 > 0) QK_TRY(qk_get_hits(ix, 1, reinterpret_cast<int64_t*>(h1.data()), 0));

  FileGuard g;
  g.f = std::fopen(path, "wb");
  if (!g.f) return io_error(std::string("qk_save: cannot open ") + path);
  if (std::fwrite(kMagic, 1, sizeof(kMagic), g.f) != sizeof(kMagic)) return io_error("qk_save: write failed");
  Writer w;
  w.f = g.f;
  qk_config cfg = ix->cfg;
  cfg.n_leaf = N0;
  cfg.n_parent = N1;
  w.val(kFormat);
  w.val((uint32_t)sizeof(qk_config));
  w.val(cfg);
  w.val(n);
  w.val(N0);
  w.val(N1);
  w.val((int64_t)ix->queries_seen.load());
  w.put(s0.data(), sizeof(int32_t) * s0.size());
  w.put(c0.data(), sizeof(float) * c0.size());
  w.put(id0.data(), sizeof(int64_t) * id0.size());
  w.put(x.data(), sizeof(float) * x.size());
  if (lpb) {
    w.put(lp.data(), lp.size());
    w.put(sc.data(), sizeof(float) * sc.size());
  }
  if (N1 > 0) {
    w.put(s1.data(), sizeof(int32_t) * s1.size());
    w.put(c1.data(), sizeof(float) * c1.size());
    w.put(mem1.data(), sizeof(int64_t) * mem1.size());
  }
  w.put(h0.data(), sizeof(uint64_t) * h0.size());
  w.put(h1.data(), sizeof(uint64_t) * h1.size());
  const uint64_t sum = w.sum.h;
  if (!w.ok || std::fwrite(&sum, 1, sizeof(sum), g.f) != sizeof(sum)) return io_error("qk_save: write failed");
  FILE* f = g.f;
  g.f = nullptr;
  if (std::fclose(f) != 0) return io_error("qk_save: close failed");
  return QK_OK;
}

static qk_status restore_impl(const char* path, qk_config* cfg_out, qk_index** out) {
  if (!path || !out) {
    set_error("qk_restore: null argument");
    return QK_ERR_ARG;
  }
  *out = nullptr;
  FileGuard g;
  g.f = std::fopen(path, "rb");
  if (!g.f) return io_error(std::string("qk_restore: cannot open ") + path);
  char magic[8];
  if (std::fread(magic, 1, sizeof(magic), g.f) != sizeof(magic) || std::memcmp(magic, kMagic, sizeof(magic)) != 0)
    return io_error("qk_restore: not an index checkpoint");
  Reader r;
  r.f = g.f;
  const uint32_t format = r.val<uint32_t>(), cbytes = r.val<uint32_t>();
  if (!r.ok || format != kFormat || cbytes != sizeof(qk_config))
    return io_error("qk_restore: unsupported checkpoint format");
  const qk_config cfg = r.val<qk_config>();
  const int64_t n = r.val<int64_t>();
  const int32_t N0 = r.val<int32_t>(), N1 = r.val<int32_t>();
  const int64_t seen = r.val<int64_t>();
  const int d = cfg.d;
  if (!r.ok || d < 1 || d > 4096 || n < 0 || N0 < 1 || N1 < 0 || N1 > N0 || cfg.n_leaf != N0 ||
      cfg.n_parent != N1 || n > (int64_t(1) << 40) / d)
    return io_error("qk_restore: invalid header");
  const int lpb = row_bytes_lp(cfg.storage);
  // the file must be exactly as long as its header says, before anything is allocated
  const long here = std::ftell(g.f);
  const double need = (double)here + 4.0 * N0 + 4.0 * N0 * d + 8.0 * n + 4.0 * n * d +
                      (lpb ? (double)n * d * lpb + 4.0 * N0 : 0.0) +
                      (N1 > 0 ? 4.0 * N1 + 4.0 * N1 * d + 8.0 * N0 : 0.0) + 8.0 * N0 + 8.0 * N1 + 8.0;
  if (here < 0 || std::fseek(g.f, 0, SEEK_END) != 0) return io_error("qk_restore: cannot seek");
  const long size = std::ftell(g.f);
  if (size < 0 || (double)size != need || std::fseek(g.f, here, SEEK_SET) != 0)
    return io_error("qk_restore: file size does not match its header (truncated or corrupt)");
  std::vector<int32_t> s0(N0), s1(N1);
  std::vector<float> c0((size_t)N0 * d), c1((size_t)N1 * d), x((size_t)n * d), sc(N0);
  std::vector<int64_t> id0(n), mem1(N1 > 0 ? N0 : 0);
  std::vector<uint8_t> lp(lpb ? (size_t)n * d * lpb : 0);
  std::vector<uint64_t> h0(N0), h1(N1);
  r.get(s0.data(), sizeof(int32_t) * s0.size());
  r.get(c0.data(), sizeof(float) * c0.size());
  r.get(id0.data(), sizeof(int64_t) * id0.size());
  r.get(x.data(), sizeof(float) * x.size());
  if (lpb) {
    r.get(lp.data(), lp.size());
    r.get(sc.data(), sizeof(float) * sc.size());
  }
  if (N1 > 0) {
    r.get(s1.data(), sizeof(int32_t) * s1.size());
    r.get(c1.data(), sizeof(float) * c1.size());
    r.get(mem1.data(), sizeof(int64_t) * mem1.size());
  }
  r.get(h0.data(), sizeof(uint64_t) * h0.size());
  r.get(h1.data(), sizeof(uint64_t) * h1.size());
  uint64_t sum = 0;
  if (!r.ok || std::fread(&sum, 1, sizeof(sum), g.f) != sizeof(sum)) return io_error("qk_restore: truncated checkpoint");
  if (sum != r.sum.h) return io_error("qk_restore: checksum mismatch");

  // labels from the grouping; every count must add up
  std::vector<int32_t> leaf_of_row(n), parent_of_leaf(N1 > 0 ? N0 : 0);
  int64_t o = 0;
  for (int32_t j = 0; j < N0; ++j) {
    if (s0[j] < 0 || o + s0[j] > n) return io_error("qk_restore: inconsistent partition sizes");
    for (int32_t t = 0; t < s0[j]; ++t) leaf_of_row[o++] = j;
  }
  if (o != n) return io_error("qk_restore: inconsistent partition sizes");
  if (N1 > 0) {
    int64_t m = 0;
    for (int32_t p = 0; p < N1; ++p) {
      if (s1[p] < 0 || m + s1[p] > N0) return io_error("qk_restore: inconsistent parent sizes");
      for (int32_t t = 0; t < s1[p]; ++t, ++m) {
        const int64_t lf = mem1[m];
        if (lf < 0 || lf >= N0) return io_error("qk_restore: invalid member leaf");
        parent_of_leaf[lf] = p;
      }
    }
    if (m != N0) return io_error("qk_restore: inconsistent parent sizes");
  }

  qk_index* ix = nullptr;
  QK_TRY(qk_create(&cfg, &ix));
  qk_status st = qk_load(ix, x.data(), id0.data(), n, c0.data(), leaf_of_row.data(), N1 > 0 ? c1.data() : nullptr,
                         N1 > 0 ? parent_of_leaf.data() : nullptr, nullptr);
  if (st == QK_OK && lpb) {
    // the stored low-precision rows, placed by id where the load put each row
    std::vector<int64_t> now(n);
    st = qk_export_level(ix, 0, nullptr, nullptr, now.data(), nullptr);
    std::unordered_map<int64_t, int64_t> at;
    at.reserve((size_t)n * 2);
    for (int64_t i = 0; i < n; ++i) at.emplace(id0[i], i);
    std::vector<uint8_t> placed(lp.size());
    const size_t rb = (size_t)d * lpb;
    for (int64_t i = 0; st == QK_OK && i < n; ++i) {
      auto it = at.find(now[i]);
      if (it == at.end()) {
        set_error("qk_restore: row order could not be matched");
        st = QK_ERR_INTERNAL;
        break;
      }
      std::memcpy(placed.data() + (size_t)i * rb, lp.data() + (size_t)it->second * rb, rb);
    }
    int64_t base = 0;
    for (int32_t j = 0; st == QK_OK && j < N0; ++j) {
      const size_t rows = (size_t)ix->h_size0[j];
      if (rows) {
        cudaError_t e = cudaMemcpy(ix->lp0 + ix->h_off0[j] * rb, placed.data() + (size_t)base * rb, rows * rb,
                                   cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_status(e, "qk_restore: codes");
      }
      base += (int64_t)rows;
    }
    if (st == QK_OK && cfg.storage == QK_STORE_FP8) {
      cudaError_t e = cudaMemcpy(ix->lp_scale0, sc.data(), sizeof(float) * N0, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) st = cuda_status(e, "qk_restore: scales");
    }
  }
  if (st == QK_OK) {
    cudaError_t e = cudaMemcpy(ix->hits0, h0.data(), sizeof(uint64_t) * N0, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && N1 > 0) e = cudaMemcpy(ix->hits1, h1.data(), sizeof(uint64_t) * N1, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_status(e, "qk_restore: statistics");
  }
  if (st != QK_OK) {
    qk_destroy(ix);
    return st;
  }
  ix->queries_seen = seen;
  if (cfg_out) *cfg_out = cfg;
  *out = ix;
  return QK_OK;
}

extern "C" qk_status qk_save(qk_index* ix, const char* path) {
  try {
    return save_impl(ix, path);   // its reads (qk_export_level, qk_get_hits) lock for themselves
  } catch (const std::bad_alloc&) {
    set_error("qk_save: out of host memory");
    return QK_ERR_OOM;
  }
}

extern "C" qk_status qk_restore(const char* path, qk_config* cfg_out, qk_index** out) {
  try {
    return restore_impl(path, cfg_out, out);
  } catch (const std::bad_alloc&) {
    set_error("qk_restore: out of host memory");
    return QK_ERR_OOM;
  }
}
