// Copy-on-write views of the index (Sec. 9, "Concurrency": readers keep the
// view they started on while an update builds the next one).
//
// A search launch captures the arena and partition-table pointers of the
// version current at launch.  An update writes only rows and tables that no
// published version reads, publishes its new table by exchanging pointers,
// and retires what the older versions used.  Every search launch records a
// completion event tagged with the version it reads; retired memory goes
// back to the free pools once every search of a version up to the retiring
// one has completed.  Nothing here waits for a search in flight unless asked
// (reclaim with wait, on destroy).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <limits>
#include <unordered_map>

#include "common.cuh"
#include "index.cuh"

namespace qk {

// The device's private stream for the index memory: allocations and frees
// are stream-ordered on it, so freeing an old version's arena does not wait
// for the rest of the device, which a cudaFree would.
static cudaStream_t mem_stream() {
  static std::mutex mu;
  static std::unordered_map<int, cudaStream_t> streams;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  streams.emplace(dev, s);
  return s;
}

qk_status mem_alloc(void** p, size_t bytes) {
  *p = nullptr;
  cudaStream_t ms = mem_stream();
  if (!ms) {
    set_error("no stream for the index memory");
    return QK_ERR_CUDA;
  }
  QK_CUDA(cudaMallocAsync(p, std::max<size_t>(bytes, 256), ms));
  QK_CUDA(cudaStreamSynchronize(ms));   // usable from every stream from here on
  return QK_OK;
}

void mem_free(void* p) {
  if (!p) return;
  if (cudaFreeAsync(p, mem_stream()) != cudaSuccess) cudaGetLastError();
}

uint64_t next_arena_id() {
  static std::atomic<uint64_t> next{1};
  return next.fetch_add(1);
}

// Drops the readers whose events have completed (view_mu held).
static void sweep_readers(qk_index* ix) {
  size_t w = 0;
  for (size_t i = 0; i < ix->readers.size(); ++i) {
    cudaError_t e = cudaEventQuery(ix->readers[i].ev);
    if (e == cudaErrorNotReady) {
      ix->readers[w++] = ix->readers[i];
    } else {
      if (e != cudaSuccess) cudaGetLastError();   // an error of the search itself surfaces in its own status
      ix->idle_events.push_back(ix->readers[i].ev);
    }
  }
  ix->readers.resize(w);
}

void note_readers(qk_index* ix, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    cs = cudaStreamCaptureStatusNone;
  }
  if (cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> g(ix->view_mu);
  // drop the oldest readers that have completed; a full sweep only when many
  // are listed (searches on several streams complete out of order)
  if (ix->readers.size() > 4096) {
    sweep_readers(ix);
  } else {
    size_t done = 0;
    while (done < ix->readers.size() && done < 16) {
      const cudaError_t e = cudaEventQuery(ix->readers[done].ev);
      if (e == cudaErrorNotReady) break;
      if (e != cudaSuccess) cudaGetLastError();
      ix->idle_events.push_back(ix->readers[done].ev);
      ++done;
    }
    ix->readers.erase(ix->readers.begin(), ix->readers.begin() + done);
  }
  cudaEvent_t ev = nullptr;
  if (!ix->idle_events.empty()) {
    ev = ix->idle_events.back();
    ix->idle_events.pop_back();
  } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    // no event to track the launch: let it finish now instead
    cudaGetLastError();
    cudaStreamSynchronize(s);
    return;
  }
  if (cudaEventRecord(ev, s) != cudaSuccess) {
    cudaGetLastError();
    ix->idle_events.push_back(ev);
    cudaStreamSynchronize(s);
    return;
  }
  ix->readers.push_back(ViewReader{ev, ix->version});
}

// Gives a free row range back to free0, merged with its neighbours; a range
// that ends at the free tail shortens the used part instead.
static void give_rows(qk_index* ix, int64_t first, int64_t rows) {
  if (rows <= 0) return;
  auto next = ix->free0.lower_bound(first);
  if (next != ix->free0.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == first) {
      first = prev->first;
      rows += prev->second;
      ix->free0.erase(prev);
    }
  }
  next = ix->free0.lower_bound(first);
  if (next != ix->free0.end() && first + rows == next->first) {
    rows += next->second;
    ix->free0.erase(next);
  }
  if (first + rows == ix->used0) {
    ix->used0 = first;
    ix->holes0 -= rows;
    return;
  }
  ix->free0[first] = rows;
}

static void release(qk_index* ix, Retired& r) {
  if (r.arena == ix->arena_id)
    for (auto& rg : r.rows) give_rows(ix, rg.first, rg.second);
  if (r.table.off) {
    if (r.table.n == ix->n_leaf) {
      ix->spare0.push_back(r.table);
    } else {
      mem_free(r.table.off);
      mem_free(r.table.size);
    }
  }
  for (void* p : r.device) mem_free(p);
  if (r.structure) {
    release_structure(r.structure);
    delete r.structure;
  }
  r = Retired{};
}

void reclaim(qk_index* ix, bool wait) {
  std::lock_guard<std::mutex> g(ix->view_mu);
  if (wait)
    for (auto& rd : ix->readers) cudaEventSynchronize(rd.ev);
  sweep_readers(ix);
  uint64_t live = std::numeric_limits<uint64_t>::max();   // oldest version a search in flight reads
  for (auto& rd : ix->readers) live = std::min(live, rd.version);
  size_t w = 0;
  for (size_t i = 0; i < ix->retired.size(); ++i) {
    if (ix->retired[i].version < live) {
      release(ix, ix->retired[i]);
    } else {
      if (w != i) ix->retired[w] = std::move(ix->retired[i]);
      ++w;
    }
  }
  ix->retired.resize(w);
  if (wait) {
    for (cudaEvent_t ev : ix->idle_events) cudaEventDestroy(ev);
    ix->idle_events.clear();
  }
}

void retire(qk_index* ix, Retired&& r) {
  std::lock_guard<std::mutex> g(ix->view_mu);
  ix->retired.push_back(std::move(r));
}

void retire_structure(qk_index* ix) {
  qk_index* old = new qk_index();
  old->cfg = ix->cfg;
  old->device = ix->device;
  swap_structure(ix, old);
  Retired r;
  r.version = ix->version;
  r.structure = old;
  retire(ix, std::move(r));
}

int64_t readers_in_flight(qk_index* ix) {
  std::lock_guard<std::mutex> g(ix->view_mu);
  sweep_readers(ix);
  return (int64_t)ix->readers.size();
}

int64_t retired_rows(qk_index* ix) {
  std::lock_guard<std::mutex> g(ix->view_mu);
  int64_t n = 0;
  for (auto& r : ix->retired)
    if (r.arena == ix->arena_id)
      for (auto& rg : r.rows) n += rg.second;
  return n;
}

int64_t take_rows(qk_index* ix, int64_t rows) {
  auto best = ix->free0.end();
  for (auto it = ix->free0.begin(); it != ix->free0.end(); ++it)
    if (it->second >= rows && (best == ix->free0.end() || it->second < best->second)) best = it;
  if (best != ix->free0.end()) {
    const int64_t first = best->first, left = best->second - rows;
    ix->free0.erase(best);
    if (left > 0) ix->free0[first + rows] = left;
    ix->holes0 -= rows;
    return first;
  }
  if (ix->used0 + rows <= ix->cap0) {
    const int64_t first = ix->used0;
    ix->used0 += rows;
    return first;
  }
  return -1;
}

qk_status take_table(qk_index* ix, Table* t) {
  while (!ix->spare0.empty()) {
    Table s = ix->spare0.back();
    ix->spare0.pop_back();
    if (s.n == ix->n_leaf) {
      *t = s;
      return QK_OK;
    }
    mem_free(s.off);
    mem_free(s.size);
  }
  Table s;
  s.n = ix->n_leaf;
  const size_t n = (size_t)std::max(ix->n_leaf, 1);
  QK_TRY(mem_alloc(reinterpret_cast<void**>(&s.off), sizeof(int64_t) * n));
  const qk_status st = mem_alloc(reinterpret_cast<void**>(&s.size), sizeof(int32_t) * n);
  if (st != QK_OK) {
    mem_free(s.off);
    return st;
  }
  *t = s;
  return QK_OK;
}

}  // namespace qk
