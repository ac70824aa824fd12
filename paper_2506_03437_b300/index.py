"""Python face of the C ABI: an `Index` object over qk_* calls.

Marshalling only: arrays are checked for dtype and contiguity and their
addresses handed to the CUDA library.  Outputs go to the device of the query
tensor (CUDA tensors in -> CUDA tensors out, stream-ordered) or to numpy
arrays for host inputs.
"""

import ctypes as C
import os

import numpy as np

from . import _lib as L


def _as(a, dtype):
    """numpy array or torch tensor, C-contiguous with the given numpy dtype."""
    if hasattr(a, "data_ptr"):
        import torch
        tdt = {np.float32: torch.float32, np.int64: torch.int64, np.int32: torch.int32,
               np.float64: torch.float64}[dtype]
        if a.dtype != tdt:
            raise TypeError(f"expected {tdt}, got {a.dtype}")
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def config(d, metric=L.METRIC_L2, n_leaf=1000, n_parent=0, kmeans_iters=10, beta_mode=L.BETA_TABLE,
           seed=1234, f_M_leaf=0.1, f_M_parent=0.25, tau_rho=0.01, upper_recall=0.99, storage=L.STORE_F32,
           rerank=4):
    c = L.QkConfig()
    L.lib.qk_config_default(C.byref(c))
    c.d, c.metric, c.n_leaf, c.n_parent = d, metric, n_leaf, n_parent
    c.kmeans_iters, c.beta_mode, c.seed = kmeans_iters, beta_mode, seed
    c.f_M_leaf, c.f_M_parent, c.tau_rho, c.upper_recall = f_M_leaf, f_M_parent, tau_rho, upper_recall
    c.storage, c.rerank = storage, rerank
    return c


def profile_scan(d, sizes, k=10, reps=3, stream=None, **cfg):
    """lambda(s) of the cost model measured on the current device (qk_profile_scan): microseconds
    of device time one more scanned partition of s rows adds per (query, partition) item, for the
    configuration's dimension, metric and storage.  Returns a float64 array beside `sizes`."""
    return _profile(config(d, **cfg), sizes, k, reps, stream)


def _profile(c, sizes, k, reps, stream):
    sz = np.ascontiguousarray(sizes, dtype=np.int64)
    out = np.empty(sz.shape[0], np.float64)
    L.check(L.lib.qk_profile_scan(C.byref(c), int(k), L.ptr(sz), int(sz.shape[0]), int(reps), L.ptr(out),
                                  L.stream_ptr(stream)))
    return out


class Index:
    """A Quake index on the current CUDA device (see include/quake_b300.h)."""

    def __init__(self, d, **kw):
        self.cfg = config(d, **kw)
        h = C.c_void_p()
        L.check(L.lib.qk_create(C.byref(self.cfg), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            L.lib.qk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def d(self):
        return self.cfg.d

    def build(self, x, ids, stream=None):
        x, ids = _as(x, np.float32), _as(ids, np.int64)
        L.check(L.lib.qk_build(self._h, L.ptr(x), L.ptr(ids), int(ids.shape[0]), L.stream_ptr(stream)))

    def load(self, x, ids, leaf_centroids, leaf_of_row, parent_centroids=None, parent_of_leaf=None,
             stream=None):
        x, ids = _as(x, np.float32), _as(ids, np.int64)
        c0, a0 = _as(leaf_centroids, np.float32), _as(leaf_of_row, np.int32)
        c1 = None if parent_centroids is None else _as(parent_centroids, np.float32)
        a1 = None if parent_of_leaf is None else _as(parent_of_leaf, np.int32)
        L.check(L.lib.qk_load(self._h, L.ptr(x), L.ptr(ids), int(ids.shape[0]), L.ptr(c0), L.ptr(a0),
                              L.ptr(c1), L.ptr(a1), L.stream_ptr(stream)))

    def set_search_upper(self, mode):
        """Where search walks the upper levels: -1 auto, 0 in each query's CTA, 1 a
        warp-per-query prepare kernel first (the same results either way)."""
        L.check(L.lib.qk_set_search_upper(self._h, int(mode)))

    def search(self, q, k, recall_target=0.9, nprobe=0, out=None, stream=None):
        """Returns (ids, dist, nprobe, recall_estimate) on the device of `q`."""
        q = _as(q, np.float32)
        nq = int(q.shape[0])
        if out is None:
            if hasattr(q, "data_ptr"):
                import torch
                dev = q.device
                out = (torch.empty((nq, k), dtype=torch.int64, device=dev),
                       torch.empty((nq, k), dtype=torch.float32, device=dev),
                       torch.empty(nq, dtype=torch.int32, device=dev),
                       torch.empty(nq, dtype=torch.float32, device=dev))
            else:
                out = (np.empty((nq, k), np.int64), np.empty((nq, k), np.float32),
                       np.empty(nq, np.int32), np.empty(nq, np.float32))
        oi, od, on, orr = out
        L.check(L.lib.qk_search(self._h, L.ptr(q), nq, int(k), float(recall_target), int(nprobe),
                                L.ptr(oi), L.ptr(od), L.ptr(on), L.ptr(orr), L.stream_ptr(stream)))
        return out

    def search_scanned(self, q, k, recall_target=0.9, nprobe=0, cap0=64, cap1=64, stream=None):
        """search() plus each query's scanned partitions in scan order: returns
        (ids, dist, nprobe, recall_estimate, scanned0 (nq x cap0), scanned1
        (nq x cap1)), -1 padded, on the device of `q`."""
        q = _as(q, np.float32)
        nq = int(q.shape[0])
        if hasattr(q, "data_ptr"):
            import torch
            dev = q.device
            out = (torch.empty((nq, k), dtype=torch.int64, device=dev),
                   torch.empty((nq, k), dtype=torch.float32, device=dev),
                   torch.empty(nq, dtype=torch.int32, device=dev),
                   torch.empty(nq, dtype=torch.float32, device=dev),
                   torch.empty((nq, cap0), dtype=torch.int32, device=dev),
                   torch.empty((nq, cap1), dtype=torch.int32, device=dev))
        else:
            out = (np.empty((nq, k), np.int64), np.empty((nq, k), np.float32),
                   np.empty(nq, np.int32), np.empty(nq, np.float32),
                   np.empty((nq, cap0), np.int32), np.empty((nq, cap1), np.int32))
        oi, od, on, orr, s0, s1 = out
        L.check(L.lib.qk_search_scanned(self._h, L.ptr(q), nq, int(k), float(recall_target), int(nprobe),
                                        L.ptr(oi), L.ptr(od), L.ptr(on), L.ptr(orr), L.ptr(s0), int(cap0),
                                        L.ptr(s1), int(cap1), L.stream_ptr(stream)))
        return out

    def stats(self):
        """Index statistics (qk_stats) as a dict."""
        st = L.QkIndexStats()
        L.check(L.lib.qk_stats(self._h, C.byref(st)))
        out = {name: getattr(st, name) for name, _ in L.QkIndexStats._fields_}
        out["n_partitions"] = list(st.n_partitions)
        out["hits"] = list(st.hits)
        return out

    def search_ratio(self, q, k, eps, cap0=0, stream=None):
        """SPANN's early-termination rule (qk_search_ratio): returns (ids, dist,
        nprobe[, scanned0]) on the device of `q`."""
        q = _as(q, np.float32)
        nq = int(q.shape[0])
        if hasattr(q, "data_ptr"):
            import torch
            dev = q.device
            out = (torch.empty((nq, k), dtype=torch.int64, device=dev),
                   torch.empty((nq, k), dtype=torch.float32, device=dev),
                   torch.empty(nq, dtype=torch.int32, device=dev))
            if cap0:
                out = out + (torch.empty((nq, cap0), dtype=torch.int32, device=dev),)
        else:
            out = (np.empty((nq, k), np.int64), np.empty((nq, k), np.float32), np.empty(nq, np.int32))
            if cap0:
                out = out + (np.empty((nq, cap0), np.int32),)
        s0 = out[3] if cap0 else None
        L.check(L.lib.qk_search_ratio(self._h, L.ptr(q), nq, int(k), float(eps), L.ptr(out[0]), L.ptr(out[1]),
                                      L.ptr(out[2]), L.ptr(s0), int(cap0), L.stream_ptr(stream)))
        return out

    def search_nprobe(self, q, k, nprobe, out=None, stream=None):
        """Fixed-nprobe search, one nprobe per query, through the per-query kernel.
        Returns (ids, dist) on the device of `q`."""
        q = _as(q, np.float32)
        nprobe = _as(nprobe, np.int32)
        nq = int(q.shape[0])
        if out is None:
            if hasattr(q, "data_ptr"):
                import torch
                out = (torch.empty((nq, k), dtype=torch.int64, device=q.device),
                       torch.empty((nq, k), dtype=torch.float32, device=q.device))
            else:
                out = (np.empty((nq, k), np.int64), np.empty((nq, k), np.float32))
        L.check(L.lib.qk_search_nprobe(self._h, L.ptr(q), nq, int(k), L.ptr(nprobe), L.ptr(out[0]), L.ptr(out[1]),
                                       L.stream_ptr(stream)))
        return out

    def _maint(self, fn, lam_sizes, lam_us, tau_us, alpha, refine_radius, refine_iters, split_iters, s_min, refine,
               window, stream, level_band=False, level_iters=10):
        ls = np.ascontiguousarray(lam_sizes, np.float64)
        lu = np.ascontiguousarray(lam_us, np.float64)
        p = L.QkMaintParams()
        p.lambda_sizes = ls.ctypes.data_as(C.POINTER(C.c_double))
        p.lambda_us = lu.ctypes.data_as(C.POINTER(C.c_double))
        p.lambda_points = int(ls.shape[0])
        p.refine_radius, p.refine_iters, p.split_iters = refine_radius, refine_iters, split_iters
        p.s_min, p.refine, p.tau_us, p.alpha, p.window = s_min, int(bool(refine)), tau_us, alpha, window
        p.level_band, p.level_iters = int(bool(level_band)), level_iters
        cap = 1 << 16
        log = (L.QkMaintAction * cap)()
        n = C.c_int32()
        L.check(fn(self._h, C.byref(p), log, cap, C.byref(n), L.stream_ptr(stream)))
        kinds = ("split", "merge", "add_level", "remove_level", "rebuild_level")
        return [dict(level=a.level, kind=kinds[a.kind], partition=a.partition,
                     committed=bool(a.committed), estimate=a.estimate, delta=a.delta)
                for a in log[:min(n.value, cap)]]

    def maintain(self, lam_sizes, lam_us, tau_us=0.25, alpha=0.9, refine_radius=50, refine_iters=1,
                 split_iters=10, s_min=0, refine=True, window=0, stream=None, level_band=False, level_iters=10):
        """Runs the maintenance pass; returns the list of considered actions as dicts."""
        return self._maint(L.lib.qk_maintain, lam_sizes, lam_us, tau_us, alpha, refine_radius, refine_iters,
                           split_iters, s_min, refine, window, stream, level_band, level_iters)

    def maintain_prepare(self, lam_sizes, lam_us, tau_us=0.25, alpha=0.9, refine_radius=50, refine_iters=1,
                         split_iters=10, s_min=0, refine=True, window=0, stream=None, level_band=False,
                         level_iters=10):
        """Plans the pass and builds its partitions aside (searches may run meanwhile);
        returns the action list.  maintain_commit() then installs it."""
        return self._maint(L.lib.qk_maintain_prepare, lam_sizes, lam_us, tau_us, alpha, refine_radius,
                           refine_iters, split_iters, s_min, refine, window, stream, level_band, level_iters)

    def save(self, path):
        """Writes a checkpoint of the index to `path` (qk_save)."""
        L.check(L.lib.qk_save(self._h, os.fsencode(path)))

    @classmethod
    def restore(cls, path):
        """An index on the current device from a checkpoint written by save() (qk_restore)."""
        cfg = L.QkConfig()
        h = C.c_void_p()
        L.check(L.lib.qk_restore(os.fsencode(path), C.byref(cfg), C.byref(h)))
        ix = cls.__new__(cls)
        ix.cfg, ix._h = cfg, h
        return ix

    def profile_scan(self, sizes, k=10, reps=3, stream=None):
        """lambda(s) for this index's dimension, metric and storage (see profile_scan)."""
        return _profile(self.cfg, sizes, k, reps, stream)

    def maintain_commit(self, stream=None):
        L.check(L.lib.qk_maintain_commit(self._h, L.stream_ptr(stream)))

    def check(self, stream=None):
        """Waits for this index's kernels on `stream`; raises if a device check failed."""
        L.check(L.lib.qk_check(self._h, L.stream_ptr(stream)))

    def info(self):
        n = C.c_int64()
        n0, n1, d = C.c_int32(), C.c_int32(), C.c_int32()
        L.check(L.lib.qk_info(self._h, C.byref(n), C.byref(n0), C.byref(n1), C.byref(d)))
        return dict(n=n.value, n_leaf=n0.value, n_parent=n1.value, d=d.value)

    def export_level(self, level, vectors=False):
        """(sizes, centroids, ids grouped by partition[, vectors]) of one level, as numpy."""
        inf = self.info()
        nparts = inf["n_leaf"] if level == 0 else inf["n_parent"]
        nrows = inf["n"] if level == 0 else inf["n_leaf"]
        sizes = np.empty(nparts, np.int32)
        cents = np.empty((nparts, self.d), np.float32)
        ids = np.empty(nrows, np.int64)
        vec = np.empty((nrows, self.d), np.float32) if vectors else None
        L.check(L.lib.qk_export_level(self._h, level, L.ptr(sizes), L.ptr(cents), L.ptr(ids), L.ptr(vec)))
        return (sizes, cents, ids, vec) if vectors else (sizes, cents, ids)

    def export_quantized(self):
        """(codes grouped like export_level's ids, scale per partition) of the low-precision copy."""
        inf = self.info()
        eb = 2 if self.cfg.storage == L.STORE_BF16 else 1
        codes = np.empty((inf["n"], self.d * eb), np.uint8)
        scales = np.empty(inf["n_leaf"], np.float32)
        L.check(L.lib.qk_export_quantized(self._h, L.ptr(codes), L.ptr(scales)))
        if eb == 2:
            codes = codes.view(np.uint16)
        return codes, scales

    def insert(self, x, ids, stream=None):
        x, ids = _as(x, np.float32), _as(ids, np.int64)
        L.check(L.lib.qk_insert(self._h, L.ptr(x), L.ptr(ids), int(ids.shape[0]), L.stream_ptr(stream)))

    def delete(self, ids, stream=None):
        """Removes the given ids; returns how many were present."""
        ids = _as(ids, np.int64)
        n = C.c_int64()
        L.check(L.lib.qk_delete(self._h, L.ptr(ids), int(ids.shape[0]), C.byref(n), L.stream_ptr(stream)))
        return n.value

    def hits(self, level=0, reset=False):
        inf = self.info()
        n = inf["n_leaf"] if level == 0 else inf["n_parent"]
        h = np.empty(n, np.int64)
        L.check(L.lib.qk_get_hits(self._h, level, L.ptr(h), 1 if reset else 0))
        return h


def cap_fraction(d, t, rho, mode=L.BETA_EXACT):
    """GPU FP64 cap volume fraction for arrays t, rho (host numpy in, numpy out)."""
    t = np.ascontiguousarray(t, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    out = np.empty_like(t)
    L.check(L.lib.qk_cap_fraction(int(d), int(mode), L.ptr(t), L.ptr(rho), int(t.shape[0]), L.ptr(out), None))
    return out


def kmeans_step(x, c):
    """One GPU Lloyd step: (new centroids, assignment, counts) as numpy."""
    x = np.ascontiguousarray(x, np.float32)
    c = np.ascontiguousarray(c, np.float32)
    n, d = x.shape
    K = c.shape[0]
    cn = np.empty_like(c)
    a = np.empty(n, np.int32)
    cnt = np.empty(K, np.int32)
    L.check(L.lib.qk_kmeans_step(L.ptr(x), n, d, L.ptr(c), K, L.ptr(cn), L.ptr(a), L.ptr(cnt), None))
    return cn, a, cnt


def nearest_centroids(x, c, k, metric=L.METRIC_L2):
    """The k nearest centroids of every row (tensor-core scoring + exact FP32 re-score), as numpy."""
    x = np.ascontiguousarray(x, np.float32)
    c = np.ascontiguousarray(c, np.float32)
    n, d = x.shape
    idx = np.empty((n, k), np.int32)
    dist = np.empty((n, k), np.float32)
    L.check(L.lib.qk_nearest_centroids(L.ptr(x), n, d, L.ptr(c), c.shape[0], metric, k, L.ptr(idx), L.ptr(dist), None))
    return idx, dist


class BatchPlan:
    """Workspace and tile shapes of the batched fixed-nprobe search of one index
    (qk_batch_* in include/quake_b300.h).  Every array is a CUDA tensor."""

    def __init__(self, index, max_nq, k, max_nprobe):
        h = C.c_void_p()
        L.check(L.lib.qk_batch_create(index._h, int(max_nq), int(k), int(max_nprobe), C.byref(h)))
        self._h, self.index, self.k = h, index, int(k)

    def close(self):
        if getattr(self, "_h", None):
            L.lib.qk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def tiles(self):
        t = L.QkBatchTiles()
        L.check(L.lib.qk_batch_get_tiles(self._h, C.byref(t)))
        return (t.queries_per_warp, t.tile_rows, t.chunk_rows, t.rows_per_thread)

    @tiles.setter
    def tiles(self, v):
        t = L.QkBatchTiles(*[int(x) for x in v])
        L.check(L.lib.qk_batch_set_tiles(self._h, C.byref(t)))

    def _out(self, q, out):
        if out is not None:
            return out
        import torch
        nq = int(q.shape[0])
        return (torch.empty((nq, self.k), dtype=torch.int64, device=q.device),
                torch.empty((nq, self.k), dtype=torch.float32, device=q.device))

    def search(self, q, nprobe, out=None, stream=None):
        """(ids, dist) of the batch; q (nq x d FP32) and nprobe (nq int32) on the GPU."""
        q, nprobe = _as(q, np.float32), _as(nprobe, np.int32)
        out = self._out(q, out)
        L.check(L.lib.qk_batch_search(self._h, L.ptr(q), int(q.shape[0]), L.ptr(nprobe), L.ptr(out[0]),
                                      L.ptr(out[1]), L.stream_ptr(stream)))
        return out

    def capture(self, q, nprobe, out, stream):
        """Records one batch over these buffers as a CUDA graph on `stream`."""
        q, nprobe = _as(q, np.float32), _as(nprobe, np.int32)
        L.check(L.lib.qk_batch_capture(self._h, L.ptr(q), int(q.shape[0]), L.ptr(nprobe), L.ptr(out[0]),
                                       L.ptr(out[1]), L.stream_ptr(stream)))

    def replay(self, stream):
        L.check(L.lib.qk_batch_replay(self._h, L.stream_ptr(stream)))

    STAGES = ("scoring", "selection", "grouping", "scan", "merge")

    def set_timing(self, on=True):
        L.check(L.lib.qk_batch_set_timing(self._h, 1 if on else 0))

    def stage_times(self):
        """Milliseconds of each step of the last timed batch (waits for it)."""
        ms = np.zeros(5, np.float32)
        L.check(L.lib.qk_batch_stage_times(self._h, L.ptr(ms)))
        return dict(zip(self.STAGES, ms.tolist()))

    def autotune(self, q, nprobe, out=None, reps=2, stream=None):
        """Times every valid tile shape on this batch and keeps the fastest; returns it."""
        q, nprobe = _as(q, np.float32), _as(nprobe, np.int32)
        out = self._out(q, out)
        t = L.QkBatchTiles()
        L.check(L.lib.qk_batch_autotune(self._h, L.ptr(q), int(q.shape[0]), L.ptr(nprobe), L.ptr(out[0]),
                                        L.ptr(out[1]), int(reps), C.byref(t), L.stream_ptr(stream)))
        return (t.queries_per_warp, t.tile_rows, t.chunk_rows, t.rows_per_thread)


class ApsBatchPlan:
    """Workspace of the batched APS search of one index (qk_aps_batch_* in
    include/quake_b300.h): Algorithm 1 for every query of a batch, with the
    leaf scans grouped by partition.  Every array is a CUDA tensor."""

    def __init__(self, index, max_nq, k, rounds=None):
        h = C.c_void_p()
        L.check(L.lib.qk_aps_batch_create(index._h, int(max_nq), int(k), C.byref(h)))
        self._h, self.index, self.k = h, index, int(k)
        self.rounds = 4
        if rounds is not None:
            self.set_rounds(rounds)

    def close(self):
        if getattr(self, "_h", None):
            L.lib.qk_aps_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_rounds(self, rounds):
        L.check(L.lib.qk_aps_batch_set_rounds(self._h, int(rounds)))
        self.rounds = int(rounds)

    def set_tiles(self, queries_per_warp, tile_rows, chunk_rows, rows_per_thread=0):
        t = L.QkBatchTiles(int(queries_per_warp), int(tile_rows), int(chunk_rows), int(rows_per_thread))
        L.check(L.lib.qk_aps_batch_set_tiles(self._h, C.byref(t)))

    def autotune(self, q, recall_target=0.9, out=None, reps=3, stream=None):
        """Times the valid tile shapes on this batch (all give the same results) and keeps
        the fastest; returns (queries_per_warp, tile_rows, chunk_rows, rows_per_thread)."""
        q = _as(q, np.float32)
        out = self.outputs(q) if out is None else out
        t = L.QkBatchTiles()
        L.check(L.lib.qk_aps_batch_autotune(self._h, L.ptr(q), int(q.shape[0]), float(recall_target),
                                            L.ptr(out[0]), L.ptr(out[1]), int(reps), C.byref(t),
                                            L.stream_ptr(stream)))
        return (t.queries_per_warp, t.tile_rows, t.chunk_rows, t.rows_per_thread)

    def outputs(self, q, cap0=0):
        """(ids, dist, nprobe, recall_estimate[, scanned0]) CUDA tensors for q's batch."""
        import torch
        nq, dev = int(q.shape[0]), q.device
        out = (torch.empty((nq, self.k), dtype=torch.int64, device=dev),
               torch.empty((nq, self.k), dtype=torch.float32, device=dev),
               torch.empty(nq, dtype=torch.int32, device=dev),
               torch.empty(nq, dtype=torch.float32, device=dev))
        if cap0:
            out = out + (torch.empty((nq, cap0), dtype=torch.int32, device=dev),)
        return out

    def search(self, q, recall_target=0.9, out=None, cap0=0, stream=None):
        """Returns (ids, dist, nprobe, recall_estimate[, scanned0]) of the batch."""
        q = _as(q, np.float32)
        out = self.outputs(q, cap0) if out is None else out
        s0 = out[4] if len(out) > 4 else None
        L.check(L.lib.qk_aps_batch_search(self._h, L.ptr(q), int(q.shape[0]), float(recall_target),
                                          L.ptr(out[0]), L.ptr(out[1]), L.ptr(out[2]), L.ptr(out[3]),
                                          L.ptr(s0), int(s0.shape[1]) if s0 is not None else 0,
                                          L.stream_ptr(stream)))
        return out

    def capture(self, q, recall_target, out, stream):
        """Records one batch over these buffers as a CUDA graph on `stream`."""
        q = _as(q, np.float32)
        L.check(L.lib.qk_aps_batch_capture(self._h, L.ptr(q), int(q.shape[0]), float(recall_target),
                                           L.ptr(out[0]), L.ptr(out[1]), L.ptr(out[2]), L.ptr(out[3]),
                                           L.stream_ptr(stream)))

    def replay(self, stream):
        L.check(L.lib.qk_aps_batch_replay(self._h, L.stream_ptr(stream)))

    def set_timing(self, on=True):
        L.check(L.lib.qk_aps_batch_set_timing(self._h, 1 if on else 0))

    def stage_times(self):
        """Milliseconds of the last timed batch: prepare, replay, grouping, scan (all
        rounds together) and the scan of every round (waits for the batch)."""
        ms = np.zeros(4 + self.rounds, np.float32)
        L.check(L.lib.qk_aps_batch_stage_times(self._h, L.ptr(ms)))
        return {"prepare": float(ms[0]), "replay": float(ms[1]), "grouping": float(ms[2]),
                "scan": float(ms[3]), "scan_per_round": ms[4:].tolist()}

    def round_stats(self):
        """Per round of the last batch: (items asked for, items Algorithm 1 took in)."""
        a = np.zeros(self.rounds, np.int64)
        t = np.zeros(self.rounds, np.int64)
        L.check(L.lib.qk_aps_batch_round_stats(self._h, L.ptr(a), L.ptr(t)))
        return a, t
