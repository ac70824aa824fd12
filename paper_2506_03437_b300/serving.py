"""Continuous-batching request loop over one index (queries, inserts, deletes).

Requests arrive on their own clock (open loop).  Searches waiting when a
stream slot is free are launched together as one batch; up to `streams`
batches are on the GPU at once, so requests that arrive while others run are
admitted as soon as a slot frees up, and their work overlaps on the device.
A batch is also held back while free device memory is below
`min_free_bytes`.

Inserts and deletes are applied between batch launches: pending updates wait
until `update_batch` of them have arrived or the oldest has waited
`update_wait_s`; then the pending group is applied, on its own stream, as one
delete call followed by one insert call.  The searches in flight are not
waited for: the index's copy-on-write views let them finish on the version
they were launched on, and batches launched afterwards see the update.
That order gives the same index as applying the group one by one, because the
group is first reduced to its net effect: an id inserted and then deleted
inside the group is dropped from both calls, and an id deleted and then
inserted again is deleted first and then inserted.  Searches may overtake
updates that arrived less than `update_wait_s` before them.

Every `maintain_every` operations the maintenance pass runs (Sec. 4; its
statistics window is the queries since the previous pass).  With
`concurrent_maintenance` (the default) the pass is prepared by a host thread
on its own stream while searches go on (qk_maintain_prepare builds the new
partitions aside); updates wait meanwhile, and once the pass is ready it is
committed.  Otherwise the whole pass runs in place.  Neither waits for the
searches in flight.  A request's latency
runs from its arrival to the moment its result is in host memory.

The index's kernels do all the work; this module only schedules calls to the
C ABI.
"""

import threading
import time

import numpy as np

SEARCH, INSERT, DELETE = 0, 1, 2


class Ops:
    """A request stream: `t` arrival times in seconds (ascending), `kind`
    (SEARCH / INSERT / DELETE), `vec` the query or inserted vector of each op
    (unused for deletes), `ref` the inserted or deleted id (unused for
    searches).  Op j's request id is j."""

    def __init__(self, t, kind, vec, ref):
        self.t = np.ascontiguousarray(t, np.float64)
        self.kind = np.ascontiguousarray(kind, np.int8)
        self.vec = np.ascontiguousarray(vec, np.float32)
        self.ref = np.ascontiguousarray(ref, np.int64)
        n = self.t.shape[0]
        assert self.kind.shape == (n,) and self.ref.shape == (n,) and self.vec.shape[0] == n
        assert n == 0 or np.all(np.diff(self.t) >= 0)

    def __len__(self):
        return self.t.shape[0]

    def count(self, kind):
        return int((self.kind == kind).sum())


def net_updates(kind, ref):
    """Net effect of a group of inserts and deletes applied in order.
    Returns (positions whose ids to delete, positions whose rows to insert)."""
    state = {}   # id -> (deleted an existing copy?, position of the live insert or -1)
    for j in range(kind.shape[0]):
        vid = int(ref[j])
        dele, ins = state.get(vid, (False, -1))
        if kind[j] == INSERT:
            state[vid] = (dele, j)
        elif ins >= 0:                       # delete of an id inserted in this group
            state[vid] = (dele, -1)
        else:
            state[vid] = (True, -1)
    seen, dpos = set(), []
    for j in range(kind.shape[0]):           # one delete per id: its first delete in the group
        vid = int(ref[j])
        if kind[j] == DELETE and state[vid][0] and vid not in seen:
            seen.add(vid)
            dpos.append(j)
    ipos = sorted(v[1] for v in state.values() if v[1] >= 0)
    return np.array(dpos, np.int64), np.array(ipos, np.int64)


class Server:
    """Schedules searches, inserts, deletes and maintenance on one index."""

    def __init__(self, index, d, k=10, recall_target=0.9, max_batch=2048, streams=4, min_free_bytes=1 << 30,
                 maintain_every=0, maint_args=None, update_batch=1024, update_wait_s=0.002,
                 concurrent_maintenance=True):
        import torch
        self.torch = torch
        self.concurrent = concurrent_maintenance
        self.device = torch.cuda.current_device()
        self.maint_stream = torch.cuda.Stream()
        self.update_stream = torch.cuda.Stream()
        self.ix, self.d, self.k, self.tau = index, d, k, recall_target
        self.max_batch, self.min_free = max_batch, min_free_bytes
        self.maintain_every, self.maint_args = maintain_every, maint_args or {}
        self.update_batch, self.update_wait = update_batch, update_wait_s
        self.slots = []
        for _ in range(streams):
            self.slots.append(dict(
                stream=torch.cuda.Stream(),
                q_host=torch.empty((max_batch, d), dtype=torch.float32).pin_memory(),
                q_dev=torch.empty((max_batch, d), dtype=torch.float32, device="cuda"),
                ids_dev=torch.empty((max_batch, k), dtype=torch.int64, device="cuda"),
                dist_dev=torch.empty((max_batch, k), dtype=torch.float32, device="cuda"),
                np_dev=torch.empty(max_batch, dtype=torch.int32, device="cuda"),
                r_dev=torch.empty(max_batch, dtype=torch.float32, device="cuda"),
                ids_host=torch.empty((max_batch, k), dtype=torch.int64).pin_memory(),
                dist_host=torch.empty((max_batch, k), dtype=torch.float32).pin_memory(),
                np_host=torch.empty(max_batch, dtype=torch.int32).pin_memory(),
                busy=False))

    # ---------------------------------------------------------------- batches
    def _launch(self, slot, rows):
        torch = self.torch
        n = rows.shape[0]
        np.take(self.ops.vec, rows, axis=0, out=slot["q_host"].numpy()[:n])
        st = slot["stream"]
        with torch.cuda.stream(st):
            slot["q_dev"][:n].copy_(slot["q_host"][:n], non_blocking=True)
            out = (slot["ids_dev"][:n], slot["dist_dev"][:n], slot["np_dev"][:n], slot["r_dev"][:n])
            self.ix.search(slot["q_dev"][:n], self.k, recall_target=self.tau, out=out, stream=st)
            slot["ids_host"][:n].copy_(slot["ids_dev"][:n], non_blocking=True)
            slot["dist_host"][:n].copy_(slot["dist_dev"][:n], non_blocking=True)
            slot["np_host"][:n].copy_(slot["np_dev"][:n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        slot["busy"] = True
        return dict(slot=slot, event=ev, rows=rows)

    def _finish(self, b, now):
        slot, rows = b["slot"], b["rows"]
        n = rows.shape[0]
        self.lat[rows] = now - self.ops.t[rows]
        self.nprobe[rows] = slot["np_host"].numpy()[:n]
        if self.out_ids is not None:
            self.out_ids[rows] = slot["ids_host"].numpy()[:n]
            self.out_dist[rows] = slot["dist_host"].numpy()[:n]
        slot["busy"] = False

    def _free_ok(self):
        if self.min_free <= 0:
            return True
        free, _ = self.torch.cuda.mem_get_info()
        return free >= self.min_free

    def _prepare(self, prep):
        try:
            self.torch.cuda.set_device(self.device)   # the CUDA device is per host thread
            self.ix.maintain_prepare(stream=self.maint_stream, **self.maint_args)
        except Exception as e:   # re-raised by the request loop
            prep[1] = e

    def _apply_updates(self, rows, clock):
        ops = self.ops
        dpos, ipos = net_updates(ops.kind[rows], ops.ref[rows])
        if dpos.shape[0]:
            self.ix.delete(ops.ref[rows[dpos]], stream=self.update_stream)
        if ipos.shape[0]:
            r = rows[ipos]
            self.ix.insert(ops.vec[r], ops.ref[r], stream=self.update_stream)
        self.lat[rows] = clock() - ops.t[rows]

    # ------------------------------------------------------------------- run
    def run(self, ops, keep_results=False):
        """Serves the stream; returns a summary of latencies (per kind, p50/p99/mean
        in ms), throughput and where the wall time went.  With keep_results the
        search results are left in self.out_ids / self.out_dist (row j = op j)."""
        self.ops = ops
        n_ops = len(ops)
        self.lat = np.full(n_ops, np.nan)
        self.nprobe = np.zeros(n_ops, np.int32)
        self.out_ids = np.full((n_ops, self.k), -1, np.int64) if keep_results else None
        self.out_dist = np.full((n_ops, self.k), np.inf, np.float32) if keep_results else None
        s_rows = np.flatnonzero(ops.kind == SEARCH)
        u_rows = np.flatnonzero(ops.kind != SEARCH)
        s_t, u_t = ops.t[s_rows], ops.t[u_rows]
        n_s, n_u = s_rows.shape[0], u_rows.shape[0]
        qs = us = 0          # next search / update not yet taken
        t_upd = t_maint = t_host = t_prep = 0.0
        batches = groups = passes = 0
        inflight = []
        prep = None          # the maintenance pass being prepared: [thread, error, start time]
        searched = 0         # queries launched since the last pass (its statistics window)
        min_window = max(1, min(1000, self.maintain_every // 10)) if self.maintain_every else 1
        t0 = time.perf_counter()

        def clock():
            return time.perf_counter() - t0

        while qs < n_s or us < n_u or inflight or prep is not None:
            now = clock()
            qa = int(np.searchsorted(s_t, now, side="right"))
            ua = int(np.searchsorted(u_t, now, side="right"))
            # results of finished batches
            while inflight and inflight[0]["event"].query():
                self._finish(inflight.pop(0), clock())
            # a prepared maintenance pass: commit, then updates may go on
            if prep is not None and not prep[0].is_alive():
                c0 = clock()
                if prep[1] is not None:
                    raise prep[1]
                self.ix.maintain_commit(stream=self.maint_stream)
                passes += 1
                searched = 0
                t_maint += clock() - c0
                t_prep += c0 - prep[2]
                prep = None
            # updates: between batch launches, beside the searches in flight
            if prep is None and ua > us and (ua - us >= self.update_batch or now - u_t[us] >= self.update_wait
                                             or qa == n_s):
                c0 = clock()
                self._apply_updates(u_rows[us:ua], clock)
                us = ua
                groups += 1
                t_upd += clock() - c0
            if (self.maintain_every and prep is None and (qa + ua) // self.maintain_every > passes
                    and searched >= min_window):
                if self.concurrent:
                    # pending updates first, so the pass plans from the current index
                    if ua > us:
                        c0 = clock()
                        self._apply_updates(u_rows[us:ua], clock)
                        us = ua
                        groups += 1
                        t_upd += clock() - c0
                    prep = [None, None, clock()]
                    prep[0] = threading.Thread(target=self._prepare, args=(prep,), daemon=True)
                    prep[0].start()
                else:
                    c0 = clock()
                    self.ix.maintain(stream=self.update_stream, **self.maint_args)
                    passes += 1
                    searched = 0
                    t_maint += clock() - c0
            # launch while a stream slot is free and memory allows
            launched = False
            while qa > qs and len(inflight) < len(self.slots) and self._free_ok():
                c0 = clock()
                slot = next(s for s in self.slots if not s["busy"])
                n = min(self.max_batch, qa - qs)
                inflight.append(self._launch(slot, s_rows[qs:qs + n]))
                qs += n
                searched += n
                batches += 1
                launched = True
                t_host += clock() - c0
            if not launched:
                if inflight:
                    time.sleep(20e-6)
                else:
                    nxt = min(s_t[qs] if qs < n_s else np.inf, u_t[us] if us < n_u else np.inf)
                    wait = nxt - clock()
                    if np.isfinite(wait) and wait > 0:
                        time.sleep(min(wait, 1e-3))
        wall = clock()
        out = {"wall_s": round(wall, 4), "batches": batches, "maintenance_passes": passes, "update_groups": groups,
               "update_s": round(t_upd, 4), "maintenance_stall_s": round(t_maint, 4),
               "maintenance_prepare_s": round(t_prep, 4), "launch_host_s": round(t_host, 4),
               "concurrent_maintenance": self.concurrent}
        for kind, name in ((SEARCH, "search"), (INSERT, "insert"), (DELETE, "delete")):
            v = self.lat[ops.kind == kind]
            if v.shape[0]:
                a = v * 1e3
                out[name] = {"n": int(v.shape[0]), "p50_ms": round(float(np.percentile(a, 50)), 4),
                             "p99_ms": round(float(np.percentile(a, 99)), 4), "mean_ms": round(float(a.mean()), 4)}
        out["search_qps"] = round(n_s / wall, 1) if wall > 0 else None
        out["mean_nprobe"] = round(float(self.nprobe[s_rows].mean()), 3) if n_s else None
        return out


def skewed_stream(centers, start_ids, n_ops, sigma, seed, hot=100, zipf=1.2, rotate=100_000,
                  p_query=0.9, p_insert=0.05, rate=None, next_id=None):
    """The dynamic skewed workload: queries Zipf(`zipf`) over a hot set of `hot`
    components that is redrawn every `rotate` ops, inserts of new samples from
    the hot components (fresh ids), deletes of uniformly chosen live ids.
    Arrivals are Poisson at `rate` ops/s, or all at t = 0 when rate is None."""
    from .synth import rng
    g = rng(seed)
    n_comp, d = centers.shape
    w = np.arange(1, hot + 1, dtype=np.float64) ** (-zipf)
    w /= w.sum()
    kind = g.choice(3, size=n_ops, p=[p_query, p_insert, 1.0 - p_query - p_insert]).astype(np.int8)
    t = np.cumsum(g.exponential(1.0 / rate, size=n_ops)) if rate else np.zeros(n_ops)
    n_epochs = max(1, (n_ops + rotate - 1) // rotate) if rotate else 1
    hot_sets = np.stack([g.choice(n_comp, hot, replace=False) for _ in range(n_epochs)])
    rank = g.choice(hot, size=n_ops, p=w)
    epoch = np.arange(n_ops) // rotate if rotate else np.zeros(n_ops, np.int64)
    comp = hot_sets[epoch, rank]
    vec = np.empty((n_ops, d), np.float32)
    for a in range(0, n_ops, 1 << 16):
        b = min(n_ops, a + (1 << 16))
        vec[a:b] = centers[comp[a:b]] + sigma * g.standard_normal((b - a, d))
    u = g.random(n_ops)
    live = [int(i) for i in start_ids]
    next_id = int(next_id if next_id is not None else max(live) + 1)
    ref = np.full(n_ops, -1, np.int64)
    for j in np.flatnonzero(kind != SEARCH):
        if kind[j] == INSERT:
            ref[j] = next_id
            live.append(next_id)
            next_id += 1
        elif live:
            pos = int(u[j] * len(live))
            ref[j] = live[pos]
            live[pos] = live[-1]
            live.pop()
        else:
            kind[j] = SEARCH
    return Ops(t, kind, vec, ref)


class NativeServer:
    """The same serving loop run by the library's scheduler thread (qk_server_* in
    include/quake_b300.h), with the open-loop arrivals played by the library as well
    (qk_server_play); this class only builds the configuration and reads the results.  A
    request's latency counts from its scheduled arrival, so a late submission counts in it."""

    def __init__(self, index, d, k=10, recall_target=0.9, max_batch=2048, streams=4, min_free_bytes=1 << 30,
                 maintain_every=0, maint_args=None, update_batch=1024, update_wait_s=0.01,
                 concurrent_maintenance=True, batched_from=None):
        import ctypes as C
        from . import _lib as L
        self.C, self.L = C, L
        self.ix, self.d, self.k = index, d, k
        cfg = L.QkServerConfig()
        L.lib.qk_server_config_default(C.byref(cfg))
        if batched_from is not None:   # batches from this size run through the batched APS plan
            cfg.batched_from = int(batched_from)
        cfg.k, cfg.recall_target, cfg.max_batch, cfg.streams = k, recall_target, max_batch, streams
        cfg.min_free_bytes, cfg.maintain_every = min_free_bytes, maintain_every
        cfg.update_batch, cfg.update_wait_s = update_batch, update_wait_s
        cfg.concurrent_maintenance = int(bool(concurrent_maintenance))
        self._keep = []
        if maintain_every:
            a = dict(tau_us=0.25, alpha=0.9, refine_radius=50, refine_iters=1, split_iters=10, s_min=0,
                     refine=True, window=0, level_band=False, level_iters=10)
            a.update(maint_args or {})
            ls = np.ascontiguousarray(a.pop("lam_sizes"), np.float64)
            lu = np.ascontiguousarray(a.pop("lam_us"), np.float64)
            p = L.QkMaintParams()
            p.lambda_sizes = ls.ctypes.data_as(C.POINTER(C.c_double))
            p.lambda_us = lu.ctypes.data_as(C.POINTER(C.c_double))
            p.lambda_points = int(ls.shape[0])
            p.refine_radius, p.refine_iters, p.split_iters = a["refine_radius"], a["refine_iters"], a["split_iters"]
            p.s_min, p.refine, p.tau_us = a["s_min"], int(bool(a["refine"])), a["tau_us"]
            p.alpha, p.window = a["alpha"], a["window"]
            p.level_band, p.level_iters = int(bool(a["level_band"])), a["level_iters"]
            self._keep += [ls, lu, p]
            cfg.maint = C.pointer(p)
        self.cfg = cfg

    def run(self, ops, keep_results=False):
        """Serves the stream (a fresh server per run, so ticket j is op j) and returns the
        same summary as Server.run."""
        C, L = self.C, self.L
        h = C.c_void_p()
        L.check(L.lib.qk_server_create(self.ix._h, C.byref(self.cfg), C.byref(h)))
        n = len(ops)
        lag = np.zeros(n)
        vec = np.ascontiguousarray(ops.vec, np.float32)
        kinds = np.ascontiguousarray(ops.kind, np.int8)
        refs = np.ascontiguousarray(ops.ref, np.int64)
        ts = np.ascontiguousarray(ops.t, np.float64)
        try:
            t0 = time.perf_counter()
            # the library plays the stream open-loop from this thread: each request
            # is submitted at its scheduled time and its latency counts from it
            L.check(L.lib.qk_server_play(h, n, L.ptr(kinds), L.ptr(refs), L.ptr(vec), L.ptr(ts), L.ptr(lag)))
            L.check(L.lib.qk_server_drain(h, 0.0))
            wall = time.perf_counter() - t0
            done = np.zeros(n, np.int32)
            lat = np.zeros(n)
            ids = np.empty((n, self.k), np.int64) if keep_results else None
            dist = np.empty((n, self.k), np.float32) if keep_results else None
            L.check(L.lib.qk_server_results(h, 0, n, L.ptr(done), L.ptr(ids), L.ptr(dist), L.ptr(lat)))
            stt = L.QkServerStats()
            L.check(L.lib.qk_server_get_stats(h, C.byref(stt)))
        finally:
            L.lib.qk_server_destroy(h)
        assert done.all()
        self.out_ids, self.out_dist = ids, dist
        out = {"wall_s": round(wall, 4), "batches": stt.batches, "maintenance_passes": stt.maintenance_passes,
               "update_groups": stt.update_groups, "update_s": round(stt.update_s, 4),
               "maintenance_stall_s": round(stt.maintenance_stall_s, 4),
               "maintenance_prepare_s": round(stt.maintenance_prepare_s, 4),
               "driver_lag_p99_ms": round(float(np.percentile(lag, 99)) * 1e3, 4),
               "concurrent_maintenance": bool(self.cfg.concurrent_maintenance), "native": True}
        for kind, name in ((SEARCH, "search"), (INSERT, "insert"), (DELETE, "delete")):
            v = lat[ops.kind == kind]
            if v.shape[0]:
                a = v * 1e3
                out[name] = {"n": int(v.shape[0]), "p50_ms": round(float(np.percentile(a, 50)), 4),
                             "p99_ms": round(float(np.percentile(a, 99)), 4), "mean_ms": round(float(a.mean()), 4)}
        n_s = int((ops.kind == SEARCH).sum())
        out["search_qps"] = round(n_s / wall, 1) if wall > 0 else None
        return out
