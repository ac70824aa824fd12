"""The continuous-batching request loop: results alone equal results in the mix; updates apply in order."""

import numpy as np
import pytest

from oracle import kmeans
from paper_2506_03437_b300 import synth

from .test_gpu_search import make_index

pytestmark = pytest.mark.gpu


def test_results_alone_equal_results_in_the_mix():
    from paper_2506_03437_b300.serving import Ops, Server
    X, ids, Q = synth.aps_search(seed=41, n=30_000, d=64, n_comp=40, sigma=1.2, nq=3000)
    levels = kmeans.build_index(X, ids, 150, 8, iters=3, seed=5)
    from paper_2506_03437_b300 import index as I
    ix = make_index(I, X, ids, levels, f_M_leaf=0.15, f_M_parent=0.5)
    # alone: every query is its own search call
    alone = [ix.search(Q[j:j + 1], 10, recall_target=0.9) for j in range(0, 3000, 7)]
    # in the mix: all 3,000 arrive at once and share batches on four streams
    ops = Ops(np.zeros(3000), np.zeros(3000, np.int8), Q, np.full(3000, -1))
    srv = Server(ix, 64, k=10, recall_target=0.9, max_batch=200, streams=4)
    st = srv.run(ops, keep_results=True)
    assert st["batches"] >= 15 and st["search"]["n"] == 3000
    for n, j in enumerate(range(0, 3000, 7)):
        assert np.array_equal(srv.out_ids[j], alone[n][0][0])
        assert np.array_equal(srv.out_dist[j], alone[n][1][0])


@pytest.mark.parametrize("concurrent", [False, True])
def test_stream_with_updates_and_maintenance(concurrent):
    from paper_2506_03437_b300.serving import Server, skewed_stream
    X, ids, Q = synth.aps_search(seed=42, n=20_000, d=64, n_comp=50, sigma=1.2, nq=1)
    levels = kmeans.build_index(X, ids, 100, 0, iters=3, seed=6)
    from paper_2506_03437_b300 import index as I
    ix = make_index(I, X, ids, levels, f_M_leaf=0.2)
    C = synth.mixture_centers(50, 64, 42)
    ops = skewed_stream(C, ids, 6000, 1.2, 7, hot=10, rotate=2000, rate=2e5)
    srv = Server(ix, 64, k=10, recall_target=0.9, max_batch=256, streams=3, maintain_every=3000,
                 concurrent_maintenance=concurrent,
                 maint_args=dict(lam_sizes=[0, 1000], lam_us=[2.0, 47.0], tau_us=0.25, alpha=0.9, refine_radius=8,
                                 s_min=20))
    st = srv.run(ops)
    assert ix.info()["n"] == 20_000 + ops.count(1) - ops.count(2)
    # in place, a pass runs every 3,000 operations; prepared beside the searches, a pass
    # also needs queries since the previous one, so the stream's end may leave one out
    assert (st["maintenance_passes"] == 2 if not concurrent else st["maintenance_passes"] >= 1)
    assert st["search"]["n"] == ops.count(0)
    # every live id is stored exactly once
    _, _, got = ix.export_level(0)
    live = set(ids.tolist())
    for kind, ref in zip(ops.kind, ops.ref):
        if kind == 1:
            live.add(int(ref))
        elif kind == 2:
            live.discard(int(ref))
    assert sorted(got.tolist()) == sorted(live)


@pytest.mark.parametrize("batched_from", [0, 1, 64])
def test_native_server_results_alone_equal_results_in_the_mix(batched_from):
    """Each search's result in a served stream equals the per-query kernel's result for the
    query alone, whether its batch ran through qk_search (batched_from 0), through the slot's
    batched APS plan (1), or either, by batch size (64)."""
    from paper_2506_03437_b300.serving import NativeServer, Ops
    X, ids, Q = synth.aps_search(seed=43, n=30_000, d=64, n_comp=40, sigma=1.2, nq=3000)
    levels = kmeans.build_index(X, ids, 150, 8, iters=3, seed=5)
    from paper_2506_03437_b300 import index as I
    ix = make_index(I, X, ids, levels, f_M_leaf=0.15, f_M_parent=0.5)
    alone = [ix.search(Q[j:j + 1], 10, recall_target=0.9) for j in range(0, 3000, 7)]
    ops = Ops(np.zeros(3000), np.zeros(3000, np.int8), Q, np.full(3000, -1))
    srv = NativeServer(ix, 64, k=10, recall_target=0.9, max_batch=200, streams=4, batched_from=batched_from)
    st = srv.run(ops, keep_results=True)
    assert st["batches"] >= 15 and st["search"]["n"] == 3000
    for n, j in enumerate(range(0, 3000, 7)):
        assert np.array_equal(srv.out_ids[j], alone[n][0][0])
        assert np.array_equal(srv.out_dist[j], alone[n][1][0])


@pytest.mark.parametrize("concurrent", [False, True])
def test_native_server_stream_with_updates_and_maintenance(concurrent):
    from paper_2506_03437_b300.serving import NativeServer, skewed_stream
    X, ids, Q = synth.aps_search(seed=44, n=20_000, d=64, n_comp=50, sigma=1.2, nq=1)
    levels = kmeans.build_index(X, ids, 100, 0, iters=3, seed=6)
    from paper_2506_03437_b300 import index as I
    ix = make_index(I, X, ids, levels, f_M_leaf=0.2)
    C = synth.mixture_centers(50, 64, 44)
    ops = skewed_stream(C, ids, 6000, 1.2, 8, hot=10, rotate=2000, rate=1e5)
    srv = NativeServer(ix, 64, k=10, recall_target=0.9, max_batch=256, streams=3, maintain_every=3000,
                       concurrent_maintenance=concurrent,
                       maint_args=dict(lam_sizes=[0, 1000], lam_us=[2.0, 47.0], tau_us=0.25, alpha=0.9,
                                       refine_radius=8, s_min=20))
    st = srv.run(ops)
    assert ix.info()["n"] == 20_000 + ops.count(1) - ops.count(2)
    assert (st["maintenance_passes"] == 2 if not concurrent else st["maintenance_passes"] >= 1)
    assert st["search"]["n"] == ops.count(0) and st["insert"]["n"] == ops.count(1)
    _, _, got = ix.export_level(0)
    live = set(ids.tolist())
    for kind, ref in zip(ops.kind, ops.ref):
        if kind == 1:
            live.add(int(ref))
        elif kind == 2:
            live.discard(int(ref))
    assert sorted(got.tolist()) == sorted(live)


def test_native_server_rejects_bad_config_and_reports_a_failed_update():
    """An invalid configuration is refused; an insert of an id the index already holds fails
    its update group, stops the server, and drain reports it."""
    import ctypes as C
    from paper_2506_03437_b300 import _lib as L
    X, ids, Q = synth.aps_search(seed=45, n=5000, d=64, n_comp=10, sigma=1.0, nq=4)
    levels = kmeans.build_index(X, ids, 20, 0, iters=2, seed=2)
    from paper_2506_03437_b300 import index as I
    ix = make_index(I, X, ids, levels)
    cfg = L.QkServerConfig()
    L.lib.qk_server_config_default(C.byref(cfg))
    h = C.c_void_p()
    bad = L.QkServerConfig.from_buffer_copy(cfg)
    bad.streams = 0
    assert L.lib.qk_server_create(ix._h, C.byref(bad), C.byref(h)) == L.ERR_ARG
    bad = L.QkServerConfig.from_buffer_copy(cfg)
    bad.maintain_every = 100   # a maintenance cadence needs pass parameters
    assert L.lib.qk_server_create(ix._h, C.byref(bad), C.byref(h)) == L.ERR_ARG
    L.check(L.lib.qk_server_create(ix._h, C.byref(cfg), C.byref(h)))
    try:
        t = C.c_int64()
        # a non-finite vector is refused at submission; the server keeps running
        nanq = np.ascontiguousarray(Q[0].copy())
        nanq[3] = np.nan
        assert L.lib.qk_server_submit_search(h, nanq.ctypes.data, C.byref(t)) == L.ERR_ARG
        infx = np.ascontiguousarray(X[0].copy())
        infx[0] = np.inf
        assert L.lib.qk_server_submit_insert(h, infx.ctypes.data, 10 ** 9, C.byref(t)) == L.ERR_ARG
        L.check(L.lib.qk_server_submit_search(h, Q.ctypes.data, C.byref(t)))
        assert L.lib.qk_server_drain(h, 30.0) == L.OK
        x = np.ascontiguousarray(X[0] + 0.5)
        L.check(L.lib.qk_server_submit_insert(h, x.ctypes.data, 7, C.byref(t)))   # id 7 exists
        assert L.lib.qk_server_drain(h, 30.0) == L.ERR_STATE
        assert b"insert" in L.lib.qk_last_error()
        assert L.lib.qk_server_submit_delete(h, 3, C.byref(t)) == L.ERR_STATE   # stopped
    finally:
        L.lib.qk_server_destroy(h)
    assert ix.info()["n"] == 5000   # the failed group inserted nothing
