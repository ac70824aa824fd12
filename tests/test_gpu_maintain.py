"""GPU parity of the maintenance pass (Sec. 4) against the oracle."""

import numpy as np
import pytest

from oracle import aps, kmeans, knn, maintenance

from .parity import compare_search, same_topk
from .test_gpu_search import make_index
from .test_oracle_maintain import example_lambda, example_level

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


def test_worked_example_on_gpu(I):
    """Sec. 4's example: P2 splits 450/50 (Delta = +5 us, rejected), P1 250/250 (Delta = -5 us, committed)."""
    g, pts = example_lambda()
    X, ids, C, lab = example_level()
    ix = I.Index(32, n_leaf=2, seed=1234)
    ix.load(X, ids, C, lab.astype(np.int32))
    # 10 queries land in each partition; with |W| = 100 that is A = 0.10 for both
    Q = np.concatenate([np.repeat(C[:1], 10, 0), np.repeat(C[1:], 10, 0)])
    ix.search(Q, 5, recall_target=0.0, nprobe=1)
    assert ix.hits(0).tolist() == [10, 10]
    log = ix.maintain(pts[:, 0], pts[:, 1], tau_us=g["tau"], alpha=g["alpha"], refine=False, window=100)
    assert [(a["kind"], a["partition"], a["committed"]) for a in log] == [("split", 0, False), ("split", 1, True)]
    assert abs(log[0]["estimate"] - g["delta_estimate"]) < 1e-9
    assert abs(log[0]["delta"] - g["P2_delta"]) < 1e-9 and abs(log[1]["delta"] - g["P1_delta"]) < 1e-9
    sizes, _, _ = ix.export_level(0)
    assert sizes.tolist() == [500, 250, 250]


def scenario(seed=3, d=32):
    g = np.random.default_rng(seed)
    cen = (3 * g.standard_normal((40, d))).astype(np.float32)
    sizes = (3000 / np.arange(1, 41) ** 0.8).astype(int) + 20
    X = np.concatenate([c + 0.05 * g.standard_normal((s, d)) for c, s in zip(cen, sizes)]).astype(np.float32)
    ids = np.arange(X.shape[0], dtype=np.int64)
    qlab = np.minimum(g.zipf(1.3, 600) - 1, 39)
    Q = (cen[qlab] + 0.05 * g.standard_normal((600, d))).astype(np.float32)
    return X, ids, Q


def test_maintenance_pass_matches_oracle(I):
    X, ids, Q = scenario()
    levels = kmeans.build_index(X, ids, 24, 5, iters=5, seed=11)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.25, f_M_parent=1.0, seed=1234)
    # Stage 0 statistics: the same queries on both sides
    ix.search(Q, 10, recall_target=0.0, nprobe=2)
    res = aps.search(levels, Q, aps.Params(k=10, recall_target=0.0, nprobe=2, f_M=(0.25, 1.0)))
    h0 = np.bincount(np.concatenate([np.array(s) for s in res["scanned"][0]]), minlength=24)
    h1 = np.bincount(np.concatenate([np.array(s) for s in res["scanned"][1]]), minlength=5)
    assert np.array_equal(ix.hits(0), h0) and np.array_equal(ix.hits(1), h1)
    lam = maintenance.Latency([0, 1000], [5.0, 55.0])
    prm = maintenance.MaintParams(lam, tau=0.01, alpha=0.9, refine_radius=4, s_min=120, split_iters=8, seed=1234)
    logs = maintenance.maintain(levels, [h0, h1], 600, prm)
    got = ix.maintain([0, 1000], [5.0, 55.0], tau_us=0.01, alpha=0.9, refine_radius=4, s_min=120, split_iters=8,
                      window=600)
    want = [(lv, k, j, ok, e, dl) for lv, lg in enumerate(logs) for k, j, e, dl, ok in lg]
    if len(got) != len(want) or any((a["level"], a["kind"], a["partition"], a["committed"]) != w[:4]
                                    for a, w in zip(got, want)):
        print("gpu   :", [(a["level"], a["kind"], a["partition"], a["committed"], a["estimate"], a["delta"]) for a in got])
        print("oracle:", want)
        print("gpu sizes", ix.export_level(0)[0].tolist(), ix.export_level(1)[0].tolist())
        print("orc sizes", levels[0].sizes().tolist(), levels[1].sizes().tolist())
    assert len(got) == len(want)
    assert any(w[3] for w in want) and any(w[1] == "merge" for w in want)
    for a, (lv, k, j, ok, e, dl) in zip(got, want):
        assert (a["level"], a["kind"], a["partition"], a["committed"]) == (lv, k, j, ok)
        assert abs(a["estimate"] - e) <= 1e-6 * max(1.0, abs(e))
        if dl is not None:
            assert abs(a["delta"] - dl) <= 1e-6 * max(1.0, abs(dl))
    # the new structure: same partitions (as id sets), centroids to FP32 rounding
    sizes, cents, gids = ix.export_level(0)
    assert sizes.tolist() == levels[0].sizes().tolist()
    off = np.concatenate([[0], np.cumsum(sizes)])
    for j in range(len(sizes)):
        assert set(gids[off[j]:off[j + 1]].tolist()) == set(levels[0].ids[j].tolist())
    np.testing.assert_allclose(cents, levels[0].centroids, rtol=1e-5, atol=1e-5)
    s1, c1, g1 = ix.export_level(1)
    assert s1.tolist() == levels[1].sizes().tolist()
    off = np.concatenate([[0], np.cumsum(s1)])
    for p in range(len(s1)):
        assert set(g1[off[p]:off[p + 1]].tolist()) == set(levels[1].ids[p].tolist())
    # every vector is still there: a full scan is exact kNN
    info = ix.info()
    assert info["n"] == X.shape[0] and info["n_leaf"] == levels[0].n_part
    gi, gd, gn, gr = ix.search(Q[:20], 10, recall_target=0.0, nprobe=info["n_leaf"])
    D, Ix = knn.knn(X, ids, Q[:20], 10)
    for j in range(20):
        assert same_topk(gi[j], gd[j], Ix[j], D[j])


def test_maintain_needs_statistics(I):
    from paper_2506_03437_b300 import _lib as L
    X, ids, Q = scenario()
    levels = kmeans.build_index(X[:3000], ids[:3000], 6, 0, iters=2, seed=1)
    ix = make_index(I, X[:3000], ids[:3000], levels)
    with pytest.raises(L.QkError) as e:
        ix.maintain([0, 1000], [5.0, 55.0])
    assert e.value.status == L.ERR_STATE
    with pytest.raises(L.QkError) as e:
        ix.maintain([10, 5], [1.0, 2.0], window=10)
    assert e.value.status == L.ERR_ARG


def test_prepare_then_commit_equals_maintain_and_searches_run_meanwhile(I):
    """qk_maintain_prepare + qk_maintain_commit give the index qk_maintain gives.  Between
    them the index still answers from its old partitions, also from another host thread,
    and a change of the index discards the prepared pass.  A prepare on a worker thread
    while this thread searches leaves those searches on the old partitions too; which of
    them its statistics count depends on when its copy of the counters runs, so that pass
    is checked for the vectors it keeps, not against qk_maintain."""
    import threading
    from paper_2506_03437_b300 import _lib as L
    X, ids, Q = scenario()
    levels = kmeans.build_index(X, ids, 24, 5, iters=5, seed=11)
    kw = dict(tau_us=0.01, alpha=0.9, refine_radius=4, s_min=120, split_iters=8, window=600)
    a = make_index(I, X, ids, levels, f_M_leaf=0.25, f_M_parent=1.0, seed=1234)
    b = make_index(I, X, ids, levels, f_M_leaf=0.25, f_M_parent=1.0, seed=1234)
    c = make_index(I, X, ids, levels, f_M_leaf=0.25, f_M_parent=1.0, seed=1234)
    for ix in (a, b, c):
        ix.search(Q, 10, recall_target=0.0, nprobe=2)
    before = b.search(Q[:50], 10, recall_target=0.9)
    log_a = a.maintain([0, 1000], [5.0, 55.0], **kw)
    # prepared here; searched from another host thread and this one until the commit
    out = {"log": b.maintain_prepare([0, 1000], [5.0, 55.0], **kw)}
    res = {}
    t = threading.Thread(target=lambda: res.update(r=[b.search(Q[:50], 10, recall_target=0.9) for _ in range(3)]))
    t.start()
    during = [b.search(Q[:50], 10, recall_target=0.9) for _ in range(3)]
    t.join()
    for r in during + res["r"] + [b.search(Q[:50], 10, recall_target=0.9)]:   # still the old partitions
        assert np.array_equal(r[0], before[0]) and np.array_equal(r[2], before[2])
    b.maintain_commit()
    # the prepare on a worker thread while this thread keeps searching
    before_c = c.search(Q[:50], 10, recall_target=0.9)
    t = threading.Thread(target=lambda: c.maintain_prepare([0, 1000], [5.0, 55.0], **kw))
    t.start()
    during = [c.search(Q[:50], 10, recall_target=0.9) for _ in range(3)]
    t.join()
    for r in during:
        assert np.array_equal(r[0], before_c[0]) and np.array_equal(r[2], before_c[2])
    c.maintain_commit()
    sc, _, ic = c.export_level(0)
    assert sorted(ic[:int(sc.sum())].tolist()) == sorted(ids.tolist())
    assert [(x["level"], x["kind"], x["partition"], x["committed"]) for x in out["log"]] == \
           [(x["level"], x["kind"], x["partition"], x["committed"]) for x in log_a]
    for lv in (0, 1):
        sa, ca, ia = a.export_level(lv)
        sb, cb, ib = b.export_level(lv)
        assert np.array_equal(sa, sb) and np.array_equal(ca, cb)
        off = np.concatenate([[0], np.cumsum(sa)])
        for j in range(len(sa)):
            assert set(ia[off[j]:off[j + 1]].tolist()) == set(ib[off[j]:off[j + 1]].tolist())
    ra, rb = a.search(Q, 10, recall_target=0.9), b.search(Q, 10, recall_target=0.9)
    assert np.array_equal(ra[0], rb[0])
    # nothing prepared, or the index changed after the prepare: refused
    with pytest.raises(L.QkError) as e:
        b.maintain_commit()
    assert e.value.status == L.ERR_STATE
    b.search(Q, 10, recall_target=0.0, nprobe=2)
    n_leaf = b.info()["n_leaf"]
    b.maintain_prepare([0, 1000], [5.0, 55.0], **kw)
    b.insert(X[:3] + 0.01, np.array([10 ** 7, 10 ** 7 + 1, 10 ** 7 + 2], np.int64))
    with pytest.raises(L.QkError) as e:
        b.maintain_commit()
    assert e.value.status == L.ERR_STATE and b.info()["n_leaf"] == n_leaf


def test_level_band_adds_and_removes_the_parent_level(I):
    """Reading M9 on the GPU: one level of 40 leaves gains round(sqrt(40)) = 6 parents, the
    oracle's (the build's k-means of the leaf centroids, seed + 1); 16 leaves lose them; and the
    new two-level index searches like the oracle's."""
    g = np.random.default_rng(0)
    X = (g.standard_normal((4000, 8)) + 4 * np.repeat(g.standard_normal((40, 8)), 100, axis=0)).astype(np.float32)
    X = np.concatenate([X, np.zeros((4000, 24), np.float32)], axis=1)   # d = 32
    ids = np.arange(4000, dtype=np.int64)
    levels = kmeans.build_index(X, ids, 40, 0, iters=3, seed=5)
    ix = make_index(I, X, ids, levels, seed=5, f_M_leaf=0.5, f_M_parent=1.0)
    Q = X[::97] + 0.01
    ix.search(Q, 10, recall_target=0.0, nprobe=2)
    lam = maintenance.Latency([0, 1000], [5.0, 55.0])
    prm = maintenance.MaintParams(lam, tau=1e9, level_band=True, level_iters=4, seed=5)
    want = maintenance.maintain(levels, [ix.hits(0)], Q.shape[0], prm)
    got = ix.maintain([0, 1000], [5.0, 55.0], tau_us=1e9, level_band=True, level_iters=4, window=Q.shape[0])
    assert [(a["level"], a["kind"], a["partition"]) for a in got if a["level"] == 1] == [(1, "add_level", 6)]
    assert want[1][0][:2] == ("add_level", 6) and ix.info()["n_parent"] == 6
    s1, c1, i1 = ix.export_level(1)
    np.testing.assert_allclose(c1, levels[1].centroids, rtol=1e-5, atol=1e-5)
    off = np.concatenate([[0], np.cumsum(s1)])
    for p in range(6):
        assert set(i1[off[p]:off[p + 1]].tolist()) == set(levels[1].ids[p].tolist())
    r = ix.search_scanned(Q, 10, recall_target=0.9, cap0=64, cap1=8)
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.9, f_M=(0.5, 1.0)))
    compare_search(r, orc, 10, label="APS after a level-band change")
    # 16 leaves: the parent level goes away again
    small = kmeans.build_index(X, ids, 16, 4, iters=3, seed=5)
    ix2 = make_index(I, X, ids, small, seed=5)
    ix2.search(Q, 10, recall_target=0.0, nprobe=2)
    got = ix2.maintain([0, 1000], [5.0, 55.0], tau_us=1e9, level_band=True, level_iters=4, window=Q.shape[0])
    assert got[-1]["kind"] == "remove_level" and ix2.info()["n_parent"] == 0
    r2 = ix2.search(Q, 10, recall_target=0.0, nprobe=16)
    D, Ix = knn.knn(X, ids, Q, 10)
    for j in range(Q.shape[0]):
        assert same_topk(r2[0][j], r2[1][j], Ix[j], D[j])


def test_level_band_rebuilds_parents_outside_the_band(I):
    """Reading M9: 40 leaves under 1 parent (below sqrt(40)/4) are regrouped under round(sqrt(40)) = 6
    new parents, the oracle's."""
    g = np.random.default_rng(1)
    X = (g.standard_normal((4000, 32)) + 4 * np.repeat(g.standard_normal((40, 32)), 100, axis=0)).astype(np.float32)
    ids = np.arange(4000, dtype=np.int64)
    levels = kmeans.build_index(X, ids, 40, 1, iters=3, seed=7)
    ix = make_index(I, X, ids, levels, seed=7, f_M_leaf=0.5, f_M_parent=1.0)
    Q = X[::50] + 0.01
    ix.search(Q, 10, recall_target=0.0, nprobe=2)
    prm = maintenance.MaintParams(maintenance.Latency([0, 1000], [5.0, 55.0]), tau=1e9, level_band=True,
                                  level_iters=4, seed=7)
    want = maintenance.maintain(levels, [ix.hits(0), ix.hits(1)], Q.shape[0], prm)
    got = ix.maintain([0, 1000], [5.0, 55.0], tau_us=1e9, level_band=True, level_iters=4, window=Q.shape[0])
    assert [(a["kind"], a["partition"]) for a in got if a["level"] == 1] == [("rebuild_level", 6)]
    assert want[1][-1][:2] == ("rebuild_level", 6) and ix.info()["n_parent"] == 6
    s1, c1, i1 = ix.export_level(1)
    np.testing.assert_allclose(c1, levels[1].centroids, rtol=1e-5, atol=1e-5)
    off = np.concatenate([[0], np.cumsum(s1)])
    for p in range(6):
        assert set(i1[off[p]:off[p + 1]].tolist()) == set(levels[1].ids[p].tolist())
    r = ix.search_scanned(Q, 10, recall_target=0.9, cap0=64, cap1=8)
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.9, f_M=(0.5, 1.0)))
    compare_search(r, orc, 10, label="APS after a level-band change")
