"""GPU parity of the search path (root scoring, APS, fused scan + top-k) against the oracle.

All inputs come from paper_2506_03437_b300.synth; every index structure used
here is built by the oracle and installed in the library with qk_load, so the
two sides search the same partitions.
"""

import numpy as np
import pytest

from oracle import aps, capvol, kmeans, knn
from paper_2506_03437_b300 import synth

from .parity import compare_search, exact_dist, same_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


def load_args(levels, n):
    lv0 = levels[0]
    leaf_of_row = np.empty(n, np.int32)
    for j, ids in enumerate(lv0.ids):
        leaf_of_row[ids] = j
    args = dict(leaf_centroids=lv0.centroids, leaf_of_row=leaf_of_row)
    if len(levels) > 1:
        pol = np.empty(lv0.n_part, np.int32)
        for p, leaves in enumerate(levels[1].ids):
            pol[leaves] = p
        args.update(parent_centroids=levels[1].centroids, parent_of_leaf=pol)
    return args


def make_index(I, X, ids, levels, **cfg):
    ix = I.Index(X.shape[1], n_leaf=levels[0].n_part,
                 n_parent=levels[1].n_part if len(levels) > 1 else 0, **cfg)
    ix.load(X, ids, **load_args(levels, X.shape[0]))
    return ix


# ------------------------------------------------------------------- estimator

@pytest.mark.parametrize("d", [1, 2, 3, 8, 64, 128, 768])
def test_cap_fraction_exact_matches_oracle(I, d):
    g = np.random.default_rng(d)
    rho = g.uniform(0.1, 10.0, 4000)
    t = rho * np.concatenate([g.uniform(0, 1.2, 3990), [0.0, 1.0, 0.999999, 1e-9, 0.5, 0.25, 2.0, 0.0, 0.7, 0.3]])
    rho[-3] = 0.0
    got = I.cap_fraction(d, t, rho, mode=1)
    want = np.array([capvol.cap_fraction([ti], ri, d)[0] for ti, ri in zip(t, rho)])
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("d", [64, 128, 768])
def test_cap_fraction_table_matches_oracle(I, d):
    g = np.random.default_rng(7 + d)
    rho = g.uniform(0.5, 5.0, 4000)
    t = rho * g.uniform(0, 1.1, 4000)
    got = I.cap_fraction(d, t, rho, mode=0)
    table = capvol.beta_table(d)
    want = np.array([capvol.cap_fraction_table([ti], ri, table)[0] for ti, ri in zip(t, rho)])
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-14)


# --------------------------------------------------------- fixed-nprobe (IVF)

def test_plain_ivf_fixed_nprobe_matches_oracle(I):
    """The plain-IVF workload at full size: 10k x 64, 100 partitions, nprobe 10, k 10."""
    X, ids, Q = synth.plain_ivf()
    levels = kmeans.build_index(X, ids, 100, 0, iters=10, seed=1234)
    ix = make_index(I, X, ids, levels)
    out = ix.search_scanned(Q, 10, recall_target=0.0, nprobe=10, cap0=16, cap1=4)
    gi, gd, gn, gr = out[:4]
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.0, nprobe=10))
    n_ok, n_exc = compare_search(out, orc, 10, check_r=False, label="plain IVF 10k x 64")
    assert n_exc == 0 and n_ok == Q.shape[0]
    assert (out[5] == -1).all()                  # one level: no parent partitions scanned
    assert np.isnan(gr).all() and (gn == 10).all()
    # recall against FP64 brute force is reported by the oracle, and must agree
    gtD, _ = knn.knn(X, ids, Q, 10)
    rg = knn.recall_at_k(gi, exact_dist(X, Q, gi), gtD, 10).mean()
    ro = knn.recall_at_k(orc["ids"], exact_dist(X, Q, orc["ids"]), gtD, 10).mean()
    assert rg == pytest.approx(ro, abs=1e-12)


@pytest.mark.parametrize("d", [32, 96, 256, 768])
def test_fixed_nprobe_dims(I, d):
    X, ids, Q = synth.plain_ivf(seed=40 + d, n=3000, d=d, n_comp=20, sigma=0.3, nq=24)
    levels = kmeans.build_index(X, ids, 37, 0, iters=3, seed=5)
    ix = make_index(I, X, ids, levels)
    for nprobe in (1, 5, 37):
        out = ix.search_scanned(Q, 7, recall_target=0.0, nprobe=nprobe, cap0=37, cap1=1)
        orc = aps.search(levels, Q, aps.Params(k=7, recall_target=0.0, nprobe=nprobe))
        n_ok, n_exc = compare_search(out, orc, 7, check_r=False, label=f"fixed nprobe {nprobe}, d = {d}")
        assert n_exc == 0


# ---------------------------------------------------------------------- APS

@pytest.mark.parametrize("mode", ["table", "exact"])
def test_aps_single_level_matches_oracle(I, mode):
    X, ids, Q = synth.aps_search(seed=11, n=20_000, d=64, n_comp=40, sigma=1.0, nq=150)
    levels = kmeans.build_index(X, ids, 150, 0, iters=5, seed=9)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.2, beta_mode=0 if mode == "table" else 1)
    out = ix.search_scanned(Q, 10, recall_target=0.9, cap0=30, cap1=1)
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.9, f_M=(0.2,), beta_mode=mode))
    compare_search(out, orc, 10, label=f"APS one level, {mode} beta")
    assert out[2].max() > 1 and out[2].min() >= 1      # APS really varied nprobe


def test_aps_two_level_matches_oracle(I):
    X, ids, Q = synth.aps_search(seed=12, n=30_000, d=128, n_comp=60, sigma=1.0, nq=120)
    levels = kmeans.build_index(X, ids, 300, 12, iters=5, seed=3)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.1, f_M_parent=0.5)
    out = ix.search_scanned(Q, 10, recall_target=0.9, cap0=30, cap1=6)
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.9, f_M=(0.1, 0.5)))
    compare_search(out, orc, 10, label="APS two levels")
    # access counts per partition are the scans the kernel reported (which
    # equal the oracle's for every query that was not excused)
    s0, s1 = out[4], out[5]
    assert np.array_equal(ix.hits(0), np.bincount(s0[s0 >= 0], minlength=300))
    assert np.array_equal(ix.hits(1), np.bincount(s1[s1 >= 0], minlength=12))
    assert ((s0 >= 0).sum(axis=1) == out[2]).all()
    st = ix.stats()
    assert st["hits"] == [int((s0 >= 0).sum()), int((s1 >= 0).sum())]
    assert st["levels"] == 2 and st["n_partitions"] == [300, 12] and st["n_vectors"] == 30_000


def test_full_scan_is_exact_knn(I):
    """f_M = 100% and an unreachable target scan everything: the result is exact kNN."""
    X, ids, Q = synth.aps_search(seed=13, n=8000, d=128, n_comp=30, sigma=1.0, nq=40)
    levels = kmeans.build_index(X, ids, 50, 5, iters=3, seed=2)
    ix = make_index(I, X, ids, levels, f_M_leaf=1.0, f_M_parent=1.0, upper_recall=2.0)
    gi, gd, gn, gr = ix.search(Q, 20, recall_target=2.0)
    D, Ix = knn.knn(X, ids, Q, 20)
    assert (gn == 50).all()
    for j in range(Q.shape[0]):
        assert same_topk(gi[j], gd[j], Ix[j], D[j])
    np.testing.assert_allclose(gr, 1.0, atol=1e-6)


# ----------------------------------------------------------------- edge cases

def test_edge_cases_padding_empty_partitions_and_device_io(I):
    import torch
    g = np.random.default_rng(3)
    d = 64
    X = g.standard_normal((300, d)).astype(np.float32)
    ids = (np.arange(300) * 7 + 11).astype(np.int64)
    C = g.standard_normal((12, d)).astype(np.float32)
    C[5] += 100.0                                      # a far centroid: its partition is empty
    a = kmeans.assign(X, C).astype(np.int32)
    assert (a != 5).all()
    ix = I.Index(d, n_leaf=12, f_M_leaf=1.0)
    ix.load(X, ids, C, a)
    Q = g.standard_normal((9, d)).astype(np.float32)
    Q[3] = X[17]                                       # a query equal to a stored vector
    # k larger than the whole index: unfilled slots are (-1, +inf)
    gi, gd, gn, gr = ix.search(Q, 400, recall_target=0.0, nprobe=12)
    assert (gi[:, 300:] == -1).all() and np.isinf(gd[:, 300:]).all()
    D, Ix = knn.knn(X, ids, Q, 400)
    for j in range(Q.shape[0]):
        assert same_topk(gi[j], gd[j], Ix[j], D[j])
    assert gi[3, 0] == ids[17] and gd[3, 0] == 0.0
    # device buffers in and out give the same answer as host buffers
    qd = torch.from_numpy(Q).cuda()
    ti, td, tn, tr = ix.search(qd, 10, recall_target=0.95)
    torch.cuda.synchronize()
    hi, hd, hn, hr = ix.search(Q, 10, recall_target=0.95)
    assert np.array_equal(ti.cpu().numpy(), hi) and np.array_equal(td.cpu().numpy(), hd)
    assert np.array_equal(tn.cpu().numpy(), hn)
    # empty query batch
    e = ix.search(np.zeros((0, d), np.float32), 10, recall_target=0.9)
    assert e[0].shape == (0, 10)


def test_invalid_arguments_are_rejected(I):
    from paper_2506_03437_b300 import _lib as L
    ix = I.Index(64, n_leaf=4)
    with pytest.raises(L.QkError) as e:
        ix.search(np.zeros((2, 64), np.float32), 5)
    assert e.value.status == L.ERR_STATE
    X = np.random.default_rng(0).standard_normal((50, 64)).astype(np.float32)
    ix.load(X, np.arange(50), X[:4].copy(), (np.arange(50) % 4).astype(np.int32))
    q = np.zeros((2, 64), np.float32)
    q[1, 3] = np.nan
    with pytest.raises(L.QkError) as e:
        ix.search(q, 5)
    assert e.value.status == L.ERR_ARG
    # device buffers: the kernel refuses the bad query, answers the other, and qk_check reports it
    import torch
    qd = torch.from_numpy(X[:2].copy()).cuda()
    qd[1, 5] = float("inf")
    gi, gd, gn, gr = ix.search(qd, 5, recall_target=0.0, nprobe=4)
    with pytest.raises(L.QkError) as e:
        ix.check()
    assert e.value.status == L.ERR_ARG
    assert int(gi[0, 0]) == 0 and float(gd[0, 0]) == 0.0 and int(gn[0]) == 4
    assert bool((gi[1] == -1).all()) and bool(torch.isnan(gd[1]).all()) and int(gn[1]) == 0
    ix.check()   # the status was cleared
    with pytest.raises(L.QkError):
        ix.search(np.zeros((2, 64), np.float32), 0)
    with pytest.raises(L.QkError) as e:
        ix.load(X, np.zeros(50, np.int64), X[:4].copy(), (np.arange(50) % 4).astype(np.int32))
    assert e.value.status == L.ERR_DUP_ID
    with pytest.raises(L.QkError) as e:
        ix.load(X, np.arange(50), X[:4].copy(), np.full(50, 9, np.int32))
    assert e.value.status == L.ERR_ARG
    with pytest.raises(L.QkError):
        I.Index(100)


def test_many_queries_per_cta_long_partitions(I):
    """Thousands of queries (each CTA runs many) over partitions of ~1,500 rows (many tiles)."""
    X, ids, Q = synth.aps_search(seed=14, n=60_000, d=128, n_comp=20, sigma=1.0, nq=3000)
    levels = kmeans.build_index(X, ids, 40, 0, iters=3, seed=4)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.5)
    out = ix.search_scanned(Q, 10, recall_target=0.9, cap0=20, cap1=1)
    gi, gd, gn, gr = out[:4]
    ix.check()
    assert ((gi >= 0) & (gi < 60_000)).all()
    assert (np.diff(gd, axis=1) >= 0).all()
    assert ((gn >= 1) & (gn <= 20)).all()
    sel = np.arange(0, 3000, 15)
    orc = aps.search(levels, Q[sel], aps.Params(k=10, recall_target=0.9, f_M=(0.5,)))
    compare_search(tuple(a[sel] for a in out), orc, 10, label="APS 3,000 queries, long partitions")


def test_per_query_nprobe_on_two_levels_equals_fixed_nprobe(I):
    """qk_search_nprobe with every query at nprobe n is the fixed-nprobe search at n (also with
    a parent level, where the leaves come from the upper level's APS), and mixed values match
    per query."""
    X, ids, Q = synth.aps_search(seed=61, n=30_000, d=64, n_comp=60, sigma=1.2, nq=120)
    levels = kmeans.build_index(X, ids, 100, 8, iters=3, seed=9)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.2, f_M_parent=0.5)
    per = np.random.default_rng(2).integers(1, 12, 120).astype(np.int32)
    gi, gd = ix.search_nprobe(Q, 10, per)
    for n in (1, 4, 11):
        fi, fd, fn, _ = ix.search(Q, 10, recall_target=0.0, nprobe=n)
        ui, ud = ix.search_nprobe(Q, 10, np.full(120, n, np.int32))
        assert np.array_equal(ui, fi) and np.array_equal(ud, fd)
        sel = per == n
        assert np.array_equal(gi[sel], fi[sel])


@pytest.mark.parametrize("two_level", [False, True])
def test_ratio_rule_matches_oracle(I, two_level):
    """SPANN's early-termination rule (reading R12): the partitions scanned, their
    number and the results equal the oracle's for several eps."""
    X, ids, Q = synth.aps_search(seed=15, n=20_000, d=64, n_comp=40, sigma=1.0, nq=120)
    levels = kmeans.build_index(X, ids, 150, 10 if two_level else 0, iters=4, seed=5)
    fm = (0.2, 0.5) if two_level else (0.2,)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.2, f_M_parent=0.5)
    counts = []
    for eps in (0.02, 0.1, 0.3):
        gi, gd, gn, s0 = ix.search_ratio(Q, 10, eps, cap0=30)
        orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.0, ratio_eps=eps, f_M=fm))
        n_ok, n_exc = compare_search((gi, gd, gn, np.full(Q.shape[0], np.nan), s0, None), orc, 10, check_r=False,
                                     label=f"ratio rule eps {eps}, {'two levels' if two_level else 'one level'}")
        assert n_exc == 0
        counts.append(gn.mean())
    assert counts[0] < counts[-1]                  # the rule really varied nprobe
