"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against a closed form, a published value,
a brute-force enumeration on a tiny input or an invariant the paper states, so
that a dropped term, a wrong sign or index, or a transposed operand in the
oracle fails at least one of them.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import aps, capvol, kmeans, knn, maintenance
from paper_2506_03437_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ exact kNN

def _rank_bruteforce(X, ids, q, k, metric):
    """Top-k by counting, for each row, how many rows precede it in (dist, id) order."""
    n = X.shape[0]
    dist = []
    for x in X:
        if metric == knn.L2:
            dist.append(sum((float(a) - float(b)) ** 2 for a, b in zip(q, x)))
        else:
            dist.append(-sum(float(a) * float(b) for a, b in zip(q, x)))
    rank = [sum(1 for j in range(n) if (dist[j], ids[j]) < (dist[i], ids[i])) for i in range(n)]
    out = sorted((rank[i], i) for i in range(n) if rank[i] < k)
    return [dist[i] for _, i in out], [int(ids[i]) for _, i in out]


@pytest.mark.parametrize("metric", [knn.L2, knn.IP])
def test_knn_matches_rank_counting(metric):
    g = np.random.default_rng(0)
    X = g.standard_normal((40, 5)).astype(np.float32)
    X[7] = X[3]            # a duplicate vector: the tie goes to the lower id
    ids = g.permutation(1000)[:40].astype(np.int64)
    Q = g.standard_normal((6, 5)).astype(np.float32)
    D, I = knn.knn(X, ids, Q, 7, metric)
    for j in range(Q.shape[0]):
        bd, bi = _rank_bruteforce(X, ids, Q[j], 7, metric)
        assert list(I[j]) == bi
        np.testing.assert_allclose(D[j], bd, rtol=1e-12, atol=1e-12)


def test_knn_hand_case_and_padding():
    X = np.array([[0.0, 0.0], [3.0, 4.0], [1.0, 0.0], [0.0, -2.0]], np.float32)
    ids = np.array([10, 11, 12, 13])
    D, I = knn.knn(X, ids, np.array([[0.0, 0.0]]), 6)
    assert list(I[0]) == [10, 12, 13, 11, -1, -1]
    assert list(D[0][:4]) == [0.0, 1.0, 4.0, 25.0]
    assert np.isinf(D[0][4:]).all()
    D2, I2 = knn.knn(X, ids, np.array([[0.0, 0.0]]), 3, bulk=True)
    assert list(I2[0]) == [10, 12, 13]


def test_recall_counts_ties():
    gt = np.array([[1.0, 2.0, 3.0]])
    assert knn.recall_at_k(np.array([[5, 6, 7]]), np.array([[1.0, 2.0, 3.0]]), gt, 3)[0] == 1.0
    assert knn.recall_at_k(np.array([[5, 6, 7]]), np.array([[1.0, 2.0, 3.5]]), gt, 3)[0] == pytest.approx(2 / 3)
    assert knn.recall_at_k(np.array([[5, -1, 7]]), np.array([[1.0, np.inf, 3.0]]), gt, 3)[0] == pytest.approx(2 / 3)


# -------------------------------------------------------------------- k-means

def test_splitmix64_published_vectors():
    with open(os.path.join(GOLDEN, "splitmix64.json")) as f:
        gold = json.load(f)
    for seq in gold["sequences"]:
        s = seq["seed"]
        for want in seq["outputs"]:
            s, z = kmeans.splitmix64_next(s)
            assert z == int(want, 0)


def test_init_rows_distinct_and_full_permutation():
    r = kmeans.init_rows(50, 50, 7)
    assert sorted(r.tolist()) == list(range(50))
    r = kmeans.init_rows(1000, 30, 9)
    assert len(set(r.tolist())) == 30 and r.min() >= 0 and r.max() < 1000


def test_kmeans_one_cluster_is_the_mean():
    g = np.random.default_rng(1)
    X = g.standard_normal((101, 3)).astype(np.float32)
    C = kmeans.lloyd(X, 1, 2, 5)
    want = np.array([sum(float(x[j]) for x in X) / 101 for j in range(3)], np.float32)
    np.testing.assert_array_equal(C[0], want)


def test_kmeans_hand_case_1d():
    X = np.array([[0.0], [1.0], [10.0], [11.0]], np.float32)
    C = np.array([[0.0], [1.0]], np.float32)
    a = kmeans.assign(X, C)
    assert a.tolist() == [0, 1, 1, 1]
    C1, counts = kmeans.update(X, a, C)
    assert counts.tolist() == [1, 3]
    assert C1[:, 0].tolist() == [0.0, np.float32(22.0 / 3.0)]
    C2 = kmeans.lloyd(X, 2, 2, 0, C0=C)
    assert C2[:, 0].tolist() == [0.5, 10.5]


def test_kmeans_ties_lower_index_and_empty_cluster_kept():
    X = np.array([[0.0], [2.0]], np.float32)
    C = np.array([[1.0], [1.0], [50.0]], np.float32)
    assert kmeans.assign(X, C).tolist() == [0, 0]
    C1, counts = kmeans.update(X, kmeans.assign(X, C), C)
    assert counts.tolist() == [2, 0, 0]
    assert C1[:, 0].tolist() == [1.0, 1.0, 50.0]


def test_kmeans_objective_non_increasing():
    X, _, _ = synth.plain_ivf(n=2000, nq=1)
    C = X[kmeans.init_rows(X.shape[0], 20, 3)].copy()
    prev = math.inf
    for _ in range(6):
        a = kmeans.assign(X, C)
        obj = kmeans.objective(X, C, a)
        assert obj <= prev * (1 + 1e-12)
        prev = obj
        C, _ = kmeans.update(X, a, C)


def test_assign_matches_direct_difference():
    g = np.random.default_rng(2)
    X = g.standard_normal((300, 16)).astype(np.float32)
    C = g.standard_normal((25, 16)).astype(np.float32)
    a = kmeans.assign(X, C)
    for i in range(0, 300, 17):
        d = [sum((float(x) - float(c)) ** 2 for x, c in zip(X[i], cc)) for cc in C]
        assert a[i] == min(range(25), key=lambda j: (d[j], j))


# --------------------------------------------------------- cap volume fraction

@pytest.mark.parametrize("s", [0.0, 0.1, 0.37, 0.5, 0.8, 0.99])
def test_cap_low_dimension_closed_forms(s):
    rho = 2.5
    t = s * rho
    # d = 1: the segment [t, rho] of [-rho, rho]
    assert capvol.cap_fraction([t], rho, 1)[0] == pytest.approx(0.5 * (1 - s), abs=1e-13)
    # d = 2: circular segment area rho^2 (theta - sin theta) / 2 over pi rho^2
    th = 2 * math.acos(s)
    assert capvol.cap_fraction([t], rho, 2)[0] == pytest.approx((th - math.sin(th)) / (2 * math.pi), abs=1e-13)
    # d = 3: spherical cap pi h^2 (3 rho - h) / 3 over 4/3 pi rho^3
    h = rho - t
    assert capvol.cap_fraction([t], rho, 3)[0] == pytest.approx(h * h * (3 * rho - h) / (4 * rho ** 3), abs=1e-13)


def test_cap_special_values():
    for d in (2, 64, 128, 768):
        assert capvol.cap_fraction([0.0], 1.0, d)[0] == pytest.approx(0.5, abs=1e-14)
        assert capvol.cap_fraction([1.0, 2.0], 1.0, d).tolist() == [0.0, 0.0]
    assert capvol.cap_fraction([0.0], 0.0, 8)[0] == 0.0


def test_cap_monte_carlo_d8():
    g = np.random.default_rng(3)
    n, d = 1_000_000, 8
    v = g.standard_normal((n, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v *= g.uniform(size=(n, 1)) ** (1.0 / d)
    for t in (0.1, 0.3, 0.6):
        frac = float((v[:, 0] > t).mean())
        want = capvol.cap_fraction([t], 1.0, d)[0]
        assert abs(frac - want) < 4.5 * math.sqrt(want * (1 - want) / n)


def test_beta_table_endpoints_and_interpolation():
    for d in (64, 128):
        T = capvol.beta_table(d)
        assert T.shape == (1024,)
        assert T[0] == 0.0 and T[-1] == pytest.approx(1.0, abs=1e-15)
        assert np.all(np.diff(T) >= 0)
        # at grid points the table equals the exact value; between them it is a chord
        x = np.array([5 / 1023, 700 / 1023])
        np.testing.assert_allclose(capvol.interp_table(T, x), T[[5, 700]], rtol=0, atol=1e-15)
        mid = (np.arange(1023) + 0.5) / 1023
        iv = capvol.interp_table(T, mid)
        np.testing.assert_allclose(iv, 0.5 * (T[:-1] + T[1:]), atol=1e-14)


# -------------------------------------------------------------- APS estimator

def test_probabilities_hand_case_2d():
    """q = 0 with four centroids; t from the bisector geometry, caps from the segment formula."""
    q = np.zeros(2)
    C = np.array([[1.0, 0.0], [-1.0, 0.0], [0.0, 3.0], [3.0, 0.0]])
    D = ((C - q) ** 2).sum(1)

    def t_geom(c0, ci):
        m = 0.5 * (c0 + ci)
        nrm = (ci - c0) / np.linalg.norm(ci - c0)
        return float(np.dot(m - q, nrm))

    t = aps.bisector_distances(D, C)
    assert t[1] == pytest.approx(0.0, abs=1e-15)
    assert t[2] == pytest.approx(t_geom(C[0], C[2]), abs=1e-14) and t[2] == pytest.approx(4 / math.sqrt(10))
    assert t[3] == pytest.approx(2.0)
    rho = 2.0
    th = 2 * math.acos(t[2] / rho)
    u = [0.5, (th - math.sin(th)) / (2 * math.pi), 0.0]
    p0 = (1 - u[0]) * (1 - u[1]) * (1 - u[2])
    p = aps.probabilities(t, rho, 2, mode="exact")
    assert p[0] == pytest.approx(p0, abs=1e-13)
    assert p[1] == pytest.approx((1 - p0) * u[0] / sum(u), abs=1e-13)
    assert p[2] == pytest.approx((1 - p0) * u[1] / sum(u), abs=1e-13)
    assert p[3] == 0.0
    assert p.sum() == pytest.approx(1.0, abs=1e-14)


def test_probabilities_degenerate():
    assert aps.probabilities(np.array([0.0]), 1.0, 4, "exact").tolist() == [1.0]
    p = aps.probabilities(np.array([0.0, 5.0, 6.0]), 1.0, 4, "exact")
    assert p.tolist() == [1.0, 0.0, 0.0]


def test_inner_product_on_the_unit_sphere_is_the_l2_search():
    # on unit-norm rows and queries -<q, x> = (||q - x||^2 - 2) / 2: same order, and
    # rho = ||q - x_k|| either way (R1, R11), so two-level APS must make the same choices
    X, ids, Q = synth.plain_ivf(seed=12, n=4000, d=16, n_comp=20, sigma=0.5, nq=25)
    X, Q = synth.unit_rows(X), synth.unit_rows(Q)
    levels = kmeans.build_index(X, ids, 40, 6, iters=4, seed=3)
    prm = aps.Params(k=10, recall_target=0.9, f_M=(0.2, 0.5), beta_mode="exact")
    r2 = aps.search(levels, Q, prm, metric=knn.L2)
    ri = aps.search(levels, Q, prm, metric=knn.IP)
    same = sum(r2["scanned"][0][j] == ri["scanned"][0][j] and np.array_equal(r2["ids"][j], ri["ids"][j])
               for j in range(Q.shape[0]))
    assert same >= Q.shape[0] - 1          # FP64 rounding may flip one near-tied decision
    # unit_rows normalises in FP32, so the norms are 1 to about 1e-7
    np.testing.assert_allclose(ri["dist"], (r2["dist"] - 2.0) / 2.0, atol=1e-6)
    # and IP recall against brute force is that of L2
    D, I = knn.knn(X, ids, Q, 10, metric=knn.IP)
    assert np.mean([len(set(ri["ids"][j]) & set(I[j])) for j in range(25)]) >= 8.0


def _small_index(seed=4, n=3000, d=8, n_leaf=30, n_parent=0):
    X, ids, Q = synth.plain_ivf(seed=seed, n=n, d=d, n_comp=12, sigma=0.6, nq=12)
    lv = kmeans.build_index(X, ids, n_leaf, n_parent, iters=4, seed=seed)
    return X, ids, Q, lv


def test_full_scan_gives_exact_knn_and_unit_recall():
    X, ids, Q, lv = _small_index()
    prm = aps.Params(k=10, recall_target=1.5, f_M=(1.0,))
    res = aps.search(lv, Q, prm)
    D, I = knn.knn(X, ids, Q, 10)
    assert (res["ids"] == I).all()
    np.testing.assert_allclose(res["dist"], D, rtol=1e-12)
    assert (res["nprobe"] == 30).all()
    # every p is spent once every candidate is scanned
    assert np.allclose(res["r"], 1.0, atol=1e-12)


def test_fixed_nprobe_equals_bruteforce_over_probed_partitions():
    X, ids, Q, lv = _small_index()
    for nprobe in (1, 3, 7):
        prm = aps.Params(k=5, recall_target=0.0, nprobe=nprobe)
        res = aps.search(lv, Q, prm)
        for j in range(Q.shape[0]):
            dc = ((lv[0].centroids.astype(np.float64) - Q[j]) ** 2).sum(1)
            probe = sorted(range(30), key=lambda c: (dc[c], c))[:nprobe]
            assert res["scanned"][0][j] == probe
            rows = np.concatenate([lv[0].vectors[c] for c in probe])
            rid = np.concatenate([lv[0].ids[c] for c in probe])
            bd, bi = _rank_bruteforce(rows, rid, Q[j], 5, knn.L2)
            assert res["ids"][j].tolist()[: len(bi)] == bi


def test_fixed_nprobe_recall_non_decreasing():
    X, ids, Q, lv = _small_index()
    gtD, _ = knn.knn(X, ids, Q, 10)
    prev = np.zeros(Q.shape[0])
    for nprobe in range(1, 31, 3):
        res = aps.search(lv, Q, aps.Params(k=10, recall_target=0.0, nprobe=nprobe))
        ex = np.array([[((X[i] - Q[j].astype(np.float64)) ** 2).sum() if i >= 0 else np.inf
                        for i in res["ids"][j]] for j in range(Q.shape[0])])
        rec = knn.recall_at_k(res["ids"], ex, gtD, 10)
        assert (rec >= prev - 1e-12).all()
        prev = rec
    assert (prev == 1.0).all()


def test_aps_order_is_descending_p_without_recompute():
    X, ids, Q, lv = _small_index()
    prm = aps.Params(k=10, recall_target=0.999, f_M=(0.5,), tau_rho=1e30, beta_mode="exact")
    for j in range(Q.shape[0]):
        q = Q[j].astype(np.float64)
        cand, cD = aps.root_candidates(q, lv[0], 0.5)
        res = aps.aps_level(q, lv[0], list(cand), cD, 10, 0.999, prm, 8, knn.L2, None)
        sc = res["scanned"]
        # find where R first held k results, then p is frozen: the rest is by descending p
        sizes = np.cumsum([lv[0].vectors[cand[p]].shape[0] for p in sc])
        first = int(np.argmax(sizes >= 10))
        R = aps._TopK(10)
        for p in sc[: first + 1]:
            c = cand[p]
            R.add(knn.distances(q, lv[0].vectors[c], knn.L2), lv[0].ids[c], lv[0].vectors[c])
        t = aps.bisector_distances(cD, lv[0].centroids[cand])
        pr = aps.probabilities(t, math.sqrt(R.dist[9]), 8, "exact")
        rest = [p for p in range(len(cand)) if p not in sc[: first + 1]]
        want = sorted(rest, key=lambda p: (-pr[p], p))
        got = sc[first + 1:]
        assert got == want[: len(got)]
        # stop rule: r crossed tau_R exactly at the last scan (or S ran out)
        r_seq = [pr[0] + sum(pr[p] for p in sc[1: i + 1] if p != 0) for i in range(len(sc))]
        if len(sc) < len(cand):
            assert r_seq[-1] >= 0.999 and all(r < 0.999 for r in r_seq[first:-1])


def test_r_non_decreasing_between_recomputes():
    X, ids, Q, lv = _small_index()
    prm = aps.Params(k=10, recall_target=0.95, f_M=(0.6,))
    res = aps.search(lv, Q, prm)
    for tr in res["traces"][0]:
        last = None
        for kind, step, val in tr:
            if kind == "recompute" and val > 0:
                last = None
            if kind == "stop":
                r = val + 0.95
                if last is not None:
                    assert r >= last - 1e-15
                last = r


def test_two_level_full_targets_equal_single_level_full_scan():
    X, ids, Q, lv = _small_index(n_leaf=30, n_parent=5)
    prm = aps.Params(k=10, recall_target=1.5, f_M=(1.0, 1.0), upper_recall=1.5)
    res = aps.search(lv, Q, prm)
    D, I = knn.knn(X, ids, Q, 10)
    assert (res["ids"] == I).all()
    assert (res["nprobe"] == 30).all()
    assert all(len(s) == 5 for s in res["scanned"][1])


def test_two_level_candidates_are_nearest_leaf_centroids():
    X, ids, Q, lv = _small_index(n_leaf=30, n_parent=5)
    prm = aps.Params(k=10, recall_target=0.0, nprobe=4, f_M=(0.2, 1.0), upper_recall=1.5)
    res = aps.search(lv, Q, prm)
    for j in range(Q.shape[0]):
        dc = ((lv[0].centroids.astype(np.float64) - Q[j]) ** 2).sum(1)
        want = sorted(range(30), key=lambda c: (dc[c], c))[:4]
        assert res["scanned"][0][j] == want


def test_n_candidates_rounding():
    assert aps.n_candidates(0.1, 1000) == 100
    assert aps.n_candidates(0.25, 32) == 8
    assert aps.n_candidates(0.001, 10) == 1
    assert aps.n_candidates(2.0, 10) == 10


# ----------------------------------------------------------------- cost model

def test_cost_model_worked_example():
    with open(os.path.join(GOLDEN, "cost_example.json")) as f:
        g = json.load(f)
    lam = maintenance.Latency(*zip(*g["lambda_points"]))
    s, A, a, dO, tau = g["s"], g["A"], g["alpha"], g["dO_plus"], g["tau"]
    assert maintenance.partition_cost(A, lam(s)) == pytest.approx(g["C_before"])
    est = maintenance.delta_split_estimate(dO, A, lam(s), lam(s / 2), a)
    assert est == pytest.approx(g["delta_estimate"])
    assert maintenance.decide(est, tau)
    for name in ("P1", "P2"):
        sl, sr = g[name + "_children"]
        dl = maintenance.delta_split_exact(dO, A, lam(s), a * A, lam(sl), a * A, lam(sr))
        assert dl == pytest.approx(g[name + "_delta"])
        assert maintenance.decide(dl, tau) == g[name + "_commit"]


def test_total_cost_and_merge_delta():
    lam = maintenance.Latency([0, 100], [0.0, 100.0])      # lambda(s) = s
    assert maintenance.total_cost([[0.5, 0.25], [1.0]], [[10, 40], [2]], lam) == pytest.approx(5 + 10 + 2)
    # merging a partition of 10 (A = 0.1) into one receiver of 30 (A = 0.2)
    d = maintenance.delta_merge_exact(-1.0, 0.1, 10.0, [(0.2, 0.1, 40.0, 30.0)])
    assert d == pytest.approx(-1.0 - 1.0 + (0.3 * 40 - 0.2 * 30))


def test_latency_interpolation_and_extension():
    lam = maintenance.Latency([50, 250, 450, 500], [250, 550, 1050, 1200])
    assert lam(150) == pytest.approx(400.0)
    assert lam(600) == pytest.approx(1500.0)        # last segment extended
    assert lam(0) == pytest.approx(175.0)           # first segment extended
    assert lam(-1000) == 0.0


# ------------------------------------------------------------- insert/delete

def test_insert_delete_live_set_and_full_scan():
    X, ids, Q, lv = _small_index(n_leaf=20, n_parent=4)
    g = np.random.default_rng(5)
    live = {int(i): X[n] for n, i in enumerate(ids)}
    newX = (X[g.integers(0, X.shape[0], 200)] + 0.05 * g.standard_normal((200, 8))).astype(np.float32)
    newI = np.arange(10_000, 10_200, dtype=np.int64)
    leaves = maintenance.insert(lv, newX, newI)
    for x, i, leaf in zip(newX, newI, leaves):
        live[int(i)] = x
        # greedy descent: nearest parent, then nearest of its children
        dp = ((lv[1].centroids.astype(np.float64) - x) ** 2).sum(1)
        par = int(np.argmin(dp))
        ch = lv[1].ids[par]
        dl = ((lv[0].centroids[ch].astype(np.float64) - x) ** 2).sum(1)
        assert leaf == ch[int(np.lexsort((ch, dl))[0])]
    dele = np.concatenate([g.choice(ids, 300, replace=False), newI[:50], np.array([99_999])])
    assert maintenance.delete(lv, dele) == 350
    for i in dele:
        live.pop(int(i), None)
    got = {}
    for v, pid in zip(lv[0].vectors, lv[0].ids):
        for row, i in zip(v, pid):
            assert int(i) not in got
            got[int(i)] = row
    assert set(got) == set(live)
    for i in list(live)[::97]:
        np.testing.assert_array_equal(got[i], live[i])
    # a full scan over the updated index equals brute force over the live set
    allI = np.array(sorted(live), dtype=np.int64)
    allX = np.stack([live[int(i)] for i in allI])
    D, I = knn.knn(allX, allI, Q, 10)
    res = aps.search(lv, Q, aps.Params(k=10, recall_target=1.5, f_M=(1.0, 1.0), upper_recall=1.5))
    assert (res["ids"] == I).all()


def test_refine_keeps_vectors_and_assigns_to_nearest():
    X, ids, Q, lv = _small_index(n_leaf=10)
    before = sorted(np.concatenate(lv[0].ids).tolist())
    maintenance.refine(lv[0], [0, 3, 4], iters=1)
    assert sorted(np.concatenate(lv[0].ids).tolist()) == before
    for j in (0, 3, 4):
        for x in lv[0].vectors[j]:
            d = ((lv[0].centroids[[0, 3, 4]].astype(np.float64) - x) ** 2).sum(1)
            assert [0, 3, 4][int(np.argmin(d))] == j


def test_oracle_does_not_import_product():
    import oracle
    src = []
    for fn in os.listdir(os.path.dirname(oracle.__file__)):
        if fn.endswith(".py"):
            with open(os.path.join(os.path.dirname(oracle.__file__), fn)) as f:
                src.append(f.read())
    assert not any("paper_2506_03437_b300" in s for s in src)
    assert itertools is not None
