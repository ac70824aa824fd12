"""Pins of the oracle's maintenance pass (Sec. 4) against the paper's worked example and invariants."""

import json
import os

import numpy as np

from oracle import kmeans, maintenance

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def example_level(d=32, seed=0):
    """Two partitions of 500: one that 2-means cuts 450/50 (index 0), one cut 250/250 (index 1)."""
    g = np.random.default_rng(seed)
    a, b, c, e = (g.standard_normal((4, d)) * 10).astype(np.float32)
    P2 = np.concatenate([a + 0.01 * g.standard_normal((450, d)), b + 0.01 * g.standard_normal((50, d))])
    P1 = np.concatenate([c + 0.01 * g.standard_normal((250, d)), e + 0.01 * g.standard_normal((250, d))])
    X = np.concatenate([P2, P1]).astype(np.float32)
    ids = np.arange(1000, dtype=np.int64)
    lab = np.repeat([0, 1], 500)
    C = np.stack([X[lab == j].astype(np.float64).mean(0) for j in (0, 1)]).astype(np.float32)
    return X, ids, C, lab


def example_lambda():
    with open(os.path.join(GOLDEN, "cost_example.json")) as f:
        g = json.load(f)
    # lambda at 2 and 3 centroids sets Delta O+ = 60 us for the two-partition level
    pts = [[2, 0.0], [3, 60.0]] + g["lambda_points"]
    return g, np.array(pts, np.float64)


def test_worked_example_end_to_end():
    g, pts = example_lambda()
    X, ids, C, lab = example_level()
    levels = kmeans.index_from_assignment(X, ids, C, lab)
    prm = maintenance.MaintParams(maintenance.Latency(pts[:, 0], pts[:, 1]), tau=g["tau"], alpha=g["alpha"],
                                  refine=False, s_min=0)
    log, keep = maintenance.maintain_level(levels[0], [g["A"], g["A"]], prm, 0)
    assert [(k, j, ok) for k, j, _, _, ok in log] == [("split", 0, False), ("split", 1, True)]
    assert abs(log[0][2] - g["delta_estimate"]) < 1e-9 and abs(log[1][2] - g["delta_estimate"]) < 1e-9
    assert abs(log[0][3] - g["P2_delta"]) < 1e-9 and abs(log[1][3] - g["P1_delta"]) < 1e-9
    assert sorted(v.shape[0] for v in levels[0].vectors) == [250, 250, 500]
    assert levels[0].vectors[0].shape[0] == 500               # the rejected partition is untouched


def test_pass_keeps_every_vector_and_lowers_modelled_cost():
    g = np.random.default_rng(3)
    cen = (3 * g.standard_normal((30, 16))).astype(np.float32)
    sizes = (2000 / np.arange(1, 31) ** 1.0).astype(int) + 5
    X = np.concatenate([c + 0.05 * g.standard_normal((s, 16)) for c, s in zip(cen, sizes)]).astype(np.float32)
    ids = np.arange(X.shape[0], dtype=np.int64)
    levels = kmeans.build_index(X, ids, 12, 0, iters=4, seed=5)
    A = np.linspace(0.5, 0.0, 12)
    lam = maintenance.Latency([0, 1000], [5.0, 55.0])
    prm = maintenance.MaintParams(lam, tau=0.01, alpha=0.9, refine_radius=4, s_min=100)
    before = maintenance.total_cost([A], [levels[0].sizes()], lam)
    log, keep = maintenance.maintain_level(levels[0], A, prm, 0)
    assert any(ok for *_, ok in log)
    for kind, j, e, dlt, ok in log:
        assert ok == (dlt is not None and dlt < -prm.tau)
    got = np.sort(np.concatenate(levels[0].ids))
    assert np.array_equal(got, ids)
    assert all(v.shape[0] == i.shape[0] for v, i in zip(levels[0].vectors, levels[0].ids))
    assert before > 0


def test_level_band_thresholds():
    f = maintenance.level_band_action
    assert f(16, 0) is None                       # 16 = 4 sqrt(16): the leaves are a valid top
    assert f(17, 0) == ("add_level", 4)           # round(sqrt(17)) = 4
    assert f(1000, 0) == ("add_level", 32)
    assert f(16, 4) == ("remove_level", 0)
    assert f(100, 10) is None
    assert f(100, 3) is None and f(100, 40) is None       # the band's ends, 2.5 and 40, are inside
    assert f(100, 2) == ("rebuild_level", 10) and f(100, 41) == ("rebuild_level", 10)
    assert f(30, 0) == ("add_level", 5) and f(42, 0) == ("add_level", 6)   # 5.48 -> 5, 6.48 -> 6
    assert f(1, 0) is None


def test_maintain_adds_a_parent_level_under_the_band():
    """One level of 40 leaves: after the pass the index has round(sqrt(40)) = 6 parents, which are
    the build's parents of the pass's leaf centroids, every leaf under exactly one."""
    from oracle import kmeans
    g = np.random.default_rng(0)
    X = (g.standard_normal((4000, 8)) + 4 * np.repeat(g.standard_normal((40, 8)), 100, axis=0)).astype(np.float32)
    ids = np.arange(4000, dtype=np.int64)
    levels = kmeans.build_index(X, ids, 40, 0, iters=3, seed=5)
    lam = maintenance.Latency([0, 1000], [5.0, 55.0])
    prm = maintenance.MaintParams(lam, tau=1e9, level_band=True, level_iters=4, seed=5)   # no split or merge
    logs = maintenance.maintain(levels, [np.ones(40)], 40, prm)
    assert len(levels) == 2 and levels[1].n_part == 6
    assert logs[1] == [("add_level", 6, logs[1][0][2], logs[1][0][3], True)]
    want = kmeans.build_index(levels[0].centroids, np.arange(40, dtype=np.int64), 6, 0, iters=4, seed=6)[0]
    np.testing.assert_array_equal(levels[1].centroids, want.centroids)
    members = np.sort(np.concatenate(levels[1].ids))
    assert np.array_equal(members, np.arange(40))
    # and with 16 leaves the parent level goes away again
    small = kmeans.build_index(X, ids, 16, 4, iters=3, seed=5)
    logs = maintenance.maintain(small, [np.ones(16), np.ones(4)], 16, prm)
    assert len(small) == 1 and logs[1][-1][0] == "remove_level"
