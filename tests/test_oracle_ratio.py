"""Pins of the oracle's SPANN early-termination rule (reading R12; Sec. 2
"Early Termination" and the comparators of Table 6): scan the candidates whose
Euclidean centroid distance is within (1 + eps) of the nearest one's."""

import numpy as np

from oracle import aps, kmeans, knn
from paper_2506_03437_b300 import synth


def test_ratio_count_hand_case():
    # Euclidean candidate distances 1.0, 1.04, 1.1, 1.5, 2.0 given as squared distances
    D = np.array([1.0, 1.04, 1.1, 1.5, 2.0]) ** 2
    assert aps.ratio_rule_count(D, 0.0) == 1
    assert aps.ratio_rule_count(D, 0.05) == 2       # on squared distances 1.0816 > 1.05 would give 1
    assert aps.ratio_rule_count(D, 0.12) == 3
    assert aps.ratio_rule_count(D, 0.6) == 4
    assert aps.ratio_rule_count(D, 2.0) == 5


def _index(two_level):
    X, ids, Q = synth.plain_ivf(seed=21, n=4000, d=8, n_comp=16, sigma=0.6, nq=20)
    return X, ids, Q, kmeans.build_index(X, ids, 40, 6 if two_level else 0, iters=4, seed=2)


def test_ratio_rule_zero_scans_the_nearest_partition_only():
    X, ids, Q, lv = _index(False)
    res = aps.search(lv, Q, aps.Params(k=5, recall_target=0.0, ratio_eps=1e-12, f_M=(0.5,)))
    assert (res["nprobe"] == 1).all()
    for j in range(Q.shape[0]):
        dc = ((lv[0].centroids.astype(np.float64) - Q[j]) ** 2).sum(1)
        p0 = int(np.lexsort((np.arange(40), dc))[0])
        assert res["scanned"][0][j] == [p0]
        D, I = knn.knn(lv[0].vectors[p0], lv[0].ids[p0], Q[j:j + 1], 5)
        assert res["ids"][j].tolist() == I[0].tolist()


def test_ratio_rule_is_monotone_and_large_eps_scans_all_candidates():
    for two_level in (False, True):
        X, ids, Q, lv = _index(two_level)
        fm = (0.5, 1.0) if two_level else (0.5,)
        prev = np.zeros(Q.shape[0])
        for eps in (0.01, 0.05, 0.2, 0.5, 1.0):
            res = aps.search(lv, Q, aps.Params(k=5, recall_target=0.0, ratio_eps=eps, f_M=fm))
            assert (res["nprobe"] >= prev).all()
            prev = res["nprobe"]
        big = aps.search(lv, Q, aps.Params(k=5, recall_target=0.0, ratio_eps=1e6, f_M=fm))
        assert (big["nprobe"] == 20).all()          # every candidate of S (M = 0.5 * 40)
        full = aps.search(lv, Q, aps.Params(k=5, recall_target=2.0, f_M=fm))   # APS until S runs out
        assert np.array_equal(big["ids"], full["ids"])
