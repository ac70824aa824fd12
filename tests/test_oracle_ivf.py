"""Pins of the oracle's per-query fixed-nprobe IVF search (R10 with one nprobe per query)."""

import numpy as np

from oracle import aps, kmeans, knn
from paper_2506_03437_b300 import synth


def hand_level():
    C = np.array([[0, 0], [10, 0], [0, 10]], np.float32)
    vecs = [np.array([[1, 0], [0, 1]], np.float32), np.array([[9, 0]], np.float32),
            np.array([[0, 9], [0, 12]], np.float32)]
    ids = [np.array([0, 1]), np.array([2]), np.array([3, 4])]
    return kmeans.Level(C, vecs, ids)


def test_hand_example():
    lv = hand_level()
    Q = np.array([[2, 0], [2, 0], [0, 7], [5, 5]], np.float32)
    D, I, scanned = aps.ivf_search(lv, Q, 3, [1, 2, 1, 1])
    # q=(2,0): centroid distances 4, 64, 104; nprobe 1 scans leaf 0 only
    assert list(scanned[0]) == [0] and list(I[0]) == [0, 1, -1]
    assert list(D[0][:2]) == [1.0, 5.0] and D[0][2] == np.inf
    assert list(scanned[1]) == [0, 1] and list(I[1]) == [0, 1, 2] and D[1][2] == 49.0
    # q=(0,7): leaf 2 is nearest (9 against 49 and 149)
    assert list(scanned[2]) == [2] and list(I[2][:2]) == [3, 4] and list(D[2][:2]) == [4.0, 25.0]
    # q=(5,5): all three centroids at 50, ties go to the lower index; the two rows tie at 41
    assert list(scanned[3]) == [0] and list(I[3][:2]) == [0, 1] and list(D[3][:2]) == [41.0, 41.0]


def test_all_partitions_equal_brute_force():
    X, ids, Q = synth.plain_ivf(seed=7, n=3000, d=16, n_comp=12, sigma=0.5, nq=20)
    lv = kmeans.build_index(X, ids, 25, 0, iters=3, seed=2)[0]
    D, I, _ = aps.ivf_search(lv, Q, 10, np.full(20, 25))
    Dk, Ik = knn.knn(X, ids, Q, 10)
    np.testing.assert_array_equal(I, Ik)
    np.testing.assert_allclose(D, Dk, rtol=1e-12)
    D2, I2, _ = aps.ivf_search(lv, Q, 10, np.full(20, 1000))   # more than the partitions there are
    np.testing.assert_array_equal(I2, Ik)


def test_uniform_nprobe_equals_fixed_nprobe_search():
    X, ids, Q = synth.plain_ivf(seed=8, n=2000, d=8, n_comp=10, sigma=0.4, nq=15)
    levels = kmeans.build_index(X, ids, 20, 0, iters=3, seed=3)
    for n in (1, 3, 7):
        D, I, scanned = aps.ivf_search(levels[0], Q, 5, n)
        r = aps.search(levels, Q, aps.Params(k=5, recall_target=0.0, nprobe=n))
        np.testing.assert_array_equal(I, r["ids"])
        for j in range(Q.shape[0]):
            assert list(scanned[j]) == r["scanned"][0][j]


def test_more_partitions_never_worse():
    X, ids, Q = synth.plain_ivf(seed=9, n=2500, d=12, n_comp=15, sigma=0.6, nq=12)
    lv = kmeans.build_index(X, ids, 30, 0, iters=3, seed=4)[0]
    prev_D, prev_s = None, None
    for n in range(1, 31):
        D, _, s = aps.ivf_search(lv, Q, 8, n)
        if prev_D is not None:
            assert np.all(D <= prev_D)
            for j in range(Q.shape[0]):
                assert list(s[j][:n - 1]) == list(prev_s[j])
        prev_D, prev_s = D, s
