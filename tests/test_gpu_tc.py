"""Tensor-core centroid scoring (tcgen05, TF32) + exact FP32 re-score against the oracle."""

import numpy as np
import pytest

from oracle import knn

from .parity import same_topk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


def check(I, n, K, d, k, metric, seed):
    g = np.random.default_rng(seed)
    C = g.standard_normal((K, d)).astype(np.float32)
    X = (C[g.integers(0, K, n)] + 0.7 * g.standard_normal((n, d))).astype(np.float32)
    idx, dist = I.nearest_centroids(X, C, k, metric=metric)
    D, Ix = knn.knn(C, np.arange(K), X, k, metric=metric)
    bad = [j for j in range(n) if not same_topk(idx[j], dist[j], Ix[j], D[j])]
    assert not bad, (bad[:5], idx[bad[0]].tolist(), Ix[bad[0]].tolist())


def test_tc_small_first():
    from paper_2506_03437_b300 import index as I
    check(I, 130, 40, 32, 1, 0, 1)


@pytest.mark.parametrize("n,K,d,k,metric", [
    (1000, 300, 64, 1, 0), (777, 513, 128, 4, 0), (300, 1000, 256, 8, 0), (257, 64, 768, 8, 0),
    (500, 700, 128, 5, 1), (129, 33, 96, 8, 1),
])
def test_tc_nearest_matches_oracle(I, n, K, d, k, metric):
    check(I, n, K, d, k, metric, n + K + d)


def test_tc_rejects_k_beyond_margin(I):
    from paper_2506_03437_b300 import _lib as L
    X = np.zeros((4, 32), np.float32)
    C = np.zeros((40, 32), np.float32)
    with pytest.raises(L.QkError):
        I.nearest_centroids(X, C, 9)
