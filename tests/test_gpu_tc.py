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


@pytest.mark.parametrize("metric", [0, 1])
def test_tc_nearest_exact_on_near_ties(I, metric):
    """k = 1 is exact even where TF32 cannot order the centroids.  The rows sit far from
    the origin, so TF32's error (about 2^-9 ||x|| ||c||, here ~600) swamps the gaps
    between 64 centroids on a sphere of radius ~2 around them (radii 2e-4 apart, in
    shuffled order); 24 centroids are exact copies of others.  Every answer must be a
    nearest centroid within the FP32 evaluation error of the FP64 brute force, a copy
    must lose to its original (ties go to the lower index), and the distance must be
    the exact one.  Keeping the 4 best approximate candidates fails here."""
    g = np.random.default_rng(5 + metric)
    n, K, d = 300, 64, 128
    X = (50.0 + 0.01 * g.standard_normal((n, d))).astype(np.float32)
    u = g.standard_normal((K, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    C = (X.mean(0) + 2.0 * (1 + 2e-4 * g.permutation(K))[:, None] * u).astype(np.float32)
    C[40:] = C[:24]
    idx, dist = I.nearest_centroids(X, C, 1, metric=metric)
    idx = idx[:, 0]
    X64, C64 = X.astype(np.float64), C.astype(np.float64)
    if metric == 0:
        D = ((X64[:, None, :] - C64[None, :, :]) ** 2).sum(-1)
        scale = D.max(1)
    else:
        D = -(X64 @ C64.T)
        scale = (np.abs(X64) @ np.abs(C64).T).max(1)
    tol = 4 * (d + 2) * 2.0 ** -24 * scale       # FP32 evaluation error, with room
    chosen = D[np.arange(n), idx]
    assert np.all(chosen <= D.min(1) + tol), np.flatnonzero(chosen > D.min(1) + tol)[:5]
    assert not np.any(idx >= 40)
    np.testing.assert_allclose(dist[:, 0], chosen, rtol=0, atol=tol.max())
