"""Exact k-nearest-neighbour search and Recall@k (oracle; test infrastructure only).

Follows Sec. 2.1 ("Vector Search Workload"): the answer to a query q is the
top-k nearest vectors of X; Recall@k = |G n R| / k.

Distance conventions used across the oracle and the library:
  L2  dist(q, x) = sum_i (q_i - x_i)^2        (squared Euclidean, smaller = nearer)
  IP  dist(q, x) = -<q, x>                     (negated inner product, smaller = nearer)
Ranking is by (dist, id) ascending, so equal distances resolve to the lower id.
"""

import numpy as np

L2 = 0
IP = 1


def distances(q, rows, metric):
    """FP64 distance from one query to each row, written out from its definition."""
    q = np.asarray(q, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.float64)
    if metric == L2:
        diff = rows - q[None, :]
        return (diff * diff).sum(axis=1)
    return -(rows @ q)


def distances_bulk(Q, X, metric):
    """FP64 distance matrix |Q| x |X|.

    For L2 the squared distance is expanded as ||q||^2 - 2<q,x> + ||x||^2 and
    the inner products come from one FP64 matmul.  The expansion is an exact
    identity; its FP64 rounding (about 1e-13 relative at the norms used here)
    is far below every tolerance in the tests.  Used only where the direct form
    would take minutes (brute force over large sets, k-means assignment).
    """
    Q = np.asarray(Q, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    G = Q @ X.T
    if metric == IP:
        return -G
    qn = (Q * Q).sum(axis=1)
    xn = (X * X).sum(axis=1)
    D = qn[:, None] - 2.0 * G + xn[None, :]
    np.maximum(D, 0.0, out=D)
    return D


def topk_by_dist_id(dist, ids, k):
    """Indices of the k smallest (dist, id) pairs, in ascending order."""
    order = np.lexsort((ids, dist))
    return order[:k]


def knn(X, ids, Q, k, metric=L2, bulk=False, chunk=256):
    """Exact top-k of every query over all rows of X.

    Returns (D, I): FP64 distances and int64 ids, shape (nq, k), rows sorted by
    (dist, id).  Slots beyond |X| are (inf, -1).
    """
    X = np.asarray(X)
    ids = np.asarray(ids, dtype=np.int64)
    Q = np.atleast_2d(np.asarray(Q))
    nq = Q.shape[0]
    D = np.full((nq, k), np.inf)
    I = np.full((nq, k), -1, dtype=np.int64)
    kk = min(k, X.shape[0])
    if bulk:
        for s in range(0, nq, chunk):
            M = distances_bulk(Q[s:s + chunk], X, metric)
            for j in range(M.shape[0]):
                sel = topk_by_dist_id(M[j], ids, kk)
                D[s + j, :kk] = M[j][sel]
                I[s + j, :kk] = ids[sel]
        return D, I
    for j in range(nq):
        dj = distances(Q[j], X, metric)
        sel = topk_by_dist_id(dj, ids, kk)
        D[j, :kk] = dj[sel]
        I[j, :kk] = ids[sel]
    return D, I


def recall_at_k(found_ids, found_dist_exact, gt_dist, k, rel_tol=1e-5):
    """Recall@k = |G n R| / k (Sec. 2.1), with distance ties counted as hits.

    A returned id is a hit when its exact distance is within the k-th ground
    truth distance (times 1 + rel_tol, plus rel_tol absolute for distances
    near zero), so that any of several equally near vectors counts.
    `found_dist_exact` must be the exact FP64 distances of the returned ids
    (inf for empty slots).  Returns the per-query recall array.
    """
    found_dist_exact = np.atleast_2d(found_dist_exact)
    gt_dist = np.atleast_2d(gt_dist)
    kth = gt_dist[:, k - 1]
    thr = kth + rel_tol * np.abs(kth) + rel_tol
    ok = (np.atleast_2d(found_ids)[:, :k] >= 0) & (found_dist_exact[:, :k] <= thr[:, None])
    return ok.sum(axis=1) / float(k)
