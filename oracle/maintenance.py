"""Cost model, maintenance actions, inserts and deletes (oracle; test infrastructure only).

Follows Sec. 3 ("Adaptive Incremental Maintenance": inserts append to the
nearest leaf found top-down, deletes compact immediately) and Sec. 4 (cost
model Eq. 1-3, exact deltas Eq. 4-5, split estimate Eq. 6, the
estimate / verify / commit workflow).  Readings where the paper defers to its
technical report:

  M1  lambda(s) is a table of profiled (size, latency) points interpolated
      linearly, extended linearly past both ends and floored at 0.
  M2  Delta O+ = lambda(N_l + 1) - lambda(N_l) and Delta O- = lambda(N_l - 1)
      - lambda(N_l): the centroid-scan latency of level l with one centroid
      more or fewer.
  M3  Merge estimate (uniform redistribution): the receivers are the
      n_R = min(r_f, N_l - 1) centroids nearest to c_j, each gaining s_j / n_R
      vectors and A_j / n_R access frequency.
  M4  A merge is considered only for partitions with s_j < s_min (a parameter).
  M5  Verified merge: every vector of j goes to its nearest remaining centroid;
      receiver m gains Delta s_m = its count and Delta A_m = A_j Delta s_m / s_j.
  M6  Verified split: the children's real sizes, each child with alpha A_j
      (the Stage-1 frequency assumption is kept, Stage 2).
  M7  Split = 2-means inside the partition (seeded rows, fixed iterations),
      then one refinement pass: a Lloyd iteration seeded by the current
      centroids over the r_f partitions nearest the two new centroids.
  M8  Partitions are processed in ascending order of their estimated delta;
      N_l is updated after every commit.  Insert descends greedily (the
      nearest centroid at each level, ties to the lower index).  Delete swaps
      the last row of the partition into the freed slot.
"""

import numpy as np

from . import kmeans as km
from .knn import L2, distances


# ----------------------------------------------------------------- cost model

class Latency:
    """lambda(s): profiled scan latency in microseconds for s vectors (M1)."""

    def __init__(self, sizes, micros):
        self.s = np.asarray(sizes, dtype=np.float64)
        self.us = np.asarray(micros, dtype=np.float64)
        order = np.argsort(self.s)
        self.s, self.us = self.s[order], self.us[order]

    def __call__(self, s):
        s = float(s)
        xs, ys = self.s, self.us
        if xs.shape[0] == 1:
            return float(ys[0])
        if s <= xs[0]:
            j = 0
        elif s >= xs[-1]:
            j = xs.shape[0] - 2
        else:
            j = int(np.searchsorted(xs, s, side="right") - 1)
        w = (s - xs[j]) / (xs[j + 1] - xs[j])
        return max(0.0, float(ys[j] + w * (ys[j + 1] - ys[j])))


def partition_cost(A, lam_s):
    """Eq. 1: C_lj = A_lj * lambda(s_lj)."""
    return A * lam_s


def total_cost(A_levels, s_levels, lam):
    """Eq. 2: C = sum over levels and partitions of A * lambda(s)."""
    c = 0.0
    for A, s in zip(A_levels, s_levels):
        for a, sz in zip(A, s):
            c += partition_cost(a, lam(sz))
    return c


def delta_split_exact(dO_plus, A, lam_s, A_L, lam_L, A_R, lam_R):
    """Eq. 4: Delta O+ - A lambda(s) + A_L lambda(s_L) + A_R lambda(s_R)."""
    return dO_plus - A * lam_s + A_L * lam_L + A_R * lam_R


def delta_split_estimate(dO_plus, A, lam_s, lam_half, alpha):
    """Eq. 6: Delta O+ - A lambda(s) + 2 alpha A lambda(s / 2)."""
    return dO_plus - A * lam_s + 2.0 * alpha * A * lam_half


def delta_merge_exact(dO_minus, A, lam_s, receivers):
    """Eq. 5: Delta O- - A lambda(s) + sum_m [(A_m + dA_m) lambda(s_m + ds_m) - A_m lambda(s_m)].

    receivers: iterable of (A_m, dA_m, lam(s_m + ds_m), lam(s_m)).
    """
    acc = dO_minus - A * lam_s
    for A_m, dA_m, lam_after, lam_before in receivers:
        acc += (A_m + dA_m) * lam_after - A_m * lam_before
    return acc


def decide(delta, tau):
    """Stage 3: commit when delta < -tau, reject otherwise."""
    return delta < -tau


# ------------------------------------------------------------ insert / delete

def descend(levels, x):
    """Leaf partition for x by greedy top-down descent (Sec. 3)."""
    x = np.asarray(x, dtype=np.float64)
    L = len(levels)
    if L == 1:
        return int(np.argmin(distances(x, levels[0].centroids, L2)))
    top = levels[1]
    p = int(np.argmin(distances(x, top.centroids, L2)))
    leaves = top.ids[p]
    if leaves.shape[0] == 0:
        raise ValueError("empty parent partition")
    dl = distances(x, levels[0].centroids[leaves], L2)
    best = np.lexsort((leaves, dl))[0]
    return int(leaves[best])


def insert(levels, X, ids):
    """Append each vector to its leaf (in batch order); returns the leaf of each."""
    lv = levels[0]
    out = []
    for x, i in zip(np.asarray(X, np.float32), np.asarray(ids, np.int64)):
        j = descend(levels, x)
        lv.vectors[j] = np.concatenate([lv.vectors[j], x[None, :]])
        lv.ids[j] = np.concatenate([lv.ids[j], np.array([i], np.int64)])
        out.append(j)
    return np.array(out, dtype=np.int64)


def delete(levels, ids):
    """Remove each id (swap-with-last compaction); unknown ids are skipped.

    Returns the number removed.
    """
    lv = levels[0]
    where = {}
    for j, pid in enumerate(lv.ids):
        for s, i in enumerate(pid):
            where[int(i)] = (j, s)
    removed = 0
    for i in np.asarray(ids, np.int64):
        i = int(i)
        if i not in where:
            continue
        j, s = where.pop(i)
        last = lv.ids[j].shape[0] - 1
        if s != last:
            lv.vectors[j][s] = lv.vectors[j][last]
            moved = int(lv.ids[j][last])
            lv.ids[j][s] = moved
            where[moved] = (j, s)
        lv.vectors[j] = lv.vectors[j][:last]
        lv.ids[j] = lv.ids[j][:last]
        removed += 1
    return removed


# ----------------------------------------------------------------- split/merge

def two_means(rows, iters, seed):
    """M7: 2-means inside one partition, seeded by two distinct rows."""
    C = km.lloyd(rows, 2, iters, seed)
    a = km.assign(rows, C)
    return C, a


def refine(level, parts, iters=1):
    """M7 refinement: Lloyd iterations over the given partitions, seeded by their centroids.

    Vectors of all listed partitions are pooled, reassigned to the nearest of
    those partitions' centroids and the centroids recomputed; after the last
    iteration the pooled vectors are redistributed.
    """
    parts = list(parts)
    rows = np.concatenate([level.vectors[j] for j in parts]) if parts else np.zeros((0, level.centroids.shape[1]), np.float32)
    rid = np.concatenate([level.ids[j] for j in parts]) if parts else np.zeros(0, np.int64)
    C = level.centroids[parts].copy()
    for _ in range(iters):
        a = km.assign(rows, C)
        C, _ = km.update(rows, a, C)
    a = km.assign(rows, C)
    for n, j in enumerate(parts):
        level.centroids[j] = C[n]
        level.vectors[j] = rows[a == n]
        level.ids[j] = rid[a == n]
