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
  M7  Split = 2-means inside the partition (fixed iterations) over its vectors
      taken in ascending id order, so that the seeded rows do not depend on
      how a partition happens to be stored; then one refinement pass: a Lloyd
      iteration seeded by the current centroids over the r_f partitions
      nearest the two new centroids.
  M8  Partitions are processed in ascending order of their estimated delta;
      N_l is updated after every commit.  Insert descends greedily (the
      nearest centroid at each level, ties to the lower index).  Delete swaps
      the last row of the partition into the freed slot.
  M9  (optional, level_band) Levels are added and removed by a size band on
      the top level, [sqrt(N0)/4, 4 sqrt(N0)] (see level_band_action): the
      paper's thresholds are in its technical report, which is not available.
"""

import math

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


# ------------------------------------------------------ the maintenance pass

MASK64 = (1 << 64) - 1


class MaintParams:
    """Maintenance parameters (Sec. 4 and Sec. 8.1 defaults where the paper gives them)."""

    def __init__(self, lam, tau=0.25, alpha=0.9, refine_radius=50, refine_iters=1, split_iters=10,
                 s_min=0, seed=1234, refine=True, level_band=False, level_iters=10):
        self.lam = lam
        self.tau = tau
        self.alpha = alpha
        self.refine_radius = refine_radius
        self.refine_iters = refine_iters
        self.split_iters = split_iters
        self.s_min = s_min
        self.seed = seed
        self.refine = refine
        self.level_band = level_band
        self.level_iters = level_iters


def split_seed(seed, level, j):
    """Seed of the 2-means that splits partition j of `level` (both sides use this rule)."""
    return (seed + 0x9E3779B97F4A7C15 * (level * 1_000_003 + j + 1)) & MASK64


def nearest(C, live, x, count, exclude=None):
    """The `count` live centroid indices nearest to x (ties to the lower index)."""
    cand = [j for j in live if j != exclude]
    if not cand:
        return []
    cand = np.array(cand, dtype=np.int64)
    d = distances(x, C[cand], L2)
    order = np.lexsort((cand, d))
    return [int(cand[i]) for i in order[:count]]


def maintain_level(level, A, prm, level_no, parent_of=None, detail=None):
    """One estimate / verify / commit pass over one level (Sec. 4 "Decision Workflow").

    level      kmeans.Level (centroids, vectors, ids), modified in place
    A          access frequency per partition (hits / |W|)
    parent_of  for level 0 of a two-level index: the parent of every leaf,
               extended and compacted together with the leaves
    detail     optional list; every verify appends a dict with the action's
               kind, partition, estimate, exact delta and decision, plus the
               children's sizes (split) or, per receiver m, (Delta s_m,
               Delta A_m) (merge, M5)
    Returns (log, keep): the actions taken and the old index of every
    surviving partition, in the new order.

    Readings: candidates are the partitions whose estimate (Eq. 6 for split,
    M3 for merge) is below -tau, processed in ascending order of the estimate
    (ties: lower index, split before merge).  A partition touched by an
    earlier committed action of the pass (a split child, a merge receiver, a
    refined neighbour) is skipped.  A split keeps the left child in place and
    appends the right child; a merge marks the partition dead and the dead
    are removed at the end of the pass, keeping the order of the rest.
    Every verify uses the current number of live partitions for Delta O.
    """
    lam, tau, alpha = prm.lam, prm.tau, prm.alpha
    C = [np.array(c, dtype=np.float32) for c in level.centroids]
    V = list(level.vectors)
    I = list(level.ids)
    A = [float(a) for a in A]
    N0 = len(C)
    live = list(range(N0))
    sizes = [v.shape[0] for v in V]
    cands = []
    for j in range(N0):
        s, a = sizes[j], A[j]
        if s >= 2:
            e = delta_split_estimate(lam(N0 + 1) - lam(N0), a, lam(s), lam(s / 2.0), alpha)
            if e < -tau:
                cands.append((e, j, 0))
        if s < prm.s_min and N0 > 1:
            nR = min(prm.refine_radius, N0 - 1)
            R = nearest(np.array(C), live, C[j].astype(np.float64), nR, exclude=j)
            rec = [(A[m], a / nR, lam(sizes[m] + s / nR), lam(sizes[m])) for m in R]
            e = delta_merge_exact(lam(N0 - 1) - lam(N0), a, lam(s), rec)
            if e < -tau:
                cands.append((e, j, 1))
    cands.sort()
    touched, dead, log = set(), set(), []
    for e, j, kind in cands:
        if j in touched or j in dead:
            continue
        n_live = len(live)
        rows, rid, s, a = V[j], I[j], sizes[j], A[j]
        if kind == 0:
            by_id = np.argsort(rid, kind="stable")
            C2 = km.lloyd(rows[by_id], 2, prm.split_iters, split_seed(prm.seed, level_no, j))
            a2 = km.assign(rows, C2)
            sL, sR = int((a2 == 0).sum()), int((a2 == 1).sum())
            if sL == 0 or sR == 0:
                log.append(("split", j, e, None, False))
                continue
            d = delta_split_exact(lam(n_live + 1) - lam(n_live), a, lam(s), alpha * a, lam(sL), alpha * a, lam(sR))
            ok = decide(d, tau)
            log.append(("split", j, e, d, ok))
            if detail is not None:
                detail.append(dict(kind="split", j=j, estimate=e, delta=d, ok=ok, sizes=(sL, sR)))
            if not ok:
                continue
            jn = len(C)
            C[j], V[j], I[j] = C2[0], rows[a2 == 0], rid[a2 == 0]
            C.append(C2[1])
            V.append(rows[a2 == 1])
            I.append(rid[a2 == 1])
            A[j] = alpha * a
            A.append(alpha * a)
            sizes[j] = sL
            sizes.append(sR)
            live.append(jn)
            if parent_of is not None:
                parent_of.append(parent_of[j])
            touched |= {j, jn}
            if prm.refine and prm.refine_iters > 0:
                Cn = np.array(C)
                P = set(nearest(Cn, live, C[j].astype(np.float64), prm.refine_radius))
                P |= set(nearest(Cn, live, C[jn].astype(np.float64), prm.refine_radius))
                P = sorted(P)
                tmp = km.Level(np.array([C[p] for p in P]), [V[p] for p in P], [I[p] for p in P])
                refine(tmp, list(range(len(P))), prm.refine_iters)
                for n, p in enumerate(P):
                    C[p], V[p], I[p] = tmp.centroids[n], tmp.vectors[n], tmp.ids[n]
                    sizes[p] = V[p].shape[0]
                touched |= set(P)
        else:
            others = [m for m in live if m != j]
            Co = np.array([C[m] for m in others])
            am = km.assign(rows, Co) if s > 0 else np.zeros(0, np.int64)
            recv = {}
            for r, k in enumerate(am):
                recv.setdefault(others[int(k)], []).append(r)
            rec = [(A[m], a * len(rs) / s, lam(sizes[m] + len(rs)), lam(sizes[m])) for m, rs in sorted(recv.items())]
            d = delta_merge_exact(lam(n_live - 1) - lam(n_live), a, lam(s), rec)
            ok = decide(d, tau)
            log.append(("merge", j, e, d, ok))
            if detail is not None:
                detail.append(dict(kind="merge", j=j, estimate=e, delta=d, ok=ok,
                                   receivers={m: (len(rs), a * len(rs) / s) for m, rs in sorted(recv.items())}))
            if not ok:
                continue
            for m, rs in sorted(recv.items()):
                rs = np.array(rs, dtype=np.int64)
                V[m] = np.concatenate([V[m], rows[rs]])
                I[m] = np.concatenate([I[m], rid[rs]])
                A[m] += a * len(rs) / s
                sizes[m] += len(rs)
                touched.add(m)
            dead.add(j)
            live.remove(j)
            touched.add(j)
    keep = [j for j in range(len(C)) if j not in dead]
    level.centroids = np.array([C[j] for j in keep], dtype=np.float32).reshape(len(keep), -1)
    level.vectors = [V[j] for j in keep]
    level.ids = [I[j] for j in keep]
    if parent_of is not None:
        parent_of[:] = [parent_of[j] for j in keep]
    return log, keep


def level_band_action(n_leaf, n_parent):
    """Reading L1 (the paper adds and removes levels, Sec. 3-4, with thresholds only in its
    technical report): the top level should hold between sqrt(N0)/4 and 4 sqrt(N0)
    centroids, N0 = n_leaf.  One level is the top itself, so it needs a parent level once
    N0 > 4 sqrt(N0), i.e. N0 > 16; two levels with N0 <= 16 drop the parents; parents
    outside the band are rebuilt.  Returns (action, new parent count) or None, the count
    being round(sqrt(N0)) (halves up)."""
    r = math.sqrt(n_leaf)
    p = max(1, int(math.floor(r + 0.5)))
    if n_parent == 0:
        return ("add_level", p) if n_leaf > 16 else None
    if n_leaf <= 16:
        return ("remove_level", 0)
    if n_parent < r / 4 or n_parent > 4 * r:
        return ("rebuild_level", p)
    return None


def apply_level_band(levels, logs, prm):
    """Applies level_band_action after a pass: new parents are k-means (seed + 1, like the
    build) of the leaf centroids, every leaf under its nearest final parent."""
    n_leaf = levels[0].n_part
    act = level_band_action(n_leaf, levels[1].n_part if len(levels) > 1 else 0)
    if act is None:
        return
    kind, p = act
    if kind == "remove_level":
        levels.pop()
    else:
        C0 = levels[0].centroids
        C1 = km.lloyd(C0, p, prm.level_iters, prm.seed + 1)
        lv1, _ = km.partition_level(C0, np.arange(n_leaf, dtype=np.int64), C1)
        if len(levels) == 1:
            levels.append(lv1)
        else:
            levels[1] = lv1
    while len(logs) < 2:
        logs.append([])
    logs[1].append((kind, p, float("nan"), float("nan"), True))


def maintain(levels, hits, window, prm):
    """The bottom-up maintenance pass of Sec. 4 over every level; returns the action logs.

    hits[l] are the access counts of level l's partitions over the last
    `window` queries (A = hits / |W|, Stage 0).  After the leaves change, the
    parent level is rebuilt from the parent of every surviving leaf (split
    children stay with their parent, merged leaves leave it), then the parent
    level runs its own pass (Stage 4).
    """
    logs = []
    if len(levels) == 1:
        log, _ = maintain_level(levels[0], np.asarray(hits[0]) / window, prm, 0)
        logs = [log]
        if prm.level_band:
            apply_level_band(levels, logs, prm)
        return logs
    n_leaf = levels[0].n_part
    parent_of = [0] * n_leaf
    for p, leaves in enumerate(levels[1].ids):
        for lf in leaves:
            parent_of[int(lf)] = p
    log0, keep = maintain_level(levels[0], np.asarray(hits[0]) / window, prm, 0, parent_of=parent_of)
    logs.append(log0)
    P1 = levels[1].n_part
    members = [[] for _ in range(P1)]
    for lf, p in enumerate(parent_of):
        members[p].append(lf)
    C0 = levels[0].centroids
    levels[1] = km.Level(levels[1].centroids, [C0[np.array(m, dtype=np.int64)] if m else np.zeros((0, C0.shape[1]), np.float32) for m in members],
                         [np.array(m, dtype=np.int64) for m in members])
    log1, _ = maintain_level(levels[1], np.asarray(hits[1]) / window, prm, 1)
    logs.append(log1)
    if prm.level_band:
        apply_level_band(levels, logs, prm)
    return logs
