"""Adaptive Partition Scanning and multi-level search (oracle; test infrastructure only).

Follows Sec. 5 (geometric model Eq. 7, half-space caps, Eq. 8-9, Algorithm 1)
and Sec. 3 ("Index Structure", top-down search).  Readings of the paper where
it is silent or garbled (each applied identically, but independently, in the
library):

  R1  rho is the Euclidean (not squared) distance from q to the current k-th
      result.  For inner product it is the Euclidean distance from q to that
      result's vector, ||q - x_k||.
  R2  t_i, the distance from q to the bisector of c_0 and c_i, is
      (D_i - D_0) / (2 ||c_i - c_0||) with D the squared Euclidean centroid
      distance, whatever the metric: the partitions are k-means cells
      (Sec. 3), whose boundaries are the Euclidean bisectors of their
      centroids.  Coincident centroids give t_i = 0.
  R3  p_0 = prod_j (1 - u_j) over the raw cap fractions u_j; the remaining
      mass 1 - p_0 is spread in proportion to the normalised v_i = u_i / sum u
      (Eq. 8-9).  With sum u = 0, p_0 = 1 and every p_i = 0.
      Params(p0_reading="normalised") takes the text of Eq. 8 literally
      instead: the caps are normalised first and p_0 = prod_j (1 - v_j) over
      the normalised v_j.  It exists to compare the two readings; the search
      defaults to R3.
  R4  Until R holds k results the estimator is not used: partitions are
      scanned in centroid-distance order.  When R first holds k results, rho is
      set and every p is computed.
  R5  r = p_0 + sum of p_i over the scanned candidates i >= 1, always with the
      current p values (the garbled update line of Algorithm 1 read as a sum
      over scanned candidates).
  R6  The next candidate is the unscanned one with the largest p_i; equal p_i
      go to the nearer centroid (lower position in S).
  R7  After each scan rho' is the new k-th distance; if |rho' - rho| > tau_rho
      rho, rho <- rho' and all p (including p_0) are recomputed.
  R8  The loop stops when r >= tau_R or S is exhausted.  nprobe counts the
      scanned candidates (empty partitions included).  If S runs out before R
      holds k results, r is reported as 1.
  R9  |S| = M = ceil(f_M * N_l) computed in double precision, clamped to
      [1, N_l].  Upper levels run APS with k' = M of the level below and the
      fixed recall target (0.99 in Sec. 5); the k' results, sorted by
      (distance, index), are the next level's S.
  R10 Fixed-nprobe search (Faiss-IVF style, used for the plain-IVF workload)
      scans the first nprobe candidates of S in centroid order.
  R11 With inner product the tree is searched in the geometry it was built
      in: centroids are scored by squared Euclidean distance at every level,
      and the upper levels' result sets are ranked the same way.  Only the
      base rows (level 0) are ranked by -<q, x>, and rho is ||q - x_k|| (R1).
      On unit-norm rows and queries -<q, x> = (||q - x||^2 - 2) / 2, so
      there the inner-product search coincides with the L2 search.
  R12 SPANN's early-termination rule (Sec. 2 "Early Termination", the
      comparator of Table 6): scan the candidates of S, nearest first, whose
      Euclidean centroid distance is at most (1 + eps) times the nearest
      one's; eps is the rule's tuned parameter.  S is the candidate set APS
      uses (the f_M nearest with one level, the upper level's APS result
      with two), and the candidates kept form a prefix of S.
"""

import math

import numpy as np

from .capvol import beta_table, cap_fraction, cap_fraction_table
from .knn import L2, distances


class Params:
    """Search parameters (defaults from Sec. 5 and Sec. 8.1)."""

    def __init__(self, k=10, recall_target=0.9, nprobe=0, f_M=(0.1, 0.25),
                 tau_rho=0.01, upper_recall=0.99, beta_mode="table", p0_reading="raw", ratio_eps=0.0):
        self.k = k
        self.recall_target = recall_target
        self.nprobe = nprobe
        self.f_M = tuple(f_M)
        self.tau_rho = tau_rho
        self.upper_recall = upper_recall
        self.beta_mode = beta_mode
        if p0_reading not in ("raw", "normalised"):
            raise ValueError("p0_reading is 'raw' (R3) or 'normalised' (Eq. 8 read literally)")
        self.p0_reading = p0_reading
        self.ratio_eps = ratio_eps      # > 0 with recall_target <= 0: SPANN's rule (R12)


def n_candidates(f, n):
    """M = ceil(f * n) in double precision, clamped to [1, n] (R9)."""
    return int(max(1, min(n, math.ceil(f * n))))


def bisector_distances(D, C):
    """t_i for every candidate (R2); D are squared Euclidean centroid distances and
    D[0], C[0] belong to the nearest centroid."""
    D = np.asarray(D, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    diff = C - C[0][None, :]
    cd = np.sqrt((diff * diff).sum(axis=1))
    num = D - D[0]
    den = 2.0 * cd
    t = np.zeros_like(D)
    nz = den > 0.0
    t[nz] = num[nz] / den[nz]
    return np.maximum(t, 0.0)


def probabilities(t, rho, d, mode="table", table=None, p0_reading="raw"):
    """p_0..p_{M-1} from Eq. 8-9 with raw caps for p_0 (R3), or with the
    normalised caps for p_0 when p0_reading is "normalised".  t[0] is unused."""
    t = np.asarray(t, dtype=np.float64)
    M = t.shape[0]
    p = np.zeros(M)
    if M == 1:
        p[0] = 1.0
        return p
    if mode == "exact":
        u = cap_fraction(t[1:], rho, d)
    else:
        u = cap_fraction_table(t[1:], rho, table)
    U = float(u.sum())
    if p0_reading == "raw":
        p0 = float(np.prod(1.0 - u))
    elif U > 0.0:
        p0 = float(np.prod(1.0 - u / U))
    else:
        p0 = 1.0
    p[0] = p0
    if U > 0.0:
        p[1:] = (1.0 - p0) * (u / U)
    return p


class _TopK:
    """The result set R of Algorithm 1: the k smallest (dist, id) pairs seen."""

    def __init__(self, k):
        self.k = k
        self.dist = np.zeros(0)
        self.ids = np.zeros(0, dtype=np.int64)
        self.rows = np.zeros((0, 0))

    def add(self, dist, ids, rows):
        if dist.shape[0] == 0:
            return
        if self.rows.shape[0] == 0:
            self.rows = np.zeros((0, rows.shape[1]))
        dd = np.concatenate([self.dist, dist])
        ii = np.concatenate([self.ids, ids])
        rr = np.concatenate([self.rows, np.asarray(rows, np.float64)])
        order = np.lexsort((ii, dd))[: self.k]
        self.dist, self.ids, self.rows = dd[order], ii[order], rr[order]

    def full(self):
        return self.dist.shape[0] >= self.k


def kth_radius(R, q, metric):
    """rho from the current k-th result (R1)."""
    if metric == L2:
        return math.sqrt(max(R.dist[R.k - 1], 0.0))
    diff = np.asarray(q, np.float64) - R.rows[R.k - 1]
    return math.sqrt(float((diff * diff).sum()))


def aps_level(q, level, cand, cand_D, k, tau_R, params, d, metric, table,
              fixed_nprobe=0):
    """Algorithm 1 on one level.

    q        query vector
    level    kmeans.Level whose partitions are scanned
    cand     candidate partition indices S, nearest first (position 0 = c_0)
    cand_D   their squared Euclidean centroid distances D_i (R11)
    metric   ranks the level's rows (L2 for upper levels, R11)
    Returns a dict: dist, ids (R sorted), scanned (positions in scan order),
    r (final estimate), trace (decision margins for parity checks) and steps:
    one record per estimator step, the first taken when R first holds k
    results, then one after every later scan, each with the position just
    scanned ("pos", None for the first), "rho" and "p" as they stand after
    the recompute decision, "recomputed" and "r".
    """
    q = np.asarray(q, dtype=np.float64)
    M = len(cand)
    R = _TopK(k)
    scanned = np.zeros(M, dtype=bool)
    order = []
    trace = []
    steps = []

    def scan(pos):
        j = cand[pos]
        rows = level.vectors[j]
        R.add(distances(q, rows, metric), level.ids[j], rows)
        scanned[pos] = True
        order.append(pos)

    if fixed_nprobe > 0:
        for pos in range(min(fixed_nprobe, M)):
            scan(pos)
        return dict(dist=R.dist, ids=R.ids, scanned=order, r=float("nan"), trace=trace, steps=steps)

    t = bisector_distances(cand_D, level.centroids[np.asarray(cand)])

    scan(0)
    while not R.full() and not scanned.all():                       # R4
        scan(int(np.argmin(scanned)))
    if not R.full():
        return dict(dist=R.dist, ids=R.ids, scanned=order, r=1.0, trace=trace, steps=steps)

    rho = kth_radius(R, q, metric)
    p = probabilities(t, rho, d, params.beta_mode, table, params.p0_reading)
    r = p[0] + p[1:][scanned[1:]].sum()                                # R5
    steps.append(dict(pos=None, rho=rho, recomputed=True, p=p.copy(), r=float(r)))
    while True:
        trace.append(("stop", len(order), r - tau_R))
        if not (r < tau_R) or scanned.all():                          # R8
            break
        un = np.nonzero(~scanned)[0]
        pu = p[un]
        best = un[int(np.argmax(pu))]                                  # R6 (first max = nearest)
        if un.shape[0] > 1:
            s = np.sort(pu)[::-1]
            gap = (s[0] - s[1]) / max(s[0], 1e-300)
        else:
            gap = float("inf")
        trace.append(("choose", len(order), gap))
        scan(int(best))
        rho_new = kth_radius(R, q, metric)
        dev = abs(rho_new - rho) - params.tau_rho * rho
        trace.append(("recompute", len(order), dev / max(rho, 1e-300)))
        recomputed = abs(rho_new - rho) > params.tau_rho * rho
        if recomputed:                                                 # R7
            rho = rho_new
            p = probabilities(t, rho, d, params.beta_mode, table, params.p0_reading)
        r = p[0] + p[1:][scanned[1:]].sum()
        steps.append(dict(pos=int(best), rho=rho, recomputed=bool(recomputed), p=p.copy(), r=float(r)))
    return dict(dist=R.dist, ids=R.ids, scanned=order, r=float(r), trace=trace, steps=steps)


def ratio_rule_count(cand_D, eps):
    """R12: how many candidates (sorted by squared distance D) lie within
    (1 + eps) of the nearest one's Euclidean distance."""
    r = np.sqrt(np.maximum(np.asarray(cand_D, np.float64), 0.0))
    return int(np.count_nonzero(r <= (1.0 + eps) * r[0])) if r.shape[0] else 0


def root_candidates(q, top_level, f):
    """Score the single top partition (all centroids of the top level, squared
    Euclidean distance, R11) and keep M."""
    D = distances(q, top_level.centroids, L2)
    idx = np.arange(D.shape[0], dtype=np.int64)
    M = n_candidates(f, D.shape[0])
    order = np.lexsort((idx, D))[:M]
    return idx[order], D[order]


def search(levels, Q, params, metric=L2):
    """Top-down Quake search of every query (Sec. 3, Sec. 5).

    levels[0] holds the base vectors; levels[1] (optional) holds the leaf
    centroids grouped under parent centroids.  Returns a dict of arrays
    dist (nq, k), ids (nq, k), nprobe (nq,), r (nq,), plus per-query lists
    scanned[l] (partition indices per level, in scan order) and traces.
    """
    Q = np.atleast_2d(np.asarray(Q))
    nq, d = Q.shape
    k = params.k
    table = beta_table(d) if params.beta_mode == "table" else None
    L = len(levels)
    out_D = np.full((nq, k), np.inf)
    out_I = np.full((nq, k), -1, dtype=np.int64)
    out_np = np.zeros(nq, dtype=np.int64)
    out_r = np.zeros(nq)
    scanned = [[None] * nq for _ in range(L)]
    traces = [[None] * nq for _ in range(L)]
    ratio = params.recall_target <= 0 and params.ratio_eps > 0
    fixed = params.nprobe if params.recall_target <= 0 and not ratio else 0
    for j in range(nq):
        q = Q[j]
        top = levels[L - 1]
        if L == 1:
            if fixed:                                                    # R10
                cand, cD = root_candidates(q, top, 1.0)
                cand, cD = cand[:fixed], cD[:fixed]
            else:
                cand, cD = root_candidates(q, top, params.f_M[0])
        else:
            cand1, cD1 = root_candidates(q, top, params.f_M[1])
            k1 = n_candidates(params.f_M[0], levels[0].n_part)
            res1 = aps_level(q, levels[1], list(cand1), cD1, k1, params.upper_recall,
                             params, d, L2, table)                      # R11
            scanned[1][j] = [int(cand1[p]) for p in res1["scanned"]]
            traces[1][j] = res1["trace"]
            cand, cD = res1["ids"], res1["dist"]
        nfix = ratio_rule_count(cD, params.ratio_eps) if ratio else fixed     # R12
        res = aps_level(q, levels[0], list(cand), cD, k, params.recall_target,
                        params, d, metric, table, fixed_nprobe=nfix)
        n = res["ids"].shape[0]
        out_D[j, :n] = res["dist"]
        out_I[j, :n] = res["ids"]
        out_np[j] = len(res["scanned"])
        out_r[j] = res["r"]
        scanned[0][j] = [int(cand[p]) for p in res["scanned"]]
        traces[0][j] = res["trace"]
    return dict(dist=out_D, ids=out_I, nprobe=out_np, r=out_r, scanned=scanned,
                traces=traces)


def ivf_search(level, Q, k, nprobe, metric=L2):
    """Fixed-nprobe IVF over one level with one nprobe per query (R10 per query).

    Query j scans its nprobe[j] nearest partitions (squared Euclidean centroid
    distance, R11; ties to the lower index; more than the partitions there are
    means all of them) and
    returns the exact top-k of their members by (distance, id).  Returns
    dist (nq, k) FP64, ids (nq, k) (inf / -1 past the scanned rows) and the
    scanned partition indices of every query, nearest first.
    """
    Q = np.atleast_2d(np.asarray(Q))
    nq = Q.shape[0]
    nprobe = np.broadcast_to(np.asarray(nprobe, dtype=np.int64), (nq,))
    out_D = np.full((nq, k), np.inf)
    out_I = np.full((nq, k), -1, dtype=np.int64)
    scanned = []
    idx = np.arange(level.n_part, dtype=np.int64)
    for j in range(nq):
        D = distances(Q[j], level.centroids, L2)
        parts = np.lexsort((idx, D))[:min(int(nprobe[j]), level.n_part)]
        scanned.append(parts)
        rows = [level.vectors[p] for p in parts if level.vectors[p].shape[0]]
        if not rows:
            continue
        X = np.concatenate(rows)
        ids = np.concatenate([level.ids[p] for p in parts if level.vectors[p].shape[0]])
        dist = distances(Q[j], X, metric)
        order = np.lexsort((ids, dist))[:k]
        out_D[j, :order.shape[0]] = dist[order]
        out_I[j, :order.shape[0]] = ids[order]
    return out_D, out_I, scanned
