"""Helpers shared by the GPU parity tests: compare the CUDA path with the oracle.

Tolerances (derived from the arithmetic of the two sides):
  distances   the GPU accumulates FP32 squared differences; over d <= 1024
              terms the relative error stays below ~1e-6 in practice, so the
              bar is the stated 1e-5 relative (plus 1e-5 absolute near 0).
  ties        result sets may differ only where two candidates' exact
              distances are within 1e-5 relative of the k-th one.
  decisions   the estimator sees FP32-derived t_i and rho (relative error
              ~1e-7), which moves a cap fraction u by up to d/(1 - s^2) times
              that, so p values agree to roughly 1e-5 relative and r to about
              1e-5 absolute.  A query may differ from the oracle only if the
              oracle's trace shows a decision inside these margins: runner-up
              p within 1e-4 relative of the best, r within 1e-4 of the target,
              or |rho' - rho| within 1e-5 rho of the recompute threshold.
              Every such query is counted, printed, and bounded by the caller
              (at most 1% of a test's queries, and at least one allowed).
  selections  the partitions scanned, in scan order, at every level
              (Algorithm 1's choices) must equal the oracle's for every query
              that is not excused.
"""

import numpy as np

from oracle import knn

DIST_RTOL = 1e-5
GAP_TOL = 1e-4
R_TOL = 1e-4
RHO_TOL = 1e-5


def near_tie(trace):
    for kind, _, val in trace or ():
        if kind == "choose" and val < GAP_TOL:
            return True
        if kind == "stop" and abs(val) < R_TOL:
            return True
        if kind == "recompute" and abs(val) < RHO_TOL:
            return True
    return False


def same_topk(gi, gd, oi, od, rtol=DIST_RTOL):
    """True if two top-k lists agree up to (distance, id) near-ties."""
    gi, gd, oi, od = map(np.asarray, (gi, gd, oi, od))
    if np.array_equal(gi, oi):
        return bool(np.allclose(gd[gi >= 0], od[oi >= 0], rtol=rtol, atol=rtol))
    # sets may differ only among entries tied with the k-th distance
    fin = od[np.isfinite(od)]
    if fin.size == 0:
        return False
    kth = fin[-1]
    thr = kth + rtol * abs(kth) + rtol
    a = {int(i) for i, d in zip(gi, gd) if i >= 0 and d < kth - rtol * abs(kth) - rtol}
    b = {int(i) for i, d in zip(oi, od) if i >= 0 and d < kth - rtol * abs(kth) - rtol}
    if a != b:
        return False
    return bool(np.all(gd[gi >= 0] <= thr + rtol * abs(thr)))


def max_excused(nq):
    """The bound on excused queries of one comparison: 1%, at least one."""
    return max(1, nq // 100)


def compare_search(gpu, orc, k, check_r=True, label="", bound=True):
    """Per-query comparison; returns (n_exact, n_excused).  Raises on a real mismatch.

    gpu is (ids, dist, nprobe, r) or, from Index.search_scanned, (ids, dist,
    nprobe, r, scanned0, scanned1): then the partitions scanned at each level,
    in order, are compared with the oracle's as well (a level given as None
    is not compared).  With bound=True the
    excused queries may be at most max_excused(nq)."""
    gi, gd, gn, gr = gpu[:4]
    scanned = gpu[4:6] if len(gpu) >= 6 else None
    nq = gi.shape[0]
    n_ok = n_exc = 0
    for j in range(nq):
        np_ok = int(gn[j]) == int(orc["nprobe"][j])
        res_ok = same_topk(gi[j], gd[j], orc["ids"][j], orc["dist"][j])
        r_ok = True
        if check_r and np.isfinite(orc["r"][j]):
            r_ok = abs(float(gr[j]) - float(orc["r"][j])) < 1e-4
        sel_ok = True
        if scanned is not None:
            for lv, rec in enumerate(scanned):
                if rec is None:
                    continue
                row = np.asarray(rec[j])
                got = [int(x) for x in row if x >= 0]
                want = orc["scanned"][lv][j] if lv < len(orc["scanned"]) else None
                want = [] if want is None else [int(x) for x in want][: row.shape[0]]
                sel_ok = sel_ok and got == want
        if np_ok and res_ok and r_ok and sel_ok:
            n_ok += 1
            continue
        traces = [orc["traces"][lv][j] for lv in range(len(orc["traces"])) if orc["traces"][lv][j] is not None]
        if any(near_tie(t) for t in traces):
            n_exc += 1
            continue
        raise AssertionError(
            f"query {j}: gpu nprobe={gn[j]} r={gr[j]:.6f} ids={list(gi[j])}\n"
            f"          oracle nprobe={orc['nprobe'][j]} r={orc['r'][j]:.6f} ids={list(orc['ids'][j])}\n"
            f"          gpu d={list(gd[j])}\n          orc d={list(orc['dist'][j])}\n"
            f"          selections equal: {sel_ok}")
    print(f"[parity] {label or 'search'}: {n_ok} identical, {n_exc} excused as near-ties, of {nq} queries")
    if bound:
        assert n_exc <= max_excused(nq), f"{n_exc} of {nq} queries excused (bound {max_excused(nq)})"
    return n_ok, n_exc


def exact_dist(X_by_id, Q, ids, metric=knn.L2):
    """FP64 distances of returned ids (inf where id < 0)."""
    out = np.full(ids.shape, np.inf)
    for j in range(ids.shape[0]):
        sel = ids[j] >= 0
        if sel.any():
            out[j, sel] = knn.distances(Q[j], X_by_id[ids[j][sel]], metric)
    return out
