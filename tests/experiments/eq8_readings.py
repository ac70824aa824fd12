"""Experiment: the two readings of Eq. 8 on the APS workload's data (oracle only).

Reading R3 (the oracle's and the library's) takes p_0 = prod (1 - u_j) over the
raw cap fractions; the literal text of Sec. 5 normalises the caps first and
takes p_0 = prod (1 - v_j) over the normalised v_j.  This script runs Algorithm
1 under both readings on a sample of the 1M x 128 APS workload (two levels, 32
parents over 1,000 leaves) at several recall targets, beside the two
comparators of Table 6: the smallest fixed nprobe whose mean recall@10 reaches
the target, and the per-query oracle nprobe (each query's smallest nprobe
whose own recall@10 reaches it).  Recall is against FP64 brute force.

    python -m tests.experiments.eq8_readings [--queries 300] [--targets 0.8,0.9,0.95,0.99]

The partitioning is the generator's 1,000 component centres with every vector
in its nearest centre's partition and the parents the oracle's k-means of the
centres (as tests/test_gpu_fullsize.py builds it), so no GPU is involved.
"""

import argparse
import json
import time

import numpy as np

from oracle import aps, kmeans, knn
from paper_2506_03437_b300 import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--queries", type=int, default=300)
    ap.add_argument("--targets", default="0.8,0.9,0.95,0.99")
    ap.add_argument("--n", type=int, default=1_000_000)
    args = ap.parse_args()
    t0 = time.time()
    X, ids, Q = synth.aps_search(n=args.n, d=128, n_comp=1000, sigma=1.5, nq=10_000)
    C0 = synth.mixture_centers(1000, 128, 1236)
    a0 = kmeans.assign(X, C0)
    C1 = kmeans.lloyd(C0, 32, 10, 1235)
    a1 = kmeans.assign(C0, C1)
    levels = kmeans.index_from_assignment(X, ids, C0, a0, C1, a1)
    sel = np.random.default_rng(7).choice(Q.shape[0], args.queries, replace=False)
    Qs = Q[sel]
    gtD, _ = knn.knn(X, ids, Qs, 10, bulk=True)

    def recall_of(found):
        ex = np.array([[((X[i].astype(np.float64) - Qs[j]) ** 2).sum() if i >= 0 else np.inf for i in found[j]]
                       for j in range(Qs.shape[0])])
        return knn.recall_at_k(found, ex, gtD, 10)

    # per-query recall as a function of a fixed nprobe (candidates = the upper level's S)
    per_q = {}
    for nprobe in range(1, 101):
        r = aps.search(levels, Qs, aps.Params(k=10, recall_target=0.0, nprobe=nprobe, f_M=(0.1, 0.25)))
        per_q[nprobe] = recall_of(r["ids"])
        if per_q[nprobe].min() >= 0.999:
            break
    out = {"n": args.n, "queries": int(Qs.shape[0]), "rows": []}
    for tau in [float(x) for x in args.targets.split(",")]:
        row = {"target": tau}
        for reading in ("raw", "normalised"):
            prm = aps.Params(k=10, recall_target=tau, f_M=(0.1, 0.25), p0_reading=reading)
            r = aps.search(levels, Qs, prm)
            row[reading] = {"recall": round(float(recall_of(r["ids"]).mean()), 4),
                            "nprobe": round(float(r["nprobe"].mean()), 2)}
        fixed = next((n for n in sorted(per_q) if per_q[n].mean() >= tau), None)
        row["fixed"] = {"nprobe": fixed, "recall": round(float(per_q[fixed].mean()), 4) if fixed else None}
        need = np.array([next((n for n in sorted(per_q) if per_q[n][j] >= tau), max(per_q))
                         for j in range(Qs.shape[0])])
        row["oracle"] = {"nprobe": round(float(need.mean()), 2),
                         "recall": round(float(np.mean([per_q[need[j]][j] for j in range(Qs.shape[0])])), 4)}
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    out["seconds"] = round(time.time() - t0, 1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
