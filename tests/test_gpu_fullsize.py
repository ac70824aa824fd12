"""Parity at the full APS workload size (1M x 128, 1,000 leaves under 32 parents, 10,000 queries).

The GPU searches the whole 10,000-query batch in one launch, as bench.py
times it; the oracle recomputes a sample of those queries one by one.  The
partitioning is fixed by the oracle: leaf centroids are the generator's
1,000 component centres with every vector in its nearest centre's partition
(exact FP64 assignment), parents are the oracle's k-means of those centres.
"""

import numpy as np
import pytest

from oracle import aps, kmeans, knn
from paper_2506_03437_b300 import synth

from .parity import compare_search, exact_dist
from .test_gpu_search import make_index

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", [0])
def test_full_size_aps_sampled_parity(storage):
    import torch
    from paper_2506_03437_b300 import index as I
    n, d, n_comp, nq = 1_000_000, 128, 1000, 10_000
    X, ids, Q = synth.aps_search(n=n, d=d, n_comp=n_comp, sigma=1.5, nq=nq)
    C0 = synth.mixture_centers(n_comp, d, 1236)
    a0 = kmeans.assign(X, C0)
    C1 = kmeans.lloyd(C0, 32, 10, 1235)
    a1 = kmeans.assign(C0, C1)
    levels = kmeans.index_from_assignment(X, ids, C0, a0, C1, a1)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.1, f_M_parent=0.25)
    out = ix.search_scanned(torch.from_numpy(Q).cuda(), 10, recall_target=0.9, cap0=100, cap1=8)
    ix.check()
    out = tuple(a.cpu().numpy() for a in out)
    gi, gd, gn, gr = out[:4]
    assert ((gi >= 0) & (gi < n)).all() and (np.diff(gd, axis=1) >= 0).all()
    sel = np.random.default_rng(0).choice(nq, 40, replace=False)
    orc = aps.search(levels, Q[sel], aps.Params(k=10, recall_target=0.9, f_M=(0.1, 0.25)))
    compare_search(tuple(a[sel] for a in out), orc, 10, label="APS 1M x 128, 40 sampled queries")
    # the batched path, in the launch configuration the benchmark times (4 rounds)
    plan = I.ApsBatchPlan(ix, nq, 10, rounds=4)
    bo = tuple(a.cpu().numpy() for a in plan.search(torch.from_numpy(Q).cuda(), 0.9, cap0=100))
    ix.check()
    compare_search(tuple(a[sel] for a in bo) + (out[5][sel],), orc, 10,
                   label="batched APS 1M x 128, 40 sampled queries")
    agree = np.mean([np.array_equal(bo[0][j], gi[j]) and bo[2][j] == gn[j] and np.array_equal(bo[4][j], out[4][j])
                     for j in range(nq)])
    print(f"[parity] batched APS vs the per-query kernel: {agree:.4f} of {nq} queries identical")
    assert agree >= 0.999
    # recall of the sample against FP64 brute force
    gtD, _ = knn.knn(X, ids, Q[sel], 10, bulk=True)
    rec = knn.recall_at_k(gi[sel], exact_dist(X, Q[sel], gi[sel]), gtD, 10).mean()
    assert rec > 0.85
