"""The batched fixed-nprobe search at the batching workload's full size (5M x 256 rows,
20,000 Zipf-sized partitions, 4,096 queries with nprobe 1..500) in the launch
configuration the benchmark times (autotuned tiles, CUDA-graph replay), checked against
the oracle on a sample of queries spread over the nprobe range."""

import numpy as np
import pytest

from oracle import aps, kmeans
from paper_2506_03437_b300 import synth

from .test_gpu_batch import check_against_oracle

pytestmark = pytest.mark.gpu


def test_full_size_sample_matches_oracle():
    import torch
    from paper_2506_03437_b300 import index as I
    n, d, n_part, nq, k = 5_000_000, 256, 20_000, 4096, 10
    X, ids, lab, Q, nprobe = synth.zipf_partitions(n=n, d=d, n_part=n_part, nq=nq, nprobe_hi=500)
    sizes = np.bincount(lab, minlength=n_part)
    Xd, labd = torch.from_numpy(X).cuda(), torch.from_numpy(lab).cuda()
    C = torch.zeros((n_part, d), dtype=torch.float64, device="cuda")
    for s in range(0, n, 1 << 20):
        C.index_add_(0, labd[s:s + (1 << 20)], Xd[s:s + (1 << 20)].double())
    C = (C / torch.from_numpy(sizes).cuda().double()[:, None]).float()
    ix = I.Index(d, n_leaf=n_part, n_parent=0)
    ix.load(Xd, torch.from_numpy(ids).cuda(), leaf_centroids=C, leaf_of_row=labd.int())
    Qd, npd = torch.from_numpy(Q).cuda(), torch.from_numpy(nprobe).cuda()
    plan = I.BatchPlan(ix, nq, k, 500)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        plan.autotune(Qd, npd, reps=1, stream=s)
        out = (torch.empty((nq, k), dtype=torch.int64, device="cuda"),
               torch.empty((nq, k), dtype=torch.float32, device="cuda"))
        plan.capture(Qd, npd, out, s)
        plan.replay(s)
        s.synchronize()
    ix.check()
    gi, gd = out[0].cpu().numpy(), out[1].cpu().numpy()
    # sample: the queries with the largest nprobe, the smallest, and a spread in between
    order = np.argsort(nprobe, kind="stable")
    pick = np.unique(np.concatenate([order[:6], order[-6:], order[np.linspace(0, nq - 1, 20).astype(int)]]))
    off = np.concatenate([[0], np.cumsum(sizes)])
    level = kmeans.Level(C.cpu().numpy(), [X[off[j]:off[j + 1]] for j in range(n_part)],
                         [ids[off[j]:off[j + 1]] for j in range(n_part)])
    check_against_oracle(level, Q[pick], nprobe[pick], gi[pick], gd[pick], k, max_excused=0.1)
    # every result id is a real row and lists are sorted by distance
    assert np.all(gi >= 0) and np.all(np.diff(gd, axis=1) >= 0)
