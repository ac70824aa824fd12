"""The parallel oracle leg of the CPU baseline: spawned workers over shared level-0 rows run the
oracle's search on every query and report a positive rate."""

import numpy as np

from oracle import aps, kmeans, pool


def test_pool_runs_every_query_in_spawned_workers():
    g = np.random.default_rng(0)
    X = g.standard_normal((3000, 16)).astype(np.float32)
    ids = np.arange(3000, dtype=np.int64) * 3
    levels = kmeans.build_index(X, ids, 12, 3, iters=2, seed=1)
    Q = X[::150] + 0.01
    prm = aps.Params(k=5, recall_target=0.9, f_M=(0.5, 1.0))
    rate, done = pool.search_rate(levels, Q, prm, 60.0, 2)
    assert done == Q.shape[0] and rate > 0
    assert pool.available_cores() >= 1
