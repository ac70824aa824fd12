"""Batched APS (qk_aps_batch_*): Algorithm 1 for every query of a batch with the
leaf scans grouped by partition, against the oracle and the per-query kernel.

The rounds speculate: a query asks for the partitions Algorithm 1 would take
if p stayed as it is, and items scanned past its stop are discarded.  The
results, nprobe, r and the sequence of partitions taken in must not depend on
that: they are compared with the oracle query by query, and must be the same
for any number of rounds.
"""

import numpy as np
import pytest

from oracle import aps, kmeans, knn
from paper_2506_03437_b300 import synth

from .parity import compare_search, same_topk
from .test_gpu_search import make_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


@pytest.fixture(scope="module")
def two_level():
    X, ids, Q = synth.aps_search(seed=12, n=30_000, d=128, n_comp=60, sigma=1.0, nq=120)
    levels = kmeans.build_index(X, ids, 300, 12, iters=5, seed=3)
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.9, f_M=(0.1, 0.5)))
    return X, ids, Q, levels, orc


def cpu(out):
    return tuple(a.cpu().numpy() for a in out)


def test_batched_aps_matches_oracle_two_levels(I, two_level):
    import torch
    X, ids, Q, levels, orc = two_level
    ix = make_index(I, X, ids, levels, f_M_leaf=0.1, f_M_parent=0.5)
    plan = I.ApsBatchPlan(ix, Q.shape[0], 10)
    out = cpu(plan.search(torch.from_numpy(Q).cuda(), 0.9, cap0=30))
    ix.check()
    _, _, _, _, _, s1 = ix.search_scanned(Q, 10, recall_target=0.9, cap0=30, cap1=6)
    compare_search(out[:4] + (out[4], s1), orc, 10, label="batched APS, two levels")
    # every partition Algorithm 1 took in was counted once per query, at both levels
    ix.hits(0, reset=True)
    ix.hits(1, reset=True)
    out = cpu(plan.search(torch.from_numpy(Q).cuda(), 0.9, cap0=30))
    s0 = out[4]
    assert np.array_equal(ix.hits(0), np.bincount(s0[s0 >= 0], minlength=300))
    assert np.array_equal(ix.hits(1), np.bincount(s1[s1 >= 0], minlength=12))
    assert ((s0 >= 0).sum(axis=1) == out[2]).all()
    asked, taken = plan.round_stats()
    assert taken.sum() == out[2].sum() and (asked >= taken).all()
    assert asked[0] >= Q.shape[0]                 # the first round asks for each P_0 (more if it holds < k rows)


@pytest.mark.parametrize("rounds", [1, 2, 3, 16])
def test_round_count_does_not_change_results(I, two_level, rounds):
    import torch
    X, ids, Q, levels, orc = two_level
    ix = make_index(I, X, ids, levels, f_M_leaf=0.1, f_M_parent=0.5)
    qd = torch.from_numpy(Q).cuda()
    base = cpu(I.ApsBatchPlan(ix, Q.shape[0], 10).search(qd, 0.9, cap0=30))
    plan = I.ApsBatchPlan(ix, Q.shape[0], 10, rounds=rounds)
    out = cpu(plan.search(qd, 0.9, cap0=30))
    # selections, nprobe and r never depend on the rounds
    assert np.array_equal(out[2], base[2]) and np.array_equal(out[4], base[4])
    np.testing.assert_allclose(out[3], base[3], rtol=1e-6)
    # every item is scanned by the same kernel whatever the rounds, so the
    # results agree bitwise
    for a, b in zip(out, base):
        assert np.array_equal(a, b)
    asked, taken = plan.round_stats()
    assert taken.sum() == base[2].sum() and (asked >= taken).all()


@pytest.mark.parametrize("mode", ["table", "exact"])
def test_batched_aps_one_level_matches_oracle_and_per_query_kernel(I, mode):
    import torch
    X, ids, Q = synth.aps_search(seed=11, n=20_000, d=64, n_comp=40, sigma=1.0, nq=150)
    levels = kmeans.build_index(X, ids, 150, 0, iters=5, seed=9)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.2, beta_mode=0 if mode == "table" else 1)
    plan = I.ApsBatchPlan(ix, Q.shape[0], 10)
    out = cpu(plan.search(torch.from_numpy(Q).cuda(), 0.9, cap0=30))
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.9, f_M=(0.2,), beta_mode=mode))
    compare_search(out[:4] + (out[4], None), orc, 10, label=f"batched APS, one level, {mode} beta")
    assert out[2].max() > 1
    # the grouped scan sums every row in the per-query kernel's order, so the batch takes
    # the per-query kernel's decisions and returns its distances bit for bit
    pi, pd, pn, pr = ix.search(Q, 10, recall_target=0.9)
    assert np.array_equal(pn, out[2]) and np.array_equal(pi, out[0])
    assert np.array_equal(pd.view(np.uint32), out[1].view(np.uint32))


@pytest.mark.parametrize("d", [32, 64, 96, 128, 192, 256, 384])
def test_every_tile_shape_gives_the_per_query_kernels_results(I, d):
    """Each tile shape splits a row over a different number of lanes (1 to 32 per row, one
    to eight of the per-query kernel's lanes per lane, or whole rows per thread); all of them
    must return the per-query kernel's ids, distances and nprobe bit for bit."""
    import torch
    X, ids, Q = synth.aps_search(seed=80 + d, n=12_000, d=d, n_comp=30, sigma=1.0, nq=200)
    levels = kmeans.build_index(X, ids, 80, 0, iters=4, seed=5)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.2)
    pi, pd, pn, _ = ix.search(Q, 10, recall_target=0.9)
    plan = I.ApsBatchPlan(ix, Q.shape[0], 10)
    Qd = torch.from_numpy(Q).cuda()
    shapes = [(qw, tr, ch) for qw in (1, 2, 4) for tr, ch in ((16, 1024), (32, 4096))
              if (qw, d) not in ((4, 192), (4, 256), (4, 768), (4, 1024))]
    if d <= 256:   # whole rows per thread in the rounds after the first
        shapes += [(1, 16, 1024, 2), (2, 32, 4096, 2)]
    for shape in shapes:
        plan.set_tiles(*shape)
        gi, gd, gn = cpu(plan.search(Qd, 0.9))[:3]
        assert np.array_equal(gn, pn), shape
        assert np.array_equal(gi, pi), shape
        assert np.array_equal(gd.view(np.uint32), pd.view(np.uint32)), shape
    plan.close()


def test_batched_aps_many_queries_long_partitions_and_graph(I):
    """3,000 queries over partitions of ~1,500 rows (several chunks and tiles), then the
    same batch replayed from a CUDA graph; an insert makes the graph stale."""
    import torch
    X, ids, Q = synth.aps_search(seed=14, n=60_000, d=128, n_comp=20, sigma=1.0, nq=3000)
    levels = kmeans.build_index(X, ids, 40, 0, iters=3, seed=4)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.5)
    plan = I.ApsBatchPlan(ix, 3000, 10)
    qd = torch.from_numpy(Q).cuda()
    out = cpu(plan.search(qd, 0.9, cap0=20))
    ix.check()
    sel = np.arange(0, 3000, 15)
    orc = aps.search(levels, Q[sel], aps.Params(k=10, recall_target=0.9, f_M=(0.5,)))
    compare_search(tuple(a[sel] for a in out[:5]) + (None,), orc, 10, label="batched APS, 3,000 queries")
    stream = torch.cuda.current_stream()
    g = plan.outputs(qd)
    plan.capture(qd, 0.9, g, stream.cuda_stream)
    for t in g:
        t.zero_()
    plan.replay(stream.cuda_stream)
    torch.cuda.synchronize()
    for a, b in zip(cpu(g), out[:4]):
        assert np.array_equal(a, b)
    ix.insert(X[:5] + 0.01, np.arange(10_000_000, 10_000_005))
    from paper_2506_03437_b300 import _lib as L
    with pytest.raises(L.QkError):
        plan.replay(stream.cuda_stream)
    out2 = cpu(plan.search(qd, 0.9))                # a plain call follows the index
    assert (out2[0] >= 0).all()


def test_batched_aps_refuses_bad_queries_and_answers_the_rest(I, two_level):
    import torch
    from paper_2506_03437_b300 import _lib as L
    X, ids, Q, levels, orc = two_level
    ix = make_index(I, X, ids, levels, f_M_leaf=0.1, f_M_parent=0.5)
    plan = I.ApsBatchPlan(ix, Q.shape[0], 10)
    Qb = Q.copy()
    Qb[3, 5] = np.nan
    Qb[7, 0] = np.inf
    out = cpu(plan.search(torch.from_numpy(Qb).cuda(), 0.9, cap0=30))
    with pytest.raises(L.QkError):
        ix.check()
    assert (out[0][[3, 7]] == -1).all() and (out[2][[3, 7]] == 0).all() and (out[4][[3, 7]] == -1).all()
    good = np.setdiff1d(np.arange(Q.shape[0]), [3, 7])
    for j in good:
        assert same_topk(out[0][j], out[1][j], orc["ids"][j], orc["dist"][j])
    # arguments the plan refuses
    with pytest.raises(L.QkError):
        plan.search(torch.from_numpy(Q).cuda(), 0.0)
    with pytest.raises(L.QkError):
        I.ApsBatchPlan(ix, 10, 64)                  # k > 32


def test_autotune_keeps_results():
    """Every shape qk_aps_batch_autotune times sums a row in the same order: the batch
    after tuning equals the batch before it, bit for bit."""
    import torch
    from paper_2506_03437_b300 import index as I, synth
    X, ids, Q = synth.aps_search(seed=71, n=60_000, d=128, n_comp=60, sigma=1.2, nq=1500)
    ix = I.Index(128, n_leaf=120, n_parent=8, kmeans_iters=3, seed=2)
    Xd, idd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(ids).cuda(), torch.from_numpy(Q).cuda()
    ix.build(Xd, idd)
    plan = I.ApsBatchPlan(ix, 1500, 10)
    before = [t.clone() for t in plan.search(Qd, 0.9)[:3]]
    chosen = plan.autotune(Qd, 0.9, reps=1)
    after = plan.search(Qd, 0.9)
    torch.cuda.synchronize()
    assert chosen[0] in (1, 2, 4) and chosen[1] in (16, 32, 64) and chosen[2] in (1024, 4096, 16384)
    assert all(bool((a == b).all()) for a, b in zip(before, after[:3]))
    plan.close()
