"""GPU parity of the batched fixed-nprobe search (one nprobe per query, Zipf-sized
partitions, grouped scan) and of the per-query kernel with per-query nprobe, against
the oracle's per-query IVF search."""

import numpy as np
import pytest

from oracle import aps, kmeans, knn, maintenance
from paper_2506_03437_b300 import synth

from .parity import DIST_RTOL, same_topk
from .test_gpu_search import load_args

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


def zipf_index(seed, n, d, n_part, hi, nq, np_hi, n_empty=0):
    """Oracle level of a Zipf-partitioned workload; partitions are the components,
    centroids their FP64 means rounded to FP32.  n_empty extra partitions hold no rows."""
    X, ids, lab, Q, nprobe = synth.zipf_partitions(seed=seed, n=n, d=d, n_part=n_part, lo=2, hi=hi, nq=nq,
                                                   nprobe_lo=1, nprobe_hi=np_hi)
    C = np.zeros((n_part + n_empty, d), np.float64)
    np.add.at(C, lab, X.astype(np.float64))
    C[:n_part] /= np.bincount(lab, minlength=n_part)[:, None]
    if n_empty:
        C[n_part:] = synth.rng(seed + 9).standard_normal((n_empty, d))
    levels = kmeans.index_from_assignment(X, ids, C.astype(np.float32), lab)
    return X, ids, Q, nprobe.astype(np.int32), levels


def make(I, X, levels):
    ix = I.Index(X.shape[1], n_leaf=levels[0].n_part, n_parent=0)
    ix.load(X, np.arange(X.shape[0], dtype=np.int64), **load_args(levels, X.shape[0]))
    return ix


def boundary_tie(level, q, n, rtol=DIST_RTOL):
    """True if the n-th and (n+1)-th nearest centroids are within rtol (selection may differ)."""
    if n >= level.n_part:
        return False
    D = np.sort(knn.distances(q, level.centroids, knn.L2))
    return D[n] - D[n - 1] <= rtol * abs(D[n]) + rtol


def check_against_oracle(level, Q, nprobe, gi, gd, k, max_excused=0.02):
    D, Io, _ = aps.ivf_search(level, Q, k, nprobe)
    excused = 0
    for j in range(Q.shape[0]):
        if same_topk(gi[j], gd[j], Io[j], D[j]):
            continue
        if boundary_tie(level, Q[j], int(nprobe[j])):
            excused += 1
            continue
        raise AssertionError(f"query {j} nprobe {nprobe[j]}: gpu {list(gi[j])} {list(gd[j])}\n"
                             f"oracle {list(Io[j])} {list(D[j])}")
    assert excused <= max_excused * Q.shape[0]


@pytest.fixture(scope="module")
def small():
    return zipf_index(seed=51, n=60_000, d=64, n_part=300, hi=5000, nq=400, np_hi=60, n_empty=4)


@pytest.mark.parametrize("tiles", [(2, 32, 4096), (1, 16, 1024), (4, 64, 1024), (2, 64, 16384), (4, 64, 1024, 2)])
def test_batch_matches_oracle(I, small, tiles):
    import torch
    X, ids, Q, nprobe, levels = small
    ix = make(I, X, levels)
    plan = I.BatchPlan(ix, 512, 10, 64)
    plan.tiles = tiles
    assert plan.tiles == tuple(tiles) + (0,) * (4 - len(tiles))
    q, npd = torch.from_numpy(Q).cuda(), torch.from_numpy(nprobe).cuda()
    gi, gd = plan.search(q, npd)
    gi2, gd2 = plan.search(q, npd)
    ix.check()
    assert torch.equal(gi, gi2) and torch.equal(gd, gd2)   # deterministic
    check_against_oracle(levels[0], Q, nprobe, gi.cpu().numpy(), gd.cpu().numpy(), 10)


def test_per_query_kernel_matches_oracle(I, small):
    X, ids, Q, nprobe, levels = small
    ix = make(I, X, levels)
    gi, gd = ix.search_nprobe(Q[:200], 10, nprobe[:200])
    check_against_oracle(levels[0], Q[:200], nprobe[:200], gi, gd, 10)


@pytest.mark.parametrize("d,rows", [(32, 0), (128, 0), (256, 0), (256, 2), (192, 2)])
def test_batch_dims(I, d, rows):
    import torch
    X, ids, Q, nprobe, levels = zipf_index(seed=52 + d, n=20_000, d=d, n_part=120, hi=3000, nq=150, np_hi=30)
    ix = make(I, X, levels)
    plan = I.BatchPlan(ix, 150, 16, 40)
    if rows:
        plan.tiles = (2, 32, 4096, 2)
    gi, gd = plan.search(torch.from_numpy(Q).cuda(), torch.from_numpy(nprobe).cuda())
    ix.check()
    check_against_oracle(levels[0], Q, nprobe, gi.cpu().numpy(), gd.cpu().numpy(), 16)


def test_every_partition_is_exact_knn_and_short_lists_pad(I, small):
    import torch
    X, ids, Q, nprobe, levels = small
    ix = make(I, X, levels)
    plan = I.BatchPlan(ix, 64, 32, 2048)
    q = torch.from_numpy(Q[:40]).cuda()
    # nprobe above the number of partitions: every leaf, so exact kNN
    gi, gd = plan.search(q, torch.full((40,), 2000, dtype=torch.int32, device="cuda"))
    Dk, Ik = knn.knn(X, ids, Q[:40], 32)
    for j in range(40):
        assert same_topk(gi[j].cpu().numpy(), gd[j].cpu().numpy(), Ik[j], Dk[j])
    # nprobe 1 into partitions smaller than k: the rest is (-1, inf)
    gi, gd = plan.search(q, torch.ones(40, dtype=torch.int32, device="cuda"))
    D, Io, scanned = aps.ivf_search(levels[0], Q[:40], 32, 1)
    gi, gd = gi.cpu().numpy(), gd.cpu().numpy()
    for j in range(40):
        n = levels[0].vectors[scanned[j][0]].shape[0]
        if n < 32:
            assert np.all(gi[j, n:] == -1) and np.all(np.isinf(gd[j, n:]))
        assert same_topk(gi[j], gd[j], Io[j], D[j]) or boundary_tie(levels[0], Q[j], 1)


def test_capture_replay_and_updates(I, small):
    import copy
    import torch
    X, ids, Q, nprobe, levels = small
    levels = copy.deepcopy(levels)   # the inserts below change the oracle's copy
    ix = make(I, X, levels)
    plan = I.BatchPlan(ix, 400, 10, 64)
    q, npd = torch.from_numpy(Q).cuda(), torch.from_numpy(nprobe).cuda()
    ref = plan.search(q, npd)
    s = torch.cuda.Stream()
    out = (torch.full_like(ref[0], 7), torch.zeros_like(ref[1]))
    plan.capture(q, npd, out, s)
    out[0].fill_(7)
    out[1].zero_()
    plan.replay(s)
    plan.replay(s)
    s.synchronize()
    assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
    # an insert changes the partitions: the graph is stale, the plan follows the index
    g = np.random.default_rng(3)
    nx = (Q[:50] + 0.01 * g.standard_normal(Q[:50].shape)).astype(np.float32)
    ni = np.arange(10_000_000, 10_000_050, dtype=np.int64)
    ix.insert(nx, ni)
    maintenance.insert(levels, nx, ni)
    from paper_2506_03437_b300 import _lib as L
    with pytest.raises(L.QkError) as e:
        plan.replay(s)
    assert e.value.status == L.ERR_STATE
    gi, gd = plan.search(q, npd)
    ix.check()
    check_against_oracle(levels[0], Q, nprobe, gi.cpu().numpy(), gd.cpu().numpy(), 10)
    # the inserted near-copies of the first queries are their nearest neighbours
    assert set(gi[:50, 0].cpu().numpy().tolist()) <= set(ni.tolist())


def test_autotune_keeps_a_valid_shape(I, small):
    import torch
    X, ids, Q, nprobe, levels = small
    ix = make(I, X, levels)
    plan = I.BatchPlan(ix, 400, 10, 64)
    q, npd = torch.from_numpy(Q).cuda(), torch.from_numpy(nprobe).cuda()
    t = plan.autotune(q, npd, reps=1)
    assert t == plan.tiles and t[0] in (1, 2, 4) and t[1] in (16, 32, 64) and t[2] in (1024, 4096, 16384)
    gi, gd = plan.search(q, npd)
    check_against_oracle(levels[0], Q, nprobe, gi.cpu().numpy(), gd.cpu().numpy(), 10)


def test_invalid_arguments(I, small):
    import torch
    from paper_2506_03437_b300 import _lib as L
    X, ids, Q, nprobe, levels = small
    ix = make(I, X, levels)
    with pytest.raises(L.QkError):
        I.BatchPlan(ix, 10, 33, 10)          # k above 32
    with pytest.raises(L.QkError):
        I.BatchPlan(ix, 10, 10, 4096)        # max_nprobe above 2048
    plan = I.BatchPlan(ix, 8, 10, 16)
    q = torch.from_numpy(Q[:8]).cuda()
    gi0, gd0 = plan.search(q[:0], torch.ones(1, dtype=torch.int32, device="cuda")[:0])   # empty batch: no-op
    assert tuple(gi0.shape) == (0, 10) and tuple(gd0.shape) == (0, 10)
    with pytest.raises(L.QkError):
        plan.search(Q[:8], nprobe[:8])       # host buffers
    with pytest.raises(L.QkError):
        plan.tiles = (3, 32, 4096)
    with pytest.raises(L.QkError):
        plan.tiles = (2, 32, 512)
    with pytest.raises(L.QkError):
        plan.tiles = (4, 64, 4096, 1)        # rows_per_thread is 0 or 2
    big = torch.from_numpy(np.repeat(Q[:1], 9, axis=0)).cuda()
    with pytest.raises(L.QkError):
        plan.search(big, torch.ones(9, dtype=torch.int32, device="cuda"))   # nq above max_nq
    # an nprobe outside [1, max_nprobe] is reported by the device status word
    bad = torch.tensor([1, 0, 2, 17, 1, 1, 1, 1], dtype=torch.int32, device="cuda")
    gi, gd = plan.search(q, bad)
    with pytest.raises(L.QkError) as e:
        ix.check()
    assert e.value.status == L.ERR_ARG
    assert int(gi[1, 0]) == -1 and int(gi[3, 0]) == -1 and int(gi[0, 0]) >= 0
    # a query with a NaN or infinite element is refused the same way; the others are unchanged
    four = torch.full((8,), 4, dtype=torch.int32, device="cuda")
    ref_i, ref_d = plan.search(q, four)
    ix.check()
    ref_i, ref_d = ref_i.clone(), ref_d.clone()
    qb = q.clone()
    qb[2, 7] = float("nan")
    qb[5, 0] = float("inf")
    gi, gd = plan.search(qb, four)
    with pytest.raises(L.QkError) as e:
        ix.check()
    assert e.value.status == L.ERR_ARG
    assert bool((gi[2] == -1).all()) and bool((gi[5] == -1).all())
    for j in (0, 1, 3, 4, 6, 7):
        assert torch.equal(gi[j], ref_i[j]) and torch.equal(gd[j], ref_d[j])
    ixi = I.Index(64, n_leaf=8, metric=L.METRIC_IP)
    ixi.build(X[:2000], ids[:2000])
    with pytest.raises(L.QkError):
        I.BatchPlan(ixi, 8, 10, 4)
