"""GPU parity of inserts and deletes (greedy descent, append, swap-with-last) against the oracle."""

import numpy as np
import pytest

from oracle import aps, kmeans, knn, maintenance
from paper_2506_03437_b300 import synth

from .parity import same_topk
from .test_gpu_search import make_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


def partitions_of(ix):
    sizes, _, ids, vec = ix.export_level(0, vectors=True)
    off = np.concatenate([[0], np.cumsum(sizes)])
    return [(ids[off[j]:off[j + 1]], vec[off[j]:off[j + 1]]) for j in range(len(sizes))]


def assert_same_partitions(ix, levels, allow_moved=()):
    got = partitions_of(ix)
    assert len(got) == levels[0].n_part
    for j, (gi, gv) in enumerate(got):
        oi, ov = levels[0].ids[j], levels[0].vectors[j]
        gs, os_ = set(gi.tolist()), set(oi.tolist())
        diff = gs ^ os_
        assert diff <= set(allow_moved), (j, sorted(diff)[:10])
        common = sorted(gs & os_)
        gmap = {int(i): v for i, v in zip(gi, gv)}
        omap = {int(i): v for i, v in zip(oi, ov)}
        for i in common[::7]:
            np.testing.assert_array_equal(gmap[i], omap[i])


def near_tied_inserts(levels, X):
    """Inserted rows whose best and second-best leaf are within FP32 noise (descent may differ)."""
    tied = []
    for r, x in enumerate(X):
        x64 = x.astype(np.float64)
        if len(levels) == 1:
            dl = ((levels[0].centroids.astype(np.float64) - x64) ** 2).sum(1)
        else:
            dp = ((levels[1].centroids.astype(np.float64) - x64) ** 2).sum(1)
            s = np.sort(dp)
            if s[1] - s[0] <= 1e-5 * s[0] + 1e-6:
                tied.append(r)
                continue
            ch = levels[1].ids[int(np.argmin(dp))]
            dl = ((levels[0].centroids[ch].astype(np.float64) - x64) ** 2).sum(1)
        s = np.sort(dl)
        if len(s) > 1 and s[1] - s[0] <= 1e-5 * s[0] + 1e-6:
            tied.append(r)
    return tied


@pytest.mark.parametrize("two_level", [False, True])
def test_insert_delete_sequence_matches_oracle(I, two_level):
    X, ids, Q = synth.aps_search(seed=21, n=12_000, d=64, n_comp=30, sigma=1.0, nq=30)
    levels = kmeans.build_index(X, ids, 60, 6 if two_level else 0, iters=4, seed=8)
    ix = make_index(I, X, ids, levels, f_M_leaf=1.0, f_M_parent=1.0, upper_recall=2.0)
    g = np.random.default_rng(9)
    live = {int(i): X[n] for n, i in enumerate(ids)}
    next_id = 1_000_000
    moved = []
    for step in range(6):
        # inserts: new samples near existing rows (write skew towards a few components)
        hot = g.choice(X.shape[0], 5)
        nx = (X[np.repeat(hot, 150)] + 0.3 * g.standard_normal((750, 64))).astype(np.float32)
        ni = np.arange(next_id, next_id + 750, dtype=np.int64)
        next_id += 750
        tied = near_tied_inserts(levels, nx)
        moved += [int(ni[r]) for r in tied]
        maintenance.insert(levels, nx, ni)
        ix.insert(nx, ni)
        for x, i in zip(nx, ni):
            live[int(i)] = x
        # deletes: random live ids, some inserted in this batch, plus unknown ids
        cand = np.array(sorted(live), dtype=np.int64)
        dl = np.concatenate([g.choice(cand, 400, replace=False), np.array([-5, 987_654_321])])
        n_or = maintenance.delete(levels, dl)
        n_gpu = ix.delete(dl)
        assert n_gpu == n_or == 400
        for i in dl:
            live.pop(int(i), None)
        assert ix.info()["n"] == len(live)
        assert_same_partitions(ix, levels, allow_moved=moved)
    # a full scan over the updated index is exact kNN over the live set
    allI = np.array(sorted(live), dtype=np.int64)
    allX = np.stack([live[int(i)] for i in allI])
    gi, gd, gn, gr = ix.search(Q, 10, recall_target=2.0)
    D, Ix = knn.knn(allX, allI, Q, 10)
    for j in range(Q.shape[0]):
        assert same_topk(gi[j], gd[j], Ix[j], D[j])


def test_insert_grows_a_full_partition_and_keeps_everything(I):
    X, ids, Q = synth.aps_search(seed=22, n=3000, d=128, n_comp=10, sigma=1.0, nq=10)
    levels = kmeans.build_index(X, ids, 20, 0, iters=3, seed=3)
    ix = make_index(I, X, ids, levels, f_M_leaf=1.0)
    c = levels[0].centroids[4]
    g = np.random.default_rng(1)
    nx = (c[None, :] + 0.01 * g.standard_normal((2000, 128))).astype(np.float32)   # all land in leaf 4
    ni = np.arange(50_000, 52_000, dtype=np.int64)
    ix.insert(nx, ni)
    maintenance.insert(levels, nx, ni)
    sizes, _, _ = ix.export_level(0)
    assert sizes[4] == levels[0].vectors[4].shape[0] >= 2000
    assert_same_partitions(ix, levels)
    allX = np.concatenate([X, nx])
    allI = np.concatenate([ids, ni])
    gi, gd, gn, gr = ix.search(Q, 5, recall_target=0.0, nprobe=20)
    D, Ix = knn.knn(allX, allI, Q, 5)
    for j in range(Q.shape[0]):
        assert same_topk(gi[j], gd[j], Ix[j], D[j])


def test_duplicate_and_nan_inserts_apply_nothing(I):
    from paper_2506_03437_b300 import _lib as L
    X, ids, Q = synth.aps_search(seed=23, n=2000, d=64, n_comp=5, sigma=1.0, nq=4)
    levels = kmeans.build_index(X, ids, 8, 0, iters=2, seed=3)
    ix = make_index(I, X, ids, levels)
    before = partitions_of(ix)
    with pytest.raises(L.QkError) as e:
        ix.insert(X[:3], np.array([9000, 9001, 5], np.int64))          # 5 exists
    assert e.value.status == L.ERR_DUP_ID
    with pytest.raises(L.QkError) as e:
        ix.insert(X[:2], np.array([9000, 9000], np.int64))             # repeated in the batch
    assert e.value.status == L.ERR_DUP_ID
    bad = X[:2].copy()
    bad[1, 7] = np.nan
    with pytest.raises(L.QkError) as e:
        ix.insert(bad, np.array([9000, 9001], np.int64))
    assert e.value.status == L.ERR_ARG
    after = partitions_of(ix)
    assert ix.info()["n"] == 2000
    for (a, _), (b, _) in zip(before, after):
        assert np.array_equal(a, b)
    assert ix.delete(np.array([], np.int64)) == 0
    assert ix.delete(np.array([123456], np.int64)) == 0


@pytest.mark.parametrize("storage", [0, 2])
def test_partitions_move_to_the_tail_and_compact(I, storage):
    """Repeated inserts into two partitions: each overflow moves the partition to the
    arena's free tail, and once the tail is used up the arena is compacted.  After every
    round the partitions hold what the oracle's do, and the FP8 codes follow their rows."""
    from oracle import quant
    X, ids, Q = synth.aps_search(seed=24, n=8000, d=64, n_comp=16, sigma=1.0, nq=12)
    levels = kmeans.build_index(X, ids, 16, 0, iters=3, seed=4)
    ix = make_index(I, X, ids, levels, f_M_leaf=1.0, storage=storage)
    scales0 = ix.export_quantized()[1].copy() if storage == 2 else None
    g = np.random.default_rng(5)
    allX, allI = [X], [ids]
    next_id = 500_000
    for rnd in range(24):
        leaf = (3, 7, 11)[rnd % 3]
        c = levels[0].centroids[leaf]
        nx = (c[None, :] + 0.01 * g.standard_normal((90, 64))).astype(np.float32)
        ni = np.arange(next_id, next_id + 90, dtype=np.int64)
        next_id += 90
        ix.insert(nx, ni)
        maintenance.insert(levels, nx, ni)
        allX.append(nx)
        allI.append(ni)
        assert_same_partitions(ix, levels)
    if storage == 2:
        sizes, _, gid = ix.export_level(0)
        codes, scales = ix.export_quantized()
        assert np.array_equal(scales, scales0)
        part = np.repeat(np.arange(len(sizes)), sizes)
        byid = {int(i): r for r, i in enumerate(gid)}
        X_all, I_all = np.concatenate(allX), np.concatenate(allI)
        for n in range(0, X_all.shape[0], 13):
            r = byid[int(I_all[n])]
            assert np.array_equal(codes[r], quant.quantize_e4m3(X_all[n][None, :], scales[part[r]])[0])
    X_all, I_all = np.concatenate(allX), np.concatenate(allI)
    gi, gd, gn, gr = ix.search(Q, 10, recall_target=0.0, nprobe=16)
    D, Ix = knn.knn(X_all, I_all, Q, 10)
    for j in range(Q.shape[0]):
        if storage == 0:
            assert same_topk(gi[j], gd[j], Ix[j], D[j])
        else:   # FP8 candidates re-ranked in FP32: every returned distance is exact
            assert np.all(np.isin(gi[j], I_all))
