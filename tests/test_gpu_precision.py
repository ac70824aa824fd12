"""Low-precision storage (BF16, FP8 E4M3 with per-partition scales), the FP32 re-rank,
and inner-product APS, against the oracle."""

import numpy as np
import pytest

from oracle import aps, kmeans, knn, quant
from paper_2506_03437_b300 import synth

from .parity import compare_search, exact_dist, same_topk
from .test_gpu_search import load_args

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


def make(I, X, ids, levels, **cfg):
    ix = I.Index(X.shape[1], n_leaf=levels[0].n_part, n_parent=levels[1].n_part if len(levels) > 1 else 0, **cfg)
    ix.load(X, ids, **load_args(levels, X.shape[0]))
    return ix


def codes_by_id(ix):
    sizes, _, ids = ix.export_level(0)
    codes, scales = ix.export_quantized()
    off = np.concatenate([[0], np.cumsum(sizes)])
    part = np.repeat(np.arange(len(sizes)), sizes)
    return {int(i): (codes[r], part[r]) for r, i in enumerate(ids)}, scales, off


@pytest.mark.parametrize("storage", [1, 2])
def test_quantized_codes_are_bit_exact(I, storage):
    X, ids, Q = synth.aps_search(seed=31, n=3000, d=64, n_comp=10, sigma=1.0, nq=4)
    X[5, 3] = 0.0
    levels = kmeans.build_index(X, ids, 12, 0, iters=2, seed=1)
    ix = make(I, X, ids, levels, storage=storage)
    got, scales, _ = codes_by_id(ix)
    for j in range(12):
        rows, rid = levels[0].vectors[j], levels[0].ids[j]
        if storage == 2:
            s = quant.partition_scale(rows)
            assert scales[j] == s
            want = quant.quantize_e4m3(rows, s)
        else:
            want = quant.quantize_bf16(rows)
        for r, i in enumerate(rid[::5]):
            assert np.array_equal(got[int(i)][0], want[::5][r]), (j, int(i))
    # inserted rows use their partition's existing scale (saturating beyond it)
    if storage == 2:
        nx = (X[:40] * 3).astype(np.float32)
        ni = np.arange(90_000, 90_040, dtype=np.int64)
        ix.insert(nx, ni)
        got, scales2, _ = codes_by_id(ix)
        assert np.array_equal(scales2, scales)
        for x, i in zip(nx, ni):
            c, part = got[int(i)]
            assert np.array_equal(c, quant.quantize_e4m3(x[None, :], scales[part])[0])


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("metric", [0, 1])
def test_rerank_of_all_candidates_is_exact(I, storage, metric):
    X, ids, Q = synth.aps_search(seed=32, n=900, d=128, n_comp=6, sigma=1.0, nq=12)
    if metric == 1:
        X, Q = synth.unit_rows(X), synth.unit_rows(Q)
    levels = kmeans.build_index(X, ids, 9, 0, iters=2, seed=2)
    ix = make(I, X, ids, levels, storage=storage, rerank=100, metric=metric, f_M_leaf=1.0)
    gi, gd, gn, gr = ix.search(Q, 10, recall_target=0.0, nprobe=9)
    D, Ix = knn.knn(X, ids, Q, 10, metric=metric)
    for j in range(Q.shape[0]):
        assert same_topk(gi[j], gd[j], Ix[j], D[j])


def test_low_precision_recall_against_fp64(I):
    X, ids, Q = synth.aps_search(seed=33, n=40_000, d=128, n_comp=40, sigma=1.5, nq=200)
    levels = kmeans.build_index(X, ids, 100, 0, iters=4, seed=3)
    gtD, _ = knn.knn(X, ids, Q, 10, bulk=True)
    rec = {}
    for storage in (0, 1, 2):
        ix = make(I, X, ids, levels, storage=storage, rerank=4, f_M_leaf=0.3)
        gi, gd, gn, gr = ix.search(Q, 10, recall_target=0.0, nprobe=20)
        ex = exact_dist(X, Q, gi)
        rec[storage] = knn.recall_at_k(gi, ex, gtD, 10).mean()
        # the distances returned are exact FP32 distances of the returned ids
        ok = gi >= 0
        np.testing.assert_allclose(gd[ok], ex[ok], rtol=1e-5, atol=1e-4)
    assert rec[1] >= rec[0] - 0.01 and rec[2] >= rec[0] - 0.03, rec


def test_inner_product_aps_matches_oracle(I):
    X, ids, Q = synth.aps_search(seed=34, n=20_000, d=128, n_comp=40, sigma=1.0, nq=100)
    X, Q = synth.unit_rows(X), synth.unit_rows(Q)
    levels = kmeans.build_index(X, ids, 120, 8, iters=4, seed=4)
    ix = make(I, X, ids, levels, metric=1, f_M_leaf=0.15, f_M_parent=0.5)
    out = ix.search_scanned(Q, 10, recall_target=0.9, cap0=18, cap1=4)
    orc = aps.search(levels, Q, aps.Params(k=10, recall_target=0.9, f_M=(0.15, 0.5)), metric=knn.IP)
    compare_search(out, orc, 10, label="APS inner product, two levels")


def test_inner_product_on_the_unit_sphere_is_the_l2_search(I):
    """Reading R11 on the GPU: with unit-norm rows and queries, the two-level inner-product
    search makes the L2 search's choices and its distances are (d_L2 - 2) / 2; recall
    against FP64 brute force is high for both."""
    X, ids, Q = synth.aps_search(seed=35, n=60_000, d=256, n_comp=300, sigma=1.0, nq=200)
    X, Q = synth.unit_rows(X), synth.unit_rows(Q)
    levels = kmeans.build_index(X, ids, 200, 12, iters=4, seed=5)
    l2 = make(I, X, ids, levels, metric=0, f_M_leaf=0.1, f_M_parent=0.25)
    ip = make(I, X, ids, levels, metric=1, f_M_leaf=0.1, f_M_parent=0.25)
    a = l2.search(Q, 10, recall_target=0.9)
    b = ip.search(Q, 10, recall_target=0.9)
    same = np.mean([np.array_equal(a[0][j], b[0][j]) and a[2][j] == b[2][j] for j in range(Q.shape[0])])
    assert same >= 0.97
    ok = a[0] >= 0
    np.testing.assert_allclose(b[1][ok], (a[1][ok] - 2.0) / 2.0, atol=2e-5)
    D, Ix = knn.knn(X, ids, Q, 10, metric=knn.IP)
    rec = np.mean([len(set(b[0][j]) & set(Ix[j])) / 10 for j in range(Q.shape[0])])
    assert rec >= 0.85


def test_precision_shaped_aps_matches_oracle(I):
    """The precision workload's shape at a size the oracle searches in seconds:
    200k unit-norm rows, d = 768, inner product, k = 100, two levels (10 parents
    over 200 leaves of ~1,000 rows), APS at target 0.9, FP32 storage.  Every
    query's selections at both levels, nprobe, r and top-100 must equal the
    oracle's."""
    X, ids, Q = synth.unit_mixture(seed=1240, n=200_000, d=768, n_comp=100, s=2.0, nq=48)
    levels = kmeans.build_index(X, ids, 200, 10, iters=3, seed=8)
    ix = make(I, X, ids, levels, metric=1, f_M_leaf=0.1, f_M_parent=0.3)
    out = ix.search_scanned(Q, 100, recall_target=0.9, cap0=20, cap1=3)
    orc = aps.search(levels, Q, aps.Params(k=100, recall_target=0.9, f_M=(0.1, 0.3)), metric=knn.IP)
    compare_search(out, orc, 100, label="APS 200k x 768 inner product, k = 100")
    assert out[2].max() > 1                      # the leaf level really adapted
    # and recall@10 / @100 of the FP32 path against FP64 brute force
    gtD, _ = knn.knn(X, ids, Q, 100, metric=knn.IP, bulk=True)
    rec = knn.recall_at_k(out[0], exact_dist(X, Q, out[0], knn.IP), gtD, 100).mean()
    assert rec > 0.5


@pytest.mark.parametrize("d,metric,storage", [(768, 1, 2), (768, 1, 0), (128, 0, 0), (128, 0, 1)])
def test_upper_levels_by_the_prepare_kernel_change_nothing(I, d, metric, storage):
    """qk_search may walk the upper levels with the warp-per-query prepare kernel and import
    its candidates and t_i (qk_set_search_upper 1) instead of walking them in each query's
    CTA (0): ids, distances, nprobe and r must be the same bit for bit, in every storage
    form and metric."""
    if metric == 1:
        X, ids, Q = synth.unit_mixture(seed=1250 + d, n=60_000, d=d, n_comp=60, s=2.0, nq=64)
    else:
        X, ids, Q = synth.aps_search(seed=1250 + d, n=60_000, d=d, n_comp=60, sigma=1.0, nq=64)
    levels = kmeans.build_index(X, ids, 240, 12, iters=3, seed=9)
    ix = make(I, X, ids, levels, metric=metric, storage=storage, f_M_leaf=0.1, f_M_parent=0.5)
    k = 100 if metric == 1 else 10
    ix.set_search_upper(0)
    a = ix.search(Q, k, recall_target=0.9)
    ix.set_search_upper(1)
    b = ix.search(Q, k, recall_target=0.9)
    ix.set_search_upper(-1)
    c = ix.search(Q, k, recall_target=0.9)
    ix.check()
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x.view(np.uint8), y.view(np.uint8))
        assert np.array_equal(x.view(np.uint8), z.view(np.uint8))
    assert a[2].max() > 1
    with pytest.raises(Exception):
        ix.set_search_upper(2)
