"""Checkpoint and resume (qk_save / qk_restore; the paper has no counterpart): an index restored
from a file searches, updates and maintains exactly as the one that was saved."""

import numpy as np
import pytest

from oracle import kmeans

from .test_gpu_maintain import scenario
from .test_gpu_search import make_index

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def I():
    from paper_2506_03437_b300 import index
    return index


def same_partitions(a, b, level):
    sa, ca, ia = a.export_level(level)
    sb, cb, ib = b.export_level(level)
    assert np.array_equal(sa, sb) and np.array_equal(ca, cb)
    off = np.concatenate([[0], np.cumsum(sa)])
    for j in range(len(sa)):
        assert set(ia[off[j]:off[j + 1]].tolist()) == set(ib[off[j]:off[j + 1]].tolist())


def codes_by_id(ix):
    _, _, ids = ix.export_level(0)
    codes, scales = ix.export_quantized()
    return {int(i): codes[r].tobytes() for r, i in enumerate(ids)}, scales


@pytest.mark.parametrize("storage", ["f32", "fp8"])
def test_restored_index_answers_and_maintains_like_the_saved_one(I, tmp_path, storage):
    from paper_2506_03437_b300 import _lib as L
    code = {"f32": L.STORE_F32, "fp8": L.STORE_FP8}[storage]
    X, ids, Q = scenario()
    levels = kmeans.build_index(X, ids, 24, 5, iters=5, seed=11)
    a = make_index(I, X, ids, levels, f_M_leaf=0.25, f_M_parent=1.0, seed=1234, storage=code)
    a.search(Q, 10, recall_target=0.0, nprobe=2)
    # updates first: FP8 rows inserted now keep their partition's current scale (some saturate)
    g = np.random.default_rng(4)
    new = (1.7 * X[:200] + 0.1 * g.standard_normal((200, X.shape[1]))).astype(np.float32)
    a.insert(new, np.arange(10 ** 6, 10 ** 6 + 200, dtype=np.int64))
    assert a.delete(ids[::7]) == ids[::7].shape[0]
    a.search(Q[:100], 10, recall_target=0.9)
    path = tmp_path / "index.qkb"
    a.save(path)
    b = I.Index.restore(path)
    assert b.info() == a.info() and b.cfg.storage == code and b.cfg.seed == a.cfg.seed
    for lv in (0, 1):
        same_partitions(a, b, lv)
        assert np.array_equal(a.hits(lv), b.hits(lv))
    if storage == "fp8":
        ka, sa = codes_by_id(a)
        kb, sb = codes_by_id(b)
        assert ka == kb and np.array_equal(sa, sb)
    ra, rb = a.search(Q, 10, recall_target=0.9), b.search(Q, 10, recall_target=0.9)
    for x, y in zip(ra, rb):
        assert np.array_equal(x, y, equal_nan=True)
    # the statistics window and counters came along: the same pass on both
    kw = dict(tau_us=0.01, alpha=0.9, refine_radius=4, s_min=120, split_iters=8)
    la = a.maintain([0, 1000], [5.0, 55.0], **kw)
    lb = b.maintain([0, 1000], [5.0, 55.0], **kw)
    assert [(x["level"], x["kind"], x["partition"], x["committed"]) for x in la] == \
           [(x["level"], x["kind"], x["partition"], x["committed"]) for x in lb]
    assert any(x["committed"] for x in la)
    for lv in (0, 1):
        same_partitions(a, b, lv)
    ra, rb = a.search(Q, 10, recall_target=0.9), b.search(Q, 10, recall_target=0.9)
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])


def test_bad_checkpoints_are_refused(I, tmp_path):
    from paper_2506_03437_b300 import _lib as L
    X, ids, Q = scenario()
    levels = kmeans.build_index(X[:3000], ids[:3000], 6, 0, iters=2, seed=1)
    a = make_index(I, X[:3000], ids[:3000], levels)
    path = tmp_path / "a.qkb"
    a.save(path)
    raw = path.read_bytes()
    cases = {"missing": None, "not a checkpoint": b"hello world" + raw[11:], "truncated": raw[:len(raw) // 2]}
    flipped = bytearray(raw)
    flipped[len(raw) // 2] ^= 0x40    # one bit inside the rows
    cases["corrupt"] = bytes(flipped)
    for name, data in cases.items():
        p = tmp_path / f"{name.replace(' ', '_')}.qkb"
        if data is not None:
            p.write_bytes(data)
        with pytest.raises(L.QkError) as e:
            I.Index.restore(p)
        assert e.value.status == L.ERR_IO, name
    with pytest.raises(L.QkError) as e:
        I.Index(X.shape[1], n_leaf=4).save(tmp_path / "empty.qkb")
    assert e.value.status == L.ERR_STATE
    b = I.Index.restore(path)     # the intact file still loads
    assert b.info() == a.info()
