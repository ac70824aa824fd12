"""Host logic of the request loop: net effect of an update group, stream generation."""

import numpy as np

from paper_2506_03437_b300 import synth
from paper_2506_03437_b300.serving import DELETE, INSERT, SEARCH, net_updates, skewed_stream


def apply_sequential(live, kind, ref):
    live = set(live)
    for k, r in zip(kind, ref):
        if k == INSERT:
            assert r not in live
            live.add(int(r))
        else:
            live.discard(int(r))
    return live


def apply_net(live, kind, ref):
    live = set(live)
    dpos, ipos = net_updates(np.array(kind, np.int8), np.array(ref, np.int64))
    for j in dpos:
        live.discard(int(ref[j]))
    for j in ipos:
        assert ref[j] not in live
        live.add(int(ref[j]))
    return live, dpos, ipos


def test_net_updates_cancel_and_reinsert():
    live = {1, 2, 3}
    kind = [INSERT, DELETE, DELETE, INSERT, DELETE, DELETE]
    ref = [10, 10, 2, 2, 3, 3]
    got, dpos, ipos = apply_net(live, kind, ref)
    assert got == apply_sequential(live, kind, ref) == {1, 2}
    assert sorted(int(ref[j]) for j in dpos) == [2, 3]   # 10 never reaches the index; 3 deleted once
    assert [int(ref[j]) for j in ipos] == [2]


def test_net_updates_random_groups_match_sequential():
    g = np.random.default_rng(3)
    for _ in range(200):
        live = set(range(20))
        kind, ref = [], []
        cur = set(live)
        for _ in range(g.integers(1, 40)):
            if g.random() < 0.5:
                pool = [i for i in range(40) if i not in cur]
                r = int(g.choice(pool))
                kind.append(INSERT)
                cur.add(r)
            else:
                r = int(g.integers(0, 40))   # may be absent: a no-op delete
                kind.append(DELETE)
                cur.discard(r)
            ref.append(r)
        got, _, _ = apply_net(live, kind, ref)
        assert got == apply_sequential(live, kind, ref) == cur


def test_skewed_stream_shape_and_ids():
    C = synth.mixture_centers(30, 8, 1)
    start = np.arange(500, dtype=np.int64)
    ops = skewed_stream(C, start, 5000, 0.01, 2, hot=5, rotate=1000, rate=1e4)
    assert len(ops) == 5000 and np.all(np.diff(ops.t) > 0)
    frac = np.bincount(ops.kind, minlength=3) / 5000
    assert abs(frac[SEARCH] - 0.9) < 0.02 and abs(frac[INSERT] - 0.05) < 0.01
    live = set(start.tolist())
    for k, r in zip(ops.kind, ops.ref):
        if k == INSERT:
            assert r not in live and r >= 500
            live.add(int(r))
        elif k == DELETE:
            assert r in live
            live.discard(int(r))
    # queries of one rotation epoch come from at most `hot` components
    q = ops.vec[:1000][ops.kind[:1000] == SEARCH]
    near = np.argmin(((q[:, None, :] - C[None]) ** 2).sum(-1), axis=1)
    assert len(set(near.tolist())) <= 5
