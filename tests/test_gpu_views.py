"""Copy-on-write views (Sec. 9, "Concurrency"): searches launched before an insert, a
delete, a re-load or a maintenance commit keep reading the version they were launched on
while the update runs on another stream; searches launched after it read the new one.
Every result is compared, bit for bit, with the same search run alone on that version."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, D, N_LEAF, N_PARENT, NQ, K = 200_000, 64, 400, 20, 4096, 10


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2506_03437_b300 import index as I
    torch.cuda.set_device(0)
    return torch, I


def mixture(torch, seed=7, n=N, nq=NQ):
    """Gaussian mixture on the device: 400 overlapping components in d = 64 (APS scans tens
    of partitions per query, so a batch keeps the GPU busy for about a millisecond),
    queries from the same."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    C = 1.5 * torch.randn(400, D, device="cuda", generator=g)
    X = (C[torch.randint(0, 400, (n,), device="cuda", generator=g)]
         + torch.randn(n, D, device="cuda", generator=g)).contiguous()
    Q = (C[torch.randint(0, 400, (nq,), device="cuda", generator=g)]
         + torch.randn(nq, D, device="cuda", generator=g)).contiguous()
    return X, torch.arange(n, dtype=torch.int64, device="cuda"), Q, g


def fresh(torch, I, X, ids, **kw):
    ix = I.Index(D, n_leaf=N_LEAF, n_parent=N_PARENT, kmeans_iters=4, seed=3, **kw)
    ix.build(X, ids)
    torch.cuda.synchronize()
    return ix


def outputs(torch):
    return (torch.empty((NQ, K), dtype=torch.int64, device="cuda"),
            torch.empty((NQ, K), dtype=torch.float32, device="cuda"),
            torch.empty(NQ, dtype=torch.int32, device="cuda"),
            torch.empty(NQ, dtype=torch.float32, device="cuda"))


def alone(torch, ix, Q):
    """The search run alone on the current version."""
    torch.cuda.synchronize()
    out = ix.search(Q, K, recall_target=0.9)
    torch.cuda.synchronize()
    return [t.clone() for t in out[:3]]


def same(a, b):
    return all(bool((x == y).all()) for x, y in zip(a, b))


def during(torch, ix, Q, update, target_ms=600.0, post=6):
    """Queues searches on a low-priority stream until about target_ms of work is queued,
    runs update(stream) on a high-priority stream, then queues `post` more searches.
    Returns (results launched before, results launched after, still in flight when the
    update returned)."""
    sa = torch.cuda.Stream(priority=0)
    sb = torch.cuda.Stream(priority=-1)
    probe = outputs(torch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sa)
    for _ in range(5):
        ix.search(Q, K, recall_target=0.9, out=probe, stream=sa)
    e1.record(sa)
    torch.cuda.synchronize()
    per = e0.elapsed_time(e1) / 5
    n_pre = int(min(1500, max(40, target_ms / max(per, 1e-3))))
    print(f"[views] {per:.3f} ms per batch, mean nprobe {probe[2].double().mean().item():.1f}, "
          f"{n_pre} batches queued")
    pre = [outputs(torch) for _ in range(n_pre)]
    aft = [outputs(torch) for _ in range(post)]
    torch.cuda.synchronize()
    for o in pre:
        ix.search(Q, K, recall_target=0.9, out=o, stream=sa)
    queued = torch.cuda.Event()
    queued.record(sa)
    update(sb)
    in_flight = not queued.query()
    for o in aft:
        ix.search(Q, K, recall_target=0.9, out=o, stream=sa)
    torch.cuda.synchronize()
    return pre, aft, in_flight


def check(torch, ix, Q, old, pre, aft, in_flight, label):
    new = alone(torch, ix, Q)
    assert not same(old, new), f"{label}: the update changed no result; the test shows nothing"
    assert in_flight, f"{label}: the searches had finished before the update returned"
    bad_pre = [i for i, o in enumerate(pre) if not same(o[:3], old)]
    bad_aft = [i for i, o in enumerate(aft) if not same(o[:3], new)]
    print(f"[views] {label}: {len(pre)} searches launched before the update all read the old "
          f"version ({len(bad_pre)} differ), {len(aft)} launched after read the new one ({len(bad_aft)} differ)")
    assert not bad_pre and not bad_aft


def test_insert_with_searches_in_flight(env):
    torch, I = env
    X, ids, Q, g = mixture(torch)
    ix = fresh(torch, I, X, ids)
    old = alone(torch, ix, Q)
    # near copies of 1,500 queries, 600 more around one query: results change, and that
    # query's partition outgrows its room and moves to free rows
    Xn = torch.cat([Q[:1500] + 0.01 * torch.randn(1500, D, device="cuda", generator=g),
                    Q[1500:1501] + 0.05 * torch.randn(600, D, device="cuda", generator=g)]).contiguous()
    idn = torch.arange(N, N + Xn.shape[0], dtype=torch.int64, device="cuda")
    used0 = ix.stats()["arena_used"]
    pre, aft, fl = during(torch, ix, Q, lambda s: ix.insert(Xn, idn, stream=s))
    st = ix.stats()
    assert st["arena_used"] > used0 and st["n_vectors"] == N + Xn.shape[0]
    check(torch, ix, Q, old, pre, aft, fl, "insert")


def test_delete_with_searches_in_flight(env):
    torch, I = env
    X, ids, Q, g = mixture(torch, seed=8)
    ix = fresh(torch, I, X, ids)
    old = alone(torch, ix, Q)
    gone = torch.unique(old[0][:, :3].reshape(-1))   # every query's three nearest
    pre, aft, fl = during(torch, ix, Q, lambda s: ix.delete(gone, stream=s))
    assert ix.stats()["n_vectors"] == N - gone.numel()
    check(torch, ix, Q, old, pre, aft, fl, "delete")
    assert not bool(torch.isin(ix.search(Q, K, recall_target=0.9)[0], gone).any())


def test_compaction_with_searches_in_flight(env):
    """An insert larger than the free tail lays the arena out again into new memory; the
    old arena stays allocated for the searches still reading it."""
    torch, I = env
    X, ids, Q, g = mixture(torch, seed=9)
    ix = fresh(torch, I, X, ids)
    rows0 = ix.stats()["arena_rows"]
    old = alone(torch, ix, Q)
    Xn, _, _, _ = mixture(torch, seed=10, n=120_000, nq=1)
    idn = torch.arange(N, N + 120_000, dtype=torch.int64, device="cuda")
    pre, aft, fl = during(torch, ix, Q, lambda s: ix.insert(Xn, idn, stream=s))
    assert ix.stats()["arena_rows"] > rows0
    check(torch, ix, Q, old, pre, aft, fl, "insert with compaction")


def test_reload_and_maintenance_commit_with_searches_in_flight(env):
    torch, I = env
    X, ids, Q, g = mixture(torch, seed=11)
    ix = fresh(torch, I, X, ids)
    old = alone(torch, ix, Q)
    # a build with other partitions replaces the whole structure
    pre, aft, fl = during(torch, ix, Q, lambda s: ix.build(X[:150_000], ids[:150_000], stream=s))
    check(torch, ix, Q, old, pre, aft, fl, "re-build")
    # a maintenance pass prepared beside the searches, committed while they run
    old = alone(torch, ix, Q)
    ix.search(Q[:512], K, recall_target=0.0, nprobe=4)
    log = ix.maintain_prepare([0, 1000], [5.0, 55.0], tau_us=0.01, alpha=0.9, refine_radius=4, s_min=200,
                              split_iters=4, window=512)
    assert any(a["committed"] for a in log)
    pre, aft, fl = during(torch, ix, Q, lambda s: ix.maintain_commit(stream=s))
    check(torch, ix, Q, old, pre, aft, fl, "maintenance commit")


def test_batched_plan_with_searches_in_flight(env):
    """The batched APS plan launched before an insert reads the old version too."""
    torch, I = env
    X, ids, Q, g = mixture(torch, seed=12)
    ix = fresh(torch, I, X, ids)
    plan = I.ApsBatchPlan(ix, NQ, K)
    torch.cuda.synchronize()
    old = [t.clone() for t in plan.search(Q, 0.9)[:3]]
    torch.cuda.synchronize()
    sa, sb = torch.cuda.Stream(priority=0), torch.cuda.Stream(priority=-1)
    # enough queued batches that some are still waiting when the insert returns
    pre = [plan.outputs(Q) for _ in range(2000)]
    torch.cuda.synchronize()
    for o in pre:
        plan.search(Q, 0.9, out=o, stream=sa)
    queued = torch.cuda.Event()
    queued.record(sa)
    Xn = (Q[:2000] + 0.01 * torch.randn(2000, D, device="cuda", generator=g)).contiguous()
    ix.insert(Xn, torch.arange(N, N + 2000, dtype=torch.int64, device="cuda"), stream=sb)
    fl = not queued.query()
    aft = [plan.search(Q, 0.9, stream=sa) for _ in range(3)]
    torch.cuda.synchronize()
    new = [t.clone() for t in plan.search(Q, 0.9)[:3]]
    torch.cuda.synchronize()
    assert not same(old, new) and fl
    assert all(same(o[:3], old) for o in pre)
    assert all(same(o[:3], new) for o in aft)
    plan.close()


def test_retired_rows_come_back(env):
    """Rows a moved partition leaves behind are reused once no search reads them: repeated
    deletes from the same four partitions do not grow the arena."""
    torch, I = env
    X, ids, Q, g = mixture(torch, seed=13)
    ix = fresh(torch, I, X, ids)
    sizes, _, grouped = ix.export_level(0)
    off = np.concatenate([[0], np.cumsum(sizes)])
    parts = np.argsort(-sizes)[:4]
    victims = [grouped[off[j]:off[j + 1]] for j in parts]
    used = []
    for r in range(10):
        batch = np.concatenate([v[r * 20:(r + 1) * 20] for v in victims])
        assert ix.delete(batch) == 80
        torch.cuda.synchronize()
        st = ix.stats()
        used.append(st["arena_used"])
        assert st["searches_in_flight"] == 0
    assert ix.stats()["n_vectors"] == N - 800
    room = int(sum(sizes[parts]) * 1.25 + 64)
    assert max(used[1:]) <= used[0] + room, used
    ix.insert((Q[:1] + 0.0).contiguous(), torch.tensor([10 ** 9], dtype=torch.int64, device="cuda"))
    assert ix.stats()["retired_rows"] == 0


def test_updates_from_another_thread(env):
    """One thread applies a sequence of inserts and deletes while another keeps searching the
    same index.  Every search must equal, bit for bit, the search run alone on one of the
    versions the sequence goes through, and the versions the searches see never go back.
    The versions' own results come from a second index loaded with the same partitions and
    given the same updates one by one."""
    import threading
    torch, I = env
    X, ids, Q, g = mixture(torch, seed=14)
    a = fresh(torch, I, X, ids)
    sizes, cents, grouped = a.export_level(0)
    lab = np.empty(N, np.int32)
    lab[grouped] = np.repeat(np.arange(N_LEAF, dtype=np.int32), sizes)
    s1, c1, g1 = a.export_level(1)
    pol = np.empty(N_LEAF, np.int32)
    pol[g1] = np.repeat(np.arange(N_PARENT, dtype=np.int32), s1)
    b = I.Index(D, n_leaf=N_LEAF, n_parent=N_PARENT, kmeans_iters=4, seed=3)
    b.load(X, ids, leaf_centroids=cents, leaf_of_row=lab, parent_centroids=c1, parent_of_leaf=pol)
    torch.cuda.synchronize()
    steps = []
    nxt = N
    for i in range(6):
        if i % 2 == 0:
            rows = (Q[i * 300:(i + 1) * 300] + 0.01 * torch.randn(300, D, device="cuda", generator=g)).contiguous()
            steps.append(("insert", rows, torch.arange(nxt, nxt + 300, dtype=torch.int64, device="cuda")))
            nxt += 300
        else:
            steps.append(("delete", torch.randperm(N, device="cuda", generator=g)[:500].contiguous()))
    want = [alone(torch, b, Q)]
    for st in steps:
        if st[0] == "insert":
            b.insert(st[1], st[2])
        else:
            b.delete(st[1])
        want.append(alone(torch, b, Q))
    assert all(not same(want[i], want[i + 1]) for i in range(len(steps)))
    assert same(alone(torch, a, Q), want[0])

    done = threading.Event()
    errors = []

    def updater():
        try:
            su = torch.cuda.Stream()
            for st in steps:
                if st[0] == "insert":
                    a.insert(st[1], st[2], stream=su)
                else:
                    a.delete(st[1], stream=su)
        except Exception as e:   # reported below
            errors.append(e)
        finally:
            done.set()

    ss = torch.cuda.Stream()
    got = []
    th = threading.Thread(target=updater)
    th.start()
    extra = 0
    while extra < 5:
        o = outputs(torch)
        a.search(Q, K, recall_target=0.9, out=o, stream=ss)
        ss.synchronize()
        got.append([t.clone() for t in o[:3]])
        if done.is_set():
            extra += 1
    th.join()
    assert not errors, errors
    seen = []
    for r in got:
        match = [i for i, w in enumerate(want) if same(r, w)]
        assert match, "a search matched no version"
        seen.append(match[0])
    print(f"[views] {len(got)} searches during {len(steps)} updates from another thread saw versions "
          f"{sorted(set(seen))}")
    assert seen == sorted(seen) and seen[-1] == len(steps)
