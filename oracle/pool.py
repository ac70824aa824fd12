"""The oracle's searches over query chunks in spawned processes (oracle; test and timing
infrastructure only).

The arithmetic is the oracle's, unchanged: every worker runs `aps.search` (or, for a fixed nprobe
per query, `aps.ivf_search`), one query at a time, on its own share of the queries.  The workers
are spawned, never forked, so a parent that has already used a GPU can start them.  Level-0 rows
and ids go through shared memory, so the workers see them without a copy.  The workers start with
OMP_NUM_THREADS / OPENBLAS_NUM_THREADS / MKL_NUM_THREADS = 1, so each holds one BLAS thread and
`workers` is the number of cores used.
"""

import contextlib
import multiprocessing as mp
import os
import time
from multiprocessing import shared_memory

import numpy as np

BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def available_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


@contextlib.contextmanager
def _one_thread_env():
    old = {v: os.environ.get(v) for v in BLAS_VARS}
    try:
        for v in BLAS_VARS:
            os.environ[v] = "1"
        yield
    finally:
        for v, x in old.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x


def _worker(job):
    from . import aps
    from . import kmeans as km

    (xname, iname, n, d, sizes, C0, upper, Q, how, seconds) = job
    xs = shared_memory.SharedMemory(name=xname)
    ish = shared_memory.SharedMemory(name=iname)
    try:
        X = np.ndarray((n, d), np.float32, buffer=xs.buf)
        I = np.ndarray((n,), np.int64, buffer=ish.buf)
        off = np.concatenate([[0], np.cumsum(sizes)])
        lv0 = km.Level(C0, [X[off[j]:off[j + 1]] for j in range(len(sizes))],
                       [I[off[j]:off[j + 1]] for j in range(len(sizes))])
        levels = [lv0] + list(upper)
        done = 0
        t0 = time.perf_counter()
        while done < Q.shape[0] and time.perf_counter() - t0 < seconds:
            if how[0] == "aps":
                aps.search(levels, Q[done:done + 1], how[1])
            else:
                aps.ivf_search(lv0, Q[done:done + 1], how[1], how[2][done:done + 1])
            done += 1
        el = time.perf_counter() - t0
        del levels, lv0, X, I
    finally:
        xs.close()
        ish.close()
    return done, el


def _run(levels, Q, hows, seconds, workers):
    lv0 = levels[0]
    sizes = lv0.sizes()
    n, d = int(sizes.sum()), lv0.centroids.shape[1]
    xs = shared_memory.SharedMemory(create=True, size=max(1, n * d * 4))
    ish = shared_memory.SharedMemory(create=True, size=max(1, n * 8))
    try:
        X = np.ndarray((n, d), np.float32, buffer=xs.buf)
        I = np.ndarray((n,), np.int64, buffer=ish.buf)
        if n:
            X[:] = np.concatenate(lv0.vectors)
            I[:] = np.concatenate(lv0.ids)
        del X, I
        jobs = [(xs.name, ish.name, n, d, sizes, lv0.centroids, levels[1:], Q[w::workers], hows[w], seconds)
                for w in range(workers)]
        with _one_thread_env():
            with mp.get_context("spawn").Pool(workers) as pool:
                res = pool.map(_worker, jobs)
    finally:
        xs.close()
        xs.unlink()
        ish.close()
        ish.unlink()
    rate = sum(dn / el for dn, el in res if el > 0)
    return rate, sum(dn for dn, _ in res)


def search_rate(levels, Q, prm, seconds, workers):
    """Queries per second of `aps.search(levels, ., prm)` over `workers` processes, each running
    for at most `seconds` on every workers-th query.  Returns (rate, queries done)."""
    return _run(levels, Q, [("aps", prm)] * workers, seconds, workers)


def ivf_rate(level, Q, k, nprobe, seconds, workers):
    """The same for the fixed-nprobe search `aps.ivf_search(level, ., k, nprobe[i])`."""
    nprobe = np.asarray(nprobe)
    return _run([level], Q, [("ivf", k, nprobe[w::workers]) for w in range(workers)], seconds, workers)
