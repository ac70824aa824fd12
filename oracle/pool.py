"""The oracle's APS search over query chunks in parallel processes (oracle; test and timing
infrastructure only).

The arithmetic is `aps.search` unchanged: every worker runs it, one query at a time, on its own
share of the queries.  The workers are spawned, never forked, so a parent that has already used a
GPU can start them.  Level-0 rows and ids go through shared memory: the workers see them without a
copy.  Each worker keeps its BLAS to one thread, so `cores` counts threads honestly.
"""

import multiprocessing as mp
import os
import time
from multiprocessing import shared_memory

import numpy as np


def available_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _worker(job):
    from threadpoolctl import threadpool_limits

    from . import aps
    from . import kmeans as km

    (xname, iname, n, d, sizes, C0, upper, Q, prm, seconds) = job
    xs = shared_memory.SharedMemory(name=xname)
    ish = shared_memory.SharedMemory(name=iname)
    try:
        X = np.ndarray((n, d), np.float32, buffer=xs.buf)
        I = np.ndarray((n,), np.int64, buffer=ish.buf)
        off = np.concatenate([[0], np.cumsum(sizes)])
        levels = [km.Level(C0, [X[off[j]:off[j + 1]] for j in range(len(sizes))],
                           [I[off[j]:off[j + 1]] for j in range(len(sizes))])] + list(upper)
        done = 0
        with threadpool_limits(1):
            t0 = time.perf_counter()
            while done < Q.shape[0] and time.perf_counter() - t0 < seconds:
                aps.search(levels, Q[done:done + 1], prm)
                done += 1
            el = time.perf_counter() - t0
        del levels, X, I
    finally:
        xs.close()
        ish.close()
    return done, el


def search_rate(levels, Q, prm, seconds, workers):
    """Queries per second of `aps.search` over `levels` with `workers` processes, each running
    for at most `seconds` on every workers-th query.  Returns (rate, queries done)."""
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
        jobs = [(xs.name, ish.name, n, d, sizes, lv0.centroids, levels[1:], Q[w::workers], prm, seconds)
                for w in range(workers)]
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_worker, jobs)
    finally:
        xs.close()
        xs.unlink()
        ish.close()
        ish.unlink()
    rate = sum(dn / el for dn, el in res if el > 0)
    return rate, sum(dn for dn, _ in res)
