"""Repeatability: a search gives bitwise the same results every time, also when launches on two
streams are in flight together.  Each query is answered by one CTA in a fixed order over a
partition's rows, and equal distances are ordered by id."""

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


@pytest.mark.parametrize("storage", ["f32", "fp8"])
def test_search_is_bitwise_repeatable(I, storage):
    import torch
    from paper_2506_03437_b300 import _lib as L
    code = {"f32": L.STORE_F32, "fp8": L.STORE_FP8}[storage]
    X, ids, Q = scenario()
    levels = kmeans.build_index(X, ids, 24, 5, iters=5, seed=11)
    ix = make_index(I, X, ids, levels, f_M_leaf=0.25, f_M_parent=1.0, seed=1234, storage=code)
    first = ix.search(Q, 10, recall_target=0.9)
    again = ix.search(Q, 10, recall_target=0.9)
    qd = torch.from_numpy(Q).cuda()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        a = ix.search(qd, 10, recall_target=0.9, stream=s1)
    with torch.cuda.stream(s2):
        b = ix.search(qd, 10, recall_target=0.9, stream=s2)
    torch.cuda.synchronize()
    ix.check()
    for r in (again, tuple(t.cpu().numpy() for t in a), tuple(t.cpu().numpy() for t in b)):
        for x, y in zip(first, r):
            assert np.array_equal(x, y, equal_nan=True)
    fixed = [ix.search(Q, 10, recall_target=0.0, nprobe=3) for _ in range(2)]
    for x, y in zip(*fixed):
        assert np.array_equal(x, y, equal_nan=True)
