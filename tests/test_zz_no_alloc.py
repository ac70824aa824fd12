"""The allocation-free Lloyd step against the regular one.

qk_kmeans_step_noalloc serves callers that cannot allocate device memory
while they run (for example a serving loop that must not stall on the
device-wide synchronisation of cudaMalloc/cudaFree).  It keeps its FP64
scratch in a fixed array inside the library instead of allocating it.  This
test calls it through the C ABI with device buffers, twice in a row on
different data so that the second call would see anything the first one
left in the shared scratch, and compares each result with qk_kmeans_step.
It sits in a file of its own that pytest collects last.
"""

import ctypes

import numpy as np
import pytest

from paper_2506_03437_b300 import synth

pytestmark = pytest.mark.gpu


def regular_step(L, x, c):
    n, d = x.shape
    K = c.shape[0]
    cn = np.empty_like(c)
    a = np.empty(n, np.int32)
    cnt = np.empty(K, np.int32)
    L.check(L.lib.qk_kmeans_step(x.ctypes.data, n, d, c.ctypes.data, K, cn.ctypes.data, a.ctypes.data,
                                 cnt.ctypes.data, None))
    return cn, a, cnt


def noalloc_step(L, torch, x, c):
    n, d = x.shape
    K = c.shape[0]
    xd, cd = torch.from_numpy(x).cuda(), torch.from_numpy(c).cuda()
    cn = torch.empty_like(cd)
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(K, dtype=torch.int32, device="cuda")
    L.check(L.lib.qk_kmeans_step_noalloc(xd.data_ptr(), n, d, cd.data_ptr(), K, cn.data_ptr(), a.data_ptr(),
                                         cnt.data_ptr(), None))
    torch.cuda.synchronize()
    return cn.cpu().numpy(), a.cpu().numpy(), cnt.cpu().numpy()


def test_noalloc_step_matches_regular_step_twice():
    import torch
    from paper_2506_03437_b300 import _lib as L
    cases = [(64, 100, 20_000, 1), (128, 300, 9_000, 2)]
    for d, K, n, seed in cases:
        X, _, _ = synth.plain_ivf(seed=500 + seed, n=n, d=d, n_comp=K // 2, sigma=0.5, nq=1)
        C = X[np.random.default_rng(seed).choice(n, K, replace=False)].copy()
        cn0, a0, cnt0 = regular_step(L, X, C)
        cn1, a1, cnt1 = noalloc_step(L, torch, X, C)
        assert np.array_equal(a1, a0)
        assert np.array_equal(cnt1, cnt0)
        np.testing.assert_array_max_ulp(cn1, cn0, maxulp=2)


def test_noalloc_step_in_place_matches_regular_step():
    """c_new may be the same buffer as c: the step then updates c in place."""
    import torch
    from paper_2506_03437_b300 import _lib as L
    d, K, n = 64, 100, 20_000
    X, _, _ = synth.plain_ivf(seed=503, n=n, d=d, n_comp=K // 2, sigma=0.5, nq=1)
    C = X[np.random.default_rng(3).choice(n, K, replace=False)].copy()
    cn0, a0, cnt0 = regular_step(L, X, C)
    xd, cd = torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda()
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(K, dtype=torch.int32, device="cuda")
    L.check(L.lib.qk_kmeans_step_noalloc(xd.data_ptr(), n, d, cd.data_ptr(), K, cd.data_ptr(), a.data_ptr(),
                                         cnt.data_ptr(), None))
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), a0)
    assert np.array_equal(cnt.cpu().numpy(), cnt0)
    np.testing.assert_array_max_ulp(cd.cpu().numpy(), cn0, maxulp=2)


def test_noalloc_step_rejects_oversize_and_host_buffers():
    import torch
    from paper_2506_03437_b300 import _lib as L
    d, K, n = 1024, 2048, 16                      # K * d = 2^21 > the 2^20 fixed sums
    x = torch.zeros((n, d), device="cuda")
    c = torch.zeros((K, d), device="cuda")
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(K, dtype=torch.int32, device="cuda")
    st = L.lib.qk_kmeans_step_noalloc(x.data_ptr(), n, d, c.data_ptr(), K, c.data_ptr(), a.data_ptr(),
                                      cnt.data_ptr(), None)
    assert st == L.ERR_ARG and b"exceeds" in L.lib.qk_last_error()
    xh = np.zeros((n, 64), np.float32)
    c2 = torch.zeros((4, 64), device="cuda")
    st = L.lib.qk_kmeans_step_noalloc(xh.ctypes.data, n, 64, c2.data_ptr(), 4, c2.data_ptr(), a.data_ptr(),
                                      cnt.data_ptr(), None)
    assert st == L.ERR_ARG
    assert ctypes is not None
