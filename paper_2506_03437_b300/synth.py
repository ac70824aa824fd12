"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it holds none of the method's
arithmetic, so both the CUDA library's tests and the CPU oracle can take their
inputs from it.  Every generator uses numpy's PCG64 with an explicit seed.

Workload shapes (the paper's datasets are not available; these stand in):
  plain IVF      10,000 x 64 from a 50-component isotropic Gaussian mixture,
                 centres ~ N(0, I), sigma 0.2; 100 queries from the mixture.
  APS search     1,000,000 x 128 from a 1,000-component mixture, sigma 1.5
                 (Sift1M-like: APS at recall target 0.9 scans ~24 of 1,000
                 partitions), 10,000 queries whose component is drawn Zipf(1.1).
  batching       5,000,000 x 256 in 20,000 components with Zipf(1.0) sizes
                 clipped to [10, 100,000]; each query has its own nprobe.
"""

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def mixture_centers(n_comp, d, seed):
    """Component centres ~ N(0, I)."""
    return rng(seed).standard_normal((n_comp, d)).astype(np.float32)


def mixture_samples(centers, n, sigma, seed, labels=None, chunk=1 << 18):
    """n rows = centre[label] + sigma * N(0, I); labels uniform unless given."""
    g = rng(seed)
    n_comp, d = centers.shape
    if labels is None:
        labels = g.integers(0, n_comp, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        X[s:e] = centers[labels[s:e]] + np.float32(sigma) * g.standard_normal((e - s, d), dtype=np.float32)
    return X, labels


def zipf_labels(n_comp, n, a, seed):
    """Component per sample with P(rank r) ~ r^-a over a seeded permutation of components."""
    g = rng(seed)
    w = np.arange(1, n_comp + 1, dtype=np.float64) ** (-a)
    w /= w.sum()
    perm = g.permutation(n_comp)
    ranks = g.choice(n_comp, size=n, p=w)
    return perm[ranks]


def zipf_sizes(n_part, total, a, lo, hi):
    """Partition sizes ~ r^-a, clipped to [lo, hi] and rescaled to sum to `total`."""
    w = np.arange(1, n_part + 1, dtype=np.float64) ** (-a)
    s = w / w.sum() * total
    for _ in range(100):
        s = np.clip(s, lo, hi)
        free = (s > lo) & (s < hi)
        deficit = total - s.sum()
        if abs(deficit) < 0.5 or not free.any():
            break
        s[free] *= 1.0 + deficit / s[free].sum()
    s = np.clip(np.floor(s).astype(np.int64), lo, hi)
    i = 0
    while s.sum() < total:
        if s[i % n_part] < hi:
            s[i % n_part] += 1
        i += 1
    while s.sum() > total:
        if s[i % n_part] > lo:
            s[i % n_part] -= 1
        i += 1
    return s


def unit_rows(X):
    n = np.linalg.norm(X, axis=1, keepdims=True)
    n[n == 0] = 1
    return (X / n).astype(np.float32)


# ----------------------------------------------------------------- workloads

def plain_ivf(seed=1235, n=10_000, d=64, n_comp=50, sigma=0.2, nq=100):
    """Single-level plain IVF workload (10k x 64, 50 components, sigma 0.2)."""
    C = mixture_centers(n_comp, d, seed)
    X, _ = mixture_samples(C, n, sigma, seed + 1)
    Q, _ = mixture_samples(C, nq, sigma, seed + 2)
    return X, np.arange(n, dtype=np.int64), Q


def aps_search(seed=1236, n=1_000_000, d=128, n_comp=1000, sigma=1.5, nq=10_000, zipf=1.1):
    """Two-level APS workload (1M x 128, 1,000 components, Zipf(1.1) queries)."""
    C = mixture_centers(n_comp, d, seed)
    X, _ = mixture_samples(C, n, sigma, seed + 1)
    Q = aps_queries(seed, d, n_comp, sigma, nq, zipf)
    return X, np.arange(n, dtype=np.int64), Q


def aps_queries(seed, d, n_comp, sigma, nq, zipf=1.1, stream=0):
    """Queries of the APS workload; stream > 0 gives further independent batches."""
    C = mixture_centers(n_comp, d, seed)
    lab = zipf_labels(n_comp, nq, zipf, seed + 2 + 1000 * stream)
    Q, _ = mixture_samples(C, nq, sigma, seed + 3 + 1000 * stream, labels=lab)
    return Q


def zipf_partitions(seed=1238, n=5_000_000, d=256, n_part=20_000, a=1.0, lo=10, hi=100_000,
                    spread=0.3, nq=4096, nprobe_lo=1, nprobe_hi=500):
    """Batching workload: rows grouped in Zipf-sized components, per-query nprobe.

    Returns X, ids, labels (the component of each row, which is its partition),
    queries, and one log-uniform nprobe per query.
    """
    sizes = zipf_sizes(n_part, n, a, lo, hi)
    C = mixture_centers(n_part, d, seed)
    lab = np.repeat(np.arange(n_part, dtype=np.int64), sizes)
    X, _ = mixture_samples(C, n, spread, seed + 1, labels=lab)
    g = rng(seed + 2)
    qlab = g.integers(0, n_part, size=nq)
    Q, _ = mixture_samples(C, nq, spread, seed + 3, labels=qlab)
    u = g.uniform(np.log(nprobe_lo), np.log(nprobe_hi + 1), size=nq)
    nprobe = np.clip(np.floor(np.exp(u)).astype(np.int32), nprobe_lo, nprobe_hi)
    return X, np.arange(n, dtype=np.int64), lab, Q, nprobe


def unit_mixture(seed=1237, n=200_000, d=768, n_comp=100, s=2.0, nq=64, chunk=1 << 16):
    """The precision workload's recipe on the host (numpy PCG64), for sizes the
    oracle can search: n unit-norm rows x = normalize(mu_c + (s / sqrt(d)) g)
    around n_comp directions mu uniform on the sphere, component uniform per
    row, and nq queries from the same mixture.  Returns FP32 (X, ids, Q)."""
    g = rng(seed)
    mu = g.standard_normal((n_comp, d))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    scale = s / d ** 0.5

    def draw(m):
        out = np.empty((m, d), dtype=np.float32)
        for a in range(0, m, chunk):
            b = min(m, a + chunk)
            lab = g.integers(0, n_comp, size=b - a)
            x = mu[lab] + scale * g.standard_normal((b - a, d))
            out[a:b] = x / np.linalg.norm(x, axis=1, keepdims=True)
        return out
    X = draw(n)
    return X, np.arange(n, dtype=np.int64), draw(nq)


def unit_mixture_cuda(seed=1237, n=10_000_000, d=768, n_comp=5000, s=1.0, nq=1024, chunk=1 << 20):
    """Precision workload, generated on the GPU (torch Philox, seeded): n unit-norm rows
    x = normalize(mu_c + (s / sqrt(d)) g) around n_comp directions mu uniform on the sphere,
    component uniform per row, and nq queries from the same mixture.  Returns CUDA tensors
    (X, Q) in FP32.  The mean cosine between a row and its direction is about 1/sqrt(1 + s^2)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    mu = torch.randn((n_comp, d), generator=g, device="cuda")
    mu /= mu.norm(dim=1, keepdim=True)
    scale = s / d ** 0.5

    def draw(m):
        out = torch.empty((m, d), dtype=torch.float32, device="cuda")
        for a in range(0, m, chunk):
            b = min(m, a + chunk)
            lab = torch.randint(0, n_comp, (b - a,), generator=g, device="cuda")
            x = mu[lab] + scale * torch.randn((b - a, d), generator=g, device="cuda")
            out[a:b] = x / x.norm(dim=1, keepdim=True)
        return out
    return draw(n), draw(nq)
