"""CPU oracle for Quake's query-time partition-scan path (Mohoney et al., OSDI'25).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
what the paper's method computes.  It exists to check the CUDA library, and it
is used only by the tests, by the package smoke check and by the CPU-baseline
leg of the benchmark.  The product path (the C-ABI library and its Python
binding) never imports, links or calls anything in here, and this package
imports nothing from the product.

Modules (each function cites the passage it follows):
  knn          exact k-nearest neighbours and Recall@k (Sec. 2.1)
  kmeans       Lloyd k-means with a SplitMix64 seeding rule, multi-level build
               (Sec. 3 "Index Structure")
  capvol       hyperspherical-cap volume fraction, exact and 1024-point table
               (Sec. 5 "Intersection Volume Approximation", Li 2010)
  aps          APS estimator (Eq. 7-9), Algorithm 1, multi-level search,
               fixed-nprobe IVF search (Sec. 3, Sec. 5)
  maintenance  cost model (Eq. 1-6), split / merge with verify, insert and
               delete (Sec. 3, Sec. 4)

Floating point: FP64 everywhere; stored vectors and centroids are FP32 values
(as in the paper's uncompressed indexes) widened to FP64 before any arithmetic.
"""

from . import knn, kmeans, capvol, aps, maintenance  # noqa: F401
